"""FP64 CPU oracle for Global QBX (test infrastructure only; see oracle.py)."""
