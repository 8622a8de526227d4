"""Values the paper prints, kept as cited text fixtures under tests/golden/,
against the library's host-side choices that follow them."""
import os

import pytest

from tests.conftest import ROOT


def _table(name):
    rows = []
    for line in open(os.path.join(ROOT, "tests", "golden", name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.fixture(scope="module")
def qbxmod():
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx


def test_default_p_add_is_table_2(qbxmod):
    rows = _table("table2_p_add.txt")
    assert [r[0] for r in rows] == [2, 4, 6, 8]
    for p, p_add in rows:
        assert qbxmod.qbx_default_p_add(p) == p_add, p


def test_default_p_add_between_and_beyond_the_table(qbxmod):
    # orders between tabulated ones take the next tabulated value; beyond p = 8
    # the last ratio p_add / p = 2.5 of the table continues, rounded up
    table = dict(_table("table2_p_add.txt"))
    for p in range(0, 9):
        nxt = min(q for q in table if q >= max(p, 2))
        assert qbxmod.qbx_default_p_add(p) == table[nxt], p
    assert table[8] / 8 == 2.5
    for p in (9, 10, 12, 16, 20):
        assert qbxmod.qbx_default_p_add(p) == -(-5 * p // 2), p
    assert qbxmod.qbx_default_p_add(12) == 30 and qbxmod.qbx_default_p_add(16) == 40
    assert qbxmod.qbx_default_p_add(-1) == -1
