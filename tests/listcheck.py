"""Brute-force quadtree checks from the definitions of Sec. 7.2 of the paper:
colleagues, U, V, W and X lists computed by testing every pair of boxes."""
from __future__ import annotations

import numpy as np


def box_squares(tree):
    """Closed squares of every box in integer units of the finest level."""
    lev = tree["level"].astype(np.int64)
    L = int(lev.max())
    sh = (L - lev)
    lo = tree["ij"].astype(np.int64) << sh[:, None]
    hi = (tree["ij"].astype(np.int64) + 1) << sh[:, None]
    return lo, hi


def brute_lists(tree):
    nb = tree["level"].shape[0]
    lev = tree["level"]
    child = tree["child"]
    leaf = np.all(child < 0, axis=1)
    parent = np.full(nb, -1)
    for b in range(nb):
        for c in child[b]:
            if c >= 0:
                parent[c] = b
    lo, hi = box_squares(tree)

    def touching(b):
        """boxes whose closed square meets b's (includes ancestors, descendants, b)."""
        return np.all((lo <= hi[b]) & (hi >= lo[b]), axis=1)

    def inside(b):
        """boxes contained in b (descendants and b)."""
        return np.all((lo >= lo[b]) & (hi <= hi[b]), axis=1)

    def contains(b):
        return np.all((lo <= lo[b]) & (hi >= hi[b]), axis=1)

    adj = []
    for b in range(nb):
        a = touching(b) & ~inside(b) & ~contains(b)
        adj.append(a)
    U, V, W = [], [], []
    for b in range(nb):
        # V: children of the parent's colleagues (same level as b) not adjacent to b
        if lev[b] >= 2:
            P = parent[b]
            coll_p = np.nonzero((lev == lev[P]) & (adj[P] | (np.arange(nb) == P)))[0]
            kids = child[coll_p].ravel()
            kids = kids[kids >= 0]
            V.append(sorted(int(d) for d in kids if d != b and not adj[b][d]))
        else:
            V.append([])
        if leaf[b]:
            U.append(sorted([b] + [int(d) for d in np.nonzero(adj[b] & leaf)[0]]))
            cand = np.nonzero((lev > lev[b]) & ~adj[b])[0]
            W.append(sorted(int(d) for d in cand if parent[d] >= 0 and adj[b][parent[d]]))
        else:
            U.append([])
            W.append([])
    X = [[] for _ in range(nb)]
    for b in range(nb):
        for d in W[b]:
            X[d].append(b)
    X = [sorted(x) for x in X]
    return dict(U=U, V=V, W=W, X=X, leaf=leaf, parent=parent)


def check_tree(tree, xy_by_class, n_max, crad=None, kappa=4.0, max_level=24):
    """Particle containment, partition of ranges and the split rule: a box is split
    iff it holds more than n_max sources + centres + targets and its children are at
    least kappa times as wide as the radius of every centre it holds."""
    nb = tree["level"].shape[0]
    x0, y0, side = tree["root"]
    lev = tree["level"]
    child = tree["child"]
    leaf = np.all(child < 0, axis=1)
    perms = [tree["perm_src"], tree["perm_ctr"], tree["perm_tgt"], None]
    for t in range(3):
        xy = xy_by_class[t]
        if xy.shape[0] == 0:
            continue
        perm = perms[t][:xy.shape[0]]
        assert np.array_equal(np.sort(perm), np.arange(xy.shape[0]))
        for b in np.nonzero(leaf)[0]:
            r0, r1 = tree["range"][b, t]
            if r1 <= r0:
                continue
            pts = xy[perm[r0:r1]]
            s = side / 2.0 ** lev[b]
            bx0 = x0 + tree["ij"][b, 0] * s
            by0 = y0 + tree["ij"][b, 1] * s
            tol = 1e-9 * side
            assert np.all(pts[:, 0] >= bx0 - tol) and np.all(pts[:, 0] <= bx0 + s + tol)
            assert np.all(pts[:, 1] >= by0 - tol) and np.all(pts[:, 1] <= by0 + s + tol)
    cnt = np.zeros(nb, np.int64)
    for t in range(3):
        cnt += tree["range"][:, t, 1] - tree["range"][:, t, 0]
    assert np.all(cnt[~leaf] > n_max)
    wide = np.ones(nb, bool)
    if crad is not None:
        pc = tree["perm_ctr"][:crad.shape[0]]
        for b in range(nb):
            r0, r1 = tree["range"][b, 1]
            if r1 > r0:
                child_side = side / 2.0 ** (lev[b] + 1)
                wide[b] = kappa * crad[pc[r0:r1]].max() <= child_side
    assert np.all(wide[~leaf])
    assert np.all((cnt[leaf] <= n_max) | (lev[leaf] >= max_level) | ~wide[leaf])
    for b in np.nonzero(~leaf)[0]:
        for t in range(4):
            tot = 0
            for c in child[b]:
                if c >= 0:
                    tot += tree["range"][c, t, 1] - tree["range"][c, t, 0]
            assert tot == tree["range"][b, t, 1] - tree["range"][b, t, 0]
