"""Seeded generators of graded block trees for tests (no method arithmetic).

A tree is a set of leaves (level, (cx, cy, cz)) covering the periodic unit
box.  ``random_graded_tree`` refines random leaves and then closes the tree
under the 2:1 rule (level difference <= 1 across faces, edges and corners) by
geometric adjacency tests written independently of both implementations.
"""
import itertools

import numpy as np


def _cells(dim, lvl, c):
    return lvl, tuple(int(x) for x in c[:dim])


def uniform_tree(dim, lvl):
    n = 1 << lvl
    rng = [range(n)] * dim
    return {(lvl, c) for c in itertools.product(*rng)}


def _touch(dim, a, b):
    """Closed cells a=(la, ca), b=(lb, cb) of the periodic unit box touch (share a point)."""
    la, ca = a
    lb, cb = b
    L = max(la, lb)
    for ax in range(dim):
        n = 1 << L
        a0 = ca[ax] << (L - la); a1 = (ca[ax] + 1) << (L - la)
        b0 = cb[ax] << (L - lb); b1 = (cb[ax] + 1) << (L - lb)
        ok = False
        for s in (-n, 0, n):
            if a0 <= b1 + s and b0 + s <= a1:
                ok = True
                break
        if not ok:
            return False
    return True


def is_graded(dim, leaves):
    ls = list(leaves)
    for i, a in enumerate(ls):
        for b in ls[i + 1:]:
            if abs(a[0] - b[0]) > 1 and _touch(dim, a, b):
                return False
    return True


def refine_leaf(dim, leaf):
    lvl, c = leaf
    out = []
    for bits in itertools.product((0, 1), repeat=dim):
        out.append((lvl + 1, tuple(2 * c[a] + bits[a] for a in range(dim))))
    return out


def random_graded_tree(dim, jmin, jmax, nref, seed):
    rng = np.random.default_rng(seed)
    leaves = set(uniform_tree(dim, jmin))
    for _ in range(nref):
        cand = sorted(x for x in leaves if x[0] < jmax)
        if not cand:
            break
        leaf = cand[rng.integers(len(cand))]
        leaves.remove(leaf)
        leaves.update(refine_leaf(dim, leaf))
        # 2:1 closure: refine any leaf that touches a leaf two levels finer
        changed = True
        while changed:
            changed = False
            ls = sorted(leaves)
            for a in ls:
                if a not in leaves:
                    continue
                for b in ls:
                    if b[0] - a[0] > 1 and _touch(dim, a, b):
                        leaves.remove(a)
                        leaves.update(refine_leaf(dim, a))
                        changed = True
                        break
    assert is_graded(dim, leaves)
    return sorted(leaves)


def as_arrays(leaves):
    lvl = np.array([x[0] for x in leaves], np.int32)
    crd = np.zeros((len(leaves), 3), np.int64)
    for n, x in enumerate(leaves):
        crd[n, :len(x[1])] = x[1]
    return lvl, crd
