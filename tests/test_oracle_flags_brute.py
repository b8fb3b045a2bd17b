"""Brute-force pin of the oracle's refinement-status rule (Sec. 2.3) and of its
+1 gradedness closure (Sec. 2.2, 2.3), on every graded 2D tree with Jmin 1 and
Jmax <= 3.

The rule, as the paper states it: a block is a coarsening candidate (-1) when
its largest detail is strictly below eps and it is above Jmin; it is coarsened
(-2) only together with all 2^d sisters (each a leaf and a candidate) and only
if no block touching it is one level finer (the merged mother must stay graded);
these vetoes are applied until nothing changes.  The reference below evaluates
that rule directly from the geometry of the leaves (closed cells that share a
point), independently of the oracle's neighbour relations and treecodes.
"""
import itertools

import numpy as np

from tests import treegen

EPS = 1e-3


def all_trees(jmin=1, jmax=3, dim=2):
    """Every leaf set reachable from the uniform level-jmin grid by refinement."""
    def expand(blk):
        res = [[blk]]
        if blk[0] < jmax:
            subs = [expand(k) for k in sorted(treegen.refine_leaf(dim, blk))]
            for combo in itertools.product(*subs):
                res.append([x for part in combo for x in part])
        return res
    per = [expand(b) for b in sorted(treegen.uniform_tree(dim, jmin))]
    for combo in itertools.product(*per):
        yield [x for part in combo for x in part]


def touch_matrix(leaves, jmax, dim=2):
    """touch[i, j]: the closed cells of leaves i and j share a point (periodic box)."""
    n = 1 << jmax
    lv = np.array([l for l, _ in leaves])
    c = np.array([cc for _, cc in leaves])
    w = 1 << (jmax - lv)
    a0 = c * w[:, None]
    a1 = a0 + w[:, None]
    t = np.ones((len(leaves), len(leaves)), bool)
    for ax in range(dim):
        x0, x1 = a0[:, ax], a1[:, ax]
        ok = np.zeros_like(t)
        for s in (-n, 0, n):
            ok |= (x0[:, None] <= x1[None, :] + s) & (x0[None, :] + s <= x1[:, None])
        t &= ok
    np.fill_diagonal(t, False)
    return t


def reference_flags(leaves, mdet, jmin, jmax, eps):
    lv = np.array([l for l, _ in leaves])
    touch = touch_matrix(leaves, jmax)
    index = {b: i for i, b in enumerate(leaves)}
    f = np.where((mdet < eps) & (lv > jmin), -1, 0)
    changed = True
    while changed:
        changed = False
        for i, (l, c) in enumerate(leaves):
            if f[i] != -1:
                continue
            keep = True
            for bits in itertools.product((0, 1), repeat=2):
                sis = (l, tuple((c[a] & ~1) | bits[a] for a in range(2)))
                j = index.get(sis)
                if j is None or f[j] != -1:
                    keep = False
            if keep and np.any(touch[i] & (lv == l + 1)):
                keep = False
            if not keep:
                f[i] = 0
                changed = True
    return np.where(f == -1, -2, f)


def reference_closure(leaves, plus, jmax):
    lv = np.array([l for l, _ in leaves])
    touch = touch_matrix(leaves, jmax)
    f = plus.copy()
    changed = True
    while changed:
        changed = False
        for i in range(len(leaves)):
            if f[i] != 1 or lv[i] >= jmax:
                continue
            up = touch[i] & (lv == lv[i] - 1) & (f != 1)
            if up.any():
                f[up] = 1
                changed = True
    return f


def ordered(o, leaves):
    """Leaves in the oracle's export (Hilbert) order."""
    ob = o.blocks(fields=False)
    order = {(int(l), (int(c[0]), int(c[1]))): n for n, (l, c) in enumerate(zip(ob["level"], ob["coords"]))}
    perm = np.array([order[b] for b in leaves])
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    return [leaves[k] for k in inv]


def test_flag_rule_brute_force_all_graded_trees(oracle_mod):
    rng = np.random.default_rng(20190201)
    jmin, jmax = 1, 3
    o = oracle_mod.Oracle(dict(dim=2, Jmin=jmin, Jmax=jmax, eps=EPS, ic="none"))
    ntrees = nties = nveto = 0
    for leaves in all_trees(jmin, jmax):
        lv0 = np.array([l for l, _ in leaves])
        if np.any(touch_matrix(leaves, jmax) & (np.abs(lv0[:, None] - lv0[None, :]) > 1)):
            continue  # not graded
        lvl, crd = treegen.as_arrays(leaves)
        o.set_blocks(lvl, crd)
        leaves = ordered(o, leaves)
        # block maxima straddling eps, eps itself included (strict <)
        mdet = rng.choice([0.25 * EPS, 0.5 * EPS, EPS, np.nextafter(EPS, 0.0), 2 * EPS],
                          size=len(leaves), p=[0.35, 0.3, 0.15, 0.1, 0.1])
        o.set_mdet(mdet)
        o.flags(0)
        got = o.blocks(fields=False)["flag"]
        ref = reference_flags(leaves, mdet, jmin, jmax, EPS)
        assert np.array_equal(got, ref), (leaves, mdet, got, ref)
        ntrees += 1
        nties += int(np.sum(mdet == EPS))
        nveto += int(np.sum((mdet < EPS) & (np.array([l for l, _ in leaves]) > jmin) & (ref == 0)))
    # the enumeration covers every graded tree, ties at eps and vetoed candidates
    assert ntrees > 60000 and nties > 10000 and nveto > 10000, (ntrees, nties, nveto)


def test_refine_closure_brute_force(oracle_mod):
    # Random graded trees (Jmin 1, Jmax 4 and 5) with random +1 statuses: the
    # oracle's closure equals the geometric rule (a +1 block below Jmax raises
    # every touching leaf one level coarser, until nothing changes), and the
    # closed set refines into a graded tree.
    rng = np.random.default_rng(7)
    n = raised = 0
    for seed in range(60):
        jmax = 4 + seed % 2
        o = oracle_mod.Oracle(dict(dim=2, Jmin=1, Jmax=jmax, eps=EPS, ic="none"))
        leaves = treegen.random_graded_tree(2, 1, jmax, 4 + seed % 5, seed)
        lvl, crd = treegen.as_arrays(leaves)
        for rep in range(3):
            o.set_blocks(lvl, crd)
            lv_ = ordered(o, leaves)
            lv = np.array([l for l, _ in lv_])
            # +1 also on blocks at Jmax: they are not refined and force nothing
            plus = np.where(rng.random(len(lv_)) < 0.08, 1, 0).astype(np.int8)
            o.set_flags(plus)
            add = o.close_refine()
            got = o.blocks(fields=False)["flag"]
            ref = reference_closure(lv_, plus, jmax)
            assert np.array_equal(got, ref), (lv_, plus, got, ref)
            assert add == int(np.sum(ref != plus))
            o.refine(1)
            ob = o.blocks(fields=False)
            after = [(int(l), (int(c[0]), int(c[1]))) for l, c in zip(ob["level"], ob["coords"])]
            assert treegen.is_graded(2, set(after))
            assert len(after) == len(lv_) + 3 * int(np.sum((ref == 1) & (lv < jmax)))
            n += 1
            raised += add
    assert n == 180 and raised > 100, (n, raised)
