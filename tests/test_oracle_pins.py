"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, index or coefficient, a transposed operand) fails it:

* prediction P exact for cubics; details of x^4 equal 9 h^4 (closed form);
* refine-then-coarsen returns the mother bit-exactly (Sec. 2.3, nested grids);
* 4th-order D1 exact for quartics; one RK4 step on a Fourier mode equals the
  closed-form amplification R(lambda dt) (Sec. 3: 4th-order FD + RK4);
* conservation on periodic uniform grids; 4th-order convergence (Fig. 4B);
* swirl reverses to its initial state at t = t_a (Sec. 3, Eq. 1);
* ghost synchronisation of a cubic on an adaptive graded tree is exact;
* neighbour table equals brute-force geometric point location; 16 / 74
  relations (Sec. 2.2);
* flag fixpoint independent of visit order; compression -> 1 as eps -> 0;
* only status +1 is refined (Sec. 2.3); the error norms weight each physical
  node once by dx^d (the L2 norm of a Gaussian in closed form).
"""
import itertools
import math

import numpy as np
import pytest

from tests import treegen


def mk(oracle_mod, **kw):
    cfg = dict(dim=2, Bs=17, ng=4, Jmin=2, Jmax=3, eps=1e-3, rhs="adv",
               rhs_params=(1.0, 0.5, 0.0), ic="none")
    cfg.update(kw)
    return oracle_mod.Oracle(cfg)


def node_xyz(B, dim, lvl, crd, L=1.0):
    """Physical coordinates (unwrapped) of the interior nodes of one block."""
    h = L / ((B - 1) * (1 << lvl))
    ax = [(crd[a] * (B - 1) + np.arange(B)) * h for a in range(dim)]
    return np.meshgrid(*ax[::-1], indexing="ij")[::-1]  # x, y(, z) arrays [z][y][x]


def fill(o, leaves, f):
    lvl, crd = treegen.as_arrays(leaves)
    B, d = o.B, o.dim
    fields = np.zeros((len(leaves), 1) + (B,) * d)
    for n in range(len(leaves)):
        X = node_xyz(B, d, lvl[n], crd[n])
        fields[n, 0] = f(*[np.mod(x, 1.0) for x in X])
    o.set_blocks(lvl, crd, fields)
    return lvl, crd


def cubic2(x, y):
    return 1.0 + 2.0 * x - 3.0 * y + x * x * y - 0.5 * x ** 3 + 0.7 * y ** 3 + x * y * y


def cubic3(x, y, z):
    return cubic2(x, y) + 0.3 * z ** 3 - x * y * z + 0.25 * z * z


# --------------------------------------------------------------- prediction --
@pytest.mark.parametrize("dim", [2, 3])
def test_refine_is_exact_for_cubics(oracle_mod, dim):
    B, g = (17, 4) if dim == 2 else (9, 2)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=2, Jmax=3)
    f = cubic2 if dim == 2 else cubic3
    fill(o, treegen.uniform_tree(dim, 2), f)
    o.refine(0)
    b = o.blocks()
    assert o.errors == 0
    checked = 0
    for n in range(o.n):
        c = b["coords"][n][:dim]
        parent = c // 2
        if np.all((parent >= 1) & (parent <= 2)):  # stencil never crosses the periodic seam
            X = node_xyz(B, dim, b["level"][n], c)
            np.testing.assert_allclose(b["fields"][n, 0], f(*X), rtol=0, atol=1e-12)
            checked += 1
    assert checked == (2 ** dim) * (2 ** dim)


def test_details_of_quartic_closed_form(oracle_mod):
    # d = f - P(R f) at a midpoint of a 4-point interpolating stencil is
    # f''''/4! * (3/2 * 1/2 * 1/2 * 3/2) H^4 = 9 h^4 for f = x^4 (H = 2h).
    o = mk(oracle_mod, Jmin=3, Jmax=3)
    fill(o, treegen.uniform_tree(2, 3), lambda x, y: x ** 4)
    o.details()
    b = o.blocks(fields=False)
    h = 1.0 / (16 * 8)
    inner = [n for n in range(o.n) if 1 <= b["coords"][n][0] <= 6]
    assert len(inner) == 6 * 8
    np.testing.assert_allclose(b["mdet"][inner], 9.0 * h ** 4, rtol=1e-6)


@pytest.mark.parametrize("dim", [2, 3])
def test_refine_then_coarsen_returns_mother_bit_exactly(oracle_mod, dim):
    B, g = (17, 4) if dim == 2 else (9, 2)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=2, Jmax=3, eps=1e300)
    # random values on the global level-2 lattice (redundant block-edge nodes
    # hold one value, as Sec. 2.5 assumes), sampled by every block
    rng = np.random.default_rng(7)
    leaves = sorted(treegen.uniform_tree(dim, 2))
    lvl, crd = treegen.as_arrays(leaves)
    n = (B - 1) * 4
    glob = rng.standard_normal((n,) * dim)
    fields = np.zeros((len(leaves), 1) + (B,) * dim)
    for q in range(len(leaves)):
        idx = [np.mod(crd[q, a] * (B - 1) + np.arange(B), n) for a in range(dim)]
        fields[q, 0] = glob[np.ix_(*idx[::-1])]
    o.set_blocks(lvl, crd, fields)
    before = o.blocks()
    o.refine(0)
    assert o.n == len(leaves) * 2 ** dim
    o.details()
    assert o.flags(0) == o.n
    o.coarsen()
    after = o.blocks()
    assert np.array_equal(before["level"], after["level"])
    assert np.array_equal(before["coords"], after["coords"])
    assert np.array_equal(before["fields"], after["fields"])


# --------------------------------------------------------------- FD + RK4 ----
def test_d1_exact_for_quartic(oracle_mod):
    o = mk(oracle_mod, Jmin=3, Jmax=3, rhs_params=(1.0, 0.5, 0.0))
    f = lambda x, y: x ** 4 - x * y ** 3 + 0.5 * y ** 4
    fill(o, treegen.uniform_tree(2, 3), f)
    k = o.rhs(0.0)
    b = o.blocks(fields=False)
    for n in range(o.n):
        c = b["coords"][n][:2]
        if np.all((c >= 1) & (c <= 6)):
            x, y = node_xyz(17, 2, 3, c)
            fx = 4 * x ** 3 - y ** 3
            fy = -3 * x * y ** 2 + 2 * y ** 3
            np.testing.assert_allclose(k[n, 0], -(1.0 * fx + 0.5 * fy), rtol=0, atol=1e-9)


def test_rk4_step_on_fourier_mode_matches_closed_form(oracle_mod):
    lvl, B, u, dt = 3, 17, 1.0, 3e-3
    o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, rhs_params=(u, 0.0, 0.0))
    w = 2 * math.pi
    fill(o, treegen.uniform_tree(2, lvl), lambda x, y: np.sin(w * x))
    o.rk4(0.0, dt)
    h = 1.0 / ((B - 1) * (1 << lvl))
    kappa = (8 * math.sin(w * h) - math.sin(2 * w * h)) / (6 * h)
    z = -1j * u * kappa * dt
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    b = o.blocks()
    for n in range(o.n):
        x, y = node_xyz(B, 2, lvl, b["coords"][n][:2])
        ex = R.real * np.sin(w * x) + R.imag * np.cos(w * x)
        np.testing.assert_allclose(b["fields"][n, 0], ex, rtol=0, atol=2e-14)


def unique_sum(o, v=0):
    b = o.blocks()
    sl = (slice(None), v) + (slice(0, o.B - 1),) * o.dim
    h = 1.0 / ((o.B - 1) * (1 << b["level"].astype(np.int64)))
    return float(np.sum(b["fields"][sl].reshape(o.n, -1).sum(1) * h ** o.dim))


def test_mass_conserved_on_uniform_periodic_grid(oracle_mod):
    o = mk(oracle_mod, Jmin=3, Jmax=3, ic="gauss", ic_params=(0.3, 0.6, 0.0, 0.08))
    o.set_blocks(*treegen.as_arrays(sorted(treegen.uniform_tree(2, 3))))
    o.set_ic(0.0)
    m0 = unique_sum(o)
    for s in range(5):
        o.rk4(s * 2e-3, 2e-3)
    assert abs(unique_sum(o) - m0) <= 1e-14 * abs(m0) * 10


def test_fourth_order_convergence_uniform(oracle_mod):
    # Fig. 4B: error decays with order ~4 in the grid spacing
    errs = []
    T = 0.05
    for lvl in (2, 3, 4):
        o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, ic="gauss", ic_params=(0.5, 0.5, 0.0, 0.1),
               rhs_params=(1.0, 0.5, 0.0))
        o.set_blocks(*treegen.as_arrays(sorted(treegen.uniform_tree(2, lvl))))
        o.set_ic(0.0)
        h = 1.0 / (16 * (1 << lvl))
        n = int(math.ceil(T / (0.5 * h / math.hypot(1.0, 0.5))))
        dt = T / n
        for s in range(n):
            o.rk4(s * dt, dt)
        errs.append(o.error(T)["linf_abs"])
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 3.5, (errs, orders)


def test_swirl_returns_to_initial_state(oracle_mod):
    # Sec. 3: the time-periodic swirl reverses the deformation at t = t_a.
    ta = 0.25
    o = mk(oracle_mod, Jmin=2, Jmax=3, eps=1e-4, rhs="swirl", rhs_params=(ta,),
           ic="gauss", ic_params=(0.5, 0.75, 0.0, math.sqrt(0.01 / 2)))
    o.init_tree()
    h = 1.0 / (16 * 8)
    n = int(math.ceil(ta / (0.5 * h)))
    dt = ta / n
    half = None
    for s in range(n):
        o.step(s * dt, dt)
        if s + 1 == n // 2:
            half = o.error(0.0)["linf"]
    end = o.error(0.0)["linf"]
    assert o.errors == 0
    assert half > 0.05 and end < half / 20, (half, end)


# ------------------------------------------------------------------ sync ----
def _adaptive_tree(dim):
    leaves = set(treegen.uniform_tree(dim, 2))
    for c in itertools.product((1, 2), repeat=dim):
        leaves.remove((2, c))
        leaves.update(treegen.refine_leaf(dim, (2, c)))
    for c in itertools.product((3, 4), repeat=dim):
        leaves.remove((3, c))
        leaves.update(treegen.refine_leaf(dim, (3, c)))
    leaves = sorted(leaves)
    assert treegen.is_graded(dim, leaves)
    return leaves


@pytest.mark.parametrize("dim", [2, 3])
def test_sync_of_cubic_is_exact_on_adaptive_tree(oracle_mod, dim):
    B, g = (17, 4) if dim == 2 else (9, 2)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=2, Jmax=4)
    f = cubic2 if dim == 2 else cubic3
    fill(o, _adaptive_tree(dim), f)
    o.sync()
    assert o.errors == 0
    t = o.tiles()
    b = o.blocks(fields=False)
    T = B + 2 * g
    for n in range(o.n):
        lv, c = b["level"][n], b["coords"][n]
        h = 1.0 / ((B - 1) * (1 << lv))
        ax = [np.mod((c[a] * (B - 1) + np.arange(-g, B + g)) * h, 1.0) for a in range(dim)]
        X = np.meshgrid(*ax[::-1], indexing="ij")[::-1]
        np.testing.assert_allclose(t[n, 0], f(*X), rtol=0, atol=1e-11)
    assert t.shape[-1] == T


# ------------------------------------------------------------ neighbours ----
def _relations(dim):
    """Relation order: faces, edges, corners (by number of nonzero components),
    directions with x fastest; non-corner directions get a full entry then one
    entry per child touching the block (x fastest among the zero axes)."""
    rel = []
    rngs = [(-1, 0, 1)] * dim
    dirs = [s[::-1] for s in itertools.product(*rngs[::-1])]
    for nnz in range(1, dim + 1):
        for s in dirs:
            if sum(1 for v in s if v) != nnz:
                continue
            rel.append((s, -1))
            if nnz < dim:
                for sub in range(1 << (dim - nnz)):
                    rel.append((s, sub))
    return rel


def _locate(dim, leaves, point):
    """Leaf whose open cell contains the point (brute force over all leaves)."""
    hits = []
    for lv, c in leaves:
        w = 1.0 / (1 << lv)
        if all(c[a] * w < point[a] % 1.0 < (c[a] + 1) * w for a in range(dim)):
            hits.append((lv, c))
    assert len(hits) == 1, (point, hits)
    return hits[0]


def _expected_neighbours(dim, leaves, leaf, rel):
    lv, c = leaf
    out = []
    for s, sub in rel:
        corner = all(v != 0 for v in s)
        # child of the neighbouring cell that touches the block, chosen by sub
        z = 0
        child = []
        for a in range(dim):
            if s[a] != 0:
                bit = 1 if s[a] < 0 else 0
            else:
                bit = ((0 if sub < 0 else sub) >> z) & 1
                z += 1
            child.append(2 * (c[a] + s[a]) + bit)
        w = 1.0 / (1 << (lv + 1))
        centre = [(child[a] + 0.5) * w for a in range(dim)]
        hit = _locate(dim, leaves, centre)
        if sub < 0:
            ok = hit[0] <= lv or corner
        else:
            ok = hit[0] == lv + 1
        out.append((hit, hit[0] - lv) if ok else None)
    return out


@pytest.mark.parametrize("dim,jmin,jmax,seed", [(2, 1, 4, 1), (2, 1, 4, 2), (2, 1, 5, 3), (3, 1, 3, 4),
                                                (2, 2, 4, 5), (3, 2, 3, 6)])
def test_neighbour_table_matches_point_location(oracle_mod, dim, jmin, jmax, seed):
    # jmin 2: leaves at Jmin itself touch finer leaves (coarser neighbours at Jmin)
    leaves = treegen.random_graded_tree(dim, jmin, jmax, 6 if dim == 2 else 3, seed)
    B, g = (17, 4) if dim == 2 else (9, 2)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=jmin, Jmax=jmax)
    o.set_blocks(*treegen.as_arrays(leaves))
    assert o.nrel == {2: 16, 3: 74}[dim]  # Sec. 2.2
    rel = _relations(dim)
    assert len(rel) == o.nrel
    nbr, dl = o.neighbors()
    b = o.blocks(fields=False)
    ids = [(int(b["level"][n]), tuple(int(x) for x in b["coords"][n][:dim])) for n in range(o.n)]
    for n, leaf in enumerate(ids):
        exp = _expected_neighbours(dim, leaves, leaf, rel)
        for r, e in enumerate(exp):
            if e is None:
                assert nbr[n, r] == -1, (leaf, rel[r])
            else:
                assert nbr[n, r] >= 0, (leaf, rel[r], e)
                assert ids[nbr[n, r]] == e[0] and dl[n, r] == e[1], (leaf, rel[r], e)


def test_treecode_digits_and_level(oracle_mod):
    # Sec. 2.2: one digit per level, so the level is the treecode length.
    leaves = treegen.random_graded_tree(2, 1, 4, 5, 11)
    o = mk(oracle_mod, Jmin=1, Jmax=4)
    o.set_blocks(*treegen.as_arrays(leaves))
    b = o.blocks(fields=False)
    for n in range(o.n):
        lv, (cx, cy) = int(b["level"][n]), b["coords"][n][:2]
        digits = [((cx >> (lv - 1 - k)) & 1) + 2 * ((cy >> (lv - 1 - k)) & 1) for k in range(lv)]
        code = 0
        for dgt in digits:
            code = code * 4 + dgt
        assert int(b["treecode"][n]) == code and len(digits) == lv


@pytest.mark.parametrize("dim,bits", [(2, 1), (2, 4), (3, 1), (3, 3)])
def test_hilbert_key_is_a_continuous_nested_curve(oracle_mod, dim, bits):
    n = 1 << bits
    cells = list(itertools.product(range(n), repeat=dim))
    keys = [oracle_mod.Oracle.hilbert(dim, bits, c) for c in cells]
    assert sorted(keys) == list(range(n ** dim))
    order = [c for _, c in sorted(zip(keys, cells))]
    for a, b2 in zip(order, order[1:]):
        assert sum(abs(x - y) for x, y in zip(a, b2)) == 1
    # every aligned 2^d group of consecutive keys is one parent cell
    for i in range(0, len(order), 1 << dim):
        par = {tuple(x >> 1 for x in c) for c in order[i:i + (1 << dim)]}
        assert len(par) == 1


# ----------------------------------------------------------------- flags ----
def test_flag_fixpoint_independent_of_visit_order(oracle_mod):
    o = mk(oracle_mod, Jmin=2, Jmax=4, eps=1e-3, ic="gauss", ic_params=(0.4, 0.55, 0.0, 0.05))
    o.init_tree()
    o.refine(0)
    o.details()
    ref = None
    for seed in (0, 1, 2, 3, 4):
        o.flags(seed)
        f = o.blocks(fields=False)["flag"]
        if ref is None:
            ref = f
            assert (f == -2).any() and (f == 0).any()
        assert np.array_equal(f, ref)


def test_graded_after_init_and_steps(oracle_mod):
    o = mk(oracle_mod, Jmin=2, Jmax=5, eps=1e-4, ic="gauss", ic_params=(0.5, 0.5, 0.0, 0.05))
    o.init_tree()
    for s in range(3):
        o.step(s * 1e-3, 1e-3)
        b = o.blocks(fields=False)
        leaves = [(int(b["level"][n]), tuple(int(x) for x in b["coords"][n][:2])) for n in range(o.n)]
        assert treegen.is_graded(2, leaves)
    assert o.errors == 0


def test_compression_tends_to_one(oracle_mod):
    counts = []
    for eps in (1e-2, 1e-4, 1e-9):
        o = mk(oracle_mod, Jmin=2, Jmax=4, eps=eps, ic="gauss", ic_params=(0.5, 0.5, 0.0, 0.2))
        o.init_tree()
        counts.append(o.n)
    assert counts[0] <= counts[1] <= counts[2]
    assert counts[2] == 4 ** 4


def test_sync_makes_redundant_edge_nodes_single_valued(oracle_mod):
    # Sec. 2.2/2.5: a node on the edge shared by blocks holds one value after a
    # synchronisation (finer block first, equal-level copies from the block that
    # holds the node at its lower edge).  Start from independent random blocks.
    rng = np.random.default_rng(3)
    leaves = treegen.random_graded_tree(2, 1, 4, 6, 9)
    lvl, crd = treegen.as_arrays(leaves)
    o = mk(oracle_mod, Jmin=1, Jmax=4)
    o.set_blocks(lvl, crd, rng.standard_normal((len(leaves), 1, 17, 17)))
    o.sync()
    b = o.blocks()
    vals = {}
    for n in range(o.n):
        lv, (cx, cy) = int(b["level"][n]), b["coords"][n][:2]
        s = 1 << (4 - lv)  # node spacing in level-4 units
        for j in (0, 16):
            for i in range(17):
                for (ii, jj) in ((i, j), (j, i)):
                    key = (((cx * 16 + ii) * s) % 256, ((cy * 16 + jj) * s) % 256)
                    v = b["fields"][n, 0, jj, ii]
                    assert vals.setdefault(key, v) == v, (key, v, vals[key])


# --------------------------------------------- refinement status, error norm --
def test_refine_flagged_refines_only_status_plus_one(oracle_mod):
    # Sec. 2.3: only blocks with status +1 are refined (not -1, -2 or 0), and
    # blocks at Jmax never
    leaves = treegen.random_graded_tree(2, 2, 4, 5, 9)
    o = mk(oracle_mod, Jmin=2, Jmax=4)
    o.set_blocks(*treegen.as_arrays(leaves))
    b = o.blocks(fields=False)
    rng = np.random.default_rng(3)
    flags = rng.choice(np.array([-2, -1, 0, 1], np.int8), o.n)
    o.set_flags(flags)
    o.refine(1)
    after = o.blocks(fields=False)
    got = sorted((int(l), tuple(int(x) for x in c[:2])) for l, c in zip(after["level"], after["coords"]))
    exp = set()
    for n in range(len(flags)):
        leaf = (int(b["level"][n]), tuple(int(x) for x in b["coords"][n][:2]))
        if flags[n] == 1 and leaf[0] < 4:
            exp.update(treegen.refine_leaf(2, leaf))
        else:
            exp.add(leaf)
    assert got == sorted(exp)
    assert np.sum((flags == 1) & (b["level"] < 4)) > 2 and np.sum(flags < 0) > 2


@pytest.mark.parametrize("dim", [2, 3])
def test_error_norms_count_each_node_once_with_cell_weights(oracle_mod, dim):
    # error against the analytic field: the L2 norms carry the weight dx^d and
    # count each physical node once (a block's last node per axis is its
    # neighbour's first); the L2 norm of the Gaussian is (pi sigma^2)^(d/4)
    sig, lvl = 0.06, 3
    B, g = (17, 4) if dim == 2 else (9, 2)
    c = (0.5, 0.375, 0.625)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=lvl, Jmax=lvl, ic="gauss", ic_params=c + (sig,))
    o.init_tree()
    e0 = o.error(0.0)
    assert e0["l2_abs"] == 0.0 and e0["linf_abs"] == 0.0
    h = 1.0 / ((B - 1) << lvl)
    b = o.blocks()
    delta = 1e-3
    for where, counted in (((1,) * dim, True), ((B - 1,) * dim, False)):
        f = b["fields"].copy()
        f[0][(0,) + where[::-1]] += delta  # block 0, node (i, j[, k]) at [z][y][x]
        o.set_blocks(b["level"], b["coords"], f)
        e = o.error(0.0)
        if counted:
            assert abs(e["l2_abs"] - delta * h ** (dim / 2)) <= 1e-12 * delta
            assert e["linf_abs"] == pytest.approx(delta, rel=1e-9)
            l2_exact = e["l2_abs"] / e["l2"]
            assert abs(l2_exact - (np.pi * sig * sig) ** (dim / 4)) <= 1e-9 * l2_exact
        else:
            assert e["l2_abs"] == 0.0 and e["linf_abs"] == 0.0
