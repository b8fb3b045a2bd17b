"""Pins of the oracle's shock-capturing filter (Bogey, de Cacqueray & Bailly
2009, applied after every step in Sec. 4).

* a uniform state, and a smooth state whose sensor stays below r_th, come
  back bit for bit (the strength is exactly zero);
* sensor and filter strength: a velocity wave of four nodes per period along
  x, u = a sin(pi n / 2), has dilatation a cos(pi n / 2) / dx, high-pass
  filtered dilatation half of it and magnitude M = (a / dx)^2 / 4 at every
  node, so r = a^2 / (4 c^2) + 1e-16 and s = 1 - r_th / r; the standard second-order
  filter multiplies a mode of k dx by 1 - s (1 - cos k dx) / 2, i.e.
  1 - s / 2 for this wave and 1 - s for the odd-even part of its energy.
  Amplitudes are chosen so that s is far from 0 and 1, which fixes the
  sensor's normalisation;
* the filter is a flux difference: on a periodic grid the sum of each
  conserved variable over the unique nodes is unchanged, while individual
  nodes change;
* mirror symmetry: filtering the mirror image of a state gives the mirror
  image of the filtered state (an off-by-one in the half-node strengths
  breaks this).
"""
import numpy as np
import pytest

from tests import treegen

GAM, PR, RTH = 1.4, 0.71, 1e-5


def make(oracle_mod, form, lvl, rth=RTH):
    return oracle_mod.Oracle(dict(dim=2, Bs=17, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs=form,
                                  rhs_params=(GAM, 0.0, PR, rth), ic="none", norm_kind=1))


def state(form, r, u, v, p):
    if form == "ns":
        return [r, r * u, r * v, p / (GAM - 1.0) + 0.5 * r * (u * u + v * v)]
    ph = np.sqrt(r)
    return [ph, ph * u, ph * v, p]


def set_nodes(o, form, lvl, prim):
    """prim(n, m) of global node indices (periodic, 16 * 2^lvl per axis)."""
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lvlv, crd = treegen.as_arrays(leaves)
    f = np.zeros((len(leaves), 4, 17, 17))
    for q in range(len(leaves)):
        n = crd[q, 0] * 16 + np.arange(17)
        m = crd[q, 1] * 16 + np.arange(17)
        Nn, Mm = np.meshgrid(n, m)
        f[q] = state(form, *prim(Nn, Mm))
    o.set_blocks(lvlv, crd, f)


def node_index(o):
    b = o.blocks()
    n = b["coords"][:, 0, None] * 16 + np.arange(17)[None, :]
    m = b["coords"][:, 1, None] * 16 + np.arange(17)[None, :]
    return b, n[:, None, :], m[:, :, None]


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
def test_uniform_and_smooth_states_unchanged(oracle_mod, form):
    for prim in (lambda n, m: (1.3 + 0 * n, 0.2 + 0 * n, -0.4 + 0 * n, 0.8 + 0 * n),
                 lambda n, m: (1.0 + 0.1 * np.sin(2 * np.pi * n / 64), 0.1 * np.cos(2 * np.pi * m / 64),
                               0.05 * np.sin(2 * np.pi * (n + m) / 64), 1.0 + 0 * n)):
        o = make(oracle_mod, form, 2)
        set_nodes(o, form, 2, prim)
        o.sync()  # the periodic wrap of the formula differs in the last bit at the shared edge nodes
        before = o.blocks()["fields"].copy()
        o.filter()
        assert np.array_equal(o.blocks()["fields"], before)


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
@pytest.mark.parametrize("s_target", [0.3, 0.75])
@pytest.mark.parametrize("axis", [0, 1])
def test_sensor_strength_and_transfer_function(oracle_mod, form, s_target, axis):
    p0 = 1.0
    c2 = GAM * p0
    r = RTH / (1.0 - s_target)
    a = np.sqrt(4.0 * r * c2)
    lvl = 2
    o = make(oracle_mod, form, lvl)
    if axis == 0:
        set_nodes(o, form, lvl, lambda n, m: (1.0 + 0 * n, a * np.sin(np.pi * n / 2), 0 * n, p0 + 0 * n))
    else:
        set_nodes(o, form, lvl, lambda n, m: (1.0 + 0 * n, 0 * n, a * np.sin(np.pi * m / 2), p0 + 0 * n))
    o.filter()
    b, n, m = node_index(o)
    k = n + 0 * m if axis == 0 else m + 0 * n
    f = b["fields"]
    s = 1.0 - RTH / (a * a / (4.0 * c2) + 1e-16)  # the sensor's floor 1e-16 moves s by ~1e-11
    wave = a * np.sin(np.pi * k / 2)
    assert np.allclose(f[:, 1 + axis], wave * (1.0 - s / 2.0), rtol=0, atol=1e-12 * a)
    assert np.all(f[:, 2 - axis] == 0.0)
    if form == "ns":
        assert np.all(f[:, 0] == 1.0)
        # E = p0/(g-1) + a^2/4 - a^2/4 cos(pi k): the odd-even part is scaled by 1 - s
        ex = p0 / (GAM - 1.0) + a * a / 4.0 - a * a / 4.0 * (1.0 - s) * np.cos(np.pi * k)
        assert np.allclose(f[:, 3], ex, rtol=0, atol=1e-13)
    else:
        assert np.all(f[:, 0] == 1.0) and np.all(f[:, 3] == p0)


def shock_like(n, m, N, w=None):
    """Periodic state with jumps about two nodes wide (w = 1.28 / N): rho, u
    across x = 0.4, 0.9; v, p across y = 0.45, 0.95 (where the sensor fires),
    smooth elsewhere."""
    x, y = n / N, m / N
    w = 1.28 / N if w is None else w
    sx, sy = np.tanh(np.sin(2 * np.pi * (x + 0.1)) / w), np.tanh(np.cos(2 * np.pi * (y - 0.2)) / w)
    r = 1.0 + 0.3 * sx + 0.05 * np.sin(2 * np.pi * y)
    u = 0.5 * sx + 0.1 * np.cos(2 * np.pi * y)
    v = 0.4 * sy * (1.0 + 0.2 * np.sin(2 * np.pi * x))
    p = 1.0 + 0.2 * sy + 0.05 * np.cos(2 * np.pi * x)
    return r, u, v, p


def test_flux_form_conserves_sums(oracle_mod):
    lvl = 3
    N = 16 << lvl
    o = make(oracle_mod, "ns", lvl)
    set_nodes(o, "ns", lvl, lambda n, m: shock_like(n, m, N))
    before = o.blocks()["fields"].copy()
    o.filter()
    after = o.blocks()["fields"]
    d = (after - before)[:, :, :16, :16]
    for var in range(4):
        a = np.abs(d[:, var]).sum()
        assert a > 1e-3, (var, a)
        assert abs(d[:, var].sum()) <= 1e-12 * np.abs(before[:, var, :16, :16]).sum(), var


def grid(o, N):
    """Fields of a uniform tree gathered onto the periodic N x N node grid."""
    b, n, m = node_index(o)
    g = np.zeros((4, N, N))
    for q in range(o.n):
        g[:, np.mod(m[q, :, 0], N)[:, None], np.mod(n[q, 0, :], N)[None, :]] = b["fields"][q]
    return g


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
def test_mirror_symmetry(oracle_mod, form):
    lvl = 3
    N = 16 << lvl

    def mirrored(n, m):
        r, u, v, p = shock_like(np.mod(-n, N), m, N)
        return r, -u, v, p

    out = []
    for prim in (lambda n, m: shock_like(n, m, N), mirrored):
        o = make(oracle_mod, form, lvl)
        set_nodes(o, form, lvl, prim)
        before = grid(o, N)
        o.filter()
        out.append((before, grid(o, N)))
    (b0, a0), (_, a1) = out
    assert np.abs(a0 - b0).max() > 1e-4
    back = a1[:, :, np.mod(-np.arange(N), N)]
    back[1] = -back[1]
    assert np.allclose(a0, back, rtol=0, atol=1e-13)


def test_filter_runs_on_adaptive_tree_inside_step(oracle_mod):
    # the double shear layer of Sec. 4 on a small adaptive grid: the step
    # (refine, RK4, filter, coarsen) keeps the tree graded and every value finite
    dsl = (2.0, 1.0, 1.0, -1.0, 8.0 / 240.0, 2.5, 0.1, 0.25, 4.0, 4.0)
    for form in ("ns", "ns_skew"):
        o = oracle_mod.Oracle(dict(dim=2, Bs=17, nvar=4, Jmin=2, Jmax=4, eps=1e-3, rhs=form,
                                   rhs_params=(GAM, 1e-6, PR, RTH), ic="shear_layer", ic_params=dsl,
                                   norm_kind=1, L=8.0))
        o.init_tree()
        n0 = o.n
        for s in range(2):
            o.step(s * 2e-3, 2e-3)
        assert o.errors == 0
        assert np.isfinite(o.blocks()["fields"]).all()
        assert o.n >= n0 // 4
