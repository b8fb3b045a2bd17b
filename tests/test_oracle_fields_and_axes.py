"""Pins of the oracle's swirl velocity (Sec. 3, Eq. 1), its initial fields, the
details along every axis and per variable, RK4 for a time-dependent velocity
and the coarsening rounds.

* swirl: the velocity of Eq. (1) is the flow of the stream function
  sin^2(pi x) sin^2(pi y) / pi (so the stream function is not advected, to
  rounding also by the discrete operator), it
  is (1, 0) at (1/2, 1/4) and (0, -1) at (1/4, 1/2), and it scales with
  cos(pi t / t_a);
* RK4 with the time-dependent swirl keeps its local order 5 (stage times
  t, t + dt/2, t + dt/2, t + dt);
* details: for y^4 (1 + x) the largest detail sits on a column of even x
  (and for z^4 (1 + x)(1 + y) on even x and y), 9 h^4 times the largest
  linear factor; with several variables each one is measured against its
  own largest magnitude, so scaling or negating a variable leaves the block
  norms unchanged;
* Gaussian initial field (nearest periodic image of the centre): unit peak,
  mass (2 pi sigma^2)^(d/2), centre and second moments sigma^2 per axis;
* temporal mixing layer: uniform pressure (U0 / Ma)^2 / gamma at rho = 1,
  velocities -+U0 away from the layer at y = 0, vorticity thickness delta,
  a perturbation with the Gaussian envelope exp(-(y / delta)^2) and zero
  mean along x;
* coarsening rounds continue until nothing merges (a flat field on a uniform
  tree returns to Jmin in one call), or stop after max_rounds.
"""
import math

import numpy as np
import pytest

from tests import treegen
from tests.test_oracle_pins import fill, mk, node_xyz


def uniform(o, lvl, f, dim=2):
    return fill(o, treegen.uniform_tree(dim, lvl), f)


def at_point(o, arr, x, y, lvl, B=17):
    """Value of a per-block array at the node (x, y) of a uniform tree."""
    h = 1.0 / ((B - 1) * (1 << lvl))
    i, j = int(round(x / h)), int(round(y / h))
    b = o.blocks(fields=False)
    for n in range(o.n):
        cx, cy = (int(c) * (B - 1) for c in b["coords"][n][:2])
        if cx <= i < cx + B - 1 and cy <= j < cy + B - 1:
            return arr[n, 0, j - cy, i - cx]
    raise AssertionError("node not found")


# ------------------------------------------------------------------ swirl ---

def test_swirl_velocity_is_the_stream_function_flow(oracle_mod):
    # u . grad(psi) = 0 for the stream function psi of Eq. (1).  Discretely too:
    # sin^2(pi x) and sin^2(pi y) are the same Fourier mode along their axes, so
    # D1 scales both derivatives by the same factor and the two terms of
    # u . D psi cancel to rounding
    psi = lambda x, y: np.sin(np.pi * x) ** 2 * np.sin(np.pi * y) ** 2
    gen = lambda x, y: np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.5 * np.cos(2 * np.pi * x)
    for lvl in (2, 3):
        o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, rhs="swirl", rhs_params=(1.0,))
        uniform(o, lvl, psi)
        r_psi = np.abs(o.rhs(0.0)).max()
        uniform(o, lvl, gen)
        r_gen = np.abs(o.rhs(0.0)).max()
        assert r_gen > 1.0  # the velocity acts on a generic field
        assert r_psi < 1e-12 * r_gen, (lvl, r_psi, r_gen)


@pytest.mark.parametrize("t", [0.0, 1.0 / 3.0])
def test_swirl_velocity_point_values_and_time_factor(oracle_mod, t):
    # u(1/2, 1/4) = (1, 0) and u(1/4, 1/2) = (0, -1) at t = 0, scaled by cos(pi t / t_a)
    lvl = 2
    c = math.cos(math.pi * t / 1.0)
    o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, rhs="swirl", rhs_params=(1.0,))
    uniform(o, lvl, lambda x, y: np.sin(2 * np.pi * x))  # grad = (-2 pi, 0) at x = 1/2
    r = at_point(o, o.rhs(t), 0.5, 0.25, lvl)
    assert abs(r - 2 * np.pi * c) <= 1e-4 * 2 * np.pi, (r, c)
    uniform(o, lvl, lambda x, y: np.sin(2 * np.pi * y))  # grad = (0, -2 pi) at y = 1/2
    r = at_point(o, o.rhs(t), 0.25, 0.5, lvl)
    assert abs(r - (-2 * np.pi * c)) <= 1e-4 * 2 * np.pi, (r, c)


def test_rk4_local_order_with_time_dependent_swirl(oracle_mod):
    # one RK4 step against 32 substeps of the same scheme from the same state:
    # the step's error falls as dt^5 when the stages are evaluated at
    # t, t + dt/2, t + dt/2, t + dt; a wrong stage time leaves dt^3 or dt^4
    lvl, t0 = 2, 0.3
    f = lambda x, y: np.exp(-((x - 0.5) ** 2 + (y - 0.7) ** 2) / (2 * 0.12 ** 2))
    o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, rhs="swirl", rhs_params=(1.0,))
    leaves = treegen.uniform_tree(2, lvl)
    errs = []
    for dt in (0.004, 0.002):
        fill(o, leaves, f)
        o.rk4(t0, dt)
        one = o.blocks()["fields"]
        fill(o, leaves, f)
        m = 32
        for s in range(m):
            o.rk4(t0 + s * dt / m, dt / m)
        ref = o.blocks()["fields"]
        errs.append(np.abs(one - ref).max())
    assert errs[0] / errs[1] > 24.0, errs


# ---------------------------------------------------------------- details ---

@pytest.mark.parametrize("axis", [0, 1])
def test_details_along_each_axis_2d(oracle_mod, axis):
    # f = s^4 (1 + r), s the chosen axis, r the other: |d| = 9 h^4 (1 + r) on the
    # nodes odd along s, largest on the block's last column along r (even index)
    lvl = 3
    h = 1.0 / (16 * 8)
    f = (lambda x, y: y ** 4 * (1 + x)) if axis == 1 else (lambda x, y: x ** 4 * (1 + y))
    o = mk(oracle_mod, Jmin=lvl, Jmax=lvl)
    uniform(o, lvl, f)
    o.details()
    b = o.blocks(fields=False)
    checked = 0
    for n in range(o.n):
        c = b["coords"][n][:2]
        if np.all((c >= 1) & (c <= 6)):
            r_last = (c[1 - axis] * 16 + 16) * h
            assert abs(b["mdet"][n] - 9.0 * h ** 4 * (1 + r_last)) <= 1e-6 * 9.0 * h ** 4, (n, b["mdet"][n])
            checked += 1
    assert checked == 36


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_details_along_each_axis_3d(oracle_mod, axis):
    lvl, B = 3, 9
    h = 1.0 / (8 * 8)
    o = mk(oracle_mod, dim=3, Bs=B, ng=2, Jmin=lvl, Jmax=lvl)

    def f(x, y, z):
        X = (x, y, z)
        others = [X[a] for a in range(3) if a != axis]
        return X[axis] ** 4 * (1 + others[0]) * (1 + others[1])

    uniform(o, lvl, f, dim=3)
    o.details()
    b = o.blocks(fields=False)
    checked = 0
    for n in range(o.n):
        c = b["coords"][n][:3]
        if np.all((c >= 1) & (c <= 6)):
            lin = [(1 + (c[a] * 8 + 8) * h) for a in range(3) if a != axis]
            ex = 9.0 * h ** 4 * lin[0] * lin[1]
            assert abs(b["mdet"][n] - ex) <= 1e-6 * ex, (n, b["mdet"][n], ex)
            checked += 1
    assert checked == 216


def test_details_normalised_by_each_variables_magnitude(oracle_mod):
    # norm_kind 1: block norm = max over variables of max|d_v| / max over the grid of |q_v|
    lvl = 3
    h = 1.0 / (16 * 8)

    def state(scale):
        fs = [lambda x, y: 1.0 + 0 * x, lambda x, y: x ** 4, lambda x, y: 2.0 + 4.0 * y ** 4,
              lambda x, y: 1.0 + 0 * x]
        o = oracle_mod.Oracle(dict(dim=2, Bs=17, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs="ns",
                                   rhs_params=(1.4, 0.0, 0.71, 0.0), ic="none", norm_kind=1))
        leaves = sorted(treegen.uniform_tree(2, lvl))
        lv, crd = treegen.as_arrays(leaves)
        F = np.zeros((len(leaves), 4, 17, 17))
        for n in range(len(leaves)):
            X, Y = node_xyz(17, 2, lv[n], crd[n])
            X, Y = np.mod(X, 1.0), np.mod(Y, 1.0)
            for v in range(4):
                F[n, v] = scale[v] * fs[v](X, Y)
        o.set_blocks(lv, crd, F)
        o.details()
        return o.blocks(fields=False)

    a = state([1.0, 1.0, 1.0, 1.0])
    b = state([3.0, 250.0, -1.0, 1e-3])  # variable 2 entirely negative
    assert np.array_equal(a["coords"], b["coords"])
    np.testing.assert_allclose(b["mdet"], a["mdet"], rtol=1e-12, atol=0)
    # away from the periodic seams the largest normalised detail is variable 1's,
    # 9 h^4 / max x^4 (variable 2's is 36 h^4 / (2 + 4 max y^4), smaller)
    xmax4 = (1.0 - h) ** 4  # largest x^4 over the periodic node grid
    inner = [n for n in range(len(a["mdet"])) if np.all((a["coords"][n][:2] >= 1) & (a["coords"][n][:2] <= 6))]
    assert len(inner) == 36
    np.testing.assert_allclose(a["mdet"][inner], 9.0 * h ** 4 / xmax4, rtol=1e-6)


# ---------------------------------------------------------- initial fields ---

@pytest.mark.parametrize("dim", [2, 3])
def test_gaussian_initial_field_moments(oracle_mod, dim):
    sig = 0.06
    c = (0.5, 0.375, 0.625)
    B, g, lvl = (17, 4, 4) if dim == 2 else (9, 2, 4)
    o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=lvl, Jmax=lvl, ic="gauss", ic_params=c + (sig,))
    o.init_tree()
    b = o.blocks()
    n = (B - 1) << lvl
    h = 1.0 / n
    phi = b["fields"][:, 0]
    sl = (slice(0, B - 1),) * dim
    mass, mom1, mom2, peak = 0.0, np.zeros(dim), np.zeros(dim), 0.0
    for q in range(o.n):
        X = node_xyz(B, dim, lvl, b["coords"][q])
        p = phi[q][sl]
        mass += p.sum() * h ** dim
        peak = max(peak, p.max())
        for a in range(dim):
            xa = np.mod(X[a][sl] - c[a] + 0.5, 1.0) - 0.5  # displacement to the nearest image of the centre
            mom1[a] += (xa * p).sum() * h ** dim
            mom2[a] += (xa ** 2 * p).sum() * h ** dim
    assert abs(peak - 1.0) < 1e-14
    assert abs(mass - (2 * np.pi * sig * sig) ** (dim / 2)) < 1e-10
    np.testing.assert_allclose(mom1 / mass, 0.0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(mom2 / mass, sig * sig, rtol=1e-9)


def test_mixing_layer_initial_field(oracle_mod):
    gam, delta, U0, Ma, amp = 1.4, 0.05, 1.0, 0.3, 0.02
    rng = np.random.default_rng(3)
    modes = list(rng.uniform(0.2, 1.0, 8)) + list(rng.uniform(0, 2 * np.pi, 8))
    lvl = 4
    o = oracle_mod.Oracle(dict(dim=2, Bs=17, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs="ns",
                               rhs_params=(gam, 1e-4, 0.71, 0.0), ic="mixing",
                               ic_params=[delta, U0, Ma, gam, amp] + modes, norm_kind=1, x0=(0.0, -0.5, 0.0)))
    o.init_tree()
    b = o.blocks()
    N = 16 << lvl
    grid = np.zeros((4, N, N))
    for q in range(o.n):
        x0, y0 = (int(c) * 16 for c in b["coords"][q][:2])
        grid[:, y0:y0 + 16, x0:x0 + 16] = b["fields"][q, :, :16, :16]
    rho, m1, m2, E = grid
    u, v = m1 / rho, m2 / rho
    y = -0.5 + np.arange(N) / N
    p = (gam - 1.0) * (E - 0.5 * (m1 * u + m2 * v))
    assert np.all(rho == 1.0)
    np.testing.assert_allclose(p, (U0 / Ma) ** 2 / gam, rtol=1e-12)
    ubar = u.mean(axis=1)
    j0 = np.argmin(np.abs(y))
    assert abs(ubar[j0]) < 1e-12
    jq = np.argmin(np.abs(y - 0.25))
    assert abs(ubar[jq] - U0) < 1e-6 and abs(ubar[np.argmin(np.abs(y + 0.25))] + U0) < 1e-6
    # vorticity thickness 2 U0 / max du/dy = delta (4th-order differences of the profile)
    hy = 1.0 / N
    du = (8 * (ubar[j0 + 1] - ubar[j0 - 1]) - (ubar[j0 + 2] - ubar[j0 - 2])) / (12 * hy)
    assert abs(2 * U0 / du - delta) < 1e-3 * delta, 2 * U0 / du
    # perturbation: Gaussian envelope across the layer, zero mean along x
    prof = np.abs(v).max(axis=1)
    for yy in (0.02, 0.05, 0.08):
        j = np.argmin(np.abs(y - yy))
        np.testing.assert_allclose(prof[j] / prof[j0], np.exp(-(y[j] / delta) ** 2), rtol=1e-9)
    assert np.abs(v.mean(axis=1)).max() < 1e-12 * np.abs(v).max()
    assert np.abs(v).max() > 0.1 * amp


# --------------------------------------------------------- coarsening rounds --

@pytest.mark.parametrize("max_rounds,level", [(0, 1), (1, 3)])
def test_coarsening_rounds_until_nothing_merges(oracle_mod, max_rounds, level):
    # a flat field has no details: every family merges in every round, so the
    # rounds take a uniform level-4 tree down to Jmin = 1 (several levels per
    # step), unless max_rounds stops them earlier
    o = mk(oracle_mod, Jmin=1, Jmax=4, max_rounds=max_rounds)
    uniform(o, 4, lambda x, y: 0.5 + 0 * x)
    o.coarsen_until_stable()
    b = o.blocks()
    assert np.all(b["level"] == level) and o.n == 4 ** level
    assert np.all(b["fields"] == 0.5)
