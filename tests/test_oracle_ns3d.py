"""Pins of the oracle's three-dimensional Navier-Stokes forms (Sec. 4's
equations in 3D, the run Sec. 5 names as the next step) and of the 3D
shock-capturing filter.

States: q = (rho, rho u, rho v, rho w, E) for the flux form and
q = (phi, psi_x, psi_y, psi_z, p), phi = sqrt(rho), psi = phi u, for the
skew-symmetric form.

* free-stream preservation: a uniform state has N(q) = 0 exactly;
* a state that does not vary along z and has w = 0 gives, in every z plane,
  the 2D right-hand side and the 2D filter bit for bit (the 2D forms carry
  their own pins);
* rotation: a cyclic permutation of the axes (and of the velocity components)
  of the state permutes the right-hand side and the filtered state the same
  way, which ties the z terms to the x and y terms (a wrong sign, index or
  missing z term breaks it);
* consistency: N(q) (through the chain rule for the skew form) converges at
  4th order to an FFT evaluation of the textbook equations written here;
* discrete invariants on a periodic grid: mass, momentum and energy rates sum
  to zero, and the skew form's convection conserves kinetic energy;
* filter: transfer function and sensor strength of a four-node velocity wave
  along each axis; conservation of every conserved variable;
* steps: RK4 + filter conserve every sum of the flux form on a periodic tree;
  a full adaptive step (refine, RK4, filter, coarsen) on an octree stays
  graded and finite.
"""
import math

import numpy as np
import pytest

from tests import treegen
from tests.test_oracle_filter import shock_like
from tests.test_oracle_ns_skew import generic

GAM, PR, RTH = 1.4, 0.71, 1e-5
FORMS = ["ns", "ns_skew"]


def oracle3(oracle_mod, form, lvl, mu=0.0, rth=0.0):
    return oracle_mod.Oracle(dict(dim=3, Bs=17, ng=4, nvar=5, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs=form,
                                  rhs_params=(GAM, mu, PR, rth), ic="none", norm_kind=1))


def oracle2(oracle_mod, form, lvl, mu=0.0, rth=0.0):
    return oracle_mod.Oracle(dict(dim=2, Bs=17, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs=form,
                                  rhs_params=(GAM, mu, PR, rth), ic="none", norm_kind=1))


def state3(form, r, u, v, w, p):
    if form == "ns":
        return [r, r * u, r * v, r * w, p / (GAM - 1.0) + 0.5 * r * (u * u + v * v + w * w)]
    ph = np.sqrt(r)
    return [ph, ph * u, ph * v, ph * w, p + 0 * r]


def set_global(o, lvl, A):
    """Uniform tree at lvl with the periodic global arrays A[v][z][y][x] (N^3 nodes)."""
    N = 16 << lvl
    leaves = sorted(treegen.uniform_tree(3, lvl))
    lv, crd = treegen.as_arrays(leaves)
    f = np.zeros((len(leaves), A.shape[0], 17, 17, 17))
    for q in range(len(leaves)):
        ix = np.mod(crd[q, 0] * 16 + np.arange(17), N)
        iy = np.mod(crd[q, 1] * 16 + np.arange(17), N)
        iz = np.mod(crd[q, 2] * 16 + np.arange(17), N)
        f[q] = A[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    o.set_blocks(lv, crd, f)


def to_global(o, arr, N):
    """Per-block arrays (Hilbert order, [block][v][z][y][x]) on the unique nodes of the global grid."""
    crd = o.blocks(fields=False)["coords"]
    G = np.zeros((arr.shape[1], N, N, N))
    for q in range(o.n):
        x0, y0, z0 = (int(c) * 16 for c in crd[q])
        G[:, z0:z0 + 16, y0:y0 + 16, x0:x0 + 16] = arr[q, :, :16, :16, :16]
    return G


def prim_fields(seed, N, uniform_p=False):
    """Smooth periodic primitives (rho, u, v, w, p) on the N^3 node grid from a few
    Fourier modes with seeded amplitudes and phases."""
    rng = np.random.default_rng(seed)
    modes = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, 0, 1), (1, -1, 1)]
    coef = rng.uniform(-1.0, 1.0, (5, len(modes)))
    phase = rng.uniform(0.0, 2 * np.pi, (5, len(modes)))
    x = np.arange(N) / N
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")

    def f(var):
        return sum(coef[var, m] * np.sin(2 * np.pi * (kx * X + ky * Y + kz * Z) + phase[var, m])
                   for m, (kx, ky, kz) in enumerate(modes))

    return (1.0 + 0.05 * f(0), 0.3 + 0.1 * f(1), -0.2 + 0.1 * f(2), 0.25 + 0.1 * f(3),
            1.0 + (0.0 * X if uniform_p else 0.05 * f(4)))


def rotate(A):
    """State or rate of the cyclically rotated flow: G(x, y, z) = F(y, z, x), vector
    components (w, u, v) of F becoming (u, v, w) of G.  A[v][z][y][x]."""
    T = lambda a: np.transpose(a, (1, 2, 0))  # out[z, y, x] = a[x, z, y]
    return np.stack([T(A[0]), T(A[3]), T(A[1]), T(A[2]), T(A[4])])


@pytest.mark.parametrize("form", FORMS)
def test_free_stream_preserved_exactly(oracle_mod, form):
    lvl = 1
    N = 16 << lvl
    o = oracle3(oracle_mod, form, lvl, mu=1e-3)
    one = np.ones((N, N, N))
    set_global(o, lvl, np.stack(state3(form, 1.2 * one, 0.3 * one, -0.1 * one, 0.2 * one, 0.9 * one)))
    assert np.all(o.rhs(0.0) == 0.0)


@pytest.mark.parametrize("form", FORMS)
def test_z_independent_state_gives_2d_rhs_bit_for_bit(oracle_mod, form):
    lvl, mu = 1, 0.02
    N = 16 << lvl
    prim = generic(21)
    x = np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    r, u, v, p = prim(X, Y)
    q3 = np.stack([np.broadcast_to(a, (N, N, N)) for a in state3(form, r, u, v, 0 * r, p)])
    o3 = oracle3(oracle_mod, form, lvl, mu)
    set_global(o3, lvl, q3)
    k3 = to_global(o3, o3.rhs(0.0), N)
    o2 = oracle2(oracle_mod, form, lvl, mu)
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lv, crd = treegen.as_arrays(leaves)
    s2 = [a for a in state3(form, r, u, v, 0 * r, p)]
    s2 = np.stack([s2[0], s2[1], s2[2], s2[4]])
    f2 = np.zeros((len(leaves), 4, 17, 17))
    for q in range(len(leaves)):
        ix = np.mod(crd[q, 0] * 16 + np.arange(17), N)
        iy = np.mod(crd[q, 1] * 16 + np.arange(17), N)
        f2[q] = s2[:, iy[:, None], ix[None, :]]
    o2.set_blocks(lv, crd, f2)
    k2b = o2.rhs(0.0)
    c2 = o2.blocks(fields=False)["coords"]
    k2 = np.zeros((4, N, N))
    for q in range(o2.n):
        x0, y0 = int(c2[q, 0]) * 16, int(c2[q, 1]) * 16
        k2[:, y0:y0 + 16, x0:x0 + 16] = k2b[q, :, :16, :16]
    assert np.abs(k2).max() > 0.01
    for z in range(N):
        for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
            assert np.array_equal(k3[v3, z], k2[v2]), (form, z, v3)
        assert np.all(k3[3, z] == 0.0)


@pytest.mark.parametrize("form", FORMS)
def test_cyclic_axis_rotation_rotates_rhs(oracle_mod, form):
    lvl, mu = 1, 0.03
    N = 16 << lvl
    q = np.stack(state3(form, *prim_fields(5, N)))
    out = []
    for A in (q, rotate(q)):
        o = oracle3(oracle_mod, form, lvl, mu)
        set_global(o, lvl, A)
        out.append(to_global(o, o.rhs(0.0), N))
    k, kr = out
    scale = np.abs(k).max(axis=(1, 2, 3))
    assert np.all(scale > 1e-3)
    d = np.abs(kr - rotate(k)).max(axis=(1, 2, 3))
    assert np.all(d <= 1e-12 * scale), (d, scale)


def spectral_rates3(N, mu, r, u, v, w, p):
    """Rates of (rho, rho u, rho v, rho w, E) of the compressible Navier-Stokes
    equations (ideal gas, constant c_p, Stokes hypothesis) on the periodic N^3
    grid, derivatives by FFT; arrays indexed [z][y][x]."""
    k = 2j * np.pi * np.fft.fftfreq(N, 1.0 / N)
    shape = [(1, 1, N), (1, N, 1), (N, 1, 1)]  # x, y, z wavenumbers
    axis = [2, 1, 0]
    D = lambda f, a: np.real(np.fft.ifft(k.reshape(shape[a]) * np.fft.fft(f, axis=axis[a]), axis=axis[a]))
    vel = [u, v, w]
    E = p / (GAM - 1.0) + 0.5 * r * (u * u + v * v + w * w)
    T_ = p / r
    du = [[D(vel[a], b) for b in range(3)] for a in range(3)]
    div = du[0][0] + du[1][1] + du[2][2]
    tau = [[mu * (du[a][b] + du[b][a]) - (2.0 / 3.0 * mu * div if a == b else 0.0) for b in range(3)]
           for a in range(3)]
    kap = mu * GAM / ((GAM - 1.0) * PR)
    rates = [0.0] * 5
    for a in range(3):
        F = [r * vel[a]]
        F += [r * vel[a] * vel[b] + (p if a == b else 0.0) - tau[a][b] for b in range(3)]
        F += [(E + p) * vel[a] - sum(vel[b] * tau[a][b] for b in range(3)) - kap * D(T_, a)]
        for n in range(5):
            rates[n] = rates[n] - D(F[n], a)
    return rates


def conserved_rates3(q, k):
    """Chain rule from the rates of (phi, psi, p) to those of (rho, rho u, E)."""
    ph, s, p = q[0], q[1:4], q[4]
    kph, ks, kp = k[0], k[1:4], k[4]
    return [2.0 * ph * kph] + [s[a] * kph + ph * ks[a] for a in range(3)] + \
           [kp / (GAM - 1.0) + s[0] * ks[0] + s[1] * ks[1] + s[2] * ks[2]]


@pytest.mark.parametrize("form", FORMS)
def test_rates_converge_to_spectral_reference(oracle_mod, form):
    mu = 0.05
    errs = []
    for lvl in (1, 2):
        N = 16 << lvl
        prim = prim_fields(7, N)
        o = oracle3(oracle_mod, form, lvl, mu)
        q = np.stack(state3(form, *prim))
        set_global(o, lvl, q)
        k = to_global(o, o.rhs(0.0), N)
        got = k if form == "ns" else conserved_rates3(q, k)
        ref = spectral_rates3(N, mu, *prim)
        errs.append(max(np.abs(got[n] - ref[n]).max() for n in range(5)))
    assert errs[1] < 2e-3 and math.log2(errs[0] / errs[1]) > 3.5, errs


@pytest.mark.parametrize("form", FORMS)
def test_discrete_conservation_on_periodic_grid(oracle_mod, form):
    lvl, mu = 1, 0.02
    N = 16 << lvl
    q = np.stack(state3(form, *prim_fields(9, N)))
    o = oracle3(oracle_mod, form, lvl, mu)
    set_global(o, lvl, q)
    k = to_global(o, o.rhs(0.0), N)
    rates = k if form == "ns" else conserved_rates3(q, k)
    for n in range(5):
        s, a = rates[n].sum(), np.abs(rates[n]).sum()
        assert a > 0.05, (n, a)
        assert abs(s) <= 1e-12 * a, (n, s, a)
    if form == "ns_skew":
        # phi, psi and p themselves are not conserved: the check above is not vacuous
        assert abs(k[0].sum()) > 1e-6 * np.abs(k[0]).sum()


def test_skew_convection_conserves_kinetic_energy(oracle_mod):
    # uniform pressure, no viscosity: only the split convective terms act on psi
    lvl = 1
    N = 16 << lvl
    q = np.stack(state3("ns_skew", *prim_fields(13, N, uniform_p=True)))
    o = oracle3(oracle_mod, "ns_skew", lvl, 0.0)
    set_global(o, lvl, q)
    k = to_global(o, o.rhs(0.0), N)
    ke = q[1] * k[1] + q[2] * k[2] + q[3] * k[3]
    assert np.abs(ke).sum() > 0.01
    assert abs(ke.sum()) <= 1e-12 * np.abs(ke).sum()


# ------------------------------------------------------------------ filter ---

@pytest.mark.parametrize("form", FORMS)
def test_filter_of_z_independent_state_equals_2d_filter(oracle_mod, form):
    lvl = 1
    N = 16 << lvl
    n = np.arange(N)
    Nn, Mm = np.meshgrid(n, n)
    r, u, v, p = shock_like(Nn, Mm, N)
    s3 = state3(form, r, u, v, 0 * r, p)
    o3 = oracle3(oracle_mod, form, lvl, rth=RTH)
    set_global(o3, lvl, np.stack([np.broadcast_to(a, (N, N, N)) for a in s3]))
    before = to_global(o3, o3.blocks()["fields"], N)
    o3.filter()
    f3 = to_global(o3, o3.blocks()["fields"], N)
    o2 = oracle2(oracle_mod, form, lvl, rth=RTH)
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lv, crd = treegen.as_arrays(leaves)
    s2 = np.stack([s3[0], s3[1], s3[2], s3[4]])
    f2 = np.zeros((len(leaves), 4, 17, 17))
    for q in range(len(leaves)):
        ix = np.mod(crd[q, 0] * 16 + np.arange(17), N)
        iy = np.mod(crd[q, 1] * 16 + np.arange(17), N)
        f2[q] = s2[:, iy[:, None], ix[None, :]]
    o2.set_blocks(lv, crd, f2)
    o2.filter()
    b2 = o2.blocks()
    g2 = np.zeros((4, N, N))
    for q in range(o2.n):
        x0, y0 = int(b2["coords"][q, 0]) * 16, int(b2["coords"][q, 1]) * 16
        g2[:, y0:y0 + 16, x0:x0 + 16] = b2["fields"][q, :, :16, :16]
    assert np.abs(f3 - before).max() > 1e-4
    for z in range(N):
        for v3, v2 in ((0, 0), (1, 1), (2, 2), (4, 3)):
            assert np.array_equal(f3[v3, z], g2[v2]), (form, z, v3)
        assert np.all(f3[3, z] == 0.0)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_filter_strength_and_transfer_function_per_axis(oracle_mod, form, axis):
    # u_axis = a sin(pi n / 2): dilatation a cos(pi n / 2) / dx, M = (a / dx)^2 / 4,
    # r = a^2 / (4 c^2) + 1e-16, s = 1 - r_th / r; the wave is multiplied by 1 - s / 2
    s_target, p0 = 0.6, 1.0
    c2 = GAM * p0
    r_ = RTH / (1.0 - s_target)
    a = np.sqrt(4.0 * r_ * c2)
    lvl = 1
    N = 16 << lvl
    n = np.arange(N)
    Z, Y, X = np.meshgrid(n, n, n, indexing="ij")
    kk = (X, Y, Z)[axis]
    vel = [0.0 * X, 0.0 * X, 0.0 * X]
    vel[axis] = a * np.sin(np.pi * kk / 2)
    o = oracle3(oracle_mod, form, lvl, rth=RTH)
    set_global(o, lvl, np.stack(state3(form, 1.0 + 0 * X, *vel, p0 + 0 * X)))
    o.filter()
    f = to_global(o, o.blocks()["fields"], N)
    s = 1.0 - RTH / (a * a / (4.0 * c2) + 1e-16)
    assert np.allclose(f[1 + axis], a * np.sin(np.pi * kk / 2) * (1.0 - s / 2.0), rtol=0, atol=1e-12 * a)
    for other in range(3):
        if other != axis:
            assert np.all(f[1 + other] == 0.0)
    assert np.all(f[0] == 1.0)
    if form == "ns":
        ex = p0 / (GAM - 1.0) + a * a / 4.0 - a * a / 4.0 * (1.0 - s) * np.cos(np.pi * kk)
        assert np.allclose(f[4], ex, rtol=0, atol=1e-13)
    else:
        assert np.all(f[4] == p0)


@pytest.mark.parametrize("form", FORMS)
def test_filter_rotation_and_conservation(oracle_mod, form):
    # steep state varying along all three axes: the filter acts, commutes with a
    # cyclic rotation of the axes, and (flux form) conserves every sum
    lvl = 1
    N = 16 << lvl
    n = np.arange(N)
    Z, Y, X = np.meshgrid(n, n, n, indexing="ij")
    r, u, v, p = shock_like(X, Y, N)
    _, w, _, _ = shock_like(Z, Y, N)
    q = np.stack(state3(form, r, u, v, 0.6 * w, p))
    out = []
    for A in (q, rotate(q)):
        o = oracle3(oracle_mod, form, lvl, rth=RTH)
        set_global(o, lvl, A)
        o.filter()
        out.append(to_global(o, o.blocks()["fields"], N))
    f, fr = out
    assert np.abs(f - q).max() > 1e-4
    assert np.abs(fr - rotate(f)).max() <= 1e-13 * np.abs(q).max()
    if form == "ns":
        for v_ in range(5):
            d = f[v_] - q[v_]
            assert np.abs(d).sum() > 1e-3, v_
            assert abs(d.sum()) <= 1e-12 * np.abs(q[v_]).sum(), v_


# ------------------------------------------------------------------- steps ---

def test_flux_form_steps_conserve_every_sum(oracle_mod):
    # two RK4 steps, each followed by the filter, on a periodic uniform tree: the
    # right-hand side is a flux divergence and the filter a flux difference, so
    # the sums of rho, rho u, rho v, rho w and E over the unique nodes stay put
    lvl = 1
    N = 16 << lvl
    n = np.arange(N)
    Z, Y, X = np.meshgrid(n, n, n, indexing="ij")
    r, u, v, p = shock_like(X, Y, N)
    _, w, _, _ = shock_like(Z, Y, N)
    q = np.stack(state3("ns", r, u, v, 0.6 * w, p))
    o = oracle3(oracle_mod, "ns", lvl, mu=0.01, rth=RTH)
    set_global(o, lvl, q)
    s0 = q.reshape(5, -1).sum(axis=1)
    dt = 0.2 / N / 2.5
    for s in range(2):
        o.rk4(s * dt, dt)
        o.filter()
    f = to_global(o, o.blocks()["fields"], N)
    assert np.abs(f - q).max() > 1e-4
    s1 = f.reshape(5, -1).sum(axis=1)
    scale = np.abs(q).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(s1 - s0) <= 1e-12 * scale), (s1 - s0, scale)


@pytest.mark.parametrize("form", FORMS)
def test_adaptive_step_in_3d(oracle_mod, form):
    # refine, RK4, filter, coarsen with five variables on an octree: graded,
    # finite, no stencil outside a tile
    lvl0 = 1
    o = oracle_mod.Oracle(dict(dim=3, Bs=17, ng=4, nvar=5, Jmin=1, Jmax=2, eps=1e-2, rhs=form,
                               rhs_params=(GAM, 1e-3, PR, RTH), ic="none", norm_kind=1))
    N = 16 << lvl0
    n = np.arange(N)
    Z, Y, X = np.meshgrid(n, n, n, indexing="ij")
    r, u, v, p = shock_like(X, Y, N, w=4.0 / N)
    set_global(o, lvl0, np.stack(state3(form, r, 0.3 * u, 0.3 * v, 0.1 + 0 * r, p)))
    dt = 0.1 / (16 << 2) / 2.5
    for s in range(2):
        o.step(s * dt, dt)
    b = o.blocks()
    leaves = {(int(l), tuple(int(x) for x in c)) for l, c in zip(b["level"], b["coords"])}
    assert o.errors == 0 and np.isfinite(b["fields"]).all()
    assert treegen.is_graded(3, leaves)
    assert set(b["level"].tolist()) <= {1, 2}
