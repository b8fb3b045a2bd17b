"""Pins of the oracle's skew-symmetric Navier-Stokes right-hand side and of the
double shear layer initial state (Sec. 4).

The state is q = (phi, psi_x, psi_y, p), phi = sqrt(rho), psi = phi u.

* free-stream preservation: a uniform state has N(q) = 0 exactly;
* consistency: mapped to the conserved variables by the chain rule
  (d rho = 2 phi d phi, d(rho u) = psi d phi + phi d psi,
  dE = dp / (gamma - 1) + psi . d psi), N(q) converges at 4th order to an FFT
  evaluation of the textbook equations (written in the NS flux-form test
  module, independently of the oracle);
* the split form's discrete invariants on a periodic grid: the semi-discrete
  rates of sum(rho), sum(rho u), sum(rho v) and sum(E) vanish up to rounding,
  and with uniform pressure and no viscosity so does the rate of the kinetic
  energy sum(psi . psi / 2); a convective term written in divergence form
  only, a dropped advective half or a wrong sign breaks one of these;
* inviscid entropy wave: an exact Euler solution, reached at 4th order after
  RK4 steps in the square-root variables.
"""
import math

import numpy as np
import pytest

from tests import treegen
from tests.test_oracle_ns import spectral_rhs

GAM, PR = 1.4, 0.71


def skew_oracle(oracle_mod, lvl, mu, Bs=17, rth=0.0, L=1.0):
    return oracle_mod.Oracle(dict(dim=2, Bs=Bs, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs="ns_skew",
                                  rhs_params=(GAM, mu, PR, rth), ic="none", norm_kind=1, L=L))


def set_skew_state(o, lvl, prim, Bs=17):
    """Uniform tree at lvl on the unit box with primitives prim(X, Y) -> (rho, u, v, p)."""
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lvlv, crd = treegen.as_arrays(leaves)
    h = 1.0 / ((Bs - 1) * (1 << lvl))
    f = np.zeros((len(leaves), 4, Bs, Bs))
    for n in range(len(leaves)):
        x = (crd[n, 0] * (Bs - 1) + np.arange(Bs)) * h
        y = (crd[n, 1] * (Bs - 1) + np.arange(Bs)) * h
        X, Y = np.meshgrid(x, y)
        r, u, v, p = prim(X, Y)
        ph = np.sqrt(r)
        f[n] = [ph, ph * u, ph * v, p + 0 * X]
    o.set_blocks(lvlv, crd, f)


def conserved_rates(q, k):
    """Chain rule from the rates of (phi, psi_x, psi_y, p) to those of (rho, rho u, rho v, E)."""
    ph, sx, sy, p = q
    kph, ksx, ksy, kp = k
    return [2.0 * ph * kph, sx * kph + ph * ksx, sy * kph + ph * ksy,
            kp / (GAM - 1.0) + sx * ksx + sy * ksy]


def test_free_stream_preserved_exactly(oracle_mod):
    o = skew_oracle(oracle_mod, 2, 1e-3)
    set_skew_state(o, 2, lambda X, Y: (1.2 + 0 * X, 0.3 + 0 * X, -0.1 + 0 * X, 0.9 + 0 * X))
    assert np.all(o.rhs(0.0) == 0.0)


SMOOTH = lambda X, Y: (1.0 + 0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
                       0.2 * np.cos(2 * np.pi * Y) + 0.05 * np.sin(2 * np.pi * X),
                       0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
                       1.0 + 0.05 * np.cos(2 * np.pi * (X + Y)))


@pytest.mark.parametrize("mu", [0.0, 0.05])
def test_chain_rule_rates_converge_to_spectral_reference(oracle_mod, mu):
    errs = []
    for lvl in (2, 3):
        o = skew_oracle(oracle_mod, lvl, mu)
        set_skew_state(o, lvl, SMOOTH)
        k = o.rhs(0.0)
        b = o.blocks()
        N = 16 * (1 << lvl)
        ref = spectral_rhs(N, mu, SMOOTH)
        e = 0.0
        for n in range(o.n):
            cx, cy = b["coords"][n][:2]
            ix = np.mod(cx * 16 + np.arange(17), N)
            iy = np.mod(cy * 16 + np.arange(17), N)
            got = conserved_rates(b["fields"][n], k[n])
            for var in range(4):
                e = max(e, np.abs(got[var] - ref[var][np.ix_(iy, ix)]).max())
        errs.append(e)
    assert errs[1] < 2e-3 and math.log2(errs[0] / errs[1]) > 3.5, errs


def generic(seed, uniform_p=False):
    """Smooth periodic primitives from a few Fourier modes with seeded random
    amplitudes and phases, so that no sum in the invariant checks vanishes by a
    symmetry of the chosen field."""
    rng = np.random.default_rng(seed)
    modes = [(1, 0), (0, 1), (1, 1), (1, -1), (2, 1)]
    coef = rng.uniform(-1.0, 1.0, (4, len(modes)))
    phase = rng.uniform(0.0, 2 * np.pi, (4, len(modes)))

    def f(var, X, Y):
        return sum(coef[var, m] * np.sin(2 * np.pi * (kx * X + ky * Y) + phase[var, m])
                   for m, (kx, ky) in enumerate(modes))

    return lambda X, Y: (1.0 + 0.05 * f(0, X, Y), 0.3 + 0.1 * f(1, X, Y), -0.2 + 0.1 * f(2, X, Y),
                         1.0 + (0.0 * X if uniform_p else 0.05 * f(3, X, Y)))


def _unique(a):
    return a[..., :16, :16]  # each block's last node per axis is its neighbour's first


def test_split_form_invariants_on_periodic_grid(oracle_mod):
    mu = 0.02
    prim = generic(11)
    lvl = 3
    o = skew_oracle(oracle_mod, lvl, mu)
    set_skew_state(o, lvl, prim)
    k = o.rhs(0.0)
    q = o.blocks()["fields"]
    rates = conserved_rates([q[:, v] for v in range(4)], [k[:, v] for v in range(4)])
    for var in range(4):
        r = _unique(rates[var])
        s, a = r.sum(), np.abs(r).sum()
        assert a > 0.05, (var, a)
        assert abs(s) <= 1e-12 * a, (var, s, a)
    # the individual state variables are not conserved (phi, psi and p are not
    # conserved quantities): the check above is not vacuous
    assert abs(_unique(k[:, 0]).sum()) > 1e-6 * np.abs(_unique(k[:, 0])).sum()


def test_kinetic_energy_of_convection_is_conserved(oracle_mod):
    # uniform pressure and mu = 0: only the convective terms act on psi, whose
    # skew-symmetric split makes sum(psi . d psi) vanish; the divergence form
    # alone does not
    prim = generic(12, uniform_p=True)
    lvl = 3
    o = skew_oracle(oracle_mod, lvl, 0.0)
    set_skew_state(o, lvl, prim)
    k = o.rhs(0.0)
    q = o.blocks()["fields"]
    ke = _unique(q[:, 1] * k[:, 1] + q[:, 2] * k[:, 2])
    assert np.abs(ke).sum() > 0.01
    assert abs(ke.sum()) <= 1e-12 * np.abs(ke).sum()


def test_inviscid_entropy_wave_converges_fourth_order(oracle_mod):
    u0, a, T = 0.5, 0.2, 0.02
    errs = []
    for lvl in (2, 3):
        o = skew_oracle(oracle_mod, lvl, 0.0)
        set_skew_state(o, lvl, lambda X, Y: (1.0 + a * np.sin(2 * np.pi * X), u0 + 0 * X, 0 * X, 1.0 + 0 * X))
        h = 1.0 / (16 * (1 << lvl))
        c = math.sqrt(GAM * 1.0 / (1.0 - a))
        n = int(math.ceil(T / (0.4 * h / (u0 + c))))
        dt = T / n
        for s in range(n):
            o.rk4(s * dt, dt)
        b = o.blocks()
        e = 0.0
        for q in range(o.n):
            x = (b["coords"][q][0] * 16 + np.arange(17)) * h
            ex = np.sqrt(1.0 + a * np.sin(2 * np.pi * (x - u0 * T)))
            ph, sx, sy, p = b["fields"][q]
            e = max(e, np.abs(ph - ex[None, :]).max())
            assert np.abs(sx / ph - u0).max() < 1e-6 and np.abs(sy).max() < 1e-12
            assert np.abs(p - 1.0).max() < 1e-6
        errs.append(e)
    assert math.log2(errs[0] / errs[1]) > 3.5, errs


# ------------------------------------------------------------------------------
# double shear layer initial state (Sec. 4)

DSL = (2.0, 1.0, 1.0, -1.0, 8.0 / 240.0, 2.5, 0.1, 0.25, 4.0, 4.0)


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
def test_shear_layer_initial_state(oracle_mod, form):
    o = oracle_mod.Oracle(dict(dim=2, Bs=17, nvar=4, Jmin=3, Jmax=3, eps=1e-3, rhs=form,
                               rhs_params=(GAM, 1e-6, PR, 1e-5), ic="shear_layer", ic_params=DSL,
                               norm_kind=1, L=8.0))
    o.init_tree()
    b = o.blocks()
    h = 8.0 / (16 * 8)
    n_mid = 0
    for n in range(o.n):
        cx, cy = b["coords"][n][:2]
        x = (cx * 16 + np.arange(17)) * h
        y = (cy * 16 + np.arange(17)) * h
        X, Y = np.meshgrid(x, y)
        f = b["fields"][n]
        if form == "ns":
            rho, u, v = f[0], f[1] / f[0], f[2] / f[0]
            p = (GAM - 1.0) * (f[3] - 0.5 * rho * (u * u + v * v))
        else:
            rho, u, v, p = f[0] ** 2, f[1] / f[0], f[2] / f[0], f[3]
        far = np.abs(X - 4.0) > 1.0
        assert np.allclose(rho[far], 1.0, rtol=0, atol=1e-12) and np.allclose(v[far], -1.0, rtol=0, atol=1e-12)
        mid = np.abs(X - 4.0) < 0.05  # between the layers (lw = 1/30): 1 - tanh(7.5) = 6.1e-7 from the plateau
        n_mid += int(mid.sum())
        assert np.allclose(rho[mid], 2.0, rtol=0, atol=1e-6) and np.allclose(v[mid], 1.0, rtol=0, atol=2e-6)
        assert np.allclose(u, 0.1 * np.sin(2 * np.pi * (Y - 4.0)), rtol=0, atol=1e-12)
        assert np.allclose(p, 2.5, rtol=0, atol=1e-12)
        # the jump sits at x = 4 -+ 0.25, halfway values there
        at = np.isclose(X, 3.75)
        assert np.allclose(rho[at], 1.5, rtol=0, atol=1e-12)
    assert n_mid > 0
