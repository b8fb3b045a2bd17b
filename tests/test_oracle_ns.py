"""Pins of the oracle's compressible Navier-Stokes right-hand side (Sec. 4).

* free-stream preservation: a uniform state has N(q) = 0 exactly;
* inviscid entropy wave: rho = 1 + a sin(2 pi (x - u0 t)), u = u0, v = 0,
  p = const is an exact Euler solution; the computed state after RK4 steps
  matches it with 4th-order convergence in the grid spacing;
* viscous and heat-flux terms: N(q) of a smooth periodic state converges at
  4th order to an FFT evaluation of the textbook equations written here
  independently of the oracle;
* conservation: N(q) of each conserved variable sums to zero over a periodic
  grid.
"""
import math

import numpy as np

from tests import treegen

GAM, PR = 1.4, 0.71


def ns_oracle(oracle_mod, lvl, mu, Bs=17):
    return oracle_mod.Oracle(dict(dim=2, Bs=Bs, ng=4, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs="ns",
                                  rhs_params=(GAM, mu, PR), ic="none", norm_kind=1))


def set_state(o, lvl, prim, Bs=17):
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lvlv, crd = treegen.as_arrays(leaves)
    h = 1.0 / ((Bs - 1) * (1 << lvl))
    f = np.zeros((len(leaves), 4, Bs, Bs))
    for n in range(len(leaves)):
        x = (crd[n, 0] * (Bs - 1) + np.arange(Bs)) * h
        y = (crd[n, 1] * (Bs - 1) + np.arange(Bs)) * h
        X, Y = np.meshgrid(x, y)
        r, u, v, p = prim(X, Y)
        f[n] = [r, r * u, r * v, p / (GAM - 1.0) + 0.5 * r * (u * u + v * v)]
    o.set_blocks(lvlv, crd, f)
    return lvlv, crd


def test_free_stream_preserved_exactly(oracle_mod):
    o = ns_oracle(oracle_mod, 2, 1e-3)
    set_state(o, 2, lambda X, Y: (1.2 + 0 * X, 0.3 + 0 * X, -0.1 + 0 * X, 0.9 + 0 * X))
    assert np.all(o.rhs(0.0) == 0.0)


def test_inviscid_entropy_wave_converges_fourth_order(oracle_mod):
    u0, a, T = 0.5, 0.2, 0.02
    errs = []
    for lvl in (2, 3):
        o = ns_oracle(oracle_mod, lvl, 0.0)
        set_state(o, lvl, lambda X, Y: (1.0 + a * np.sin(2 * np.pi * X), u0 + 0 * X, 0 * X, 1.0 + 0 * X))
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
            ex = 1.0 + a * np.sin(2 * np.pi * (x - u0 * T))
            e = max(e, np.abs(b["fields"][q, 0] - ex[None, :]).max())
            # velocity and pressure stay uniform
            r, m1, m2 = b["fields"][q, 0], b["fields"][q, 1], b["fields"][q, 2]
            assert np.abs(m1 / r - u0).max() < 1e-6 and np.abs(m2).max() < 1e-12
        errs.append(e)
    assert math.log2(errs[0] / errs[1]) > 3.5, errs


def spectral_rhs(N, mu, prim):
    """Navier-Stokes N(q) on a uniform periodic N x N grid, derivatives by FFT."""
    x = np.arange(N) / N
    X, Y = np.meshgrid(x, x)
    r, u, v, p = prim(X, Y)
    k = 2j * np.pi * np.fft.fftfreq(N, 1.0 / N)
    ddx = lambda f: np.real(np.fft.ifft(k[None, :] * np.fft.fft(f, axis=1), axis=1))
    ddy = lambda f: np.real(np.fft.ifft(k[:, None] * np.fft.fft(f, axis=0), axis=0))
    E = p / (GAM - 1.0) + 0.5 * r * (u * u + v * v)
    T_ = p / r
    ux, uy, vx, vy = ddx(u), ddy(u), ddx(v), ddy(v)
    div = ux + vy
    sxx = mu * (2 * ux - 2.0 / 3.0 * div)
    syy = mu * (2 * vy - 2.0 / 3.0 * div)
    sxy = mu * (uy + vx)
    kap = mu * GAM / ((GAM - 1.0) * PR)
    Fx = [r * u, r * u * u + p - sxx, r * u * v - sxy, (E + p) * u - u * sxx - v * sxy - kap * ddx(T_)]
    Fy = [r * v, r * u * v - sxy, r * v * v + p - syy, (E + p) * v - u * sxy - v * syy - kap * ddy(T_)]
    return [-(ddx(fx) + ddy(fy)) for fx, fy in zip(Fx, Fy)]


def test_viscous_rhs_converges_to_spectral_reference(oracle_mod):
    mu = 0.05
    prim = lambda X, Y: (1.0 + 0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
                         0.2 * np.cos(2 * np.pi * Y) + 0.05 * np.sin(2 * np.pi * X),
                         0.1 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
                         1.0 + 0.05 * np.cos(2 * np.pi * (X + Y)))
    errs = []
    for lvl in (2, 3):
        o = ns_oracle(oracle_mod, lvl, mu)
        set_state(o, lvl, prim)
        k = o.rhs(0.0)
        b = o.blocks(fields=False)
        N = 16 * (1 << lvl)
        ref = spectral_rhs(N, mu, prim)
        e = 0.0
        for q in range(o.n):
            cx, cy = b["coords"][q][:2]
            ix = np.mod(cx * 16 + np.arange(17), N)
            iy = np.mod(cy * 16 + np.arange(17), N)
            for var in range(4):
                e = max(e, np.abs(k[q, var] - ref[var][np.ix_(iy, ix)]).max())
        errs.append(e)
    assert errs[1] < 1e-3 and math.log2(errs[0] / errs[1]) > 3.5, errs


def test_conservative_form_sums_to_zero_on_periodic_grid(oracle_mod):
    # The right-hand side is written as a flux divergence, N(q) = -(dF/dx + dG/dy)
    # with the compressible Navier-Stokes fluxes of Sec. 4, so it conserves mass,
    # momentum and energy: on a uniform periodic grid every flux difference telescopes, so the sum of N(q)
    # over the unique nodes vanishes for each conserved variable up to rounding,
    # while the individual terms do not.  An asymmetric stencil or a term taken
    # outside the flux divergence breaks this.
    mu = 0.02
    prim = lambda X, Y: (1.0 + 0.2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y),
                         0.3 + 0.1 * np.sin(2 * np.pi * Y),
                         -0.2 + 0.1 * np.cos(2 * np.pi * X),
                         1.0 + 0.1 * np.sin(2 * np.pi * (X + Y)))
    lvl = 3
    o = ns_oracle(oracle_mod, lvl, mu)
    set_state(o, lvl, prim)
    k = o.rhs(0.0)[:, :, :16, :16]  # unique nodes: each block's last node per axis is its neighbour's first
    for var in range(4):
        s, a = k[:, var].sum(), np.abs(k[:, var]).sum()
        assert a > 1.0, (var, a)
        assert abs(s) <= 1e-12 * a, (var, s, a)
