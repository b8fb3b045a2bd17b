"""The numbers the paper prints for its grid and its two test cases
(`tests/golden/paper_values.txt`, each with its passage) against the oracle and
the benchmark's workload definitions."""
import math
import os

import numpy as np

import bench
from tests.test_oracle_pins import mk


def golden():
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, val = line.split()[:2]
                vals[key] = float(val)
    return vals


G = golden()


def test_neighbour_relation_counts(oracle_mod):
    for dim, key in ((2, "relations_2d"), (3, "relations_3d")):
        B, g = (17, 4) if dim == 2 else (9, 2)
        o = mk(oracle_mod, dim=dim, Bs=B, ng=g, Jmin=1, Jmax=2)
        assert o.nrel == G[key]


def test_swirl_blob_is_the_printed_gaussian(oracle_mod):
    # exp(-((x - c)^2 + (y - d)^2) / beta) with the printed c, d, beta on the
    # periodic unit square (nearest image): the oracle's Gaussian with
    # sigma^2 = beta / 2
    beta, c, d = G["swirl_beta"], G["swirl_c"], G["swirl_d"]
    lvl = 3
    o = mk(oracle_mod, Jmin=lvl, Jmax=lvl, ic="gauss", ic_params=(c, d, 0.0, math.sqrt(beta / 2)))
    o.init_tree()
    b = o.blocks()
    h = G["swirl_domain"] / (16 << lvl)
    wrap = lambda s: np.mod(s + 0.5, 1.0) - 0.5
    for n in range(o.n):
        x = (b["coords"][n][0] * 16 + np.arange(17)) * h
        y = (b["coords"][n][1] * 16 + np.arange(17)) * h
        X, Y = np.meshgrid(x, y)
        ex = np.exp(-(wrap(X - c) ** 2 + wrap(Y - d) ** 2) / beta)
        np.testing.assert_allclose(b["fields"][n, 0], ex, rtol=1e-13, atol=1e-300)


def test_swirl_workload_uses_the_printed_setup():
    w = bench.WORKLOADS["swirl"]
    t = w["tree"]
    assert t["ic_params"][:2] == (G["swirl_c"], G["swirl_d"])
    assert abs(2 * t["ic_params"][3] ** 2 - G["swirl_beta"]) < 1e-15
    assert t["rhs_params"][0] == G["swirl_t_a"] and w["full_time"] == G["swirl_t_a"]
    assert G["swirl_t_half"] == G["swirl_t_a"] / 2


def test_double_shear_layer_workload_uses_the_printed_setup():
    w = bench.WORKLOADS["dsl"]
    L = G["dsl_L"]
    assert w["L"] == L
    ic = w["tree"]["ic_params"]
    assert ic == (G["dsl_rho1"], G["dsl_rho0"], G["dsl_v1"], G["dsl_v0"], L / G["dsl_width_divisor"],
                  G["dsl_p0"], G["dsl_u_amplitude"], G["dsl_layer_offset"], L / 2, L / 2)
    assert w["tree"]["rhs_params"] == (G["dsl_gamma"], G["dsl_mu"], G["dsl_Pr"], G["dsl_r_th"])


def test_double_shear_layer_initial_state_from_printed_values(oracle_mod):
    L = G["dsl_L"]
    ic = (G["dsl_rho1"], G["dsl_rho0"], G["dsl_v1"], G["dsl_v0"], L / G["dsl_width_divisor"], G["dsl_p0"],
          G["dsl_u_amplitude"], G["dsl_layer_offset"], L / 2, L / 2)
    lvl = 3
    o = oracle_mod.Oracle(dict(dim=2, Bs=17, nvar=4, Jmin=lvl, Jmax=lvl, eps=1e-3, rhs="ns_skew",
                               rhs_params=(G["dsl_gamma"], G["dsl_mu"], G["dsl_Pr"], G["dsl_r_th"]),
                               ic="shear_layer", ic_params=ic, norm_kind=1, L=L))
    o.init_tree()
    b = o.blocks()
    h = L / (16 << lvl)
    umax, n_in = 0.0, 0
    for n in range(o.n):
        x = (b["coords"][n][0] * 16 + np.arange(17)) * h
        X = np.meshgrid(x, x)[0]
        ph, sx, sy, p = b["fields"][n]
        rho, u, v = ph * ph, sx / ph, sy / ph
        inside, outside = np.abs(X - L / 2) < 0.05, np.abs(X - L / 2) > 1.0
        # between the layers the tanh profiles leave 1 - tanh(0.25 / lw) = 6.1e-7
        assert np.allclose(rho[inside], G["dsl_rho1"], rtol=0, atol=1e-6)
        assert np.allclose(v[inside], G["dsl_v1"], rtol=0, atol=2e-6)
        assert np.allclose(rho[outside], G["dsl_rho0"], rtol=0, atol=1e-12)
        assert np.allclose(v[outside], G["dsl_v0"], rtol=0, atol=1e-12)
        n_in += int(inside.sum())
        assert np.all(p == G["dsl_p0"])
        umax = max(umax, np.abs(u).max())
    assert n_in > 0
    assert abs(umax - G["dsl_u_amplitude"]) < 1e-12  # sin reaches 1 on the node y = L/2 + 1/4
