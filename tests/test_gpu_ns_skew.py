"""GPU path against the FP64 oracle for the double shear layer run of Sec. 4:
the skew-symmetric Navier-Stokes stage, the shock-capturing filter and the
full step (refine, RK4, filter, coarsen), through the C ABI.

FP64 is compared bit for bit (same IEEE operations in the same order, no FMA
contraction); the FP32-stage / FP64-state form within the tolerance stated
in its test.
"""
import numpy as np
import pytest

from tests import treegen
from tests.test_gpu_parity import assert_same_tree
from tests.test_oracle_filter import shock_like, state

pytestmark = pytest.mark.gpu

GAM, PR, RTH = 1.4, 0.71, 1e-5
DSL = (2.0, 1.0, 1.0, -1.0, 8.0 / 240.0, 2.5, 0.1, 0.25, 4.0, 4.0)


@pytest.fixture(scope="module")
def mr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_00088_gb300 import build as b
    b.build()
    import paper_1902_00088_gb300 as m
    return m


def dsl_cfg(form, Bs=17, Jmin=2, Jmax=4, eps=1e-3, rth=RTH, mu=1e-6):
    return dict(dim=2, Bs=Bs, nvar=4, Jmin=Jmin, Jmax=Jmax, eps=eps, rhs=form,
                rhs_params=(GAM, mu, PR, rth), ic="shear_layer", ic_params=DSL, norm_kind=1, L=8.0)


def make(mr, oracle_mod, c, precision="fp64", **kw):
    o = oracle_mod.Oracle(c)
    tree = dict(Jmin=c["Jmin"], Jmax=c["Jmax"], eps=c["eps"], ic=c["ic"], ic_params=c["ic_params"],
                rhs_params=c["rhs_params"])
    g = mr.Forest(dim=2, Bs=c["Bs"], nvar=4, precision=precision, rhs=c["rhs"], trees=[tree],
                  capacity=1 << 15, norm_kind=1, L=c["L"], **kw)
    return o, g


def dsl_dt(c):
    dx = c["L"] / ((c["Bs"] - 1) * (1 << c["Jmax"]))
    return 0.5 * dx / (1.0 + np.sqrt(GAM * 2.5 / 1.0))


@pytest.mark.parametrize("form,Bs", [("ns_skew", 17), ("ns_skew", 33), ("ns", 17)])
def test_shear_layer_steps_bit_exact_fp64(mr, oracle_mod, form, Bs):
    # the paper's double shear layer (L = 8, lw = L/240) on a coarse adaptive
    # grid, so that the layers are steep and the filter acts; three full steps
    c = dsl_cfg(form, Bs=Bs, Jmin=2, Jmax=4 if Bs == 17 else 3)
    o, g = make(mr, oracle_mod, c)
    o.init_tree()
    g.init_tree()
    ob, f = assert_same_tree(o, g)
    assert np.array_equal(f, ob["fields"])
    dt = dsl_dt(c)
    for s in range(3):
        o.step(s * dt, dt)
        g.step(s * dt, dt)
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"]), (s, np.abs(f - ob["fields"]).max())
    o.details()
    o.flags(0)
    g.adapt("flags_only")
    gf, gm = g.get_flags()
    ob = o.blocks(fields=False)
    assert np.array_equal(gm, ob["mdet"]) and np.array_equal(gf, ob["flag"])


@pytest.mark.parametrize("form", ["ns_skew", "ns"])
@pytest.mark.parametrize("seed", [1, 2])
def test_filter_bit_exact_on_random_adaptive_tree(mr, oracle_mod, form, seed):
    # steep state on a random graded tree: uniform and mixed neighbourhoods,
    # strengths between 0 and 1 near the jumps
    leaves = sorted(treegen.random_graded_tree(2, 2, 5, 6, seed))
    lvl, crd = treegen.as_arrays(leaves)
    c = dsl_cfg(form, Jmin=2, Jmax=5)
    c["ic"] = "none"
    o, g = make(mr, oracle_mod, c)
    f = np.zeros((len(leaves), 4, 17, 17))
    N = 16 << 5
    for q in range(len(leaves)):
        s = 1 << (5 - lvl[q])
        n = (crd[q, 0] * 16 + np.arange(17)) * s
        m = (crd[q, 1] * 16 + np.arange(17)) * s
        Nn, Mm = np.meshgrid(n, m)
        f[q] = state(form, *shock_like(Nn, Mm, N))
    o.set_blocks(lvl, crd, f)
    g.set_blocks(lvl, crd, f)
    before = o.blocks()["fields"].copy()
    o.filter()
    g.filter()
    ob, gf = assert_same_tree(o, g)
    assert np.abs(ob["fields"] - before).max() > 1e-4  # the filter acted
    assert np.array_equal(gf, ob["fields"]), np.abs(gf - ob["fields"]).max()


def test_skew_fp32_acc64_within_tolerance(mr, oracle_mod):
    # FP32 stencils and filter strengths, FP64 state and accumulator, three
    # RK steps and filters on a uniform grid; relative L2 per variable group
    # (phi, psi vector, p) <= 1e-5
    c = dsl_cfg("ns_skew", Jmin=4, Jmax=4)
    o, g = make(mr, oracle_mod, c, precision="fp32_acc64", detail_fp64=True)
    o.init_tree()
    g.init_tree()
    dt = dsl_dt(c)
    for s in range(3):
        o.rk4(s * dt, dt)
        o.filter()
        g.rk_step(s * dt, dt)
        g.filter()
    ob, f = assert_same_tree(o, g)
    ref = ob["fields"]
    scale = [np.linalg.norm(ref[:, 0]), np.linalg.norm(ref[:, 1:3]), np.linalg.norm(ref[:, 1:3]),
             np.linalg.norm(ref[:, 3])]
    for v in range(4):
        rel = np.linalg.norm(f[:, v] - ref[:, v]) / scale[v]
        assert rel < 1e-5, (v, rel)


@pytest.mark.parametrize("form", ["ns_skew", "ns"])
def test_fp32_state_within_tolerance(mr, oracle_mod, form):
    # FP32 state, stages and filter (no FP64 anywhere on the field path):
    # three RK steps each followed by the filter on a uniform grid; relative
    # L2 per variable group <= 1e-5 (each step adds a few u = 2^-24)
    c = dsl_cfg(form, Jmin=4, Jmax=4)
    o, g = make(mr, oracle_mod, c, precision="fp32", detail_fp64=True)
    o.init_tree()
    g.init_tree()
    dt = dsl_dt(c)
    for s in range(3):
        o.rk4(s * dt, dt)
        o.filter()
        g.rk_step(s * dt, dt)
        g.filter()
    ob, f = assert_same_tree(o, g)
    ref = ob["fields"]
    scale = [np.linalg.norm(ref[:, 0]), np.linalg.norm(ref[:, 1:3]), np.linalg.norm(ref[:, 1:3]),
             np.linalg.norm(ref[:, 3])]
    for v in range(4):
        rel = np.linalg.norm(f[:, v] - ref[:, v]) / scale[v]
        assert rel < 1e-5, (form, v, rel)


def test_graph_steps_equal_eager_steps_with_filter(mr):
    c = dsl_cfg("ns_skew", Jmin=2, Jmax=5)
    runs = []
    for graph in (False, True):
        tree = dict(Jmin=c["Jmin"], Jmax=c["Jmax"], eps=c["eps"], ic=c["ic"], ic_params=c["ic_params"],
                    rhs_params=c["rhs_params"])
        g = mr.Forest(dim=2, Bs=17, nvar=4, precision="fp64", rhs="ns_skew", trees=[tree],
                      capacity=1 << 15, norm_kind=1, L=8.0)
        g.init_tree()
        dt = dsl_dt(c)
        if graph:
            g.set_time(0.0, dt)
            g.step_graph(4)
        else:
            for s in range(4):
                g.step(s * dt, dt)
        runs.append(g.get_blocks())
    (ia, fa), (ib, fb) = runs
    assert np.array_equal(ia["level"], ib["level"]) and np.array_equal(fa, fb)


def test_filter_properties_at_full_size(mr):
    # 128^2 blocks of 17^2 at one level (beyond the oracle's reach): a uniform
    # state comes back unchanged bit for bit; the flux-form filter conserves the
    # sum of every conserved variable over the unique nodes of a steep periodic
    # state
    lvl = 7
    N = 16 << lvl
    leaves = sorted(treegen.uniform_tree(2, lvl))
    lv, crd = treegen.as_arrays(leaves)
    n = crd[:, 0, None, None] * 16 + np.arange(17)[None, None, :] + 0 * np.arange(17)[None, :, None]
    m = crd[:, 1, None, None] * 16 + np.arange(17)[None, :, None] + 0 * np.arange(17)[None, None, :]
    tree = dict(Jmin=lvl, Jmax=lvl, eps=1e-3, ic="none", rhs_params=(GAM, 0.0, PR, RTH))
    g = mr.Forest(dim=2, Bs=17, nvar=4, precision="fp64", rhs="ns", trees=[tree], capacity=1 << 15,
                  norm_kind=1)
    for prim, changes in ((lambda a, b: (1.3 + 0 * a, 0.2 + 0 * a, -0.4 + 0 * a, 0.8 + 0 * a), False),
                          (lambda a, b: shock_like(a, b, N), True)):
        f = np.stack(state("ns", *prim(n, m)), axis=1)
        g.set_blocks(lv, crd, f)
        g.sync_ghosts()
        _, f0 = g.get_blocks()
        g.filter()
        _, f1 = g.get_blocks()
        if not changes:
            assert np.array_equal(f1, f0)
        else:
            d = (f1 - f0)[:, :, :16, :16]
            for v in range(4):
                assert np.abs(d[:, v]).sum() > 1e-3
                assert abs(d[:, v].sum()) <= 1e-12 * np.abs(f0[:, v, :16, :16]).sum(), v


@pytest.mark.parametrize("seed", [3, 4])
def test_skew_fp32_acc64_with_filter_on_adaptive_tree(mr, oracle_mod, seed):
    # the benchmarked form (FP32 stages and filter, FP64 state) on a random graded
    # tree with coarse-fine interfaces: two RK steps each followed by the filter,
    # then a synchronisation on both sides (block-edge nodes owned by a finer
    # block take the owner's value); relative L2 per variable group <= 1e-5
    leaves = sorted(treegen.random_graded_tree(2, 2, 5, 6, seed))
    lvl, crd = treegen.as_arrays(leaves)
    c = dsl_cfg("ns_skew", Jmin=2, Jmax=5)
    c["ic"] = "none"
    o, g = make(mr, oracle_mod, c, precision="fp32_acc64", detail_fp64=True)
    N = 16 << 5
    f = np.zeros((len(leaves), 4, 17, 17))
    for q in range(len(leaves)):
        s = 1 << (5 - lvl[q])
        n = (crd[q, 0] * 16 + np.arange(17)) * s
        m = (crd[q, 1] * 16 + np.arange(17)) * s
        Nn, Mm = np.meshgrid(n, m)
        r, u, v, p = shock_like(Nn, Mm, N, w=4.0 / N)
        f[q] = state("ns_skew", 1.0 + 0 * r + 0.3 * (r - 1.0), 0.3 * u, 0.3 * v, 2.0 + 0.5 * (p - 1.0))
    o.set_blocks(lvl, crd, f)
    g.set_blocks(lvl, crd, f)
    dt = 0.25 * (8.0 / (16 << 5)) / 2.0
    for s in range(2):
        o.rk4(s * dt, dt)
        o.filter()
        g.rk_step(s * dt, dt)
        g.filter()
    o.sync()
    g.sync_ghosts()
    ob, gf = assert_same_tree(o, g)
    ref = ob["fields"]
    scale = [np.linalg.norm(ref[:, 0]), np.linalg.norm(ref[:, 1:3]), np.linalg.norm(ref[:, 1:3]),
             np.linalg.norm(ref[:, 3])]
    for v in range(4):
        rel = np.linalg.norm(gf[:, v] - ref[:, v]) / scale[v]
        assert rel < 1e-5, (v, rel)
