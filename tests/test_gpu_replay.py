"""The benchmarked arithmetic forms against the FP64 oracle, replays of the
GPU's own decisions through the oracle, and the refinement-indicator and
single-round variants (Sec. 2.3), all through the C ABI.

Tolerances.  FP64 fields are compared bit for bit.  FP32 forms store the field
and run the stencils and RK stages in FP32: each stage adds a few units of
FP32 rounding (u = 2^-24, about 6e-8) relative to the field's scale, so a few
steps stay within a relative L2 difference of 1e-5 from the FP64 oracle, the
bound used here.  Trees and flags are compared bit for bit: the FP32 forms take
their threshold decisions on FP64 evaluations of the stored FP32 values (or on
FP32 evaluations certified to give the same decision), and a replay hands the
oracle exactly those stored values.
"""
import math

import numpy as np
import pytest

import synthetic
from oracle import cnn
from tests import treegen
from tests.test_gpu_parity import _bench, assert_same_tree, make_pair

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module")
def mr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_00088_gb300 import build as b
    b.build()
    import paper_1902_00088_gb300 as m
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def workload_cfg(w):
    t = w["tree"]
    return dict(dim=w["dim"], Bs=w["Bs"], Jmin=t["Jmin"], Jmax=t["Jmax"], eps=t["eps"], rhs=w["rhs"],
                rhs_params=t["rhs_params"], ic="gauss", ic_params=t["ic_params"])


def compare_flags(o, g):
    o.details()
    o.flags(0)
    g.adapt("flags_only")
    ob = o.blocks(fields=False)
    gf, gm = g.get_flags()
    assert np.array_equal(gf, ob["flag"]), np.flatnonzero(gf != ob["flag"])[:10]
    return ob, gf, gm


def start_from_gpu_state(o, g):
    """Loads the GPU's current tree and fields (exported exactly as doubles) into the oracle."""
    info, f = g.get_blocks()
    o.set_blocks(info["level"], info["coords"].astype(np.int64), f)
    return info, f


@pytest.mark.parametrize("form", ["cta", "warp"])
def test_fp32_swirl_full_size_matches_oracle(mr, oracle_mod, form):
    # The swirl workload as benchmarked: 17^2 blocks, Jmax 8, eps 1e-4, FP32
    # stencils and RK stages, FP64 threshold decisions; in both forms of the
    # stage and details kernels.  From the initial grid, and from a state in
    # the middle of the run (where the grid is largest) handed to the oracle.
    bench = _bench()
    w = bench.WORKLOADS["swirl"]
    c = workload_cfg(w)
    o, g = make_pair(mr, oracle_mod, c, precision="fp32", capacity=w["capacity"], detail_fp64=True)
    g.set_tuning(0, 1 if form == "warp" else 0)
    o.init_tree()
    g.init_tree()
    dt = bench.dt_of(w)
    for s in range(3):
        o.step(s * dt, dt)
        g.step(s * dt, dt)
        ob, f = assert_same_tree(o, g)
        assert rel_l2(f, ob["fields"]) <= REL
    compare_flags(o, g)
    # mid-run: the GPU advances alone (graph replays), then both continue
    # from the GPU's state
    n_mid = 20000  # the grid is largest near t_a / 2 (40960 steps to t_a)
    g.set_time(3 * dt, dt)
    g.step_graph(n_mid)
    t0 = float(g.get_time()[0])
    start_from_gpu_state(o, g)
    assert o.n > 150
    for s in range(3):
        o.step(t0 + s * dt, dt)
        g.step(np.array([t0 + s * dt]), np.array([dt]))
        ob, f = assert_same_tree(o, g)
        assert rel_l2(f, ob["fields"]) <= REL
    compare_flags(o, g)
    assert o.errors == 0


def test_fp32_adv3d_full_size_matches_oracle(mr, oracle_mod):
    # The 3D workload as benchmarked (17^3 blocks, Jmax 6, eps 1e-4, FP32 +
    # FP64 decisions): one full step (refinement, four RK stages, coarsening
    # rounds) from the GPU's initial grid, handed to the oracle exactly.  (The
    # oracle's own 3D initialisation takes minutes at this size; the initial
    # grid is compared with it in the FP64 tests at smaller Jmax.)
    bench = _bench()
    w = bench.WORKLOADS["adv3d"]
    c = workload_cfg(w)
    o, g = make_pair(mr, oracle_mod, c, precision="fp32", capacity=w["capacity"], detail_fp64=True)
    g.init_tree()
    start_from_gpu_state(o, g)
    assert o.n > 100
    dt = bench.dt_of(w)
    o.step(0.0, dt)
    g.step(0.0, dt)
    ob, f = assert_same_tree(o, g)
    assert rel_l2(f, ob["fields"]) <= REL
    compare_flags(o, g)
    assert o.errors == 0


def test_fp32_warp_form_on_a_grid_that_selects_it(mr, oracle_mod):
    # 64^2 blocks (more than 8 per SM): the default launch picks the
    # warp-per-block stage and details kernels.  Two RK4 steps and the details
    # of the result against the oracle.
    c = dict(dim=2, Jmin=6, Jmax=6, eps=1e-3, rhs="adv", rhs_params=(1.0, 0.5, 0.0), ic="gauss",
             ic_params=(0.5, 0.5, 0.0, 0.05))
    o, g = make_pair(mr, oracle_mod, c, precision="fp32", capacity=5000, detail_fp64=True)
    o.init_tree()
    g.init_tree()
    assert g.num_blocks() == 4096
    dt = 0.5 / (16 * 64) / math.hypot(1.0, 0.5)
    for s in range(2):
        o.rk4(s * dt, dt)
        g.rk_step(s * dt, dt)
    ob, f = assert_same_tree(o, g)
    assert rel_l2(f, ob["fields"]) <= REL
    ob, gf, gm = compare_flags(o, g)
    scale = np.abs(f).max()
    assert np.abs(gm - ob["mdet"]).max() <= 32 * 2.0 ** -24 * scale + 1e-5 * np.abs(ob["mdet"]).max()


@pytest.mark.parametrize("workload", ["swirl", "adv3d"])
def test_replay_of_fp32_fields_through_oracle_adapt(mr, oracle_mod, workload):
    # The GPU's own FP32 fields after its refinement and RK4 stages go to the
    # oracle; the oracle's details, flags and coarsening rounds on exactly those
    # values reproduce the GPU's flags, next tree and fields bit for bit.
    bench = _bench()
    w = bench.WORKLOADS[workload]
    c = workload_cfg(w)
    o, g = make_pair(mr, oracle_mod, c, precision="fp32", capacity=w["capacity"], detail_fp64=True)
    g.init_tree()
    dt = bench.dt_of(w)
    nspin = 20000 if workload == "swirl" else 20
    g.set_time(0.0, dt)
    g.step_graph(nspin)
    t0 = float(g.get_time()[0])
    for rep in range(2 if workload == "swirl" else 1):
        g.adapt("refine_all")
        g.rk_step(np.array([t0]), np.array([dt]))
        t0 += dt
        start_from_gpu_state(o, g)
        ob, gf, gm = compare_flags(o, g)
        assert (gf == -2).any() and (gf == 0).any()
        # block maxima: FP64 where the decision needed it, else the FP32 value
        scale = max(1.0, float(np.abs(g.get_blocks()[1]).max()))
        assert np.abs(gm - ob["mdet"]).max() <= 32 * 2.0 ** -24 * scale
        o.coarsen_until_stable()
        g.adapt("coarsen")
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"])
    assert o.errors == 0


def test_replay_of_learned_refinement_through_oracle(mr, oracle_mod):
    # The learned step's refinement: the GPU's proposal (network or exact
    # fallback, before the closure) is exported; the oracle applies the +1
    # gradedness closure (Sec. 2.2, 2.3) and refines; the GPU's own learned
    # refinement gives the same tree and fields bit for bit.  The network is
    # trained briefly on the run's own decisions, so that it proposes blocks
    # at the moving front of the pulse and leaves their coarser neighbours to
    # the closure.
    tree = dict(Jmin=2, Jmax=6, eps=1e-4, ic="gauss", ic_params=(0.4, 0.6, 0.0, 0.04),
                rhs_params=(1.0, 0.5, 0.0))
    cfg = dict(dim=2, Jmin=2, Jmax=6, eps=1e-4, rhs="adv", rhs_params=(1.0, 0.5, 0.0), ic="gauss",
               ic_params=(0.4, 0.6, 0.0, 0.04))
    g = mr.Forest(dim=2, precision="fp64", trees=[tree], capacity=100000)
    g.init_tree()
    dt = 0.5 / (16 * 64) / math.hypot(1.0, 0.5)
    t = 0.0
    g.proposal_collect(True, 200000)
    for _ in range(300):
        g.step(np.array([t]), np.array([dt]))
        t += dt
    g.proposal_collect(False)
    tau, _ = g.proposal_train(synthetic.cnn_init_params(cnn.SHAPES, seed=20190201), epochs=3, batch=256,
                              lr=1e-3, w_pos=0.0, recall=0.999, holdout=0.2)
    g.set_refine_mode("learned")
    o = oracle_mod.Oracle(cfg)
    proposed = added = 0
    for rep in range(6):
        for _ in range(5):
            g.step(np.array([t]), np.array([dt]))
            t += dt
        start_from_gpu_state(o, g)
        g.adapt("propose")
        prop, _ = g.get_flags()
        assert set(np.unique(prop)) <= {0, 1}
        o.set_flags(prop)
        added += o.close_refine()
        proposed += int(prop.sum())
        o.refine(1)
        g.adapt("refine_step")
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"])
        # finish the step on both sides from the refined grid
        o.rk4(t, dt)
        g.rk_step(np.array([t]), np.array([dt]))
        t += dt
        o.coarsen_until_stable()
        g.adapt("coarsen")
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"])
    assert proposed > 0 and added > 0, (proposed, added, tau)


@pytest.mark.parametrize("dim", [2, 3])
def test_refinement_indicators_with_closure_match_oracle(mr, oracle_mod, dim):
    # Caller-given refinement indicators (status +1): closed under gradedness
    # and refined; the oracle's closure and refinement agree bit for bit.
    rng = np.random.default_rng(3 + dim)
    jmax = 6 if dim == 2 else 4
    leaves = treegen.random_graded_tree(dim, 2, jmax - 1, 6 if dim == 2 else 3, 11 + dim)
    lvl, crd = treegen.as_arrays(leaves)
    c = dict(dim=dim, Jmin=2, Jmax=jmax, eps=1e-3, rhs="adv", ic="none")
    o, g = make_pair(mr, oracle_mod, c, capacity=200000)
    fields = rng.standard_normal((len(leaves), 1) + (17,) * dim)
    o.set_blocks(lvl, crd, fields)
    g.set_blocks(lvl, crd, fields)
    assert_same_tree(o, g)
    # random fields: copies of a shared block-edge node differ until a
    # synchronisation gives each the owner's value (the oracle's refinement
    # synchronises every block, the GPU's only the refined ones)
    o.sync()
    g.sync_ghosts()
    added = 0
    for rep in range(3):
        n = g.num_blocks()
        info, _ = g.get_blocks(fields=False)
        mask = ((rng.random(n) < 0.1) & (info["level"] < jmax)).astype(np.int8)
        mask[int(np.argmin(info["level"]))] = 1  # at least one indicator below Jmax
        o.set_flags(mask)
        added += o.close_refine()
        o.refine(1)
        g.set_refine_mask(mask)
        g.adapt("refine_flagged")
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"])
        o.sync()
        g.sync_ghosts()
        ob, f = assert_same_tree(o, g)
        assert np.array_equal(f, ob["fields"])
    assert added > 0
    assert o.errors == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_single_coarsening_round_matches_oracle(mr, oracle_mod, precision):
    # max_rounds = 1: one coarsening round per step (Sec. 2.1 step 3 read as
    # a single pass); trees bit for bit, FP64 fields bit for bit.
    c = dict(dim=2, Jmin=2, Jmax=6, eps=1e-4, rhs="adv", rhs_params=(1.0, 0.5, 0.0), ic="gauss",
             ic_params=(0.4, 0.6, 0.0, 0.04), max_rounds=1)
    o, g = make_pair(mr, oracle_mod, c, precision=precision, capacity=60000, detail_fp64=True)
    o.init_tree()
    g.init_tree()
    dt = 0.5 / (16 * 64) / math.hypot(1.0, 0.5)
    for s in range(4):
        o.step(s * dt, dt)
        g.step(s * dt, dt)
        ob, f = assert_same_tree(o, g)
        if precision == "fp64":
            assert np.array_equal(f, ob["fields"])
        else:
            assert rel_l2(f, ob["fields"]) <= REL
    # rounds until stable never leave more blocks than a single round
    o2 = oracle_mod.Oracle(dict(c, max_rounds=0))
    o2.init_tree()
    for s in range(4):
        o2.step(s * dt, dt)
    assert o2.n <= o.n


def test_fp64_swirl_33_long_run_bit_exact(mr, oracle_mod):
    # The paper's swirl study case (Sec. 3: 33^2 blocks, beta 1e-2, t_a 5), Jmax 4,
    # eps 1e-4, plain FP64: 512 host-driven steps (a tenth of the run to t_a,
    # through the first refinements of the filament) stay bit-exact with the
    # oracle, tree and fields, at every 128th step.
    t_a = 5.0
    c = dict(dim=2, Bs=33, Jmin=1, Jmax=4, eps=1e-4, rhs="swirl", rhs_params=(t_a,), ic="gauss",
             ic_params=(0.5, 0.75, 0.0, math.sqrt(0.005)))
    o, g = make_pair(mr, oracle_mod, c, capacity=20000)
    o.init_tree()
    g.init_tree()
    n = int(math.ceil(t_a / (0.5 / (32 * 16))))
    dt = t_a / n
    for s in range(512):
        o.step(s * dt, dt)
        g.step(s * dt, dt)
        if (s + 1) % 128 == 0:
            ob, f = assert_same_tree(o, g)
            assert np.array_equal(f, ob["fields"]), (s, np.abs(f - ob["fields"]).max())
    assert o.n > 10 and o.errors == 0


def test_warp_form_variants_give_identical_steps(mr):
    # The tuning axes of the FP32 warp-per-block stage (blocks per CTA, rows
    # staged by bulk copies or loaded) and the CTA form change the launch, not
    # the arithmetic: the same grid and fields bit for bit.
    tree = dict(Jmin=2, Jmax=7, eps=1e-4, ic="gauss", ic_params=(0.5, 0.75, 0.0, 0.05), rhs_params=(5.0,))
    dt = 0.5 / (16 * 128)
    runs = []
    for form, wb, stg in ((0, 4, 1), (1, 4, 1), (1, 2, 0), (1, 8, 1), (1, 2, 1), (1, 8, 0)):
        g = mr.Forest(dim=2, precision="fp32", detail_fp64=True, rhs="swirl", trees=[tree], capacity=40000)
        g.set_tuning(0, form)
        g.set_warp_form(wb, stg)
        g.init_tree()
        for s in range(3):
            g.step(s * dt, dt)
        g.set_time(3 * dt, dt)
        g.step_graph(10)
        runs.append(g.get_blocks())
    for info, f in runs[1:]:
        assert np.array_equal(info, runs[0][0]) and np.array_equal(f, runs[0][1])
    assert len(runs[0][0]) > 20
    with pytest.raises(mr.MRError):
        mr.Forest(dim=2, trees=[dict(Jmin=2, Jmax=4)]).set_warp_form(3, 1)
