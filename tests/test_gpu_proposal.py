"""Learned refinement proposal: GPU forward/backward against the FP64 reference
network (oracle/cnn.py), and what the trained network gains over refine-all."""
import math

import numpy as np
import pytest

import synthetic
from oracle import cnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_00088_gb300 import build as b
    b.build()
    import paper_1902_00088_gb300 as m
    return m


def test_cnn_forward_backward_matches_fp64_reference(mr):
    g = mr.Forest(dim=2, trees=[dict(Jmin=2, Jmax=4, ic="none")], capacity=1000)
    rng = np.random.default_rng(4)
    theta = synthetic.cnn_init_params(cnn.SHAPES, seed=9) + 0.02 * rng.standard_normal(cnn.NPARAM)
    T = 25
    n = 6
    x = rng.standard_normal((n, 2, T, T))
    y = np.array([1, 0, 1, 1, 0, 0], np.float64)
    p, gr, loss = g.cnn_eval(theta, x, y, w_pos=4.0)
    L, gref = cnn.loss_and_grad(theta, list(x), list(y), 4.0)
    pref = np.array([cnn.forward(theta, xi)[0] for xi in x])
    # FP32 arithmetic against FP64: probabilities to 1e-5, loss and gradient to
    # 1e-4 of the gradient's scale
    np.testing.assert_allclose(p, pref, rtol=0, atol=1e-5)
    assert abs(loss - L) <= 1e-4 * max(1.0, abs(L))
    assert np.abs(gr - gref).max() <= 1e-4 * np.abs(gref).max(), np.abs(gr - gref).max()


def run_adv(mr, mode, nsteps, params=None, tau=0.5, collect=False):
    tree = dict(Jmin=2, Jmax=6, eps=1e-4, ic="gauss", ic_params=(0.4, 0.6, 0.0, 0.04),
                rhs_params=(1.0, 0.5, 0.0))
    g = mr.Forest(dim=2, precision="fp32", detail_fp64=True, trees=[tree], capacity=200000)
    g.init_tree()
    if collect:
        g.proposal_collect(True, 600000)
    if mode == "learned":
        g.proposal_set(params, tau)
        g.set_refine_mode("learned")
    dt = 0.5 / (16 * 64) / math.hypot(1.0, 0.5)
    g.reset_stats()
    for s in range(nsteps):
        g.step(s * dt, dt)
    st = g.stats()
    err = g.error(0, nsteps * dt)
    return g, st, err


def test_learned_proposal_gain_over_refine_all(mr):
    # The method without the network refines every block each step (Sec. 2.1).
    # Trained on this run's own decisions, the network + exact fallback advance
    # far fewer blocks at the same error, and the network removes most misses of
    # the fallback alone (tau = 2 disables the network).
    n = 1000
    plain, st0, e0 = run_adv(mr, "all", n, collect=True)
    ns, npos = plain.proposal_dataset()
    assert ns > 1000 and 0 < npos < ns
    init = synthetic.cnn_init_params(cnn.SHAPES, seed=20190201)
    tau, loss = plain.proposal_train(init, epochs=6, batch=256, lr=1e-3, w_pos=0.0, recall=0.999,
                                     holdout=0.2)
    params, _ = plain.proposal_get()
    learned, st1, e1 = run_adv(mr, "learned", n, params=params, tau=tau)
    fb, st2, e2 = run_adv(mr, "learned", n, params=params, tau=2.0)
    pl, pf = learned.proposal_stats(), fb.proposal_stats()
    ratio = st1["stage_blocks"] / st0["stage_blocks"]
    assert ratio < 0.8, (ratio, pl)
    assert e1["l2"] <= 1.1 * e0["l2"] + 1e-5, (e0, e1)
    assert pl["network"] > 0 and pl["misses"] < pf["misses"], (pl, pf)


def test_learned_graph_steps_equal_eager_steps(mr):
    # The captured step runs the proposal, its closure (fixed passes) and the
    # miss check on the device: same grid, fields and counters as host-driven steps.
    params = synthetic.cnn_init_params(cnn.SHAPES, seed=7)
    tree = dict(Jmin=2, Jmax=6, eps=1e-4, ic="gauss", ic_params=(0.4, 0.6, 0.0, 0.04),
                rhs_params=(1.0, 0.5, 0.0))
    dt = 0.5 / (16 * 64) / math.hypot(1.0, 0.5)
    runs = []
    for graph in (False, True):
        g = mr.Forest(dim=2, precision="fp32", detail_fp64=True, trees=[tree], capacity=40000)
        g.init_tree()
        g.proposal_set(params, 0.5)
        g.set_refine_mode("learned")
        if graph:
            g.set_time(0.0, dt)
            g.step_graph(12)
        else:
            for s in range(12):
                g.step(s * dt, dt)
        info, f = g.get_blocks()
        runs.append((info, f, g.proposal_stats()))
    (ia, fa, sa), (ib, fb, sb) = runs
    assert np.array_equal(ia, ib) and np.array_equal(fa, fb)
    assert sa == sb and sa["considered"] > 0, (sa, sb)
