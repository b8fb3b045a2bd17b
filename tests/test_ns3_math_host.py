"""The library's 3D Navier-Stokes node arithmetic (csrc/mr_ns3_math.cuh, written
for the device) compiled as host code and run on the oracle's synchronised
tiles: its right-hand sides and its shock-capturing filter equal the oracle's 3D
forms bit for bit (flux and skew-symmetric, uniform and adaptive trees, smooth
and steep states).  The header evaluates the same
IEEE operations in the same order without fused multiply-adds, so the device
build of the same functions gives the same values; the staging kernel that
will feed it is not built yet."""
import os
import subprocess

import numpy as np
import pytest

from tests import treegen
from tests.test_oracle_ns3d import oracle3, prim_fields, state3

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1902_00088_gb300", "csrc")
GAM, MU, PR, RTH = 1.4, 0.03, 0.71, 1e-5


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("ns3") / "ns3_math_harness")
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "ns3_math_harness.cpp")])
    return exe


def run(exe, form, o, B=17, g=4, L=1.0, filt=False):
    tiles = o.tiles()
    b = o.blocks(fields=False)
    mode = {"ns": 2, "ns_skew": 3}[form] + (10 if filt else 0)
    parts = [np.array([mode, B, g, o.n], np.int32).tobytes(), np.array([GAM, MU, PR, RTH], np.float64).tobytes()]
    for n in range(o.n):
        dx = L / ((B - 1) << int(b["level"][n]))
        parts.append(np.array([dx], np.float64).tobytes())
        parts.append(np.ascontiguousarray(tiles[n], np.float64).tobytes())
    r = subprocess.run([exe], input=b"".join(parts), capture_output=True, check=True)
    return np.frombuffer(r.stdout, np.float64).reshape((o.n, 5, B, B, B))


def uniform_state(o, form, lvl, seed):
    N = 16 << lvl
    q = np.stack(state3(form, *prim_fields(seed, N)))
    leaves = sorted(treegen.uniform_tree(3, lvl))
    lv, crd = treegen.as_arrays(leaves)
    f = np.zeros((len(leaves), 5, 17, 17, 17))
    for n in range(len(leaves)):
        ix, iy, iz = (np.mod(crd[n, a] * 16 + np.arange(17), N) for a in range(3))
        f[n] = q[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    o.set_blocks(lv, crd, f)


def adaptive_state(o, form, seed):
    # levels 1 and 2: ghost layers from equal, finer and coarser neighbours
    leaves = treegen.random_graded_tree(3, 1, 2, 1, seed)
    lv, crd = treegen.as_arrays(leaves)
    rng = np.random.default_rng(seed)
    f = np.zeros((len(leaves), 5, 17, 17, 17))
    for n in range(len(leaves)):
        h = 1.0 / (16 << int(lv[n]))
        x, y, z = ((crd[n, a] * 16 + np.arange(17)) * h for a in range(3))
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        s = np.sin(2 * np.pi * (X + 2 * Y - Z)) + 0.5 * np.cos(2 * np.pi * (Y + Z))
        f[n] = state3(form, 1.0 + 0.1 * s, 0.2 + 0.1 * s, -0.1 * s, 0.3 + 0 * s, 1.0 + 0.05 * s)
    o.set_blocks(lv, crd, f)
    assert len(set(lv.tolist())) == 2 and rng is not None


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
@pytest.mark.parametrize("tree", ["uniform", "adaptive"])
def test_node_arithmetic_equals_oracle_bit_for_bit(harness, oracle_mod, form, tree):
    if tree == "uniform":
        o = oracle3(oracle_mod, form, 1, mu=MU)
        uniform_state(o, form, 1, 31)
    else:
        o = oracle_mod.Oracle(dict(dim=3, Bs=17, ng=4, nvar=5, Jmin=1, Jmax=2, eps=1e-3, rhs=form,
                                   rhs_params=(GAM, MU, PR, 0.0), ic="none", norm_kind=1))
        adaptive_state(o, form, 5)
    ref = o.rhs(0.0)  # synchronises, then the oracle's right-hand side (export order)
    got = run(harness, form, o)  # the same synchronised tiles through the header's functions
    assert o.errors == 0
    assert np.abs(ref).max() > 0.1
    bad = np.argwhere(got != ref)
    assert len(bad) == 0, (bad[:5], np.abs(got - ref).max())


@pytest.mark.parametrize("form", ["ns", "ns_skew"])
def test_filter_arithmetic_equals_oracle_bit_for_bit(harness, oracle_mod, form):
    # a steep periodic state on a uniform level-1 tree (strengths between 0 and 1
    # near the jumps, 0 elsewhere) and a smooth one on an adaptive tree
    from tests.test_oracle_filter import shock_like
    N = 32
    n = np.arange(N)
    Z, Y, X = np.meshgrid(n, n, n, indexing="ij")
    r, u, v, p = shock_like(X, Y, N)
    _, w, _, _ = shock_like(Z, Y, N)
    q = np.stack(state3(form, r, u, v, 0.6 * w, p))
    o = oracle3(oracle_mod, form, 1, rth=RTH)
    leaves = sorted(treegen.uniform_tree(3, 1))
    lv, crd = treegen.as_arrays(leaves)
    f = np.zeros((len(leaves), 5, 17, 17, 17))
    for m in range(len(leaves)):
        ix, iy, iz = (np.mod(crd[m, a] * 16 + np.arange(17), N) for a in range(3))
        f[m] = q[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    o.set_blocks(lv, crd, f)
    trees = [o]
    oa = oracle_mod.Oracle(dict(dim=3, Bs=17, ng=4, nvar=5, Jmin=1, Jmax=2, eps=1e-3, rhs=form,
                                rhs_params=(GAM, MU, PR, RTH), ic="none", norm_kind=1))
    adaptive_state(oa, form, 5)
    trees.append(oa)
    acted = []
    for t in trees:
        t.sync()
        before = t.blocks()["fields"].copy()
        got = run(harness, form, t, filt=True)  # the synchronised tiles through the header's filter
        t.filter()
        ref = t.blocks()["fields"]
        bad = np.argwhere(got != ref)
        assert len(bad) == 0, (bad[:5], np.abs(got - ref).max())
        acted.append(np.abs(ref - before).max())
    assert acted[0] > 1e-4, acted  # the steep state is filtered: the comparison is not vacuous
