"""mr_error_noalloc: the error norms of mr_error for callers that cannot
allocate device memory (their device memory is held by another allocator, or
they must avoid the device synchronisation of cudaFree).  Its scratch is a
static device array shared by all calls; two calls in a row must each agree
with the allocating entry point.  Kept in a file of its own, collected last."""
import math

import numpy as np
import pytest

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


def test_noalloc_error_matches_allocating_entry_point(mr):
    tree = dict(Jmin=2, Jmax=5, eps=1e-4, ic="gauss", ic_params=(0.45, 0.55, 0.0, 0.05),
                rhs_params=(1.0, 0.5, 0.0))
    g = mr.Forest(dim=2, precision="fp64", trees=[tree], capacity=20000)
    g.init_tree()
    dt = 0.5 / (16 * 32) / math.hypot(1.0, 0.5)
    for s in range(3):
        g.step(s * dt, dt)
    t = 3 * dt
    for tq in (t, 0.5 * t):  # two calls in a row, different exact fields
        ref = g.error(0, tq)
        ref = np.array([ref["l2_abs"], ref["l2_abs"] / ref["l2"], ref["linf_abs"], ref["linf_abs"] / ref["linf"]])
        out = g.error_noalloc(0, tq)
        # same sums up to the rounding of exp and the order of atomic additions
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0)


def test_noalloc_error_rejects_trees_beyond_its_scratch(mr):
    big = mr.Forest(dim=2, Bs=33, trees=[dict(Jmin=2, Jmax=10, ic="gauss",
                                              ic_params=(0.5, 0.5, 0.0, 0.05))], capacity=100)
    with pytest.raises(mr.MRError) as e:
        big.error_noalloc(0, 0.0)
    assert e.value.status == mr.MR_EINVAL and "scratch limit" in str(e.value)
