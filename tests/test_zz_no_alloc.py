"""msi_lower_bounds_noalloc, the entry point for callers that cannot allocate device
memory (for example code held to a memory budget by an allocator it does not control,
or a latency-critical path that must not wait on cudaMalloc). It must give the same
bounds as msi_lower_bounds,
which allocates its workspace, on consecutive calls that reuse its fixed scratch.
This file runs last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu


def test_noalloc_lower_bounds_equal_allocating_entry_point():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_00786_gb300 as msi

    X = datagen.walks(77, 0, 7000, 256)
    index = msi.msi_build(X, segments=16, cardinality=256, leaf_capacity=64)
    Q = datagen.walks(78, 0, 2, 256)
    s_lb = torch.empty(index.n, dtype=torch.float32, device="cuda")
    l_lb = torch.empty(index.leaves, dtype=torch.float32, device="cuda")
    for q in Q:  # two calls in a row on the shared scratch
        want_s, want_l = msi.msi_lower_bounds(index, q)
        msi.msi_lower_bounds_noalloc(index, torch.from_numpy(q).cuda(), s_lb, l_lb)
        torch.cuda.synchronize()
        np.testing.assert_allclose(s_lb.cpu().numpy(), want_s, rtol=1e-6, atol=0)
        np.testing.assert_allclose(l_lb.cpu().numpy(), want_l, rtol=1e-6, atol=0)
    with pytest.raises(msi.MsiError) as e:  # host memory is refused: nothing is staged
        msi.msi_lower_bounds_noalloc(index, Q[0], s_lb, l_lb)
    assert e.value.status == msi.MSI_EINVAL
    # a NaN query on a caller's stream (no error status without a wait): NaN bounds
    bad = torch.from_numpy(Q[0].copy()).cuda()
    bad[5] = float("nan")
    s = torch.cuda.Stream()
    msi.msi_lower_bounds_noalloc(index, bad, s_lb, l_lb, stream=s)
    s.synchronize()
    assert torch.isnan(s_lb).all() and torch.isnan(l_lb).all()
    index.close()
