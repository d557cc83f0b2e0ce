"""rbffd_build_stencils_static: the clouds without any device allocation.

For callers that cannot allocate device memory once they run (a fixed
footprint, or no implicit device synchronisation from cudaMalloc/cudaFree).
Checked through the C ABI against rbffd_build_stencils, which allocates its
workspace per call: two calls in a row (the second must not see leftovers
of the first), bit-exact like every cloud comparison in this suite.
This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2106_07616_gb300 import clouds, rbffd

pytestmark = pytest.mark.gpu


def _both(ctx, x, y, tag, q):
    n = x.size
    dx = torch.from_numpy(x).cuda()
    dy = torch.from_numpy(y).cuda()
    dt = None if tag is None else torch.from_numpy(tag).cuda()
    a = torch.full((n * q,), -7, dtype=torch.int32, device="cuda")
    b = torch.full((n * q,), -9, dtype=torch.int32, device="cuda")
    rbffd.rbffd_build_stencils_static(ctx, dx, dy, dt, q, a)
    rbffd.rbffd_build_stencils(ctx, dx, dy, dt, q, b)
    torch.cuda.synchronize()
    return a.cpu().numpy(), b.cpu().numpy()


def test_static_matches_allocating_entry_point_twice():
    from paper_2106_07616_gb300 import _build
    _build.build()
    ctx = rbffd.Context(0)
    fp = clouds.cavity(120)                     # 14 400 points, one-sided boundary clouds
    a, b = _both(ctx, fp.x, fp.y, fp.tag, fp.q)
    assert np.array_equal(a, b)
    x, y = clouds.random_cloud(5000, seed=31)   # smaller problem second: stale data would show
    a, b = _both(ctx, x, y, None, 20)
    assert np.array_equal(a, b)
    ctx.close()


def test_static_rejects_too_many_points():
    ctx = rbffd.Context(0)
    n = rbffd.STATIC_MAX_POINTS + 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    idx = torch.zeros(n * 4, dtype=torch.int32, device="cuda")
    with pytest.raises(rbffd.RbffdError) as e:
        rbffd.rbffd_build_stencils_static(ctx, x, x, None, 4, idx)
    assert e.value.code == rbffd.EINVAL
    assert "static limit" in str(e.value)
    ctx.close()
