"""The batch render that allocates nothing, for callers that cannot let the
library allocate device memory while they render (an application that owns
the whole device through its own allocator, or a latency-critical loop that
must not pay for cudaMalloc / cudaFree).

It is called through the C ABI and compared with the allocating batch render
on two calls in a row; the second call uses different views, so a table or
tile counter left over from the first call would show.  This file is
collected last, and passes both alone in a fresh process and after the
other tests.
"""
import numpy as np
import pytest

import gen
from tests._parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields(seed):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=(30, 26, 34), origin=(-2.0, 1.0, 0.0), dx=(1.0, 0.9, 1.1), n_epochs=5, t0=0.0, dt=2.0)
    nx, ny, nz = grid.n
    j = (rng.random((5, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(5, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, 0.9, size=(5, nz, ny, nx, 1))).astype(np.float32)
    return grid, j, beta


def test_noalloc_batch_matches_allocating_batch():
    import paper_2609_09322_gb300 as g
    grid, j, beta = _fields(7)
    with g.Context(0) as ctx:
        vol = ctx.load_snapshots(grid, j, beta)
        dirs = gen.fibonacci_directions(10)
        first = [gen.view_from_direction(grid, -d, size=48, c=1.1, t_obs=4.0) for d in dirs]
        second = [gen.view_from_direction(grid, -d, size=48, c=0.8, t_obs=6.5, beaming=(k % 2 == 0))
                  for k, d in enumerate(dirs[:7])]
        for views in (first, second):
            ref = ctx.render_batch(vol, views)
            out = torch.full((len(views), 48, 48), float("nan"), dtype=torch.float32, device="cuda:0")
            ctx.render_batch_noalloc(vol, views, out)
            torch.cuda.synchronize()
            assert ctx.last_launch_count() == 1
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            for k in range(len(views)):
                assert_parity(got[k], want[k], what=f"no-alloc view {k}")
        ctx.unload(vol)


def test_noalloc_rejects_oversized_batches_and_host_output():
    import paper_2609_09322_gb300 as g
    grid, j, beta = _fields(8)
    with g.Context(0) as ctx:
        vol = ctx.load_snapshots(grid, j, beta)
        view = gen.view_from_angles(grid, 30.0, size=8, c=1.0, t_obs=4.0)
        out = torch.empty((1025, 8, 8), dtype=torch.float32, device="cuda:0")
        with pytest.raises(g.GbdError) as e:
            ctx.render_batch_noalloc(vol, [view] * 1025, out)
        assert e.value.code == g.gbdart.ERR_INVALID and "1024" in str(e.value)
        host = torch.empty((1, 8, 8), dtype=torch.float32)
        lib = ctx.lib
        arr = (g.gbdart.CView * 1)(g.gbdart._cview(view))
        spec = ctx._spec(view, host.data_ptr(), None, on_host=True)
        rc = lib.gbd_render_batch_noalloc(ctx.handle, vol, arr, 1, spec, None, None)
        assert rc == g.gbdart.ERR_INVALID
        ctx.unload(vol)
