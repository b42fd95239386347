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


@pytest.mark.parametrize("n_views", [129, 300, 1024])
def test_noalloc_many_launches_bitwise(n_views):
    """Batches past one launch's 128 views run as several launches, each with
    its own slice of the fixed tile-counter array: every image equals the
    allocating batch render bit for bit, and one equals the oracle."""
    import oracle
    import paper_2609_09322_gb300 as g
    grid, j, beta = _fields(9)
    size = 8 if n_views > 300 else 20
    with g.Context(0) as ctx:
        vol = ctx.load_snapshots(grid, j, beta)
        dirs = gen.fibonacci_directions(n_views)
        views = [gen.view_from_direction(grid, -d, size=size, c=1.0, t_obs=2.0 + 0.01 * (k % 300),
                                         beaming=(k % 3 != 0)) for k, d in enumerate(dirs)]
        for rep in range(2):
            ref = ctx.render_batch(vol, views)
            out = torch.full((n_views, size, size), float("nan"), dtype=torch.float32, device="cuda:0")
            ctx.render_batch_noalloc(vol, views, out)
            torch.cuda.synchronize()
            assert ctx.last_launch_count() == (n_views + 127) // 128
            assert torch.equal(out, ref), f"no-alloc batch of {n_views} differs from render_batch (call {rep})"
        k = n_views - 1   # the last view sits in the last launch
        want = oracle.render(grid, j.astype(np.float64), beta.astype(np.float64), views[k])
        assert_parity(out[k].cpu().numpy(), want, what=f"no-alloc view {k} vs oracle")
        ctx.unload(vol)


def test_noalloc_time_groups_bitwise():
    """A time series (one direction, many observer times) is marched in time
    groups by both entry points: the images agree bit for bit."""
    import paper_2609_09322_gb300 as g
    grid, j, beta = _fields(10)
    with g.Context(0) as ctx:
        vol = ctx.load_snapshots(grid, j, beta)
        views = [gen.view_from_angles(grid, 35.0, 15.0, size=40, c=1.2, t_obs=1.0 + 0.7 * k) for k in range(11)]
        ref = ctx.render_batch(vol, views)
        out = torch.empty((11, 40, 40), dtype=torch.float32, device="cuda:0")
        ctx.render_batch_noalloc(vol, views, out)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        ctx.unload(vol)


def test_noalloc_checks_its_output_and_launch():
    """A short, mistyped, strided or foreign-device output, mixed image
    geometries and a region-schedule launch are refused before any work."""
    import paper_2609_09322_gb300 as g
    grid, j, beta = _fields(8)
    with g.Context(0) as ctx:
        vol = ctx.load_snapshots(grid, j, beta)
        views = [gen.view_from_angles(grid, 30.0 + k, size=16, c=1.0, t_obs=4.0) for k in range(3)]
        dev = "cuda:0"
        bad = [torch.empty((2, 16, 16), dtype=torch.float32, device=dev),
               torch.empty((3, 16, 16), dtype=torch.float64, device=dev),
               torch.empty((3, 16, 32), dtype=torch.float32, device=dev)[:, :, ::2],
               torch.empty((3, 16, 16), dtype=torch.float32)]
        for out in bad:
            with pytest.raises(ValueError):
                ctx.render_batch_noalloc(vol, views, out)
        mixed = views[:2] + [gen.view_from_angles(grid, 30.0, size=8, c=1.0, t_obs=4.0)]
        with pytest.raises(ValueError):
            ctx.render_batch_noalloc(vol, mixed, torch.empty((3, 16, 16), dtype=torch.float32, device=dev))
        out = torch.empty((3, 16, 16), dtype=torch.float32, device=dev)
        launch = {"packet": (4, 8), "cta_warps": 4, "depth": 2, "persistent": 0, "regcap": 1, "region": 32}
        with pytest.raises(g.GbdError) as e:
            ctx.render_batch_noalloc(vol, views, out, launch=launch)
        assert e.value.code == g.gbdart.ERR_INVALID and "region" in str(e.value)
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
