"""The region schedule of batched renders (gbd_launch.region).

A batch marched region by region must give, for every view and pixel, the
sum the whole-ray march gives, up to rounding (each ray restarts its anchor
at every region it enters and its region sums are added in order): held to
the oracle at the FP32 1e-5 bound (on the values the GPU stores), to the
whole-ray march within the sum of their bounds, and to itself bitwise from
run to run.  Cases cover mirrored and parallel axes, grids that
are not multiples of the region edge, both storages, paired snapshots, every
lookback/beaming routine, and host output.
"""
import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity, beta_from_u, bf16_round, four_velocity_f16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _fields(seed, n, M, bmax=0.9):
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) * rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, bmax, size=(M, nz, ny, nx, 1))).astype(np.float32)
    return j, beta


def _views(grid, count, seed, size, *, lookback=True, beaming=True, c=1.3):
    """Directions on a Fibonacci sphere plus three axis-parallel ones (the
    view then runs parallel to two axes and is mirrored on the third)."""
    rng = np.random.default_rng(seed)
    dirs = list(gen.fibonacci_directions(count - 3)) + [np.array([0.0, 0.0, -1.0]), np.array([1.0, 0.0, 0.0]),
                                                        np.array([0.0, -1.0, 0.0])]
    u_span = grid.dt * (grid.n_epochs - 1)
    out = []
    for d in dirs:
        t_obs = float(grid.t0 + rng.uniform(0.2, 0.8) * u_span)
        out.append(gen.view_from_direction(grid, d, size=size, c=c, t_obs=t_obs, lookback=lookback,
                                           beaming=beaming))
    return out


def _batch(ctx, vol, views, **launch):
    base = {"packet": (8, 4), "cta_warps": 4, "depth": 2, "persistent": 1, "regcap": 0}
    base.update(launch)
    img = ctx.render_batch(vol, views, launch=base)
    torch.cuda.synchronize()
    return img.cpu().numpy()


CASES = [
    # (seed, n, M, store, paired, lookback, beaming, region, views, size)
    (1, (40, 33, 37), 5, "f32", False, True, True, 16, 12, 40),
    (2, (48, 48, 48), 4, "f32", True, True, True, 32, 10, 32),
    (3, (35, 20, 50), 3, "bf16", False, True, False, 16, 9, 36),
    (4, (64, 17, 30), 6, "bf16", True, False, True, 16, 11, 28),
    (5, (30, 30, 30), 1, "f32", False, False, False, 64, 8, 48),
]


@pytest.mark.parametrize("seed,n,M,store,paired,lookback,beaming,region,nv,size", CASES)
def test_region_schedule_matches_whole_rays(ctx, seed, n, M, store, paired, lookback, beaming, region, nv, size):
    grid = gen.Grid(n=n, origin=(-2.0, 1.0, 0.5), dx=(1.0, 0.9, 1.2), n_epochs=M, t0=0.3, dt=2.1)
    j, beta = _fields(seed, n, M)
    vol = ctx.load_snapshots(grid, j, beta, store=store, brick=4, super_brick=2, paired=paired)
    views = _views(grid, nv, seed, size, lookback=lookback, beaming=beaming)
    whole = _batch(ctx, vol, views, region=0)
    reg = _batch(ctx, vol, views, region=region, persistent=0)
    again = _batch(ctx, vol, views, region=region, persistent=0)
    assert np.array_equal(reg, again), "region schedule is not reproducible"
    # the oracle reads exactly what the GPU stores
    js, bs = (j, beta) if store == "f32" else (bf16_round(j), beta_from_u(four_velocity_f16(beta)))
    # BF16/FP16 records: the kernel boosts from the stored u in float32 (1e-4, as for whole rays)
    rel = 1e-5 if store == "f32" else 1e-4
    for k in range(len(views)):
        assert_parity(reg[k], oracle.render(grid, js, bs, views[k]), rel=rel, what=f"view {k} region vs oracle")
        # both schedules sit within 1e-5 of the oracle
        assert_parity(reg[k], whole[k], rel=2e-5, what=f"view {k} region vs whole ray")
    assert ctx.bounds_violations() == 0
    ctx.unload(vol)


@pytest.mark.parametrize("warps", [1, 4, 8])
def test_region_ray_lists_hold_every_crossing_ray(ctx, warps):
    """Fine pixels (0.3-0.7 cells), stretched cells, a wide non-square
    image zoomed in past the grid's edges, and CTAs of 1 to 8 warps: each
    region's ray list (sized by the bound on the pixels the region's box can
    cover) takes every crossing ray, so the images equal the whole-ray march
    and no list overflows."""
    grid = gen.Grid(n=(37, 29, 41), origin=(1.0, -3.0, 0.0), dx=(0.7, 1.3, 1.0), n_epochs=3, t0=0.0, dt=4.0)
    j, beta = _fields(31, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    for fov in (20.0, 45.0):
        views = [gen.view_from_direction(grid, d, size=112, height=72, fov=fov, c=1.1, t_obs=3.0)
                 for d in gen.fibonacci_directions(7)]
        whole = _batch(ctx, vol, views, region=0)
        got = _batch(ctx, vol, views, region=16, cta_warps=warps, persistent=0)
        for k in range(len(views)):
            assert_parity(got[k], whole[k], rel=2e-5, what=f"{warps} warps fov {fov} view {k}")
        assert ctx.bounds_violations() == 0
    ctx.unload(vol)


def test_region_schedule_many_launches(ctx):
    """200 views in one region launch (in direction order, so that each
    image's view sits elsewhere in the march than in the batch) and three
    reductions in batch order; every image equals the whole-ray march, to
    device and host memory."""
    grid = gen.Grid(n=(40, 36, 33), origin=(0.5, 0.0, -1.0), dx=(1.0, 1.1, 0.9), n_epochs=4, t0=0.0, dt=3.0)
    j, beta = _fields(41, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    rng = np.random.default_rng(41)
    views = [gen.view_from_direction(grid, d, size=20, c=1.2, t_obs=float(rng.uniform(2.0, 8.0)))
             for d in gen.fibonacci_directions(200)]
    whole = _batch(ctx, vol, views, region=0)
    got = _batch(ctx, vol, views, region=16, cta_warps=8, persistent=0)
    for k in range(len(views)):
        assert_parity(got[k], whole[k], rel=2e-5, what=f"view {k}")
    host = torch.empty((len(views), 20, 20), dtype=torch.float32, pin_memory=True)
    ctx.render_batch_host(vol, views, host, launch={"packet": (4, 8), "cta_warps": 4, "depth": 2, "persistent": 0,
                                                    "regcap": 1, "region": 16})
    torch.cuda.synchronize()
    for k in range(len(views)):
        assert_parity(host[k].numpy(), whole[k], rel=2e-5, what=f"host output view {k}")
    assert ctx.bounds_violations() == 0
    ctx.unload(vol)


@pytest.mark.parametrize("n_views", [1, 2])
def test_region_schedule_one_or_two_views(ctx, n_views):
    """The smallest batches: one and two views (one region launch, one
    reduction) equal the whole-ray march."""
    grid = gen.Grid(n=(33, 35, 31), n_epochs=2, t0=0.0, dt=4.0)
    j, beta = _fields(45 + n_views, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    views = [gen.view_from_angles(grid, 40.0 + 25.0 * k, 15.0, size=36, c=1.1, t_obs=2.0) for k in range(n_views)]
    whole = _batch(ctx, vol, views, region=0)
    got = _batch(ctx, vol, views, region=16, persistent=0)
    for k in range(n_views):
        assert_parity(got[k], whole[k], rel=2e-5, what=f"view {k}")
    assert ctx.bounds_violations() == 0
    ctx.unload(vol)


def test_region_schedule_without_graphs_equals_graphs(ctx, monkeypatch):
    """With graph replay off (GBD_GRAPHS=0) a region batch is enqueued
    directly, with stream-ordered scratch and its tables uploaded on the
    caller's stream: the same kernels in the same order, so the images equal
    the graph replay's bit for bit, to device and to host memory."""
    grid = gen.Grid(n=(36, 30, 42), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=3, t0=0.0, dt=2.5)
    j, beta = _fields(43, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    views = _views(grid, 14, 43, 24)
    launch = {"packet": (4, 8), "cta_warps": 4, "depth": 2, "persistent": 0, "regcap": 1, "region": 16}
    graphed = ctx.render_batch(vol, views, launch=launch)
    torch.cuda.synchronize()
    graphed = graphed.cpu().numpy()
    monkeypatch.setenv("GBD_GRAPHS", "0")
    direct = ctx.render_batch(vol, views, launch=launch)
    host = torch.empty((len(views), 24, 24), dtype=torch.float32, pin_memory=True)
    ctx.render_batch_host(vol, views, host, launch=launch)
    torch.cuda.synchronize()
    assert np.array_equal(direct.cpu().numpy(), graphed)
    assert np.array_equal(host.numpy(), graphed)
    assert ctx.bounds_violations() == 0
    ctx.unload(vol)


def test_tuner_times_region_schedules(ctx):
    """A batch of 12 views: the autotuner also times region schedules (edges 32
    and 64), and the render it then picks equals the untuned one to FP32
    rounding."""
    grid = gen.Grid(n=(40, 36, 44), n_epochs=4, t0=0.0, dt=3.0)
    j, beta = _fields(44, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    views = _views(grid, 12, 44, 48)
    before = _batch(ctx, vol, views, region=0)
    res = ctx.tune(vol, views, launch=True)
    # the default, 72 whole-ray shapes and the flat one, then 2 edges x 16 region shapes
    assert res["candidates"] >= 1 + 72 + 1 + 32
    after = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    after = after.cpu().numpy()
    for k in range(len(views)):
        assert_parity(after[k], before[k], rel=2e-5, what=f"tuned view {k}")
    ctx.unload(vol)


def test_region_schedule_host_output_and_depths(ctx):
    grid = gen.Grid(n=(33, 41, 29), origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=4, t0=0.0, dt=3.0)
    j, beta = _fields(7, grid.n, grid.n_epochs)
    vol = ctx.load_snapshots(grid, j, beta)
    views = _views(grid, 10, 7, 30)
    whole = _batch(ctx, vol, views, region=0)
    for depth in (1, 2):
        for regcap in (0, 1):
            got = _batch(ctx, vol, views, region=32, depth=depth, regcap=regcap, persistent=0)
            for k in range(len(views)):
                assert_parity(got[k], whole[k], rel=2e-5, what=f"depth {depth} regcap {regcap} view {k}")
    host = torch.empty((len(views), 30, 30), dtype=torch.float32, pin_memory=True)
    ctx.render_batch_host(vol, views, host, launch={"packet": (4, 8), "cta_warps": 8, "depth": 2, "persistent": 0,
                                                    "regcap": 1, "region": 16})
    torch.cuda.synchronize()
    for k in range(len(views)):
        assert_parity(host[k].numpy(), whole[k], rel=2e-5, what=f"host output view {k}")
    ctx.unload(vol)


def test_region_schedule_rejects_bad_edges(ctx):
    import paper_2609_09322_gb300 as g
    grid = gen.Grid(n=(8, 8, 8), n_epochs=1)
    j, beta = _fields(8, grid.n, 1)
    vol = ctx.load_snapshots(grid, j, beta)
    views = _views(grid, 4, 8, 8, lookback=False)
    for bad in (8, 48, 256):
        with pytest.raises(g.GbdError):
            _batch(ctx, vol, views, region=bad)
    with pytest.raises(g.GbdError):
        _batch(ctx, vol, views, region=16, depth=4)
    ctx.unload(vol)
