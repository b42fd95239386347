"""GPU parity of time groups: batches of views that differ only in observer
time are marched together (one traversal per ray, one compensated sum per
view).  Each grouped image is held to the FP64 oracle at the FP32 tolerance,
its sample counts to the oracle's, and to the same view marched on its own
(launch group 1)."""
import math

import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity, beta_from_u, bf16_round, four_velocity_f16, parity_report
from tests.test_gpu_parity import f32, random_grid

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def batch(ctx, vol, views, launch=None):
    img, cnt = ctx.render_batch(vol, views, samples=True, launch=launch)
    torch.cuda.synchronize()
    return img.cpu().numpy(), cnt.cpu().numpy().astype(np.int64)


def time_series(base, t_list):
    return [base.with_(t_obs=float(t)) for t in t_list]


# Observer times: windows that overlap, coincide (a repeated time), lie before
# and after the box, and more views than one group takes (split into groups).
T_SERIES = (-6.0, -1.5, 0.2, 0.2, 1.1, 2.6, 3.0, 4.4, 6.9, 9.5, 14.0, 30.0)
CASES = [
    # (seed, theta, phi, c, lookback, size)
    (11, 33.0, 17.0, 1.1, True, (29, 23)),
    (12, 0.0, 0.0, 0.7, True, (21, 19)),       # along -z: two axes parallel
    (13, 54.7356, 45.0, 2.0, True, (24, 24)),  # body diagonal: crossing ties
    (14, 118.0, 250.0, 1.4, True, (17, 31)),
    (15, 70.0, 30.0, 1.0, False, (20, 20)),    # no lookback: one epoch pair per view
    (16, 25.0, 300.0, math.inf, True, (16, 16)),  # fast light: whole windows in or out
]


@pytest.mark.parametrize("seed,theta,phi,c,lookback,size", CASES)
def test_groups_match_oracle_and_lone_march(ctx, seed, theta, phi, c, lookback, size):
    grid, j, beta = random_grid(seed, n=(15, 11, 13), M=6)
    vol = ctx.load_snapshots(grid, j, beta)
    w, h = size
    fov = 1.9 * float(np.max(grid.extent))
    base = gen.view_from_angles(grid, theta, phi, size=w, fov=fov, c=c, lookback=lookback, beaming=True)
    base = base.with_(height=h, fov_v=fov * h / w, alpha=-0.6)
    views = time_series(base, T_SERIES)
    grouped, gcnt = batch(ctx, vol, views)
    lone, lcnt = batch(ctx, vol, views, launch={"group": 1})
    for k, v in enumerate(views):
        ref, rcnt = oracle.render(grid, j, beta, v, counts=True)
        assert_parity(grouped[k], ref, what=f"seed {seed} view {k} grouped vs oracle")
        assert np.abs(gcnt[k] - rcnt).max() <= 1
        # the lone march measures crossings from the view's own window start
        assert_parity(grouped[k], lone[k], rel=1e-5, what=f"seed {seed} view {k} grouped vs lone")
        assert np.abs(gcnt[k] - lcnt[k]).max() <= 1
    ctx.unload(vol)


@pytest.mark.parametrize("group,depth,regcap", [(2, 1, 0), (3, 2, 1), (4, 1, 1), (4, 2, 0), (5, 1, 0), (8, 2, 1),
                                                (8, 1, 1)])
def test_group_sizes_and_depths(ctx, group, depth, regcap):
    grid, j, beta = random_grid(21, n=(14, 12, 10), M=5)
    vol = ctx.load_snapshots(grid, j, beta, brick=4, super_brick=2, paired=True)
    base = gen.view_from_angles(grid, 41.0, 73.0, size=26, fov=1.9 * float(np.max(grid.extent)), c=1.2)
    views = time_series(base, np.linspace(-2.0, 9.0, 11))
    img, cnt = batch(ctx, vol, views, launch={"group": group, "depth": depth, "regcap": regcap, "packet": (4, 8)})
    for k, v in enumerate(views):
        ref, rcnt = oracle.render(grid, j, beta, v, counts=True)
        assert_parity(img[k], ref, what=f"group {group} depth {depth} view {k}")
        assert np.abs(cnt[k] - rcnt).max() <= 1
    ctx.unload(vol)


def test_groups_bf16_records(ctx):
    grid, j, beta, views = gen.config_precision(n=48, n_epochs=6, size=64)
    base = views[0]
    series = time_series(base, base.t_obs + np.linspace(-2.5, 2.5, 7) * grid.dt)
    vol = ctx.load_snapshots(grid, j, beta, store="bf16", paired=True)
    img, _ = batch(ctx, vol, series)
    lone, _ = batch(ctx, vol, series, launch={"group": 1})
    j_r = bf16_round(j).astype(np.float64)
    b_r = beta_from_u(four_velocity_f16(beta))
    for k, v in enumerate(series):
        assert_parity(img[k], oracle.render(grid, j_r, b_r, v), rel=1e-4, what=f"bf16 view {k} decoded inputs")
        ref = oracle.render(grid, j, beta, v)
        assert_parity(img[k], ref, rel=1e-2, what=f"bf16 view {k} vs float32 truth")
        assert abs(img[k].astype(np.float64).sum() - ref.sum()) <= 1e-3 * ref.sum()
        assert_parity(img[k], lone[k], rel=1e-5, what=f"bf16 view {k} grouped vs lone")
    ctx.unload(vol)


def test_interleaved_directions_group_by_runs(ctx):
    """Only consecutive views with the same rays group; the others march alone
    (and so equal single renders bit for bit)."""
    grid, j, beta = random_grid(31, n=(12, 14, 9), M=5)
    vol = ctx.load_snapshots(grid, j, beta)
    fov = 1.9 * float(np.max(grid.extent))
    a = gen.view_from_angles(grid, 30.0, 10.0, size=20, fov=fov, c=1.0)
    b = gen.view_from_angles(grid, 75.0, 160.0, size=20, fov=fov, c=1.0)
    views = [a.with_(t_obs=1.0), a.with_(t_obs=2.5), b.with_(t_obs=1.0), a.with_(t_obs=4.0), b.with_(t_obs=2.0),
             b.with_(t_obs=3.5), b.with_(t_obs=3.5, nu_ratio=2.0)]
    img, cnt = batch(ctx, vol, views)
    for k, v in enumerate(views):
        ref, rcnt = oracle.render(grid, j, beta, v, counts=True)
        assert_parity(img[k], ref, what=f"interleaved view {k}")
        assert np.abs(cnt[k] - rcnt).max() <= 1
    for k in (2, 3):  # runs of one view
        single = ctx.render(vol, views[k])
        torch.cuda.synchronize()
        assert np.array_equal(img[k], single.cpu().numpy())
    # a prefactor is per view: the last two differ by nu_ratio^alpha only
    pf = 2.0 ** views[6].alpha
    assert_parity(img[6], pf * img[5].astype(np.float64), rel=1e-6, what="prefactor within a group")
    ctx.unload(vol)


def test_graph_regroups_when_views_change(ctx):
    """A cached batch graph replayed with views that group differently runs
    the other kernel and gives what a fresh render gives."""
    grid, j, beta = random_grid(41, n=(13, 10, 12), M=4)
    vol = ctx.load_snapshots(grid, j, beta)
    fov = 1.9 * float(np.max(grid.extent))
    base = gen.view_from_angles(grid, 50.0, 20.0, size=18, fov=fov, c=1.3)
    same = time_series(base, (0.5, 1.5, 2.5, 3.5, 4.5, 5.5))
    dirs = gen.fibonacci_directions(6)
    spread = [gen.view_from_direction(grid, -d, size=18, fov=fov, c=1.3, t_obs=2.0) for d in dirs]
    first = ctx.render_batch(vol, same).cpu().numpy()
    other = ctx.render_batch(vol, spread).cpu().numpy()
    again = ctx.render_batch(vol, same).cpu().numpy()
    shifted = ctx.render_batch(vol, time_series(base, (1.0, 2.0, 3.0, 4.0, 5.0, 6.0))).cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(first, again)
    for k, v in enumerate(spread):
        single = ctx.render(vol, v)
        torch.cuda.synchronize()
        assert np.array_equal(other[k], single.cpu().numpy())
    for k, t in enumerate((1.0, 2.0, 3.0, 4.0, 5.0, 6.0)):
        assert_parity(shifted[k], oracle.render(grid, j, beta, base.with_(t_obs=t)), what=f"shifted view {k}")
    ctx.unload(vol)


def test_checked_library_groups():
    import paper_2609_09322_gb300 as g
    c = g.Context(0, checked=True)
    try:
        grid, j, beta = random_grid(51, n=(11, 9, 13), M=5)
        vol = c.load_snapshots(grid, j, beta, paired=True)
        base = gen.view_from_angles(grid, 64.0, 121.0, size=22, fov=1.9 * float(np.max(grid.extent)), c=0.9)
        views = time_series(base, np.linspace(-3.0, 10.0, 9))
        img = c.render_batch(vol, views)
        torch.cuda.synchronize()
        assert c.bounds_violations() == 0
        img = img.cpu().numpy()
        for k, v in enumerate(views):
            # Rays grazing a box corner here have one chord of a few
            # thousandths of a cell, whose two float32 crossings resolve about
            # 1e-7 of a unit (the same pixels are off by the same amount when
            # each view is marched alone): absolute floor 2e-7 of the peak.
            assert_parity(img[k], oracle.render(grid, j, beta, v), floor_frac=0.02, what=f"checked view {k}")
        c.unload(vol)
    finally:
        c.close()


def test_time_series_at_bench_shape_sampled(ctx):
    """The time-delay workload's shape at half size (two directions x nine
    observer times, grouped), sampled pixels against the oracle."""
    grid, j, beta, views = gen.config_time_delay(n=128, size=256, dtype=np.float32)
    vol = ctx.load_snapshots(grid, j, beta, paired=True)
    img, cnt = batch(ctx, vol, views)
    lone, lcnt = batch(ctx, vol, views, launch={"group": 1})
    rng = np.random.default_rng(5)
    for k in (0, 4, 8, 9, 13, 17):
        r = parity_report(img[k], lone[k], rel=1e-5)
        assert r["n_bad"] == 0, f"view {k} grouped vs lone: {r}"
        assert np.abs(cnt[k] - lcnt[k]).max() <= 1
        px = rng.integers(0, 256, size=(24, 2))
        sub = oracle.render_pixels(grid, j, beta, views[k], px)
        assert_parity(img[k][px[:, 1], px[:, 0]], sub, what=f"time-delay view {k} sampled")
    ctx.unload(vol)


def test_groups_with_host_output_and_many_launches(ctx):
    """Grouped batches to host memory equal the device images; a time series
    longer than one launch (130 views: 128 + 2, a run cut at the launch
    boundary) still matches the oracle view by view."""
    grid, j, beta = random_grid(61, n=(10, 12, 9), M=5)
    vol = ctx.load_snapshots(grid, j, beta, paired=True)
    base = gen.view_from_angles(grid, 28.0, 64.0, size=10, fov=1.9 * float(np.max(grid.extent)), c=0.8)
    views = time_series(base, np.linspace(-2.0, 11.0, 130))
    dev, cnt = batch(ctx, vol, views)
    host = torch.empty((130, 10, 10), dtype=torch.float32, pin_memory=True)
    ctx.render_batch_host(vol, views, host)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), dev)
    for k in (0, 1, 63, 126, 127, 128, 129):
        ref, rcnt = oracle.render(grid, j, beta, views[k], counts=True)
        assert_parity(dev[k], ref, what=f"long series view {k}")
        assert np.abs(cnt[k] - rcnt).max() <= 1
    ctx.unload(vol)
