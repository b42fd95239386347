"""GPU parity: the sm_103a library against the FP64 oracle on seeded inputs.

Every comparison feeds the oracle the values the GPU stores (float32 fields,
or bfloat16 j' and float16 four-velocity decoded in float64), so the FP32
tolerance measures kernel arithmetic alone: |I_gpu - I_ref| <= 1e-5 |I_ref|
+ 1e-8 max(I_ref) per pixel.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity, beta_from_u, bf16_round, four_velocity_f16, parity_report

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def render_cpu(ctx, vol, view, **kw):
    img = ctx.render(vol, view, **kw)
    torch.cuda.synchronize()
    if isinstance(img, tuple):
        return tuple(x.cpu().numpy() for x in img)
    return img.cpu().numpy()


def random_grid(seed, *, n=(13, 9, 11), M=5, dx=(1.0, 0.8, 1.3), origin=(-3.0, 2.0, 0.5), bmax=0.9,
                dt=1.7, t0=-0.4):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=n, origin=origin, dx=dx, n_epochs=M, t0=t0, dt=dt)
    nx, ny, nz = n
    j = f32(rng.random((M, nz, ny, nx)) * rng.random((M, nz, ny, nx)) + 0.05)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = f32(d * rng.uniform(0.0, bmax, size=(M, nz, ny, nx, 1)))
    return grid, j, beta


# ------------------------------------------------------------- the tiny case
def test_tiny_jet_fp64_input(ctx):
    """32^3 seeded conical jet, one epoch, beta = 0.9 z, 64x64 at theta = 30,
    no light-travel delay (the plain-method configuration)."""
    grid, j, beta, views = gen.config_tiny()
    vol = ctx.load_snapshots(grid, j, beta)          # float64 in, float32 stored
    img, cnt = render_cpu(ctx, vol, views[0], samples=True)
    ref, rcnt = oracle.render(grid, f32(j), f32(beta), views[0], counts=True)
    assert_parity(img, ref, what="tiny")
    assert np.abs(cnt.astype(np.int64) - rcnt).max() <= 1
    assert abs(int(cnt.sum()) - int(rcnt.sum())) <= max(2, 1e-4 * rcnt.sum())
    # end to end against the float64 fields: float32 storage of j' and beta
    full = oracle.render(grid, j, beta, views[0])
    r = parity_report(img, full, rel=1e-5)
    assert r["worst_rel"] < 1e-5
    ctx.unload(vol)


# ------------------------------------------------- random grids, all routines
CASES = [
    # (seed, theta, phi, lookback, beaming, c, size)
    (1, 33.0, 17.0, True, True, 1.1, (37, 23)),
    (2, 71.0, 200.0, True, True, 2.5, (16, 16)),
    (3, 0.0, 0.0, True, True, 0.7, (21, 19)),      # along -z: s_hat has zero x, y
    (4, 90.0, 0.0, True, False, 1.3, (24, 40)),    # along -x: zero y, z
    (5, 125.0, 45.0, False, True, 1.0, (29, 31)),
    (6, 54.7356, 45.0, False, False, 1.0, (32, 32)),  # body diagonal: ties at corners
    (7, 180.0, 0.0, True, True, 0.9, (17, 13)),    # along +z
    (8, 12.0, 300.0, True, True, math.inf, (20, 20)),  # fast-light limit of lookback
]


@pytest.mark.parametrize("seed,theta,phi,lookback,beaming,c,size", CASES)
def test_random_grids(ctx, seed, theta, phi, lookback, beaming, c, size):
    grid, j, beta = random_grid(seed)
    vol = ctx.load_snapshots(grid, j, beta)
    w, h = size
    fov = 1.9 * float(np.max(grid.extent))
    base = gen.view_from_angles(grid, theta, phi, size=w, fov=fov, c=c, lookback=lookback, beaming=beaming)
    base = base.with_(height=h, fov_v=fov * h / w)
    # sweep t_obs so the lookback window enters, covers and leaves the box
    for t_obs in (-9.0, -2.0, 1.3, 4.0, 7.7, 12.0, 40.0):
        v = base.with_(t_obs=t_obs, alpha=-0.6 if seed % 2 else 0.3, nu_ratio=1.0 if seed % 3 else 1.7)
        img, cnt = render_cpu(ctx, vol, v, samples=True)
        ref, rcnt = oracle.render(grid, j, beta, v, counts=True)
        assert_parity(img, ref, what=f"seed {seed} t_obs {t_obs}")
        assert np.abs(cnt.astype(np.int64) - rcnt).max() <= 1
    ctx.unload(vol)


def test_anisotropic_single_cell_and_tiny_grids(ctx):
    for n in ((1, 1, 1), (1, 5, 1), (2, 1, 3), (4, 4, 4)):
        grid, j, beta = random_grid(20 + n[0] + 2 * n[1], n=n, M=3)
        vol = ctx.load_snapshots(grid, j, beta)
        v = gen.view_from_angles(grid, 41.0, 13.0, size=9, fov=2.0 * float(np.max(grid.extent)) + 1, c=1.0,
                                 t_obs=1.0)
        assert_parity(render_cpu(ctx, vol, v), oracle.render(grid, j, beta, v), what=f"n={n}")
        ctx.unload(vol)


def test_single_epoch_lookback_and_window_edges(ctx):
    """M = 1 under lookback keeps only the fading weight of the one snapshot;
    views whose window edge cuts the box exercise the continuity at the
    ends of the stored range."""
    for M in (1, 2):
        grid, j, beta = random_grid(30 + M, M=M, n=(10, 10, 10), dt=3.0, t0=0.0)
        vol = ctx.load_snapshots(grid, j, beta)
        for t_obs in (-1.0, 0.0, 2.0, 3.5, 6.0):
            v = gen.view_from_angles(grid, 63.0, 31.0, size=24, c=1.2, t_obs=t_obs)
            assert_parity(render_cpu(ctx, vol, v), oracle.render(grid, j, beta, v), what=f"M={M} t={t_obs}")
        ctx.unload(vol)


def test_rays_missing_the_box_are_zero(ctx):
    grid, j, beta = random_grid(40)
    vol = ctx.load_snapshots(grid, j, beta)
    v = gen.view_from_angles(grid, 50.0, 10.0, size=16, fov=5.0, c=1.0, t_obs=2.0)
    far = v.with_(center=tuple(np.asarray(v.center) + 100.0 * np.asarray((0.0, 1.0, 0.0))))
    img = render_cpu(ctx, vol, far)
    assert np.all(img == 0.0)
    ctx.unload(vol)


# ---------------------------------------------- batching and launch invariance
def test_batch_equals_single_bitwise(ctx):
    grid, j, beta = random_grid(50, n=(24, 20, 28), M=6)
    vol = ctx.load_snapshots(grid, j, beta)
    dirs = gen.fibonacci_directions(12)
    views = [gen.view_from_direction(grid, -d, size=40, c=1.3, t_obs=4.0 + 0.3 * k) for k, d in enumerate(dirs)]
    batch = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    batch = batch.cpu().numpy()
    for k, v in enumerate(views):
        single = render_cpu(ctx, vol, v)
        assert np.array_equal(batch[k], single), f"view {k} differs between batch and single render"
    for launch in ({"packet": (4, 8), "depth": 1}, {"packet": (16, 2), "depth": 4, "cta_warps": 4},
                   {"packet": (32, 1), "depth": 2, "persistent": 0}, {"packet": (8, 4), "cta_warps": 8, "depth": 4}):
        other = ctx.render_batch(vol, views, launch=launch)
        torch.cuda.synchronize()
        assert np.array_equal(other.cpu().numpy(), batch), f"launch {launch} changed the result"
    # graph replay with changed views, then the original views again
    moved = [v.with_(t_obs=v.t_obs + 1.0) for v in views]
    b2 = ctx.render_batch(vol, moved)
    b3 = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    assert np.array_equal(b3.cpu().numpy(), batch)
    assert_parity(b2.cpu().numpy()[3], oracle.render(grid, j, beta, moved[3]), what="moved view")
    ctx.unload(vol)


@pytest.mark.parametrize("brick,super_brick,paired,morton", [(1, 1, 0, 0), (4, 1, 0, 0), (4, 4, 0, 0), (8, 2, 0, 0),
                                                            (2, 2, 0, 0), (8, 4, 1, 0), (4, 2, 1, 0), (1, 1, 1, 0),
                                                            (8, 4, 0, 1), (4, 2, 1, 1)])
@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_layouts_bitwise_identical(ctx, brick, super_brick, paired, morton, store):
    """Every layout, paired snapshots included, gives the same image; the
    windows of the views reach both ends of the stored snapshots."""
    grid, j, beta = random_grid(60, n=(19, 26, 33), M=4)
    ref_vol = ctx.load_snapshots(grid, j, beta, store=store)
    vol = ctx.load_snapshots(grid, j, beta, store=store, brick=brick, super_brick=super_brick, paired=paired,
                             morton_cells=morton)
    for t_obs in (-3.0, 3.0, 9.0):
        v = gen.view_from_angles(grid, 37.0, 120.0, size=48, c=1.5, t_obs=t_obs)
        a = render_cpu(ctx, ref_vol, v)
        b = render_cpu(ctx, vol, v)
        assert np.array_equal(a, b)
    info = ctx.volume_info(vol)
    assert (info["brick"], info["super_brick"], info["paired"], info["morton_cells"]) == \
        (brick, super_brick, paired, morton)
    # re-layout in place, in and out of the paired form and the Morton cells
    ctx.relayout(vol, 8, 2, not paired, not morton)
    assert np.array_equal(render_cpu(ctx, vol, v), a)
    ctx.unload(vol)
    ctx.unload(ref_vol)


def test_host_output_matches_device(ctx):
    grid, j, beta = random_grid(70, n=(16, 16, 16), M=3)
    vol = ctx.load_snapshots(grid, j, beta)
    views = [gen.view_from_angles(grid, 20.0 * k, 15.0, size=33, c=1.0, t_obs=2.0) for k in range(5)]
    dev = ctx.render_batch(vol, views)
    host = torch.empty((5, 33, 33), dtype=torch.float32, pin_memory=True)
    ctx.render_batch_host(vol, views, host)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), dev.cpu().numpy())
    ctx.unload(vol)


# ------------------------------------------------------ the time-delay path
def test_time_delay_reduced(ctx):
    """Moving blob over a steady jet (the time-delay configuration at 64^3 x
    16, 128^2): full images against the oracle for every view."""
    grid, j, beta, views = gen.config_time_delay(n=64, size=128, n_tobs=3, dtype=np.float32)
    vol = ctx.load_snapshots(grid, j, beta)
    imgs = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    imgs = imgs.cpu().numpy()
    for k, v in enumerate(views):
        assert_parity(imgs[k], oracle.render(grid, j, beta, v), what=f"view {k}")
    ctx.unload(vol)


def test_apparent_speed_on_gpu(ctx):
    """The GPU images of a blob at beta = 0.95 move across the sky at
    beta sin(theta) / (1 - beta cos(theta)) (Sec. 3.2)."""
    from tests.test_oracle_pins import blob_worldline
    for theta, expect in ((10.0, 2.5603), (45.0, 2.0465)):
        grid, j, b, v0, times = blob_worldline(theta)
        vol = ctx.load_snapshots(grid, j, b)
        views = [v0.with_(t_obs=t) for t in times]
        imgs = ctx.render_batch(vol, views)
        torch.cuda.synchronize()
        imgs = imgs.cpu().numpy().astype(np.float64)
        q = (np.arange(v0.height) + 0.5 - v0.height / 2) * v0.fov_v / v0.height
        cents = [float((im.sum(axis=1) * q).sum() / im.sum()) for im in imgs]
        speed = np.polyfit(times, cents, 1)[0] / v0.c
        assert speed == pytest.approx(expect, rel=0.02)
        for k in (0, 3):
            assert_parity(imgs[k], oracle.render(grid, j, b, views[k]), what=f"theta {theta}")
        ctx.unload(vol)


# ----------------------------------------------------------- BF16/FP16 path
def test_bf16_f16u_path(ctx):
    """bfloat16 j' and float16 four-velocity with float32 accumulation:
    against the oracle on the decoded stored values (kernel arithmetic) and on
    the float32 fields (end-to-end storage error: <= 1e-2 per pixel and
    <= 1e-3 in total flux)."""
    grid, j, beta, views = gen.config_precision(n=64, n_epochs=4, size=96)
    vol = ctx.load_snapshots(grid, j, beta, store="bf16")
    assert ctx.volume_info(vol)["record_bytes"] == 8
    img = render_cpu(ctx, vol, views[0])
    j_r = bf16_round(j).astype(np.float64)
    b_r = beta_from_u(four_velocity_f16(beta))
    ref_r = oracle.render(grid, j_r, b_r, views[0])
    assert_parity(img, ref_r, rel=1e-4, what="bf16 decoded inputs")
    ref = oracle.render(grid, j, beta, views[0])
    assert_parity(img, ref, rel=1e-2, what="bf16 vs float32 truth")
    assert abs(img.astype(np.float64).sum() - ref.sum()) <= 1e-3 * ref.sum()
    ctx.unload(vol)


# ------------------------------------------------------ the checked library
def test_checked_library_records_no_violation():
    import paper_2609_09322_gb300 as g
    c = g.Context(0, checked=True)
    try:
        for seed in (1, 3, 6, 7):
            grid, j, beta = random_grid(seed)
            vol = c.load_snapshots(grid, j, beta)
            for t_obs in (-2.0, 4.0, 12.0):
                v = gen.view_from_angles(grid, 10.0 * seed, 30.0 * seed, size=24, c=1.1, t_obs=t_obs)
                img = render_cpu(c, vol, v)
                assert_parity(img, oracle.render(grid, j, beta, v), what="checked")
            c.unload(vol)
        assert c.bounds_violations() == 0
    finally:
        c.close()


# --------------------------------------------------------- error behaviour
def test_invalid_fields_are_rejected(ctx):
    import paper_2609_09322_gb300 as g
    grid, j, beta = random_grid(80, n=(4, 4, 4), M=2)
    bad_j = j.copy()
    bad_j[1, 2, 2, 2] = -1.0
    bad_b = beta.copy()
    bad_b[0, 1, 1, 1] = (0.6, 0.6, 0.6)
    nan_j = j.copy()
    nan_j[0, 0, 0, 0] = np.nan
    for jj, bb in ((bad_j, beta), (j, bad_b), (nan_j, beta)):
        with pytest.raises(g.GbdError) as e:
            ctx.load_snapshots(grid, jj, bb)
        assert e.value.code == g.gbdart.ERR_INVALID
    with pytest.raises(g.GbdError) as e:
        ctx.load_snapshots(gen.Grid(n=(4, 4, 4), dx=(1.0, -1.0, 1.0), n_epochs=2), j, beta)
    assert e.value.code == g.gbdart.ERR_INVALID
    with pytest.raises(g.GbdError) as e:
        ctx.load_snapshots(gen.Grid(n=(4, 4, 4), n_epochs=2, dt=0.0), j, beta)
    assert e.value.code == g.gbdart.ERR_INVALID
    with pytest.raises(g.GbdError) as e:
        ctx.render(12345, gen.view_from_angles(grid, 10.0))
    assert e.value.code == g.gbdart.ERR_NOTFOUND


def test_budget_and_injected_allocation_failure(monkeypatch):
    import paper_2609_09322_gb300 as g
    grid, j, beta = random_grid(81, n=(8, 8, 8), M=2)
    small = g.Context(0, budget_bytes=4096)
    try:
        with pytest.raises(g.GbdError) as e:
            small.load_snapshots(grid, j, beta)
        assert e.value.code == g.gbdart.ERR_BUDGET
    finally:
        small.close()
    monkeypatch.setenv("GBD_FAULT", "alloc:1")
    c = g.Context(0)
    try:
        with pytest.raises(g.GbdError) as e:
            c.load_snapshots(grid, j, beta)
        assert e.value.code == g.gbdart.ERR_NOMEM
        vol = c.load_snapshots(grid, j, beta)   # the second allocation succeeds
        c.unload(vol)
    finally:
        c.close()


# ---------------------------------------------------------------- autotuner
def test_tune_and_relayout_keep_results(ctx):
    """Tuning picks a launch and a layout by timing; neither may change the
    images, and later renders without a launch use the tuned configuration."""
    grid, j, beta = random_grid(90, n=(40, 36, 44), M=6)
    vol = ctx.load_snapshots(grid, j, beta)
    views = [gen.view_from_direction(grid, -d, size=64, c=1.2, t_obs=5.0) for d in gen.fibonacci_directions(6)]
    before = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    before = before.cpu().numpy()
    res = ctx.tune(vol, views, launch=True, layout=True)
    assert res["candidates"] >= 20 and res["ms"] > 0
    assert (res["brick"], res["super_brick"]) == (ctx.volume_info(vol)["brick"], ctx.volume_info(vol)["super_brick"])
    after = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    assert np.array_equal(after.cpu().numpy(), before)
    ctx.relayout(vol, 4, 2, True)
    again = ctx.render_batch(vol, views)
    torch.cuda.synchronize()
    assert np.array_equal(again.cpu().numpy(), before)
    assert_parity(before[2], oracle.render(grid, j, beta, views[2]), what="tuned")
    ctx.unload(vol)


def test_device_inputs_written_by_pending_work(ctx):
    """Fields still being produced by queued GPU work on another stream are
    read only after that work finishes."""
    grid, j, beta = random_grid(91, n=(48, 40, 44), M=3)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        jd = torch.zeros(j.shape, dtype=torch.float32, device="cuda:0")
        bd = torch.zeros(beta.shape, dtype=torch.float32, device="cuda:0")
        torch.cuda._sleep(50_000_000)   # keep the stream busy before the writes land
        jd.copy_(torch.from_numpy(j).pin_memory(), non_blocking=True)
        bd.copy_(torch.from_numpy(beta).pin_memory(), non_blocking=True)
    vol = ctx.load_snapshots(grid, jd, bd)
    ref_vol = ctx.load_snapshots(grid, j, beta)
    v = gen.view_from_angles(grid, 33.0, 21.0, size=32, c=1.0, t_obs=2.0)
    assert np.array_equal(render_cpu(ctx, vol, v), render_cpu(ctx, ref_vol, v))
    ctx.unload(vol)
    ctx.unload(ref_vol)
