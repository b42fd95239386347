"""Out-of-core rendering (gbd_render_streamed): a volume kept in host memory,
uploaded and marched slab by slab along z with only the snapshots each slab's
rays can reach (the paper's partial sub-region renders and selective snapshot
loading, Secs. 5.2 and 6.2).

The slabs' sums must add up to the in-core render of the whole volume (to
float32 rounding: each slab restarts the ray's anchor), and to the oracle at
the FP32 1e-5 bound; flexload must upload fewer bytes than the series holds
when the views' light-cone slices leave snapshots unread, and every byte
without it.
"""
import numpy as np
import pytest

import gen
import oracle
from tests._parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


def _case(seed, n, M, dt, c, lookback=True, beaming=True, size=40, count=5):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=n, origin=(-1.0, 2.0, -3.0), dx=(1.0, 1.1, 0.9), n_epochs=M, t0=0.5, dt=dt)
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) * rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, 0.9, size=(M, nz, ny, nx, 1))).astype(np.float32)
    dirs = list(gen.fibonacci_directions(count - 1)) + [np.array([0.0, 0.0, 1.0])]
    views = []
    for k, dv in enumerate(dirs):
        t_obs = float(grid.t0 + rng.uniform(0.3, 0.7) * dt * (M - 1))
        views.append(gen.view_from_direction(grid, dv, size=size, c=c, t_obs=t_obs, lookback=lookback,
                                             beaming=beaming))
    return grid, j, beta, views


@pytest.mark.parametrize("slab", [7, 16, 64])
def test_streamed_equals_in_core(ctx, slab):
    grid, j, beta, views = _case(1, (30, 26, 45), 12, 2.0, 1.4)
    vol = ctx.load_snapshots(grid, j, beta)
    ref = ctx.render_batch(vol, views)
    got, info = ctx.render_streamed(grid, j, beta, views, slab=slab)
    torch.cuda.synchronize()
    ref, got = ref.cpu().numpy(), got.cpu().numpy()
    assert info["slabs"] <= -(-45 // slab)
    for k in range(len(views)):
        assert_parity(got[k], oracle.render(grid, j, beta, views[k]), what=f"slab {slab} view {k} vs oracle")
        assert_parity(got[k], ref[k], rel=2e-5, what=f"slab {slab} view {k} vs in-core")
    ctx.unload(vol)


def test_flexload_uploads_only_reachable_snapshots(ctx):
    """Light crosses the whole box in a few snapshot intervals here, so each
    slab needs a few of the 40 snapshots: flexload uploads a fraction, and
    without it every byte goes up; both give the same images."""
    grid, j, beta, views = _case(2, (24, 24, 60), 40, 1.0, 4.0, count=3)
    views = [v.with_(t_obs=float(grid.t0 + 20.0)) for v in views]
    flex, fi = ctx.render_streamed(grid, j, beta, views, slab=12, flexload=True)
    full, ni = ctx.render_streamed(grid, j, beta, views, slab=12, flexload=False)
    torch.cuda.synchronize()
    assert ni["bytes_uploaded"] == ni["bytes_total"]
    assert fi["bytes_uploaded"] < 0.6 * fi["bytes_total"]
    flex, full = flex.cpu().numpy(), full.cpu().numpy()
    for k in range(len(views)):
        assert_parity(flex[k], full[k], rel=2e-5, what=f"flexload view {k}")
        assert_parity(flex[k], oracle.render(grid, j, beta, views[k]), what=f"flexload view {k} vs oracle")


def test_streamed_fast_light_and_bf16(ctx):
    grid, j, beta, views = _case(3, (20, 33, 28), 5, 3.0, 1.0, lookback=False, count=4)
    # one observer time between snapshots 0 and 1
    views = [v.with_(t_obs=float(grid.t0 + 0.4 * grid.dt)) for v in views]
    got, info = ctx.render_streamed(grid, j, beta, views, slab=9)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    for k in range(len(views)):
        assert_parity(got[k], oracle.render(grid, j, beta, views[k]), what=f"fast light view {k}")
    # without lookback each slab reads the pair (0, 1), kept with one snapshot of margin: 3 of 5
    assert info["bytes_uploaded"] == info["bytes_total"] * 3 // 5
    vol = ctx.load_snapshots(grid, j, beta, store="bf16")
    ref = ctx.render_batch(vol, views).cpu().numpy()
    bf, _ = ctx.render_streamed(grid, j, beta, views, slab=9, store="bf16")
    torch.cuda.synchronize()
    for k in range(len(views)):
        assert_parity(bf.cpu().numpy()[k], ref[k], rel=2e-5, what=f"bf16 streamed view {k}")
    ctx.unload(vol)


def test_streamed_budget_and_arguments():
    import paper_2609_09322_gb300 as g
    grid, j, beta, views = _case(4, (16, 16, 16), 3, 1.0, 1.0, count=2)
    small = g.Context(0, budget_bytes=64 * 1024)
    with pytest.raises(g.GbdError) as e:
        small.render_streamed(grid, j, beta, views, slab=16)
    assert e.value.code == g.gbdart.ERR_BUDGET
    small.close()
    c = g.Context(0)
    with pytest.raises(g.GbdError):
        c.render_streamed(grid, j, beta, views, slab=-1)
    c.close()
