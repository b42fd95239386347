"""The memory-analysis march (gbd_touched_records): the distinct (cell,
snapshot) records a batch render reads, the compulsory floor of its traffic.

Closed form: a view along -z with one pixel per cell column (pixel centres on
cell centres) crosses every cell once; without lookback it reads one snapshot
when t_obs falls on a snapshot and two in between.  A second view adds no new
records when it crosses the same cells at the same snapshots, and the count
never exceeds two records per cell-sample.
"""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2609_09322_gb300 as g
    c = g.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("paired", [False, True])
def test_axis_aligned_view_reads_every_cell_once(ctx, paired):
    n = (12, 10, 7)
    grid = gen.Grid(n=n, origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=4, t0=0.0, dt=1.0)
    rng = np.random.default_rng(1)
    M, (nx, ny, nz) = grid.n_epochs, n
    j = rng.random((M, nz, ny, nx)).astype(np.float32) + 0.1
    beta = np.zeros((M, nz, ny, nx, 3), np.float32)
    vol = ctx.load_snapshots(grid, j, beta, brick=4, super_brick=2, paired=paired)
    base = gen.View(dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), center=grid.center, width=nx, height=ny,
                    fov_u=float(nx), fov_v=float(ny), lookback=False, beaming=False)
    cells = nx * ny * nz
    assert ctx.touched_records(vol, [base.with_(t_obs=2.0)]) == cells          # on snapshot 2
    assert ctx.touched_records(vol, [base.with_(t_obs=1.5)]) == 2 * cells      # between 1 and 2
    # the same cells and snapshots seen twice are counted once
    assert ctx.touched_records(vol, [base.with_(t_obs=1.5), base.with_(t_obs=1.25)]) == 2 * cells
    # another snapshot pair adds its records
    assert ctx.touched_records(vol, [base.with_(t_obs=1.5), base.with_(t_obs=2.5)]) == 3 * cells
    ctx.unload(vol)


def test_large_batch_covers_every_tile(ctx):
    """Many views of many packets (more than one wave of CTAs): the same
    axis-aligned closed form, each view at its own snapshot."""
    n = (64, 48, 20)
    grid = gen.Grid(n=n, origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=40, t0=0.0, dt=1.0)
    M, (nx, ny, nz) = grid.n_epochs, n
    j = np.ones((M, nz, ny, nx), np.float32)
    beta = np.zeros((M, nz, ny, nx, 3), np.float32)
    vol = ctx.load_snapshots(grid, j, beta)
    base = gen.View(dir=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), center=grid.center, width=nx, height=ny,
                    fov_u=float(nx), fov_v=float(ny), lookback=False, beaming=False)
    views = [base.with_(t_obs=float(m)) for m in range(0, 40, 2)]  # 20 views, 20 distinct snapshots
    assert ctx.touched_records(vol, views) == 20 * nx * ny * nz
    ctx.unload(vol)


def test_bounded_by_two_records_per_sample(ctx):
    grid, j, beta, views = gen.config_tiny()
    vol = ctx.load_snapshots(grid, j, beta)
    _, cnt = ctx.render_batch(vol, views, samples=True)
    torch.cuda.synchronize()
    samples = int(cnt.to(torch.int64).sum().item())
    touched = ctx.touched_records(vol, views)
    assert 0 < touched <= 2 * samples
    assert touched <= int(np.prod(grid.n)) * grid.n_epochs
    ctx.unload(vol)
