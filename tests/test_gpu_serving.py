"""Serving: continuous batching of mixed requests against resident volumes.

A request's image must be the same whether it is served alone or in a mix
of other volumes, storages, image sizes and orientations, and the same as
the direct render of its view; requests that arrive while others run must be
admitted as request slots and device memory free up, with several waves on
the GPU at once.  Failure paths are driven from the host only.
"""
import time

import numpy as np
import pytest

import gen
from tests._parity import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _volume(ctx, seed, n, M, store):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=n, origin=(0.0, 0.0, 0.0), dx=(1.0, 1.0, 1.0), n_epochs=M, t0=0.0, dt=3.0)
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, 0.95, size=(M, nz, ny, nx, 1))).astype(np.float32)
    return grid, ctx.load_snapshots(grid, j, beta, store=store)


def _requests(rng, vols, count):
    out = []
    for k in range(count):
        grid, vol = vols[int(rng.integers(len(vols)))]
        size = int(rng.choice([16, 40, 64, 96]))
        d = rng.normal(size=3)
        t_obs = float(rng.uniform(0.0, 3.0 * (grid.n_epochs - 1)))
        out.append((vol, gen.view_from_direction(grid, -d, size=size, c=1.0, t_obs=t_obs,
                                                 beaming=bool(k % 3), lookback=bool(k % 4))))
    return out


@pytest.fixture
def served():
    import paper_2609_09322_gb300 as g
    ctx = g.Context(0)
    vols = [_volume(ctx, 1, (24, 20, 28), 5, "f32"), _volume(ctx, 2, (40, 33, 37), 3, "bf16"),
            _volume(ctx, 3, (16, 16, 16), 8, "f32")]
    yield ctx, vols
    ctx.close()


def test_alone_equals_mix_and_direct_render(served):
    ctx, vols = served
    ctx.serve_start(max_waves=3, max_requests_per_wave=8)
    rng = np.random.default_rng(5)
    reqs = _requests(rng, vols, 40)
    probe_vol, probe_view = reqs[7]
    # alone
    alone = torch.empty((probe_view.height, probe_view.width), device="cuda:0")
    st = ctx.wait(ctx.submit(probe_vol, probe_view, alone), 60000)
    assert st["status"] == 0 and st["latency_ms"] > 0
    # in a mix of 40 requests submitted back to back
    outs, tickets = [], []
    for vol, view in reqs:
        o = torch.empty((view.height, view.width), device="cuda:0")
        outs.append(o)
        tickets.append(ctx.submit(vol, view, o, priority=int(rng.integers(3))))
    for t in tickets:
        ctx.wait(t, 60000)
    torch.cuda.synchronize()
    assert torch.equal(outs[7], alone), "a request differs between alone and in the mix"
    # every request alone, afterwards: the same image bit for bit as in the
    # mix and as the direct render of its view
    for k, ((vol, view), o) in enumerate(zip(reqs, outs)):
        solo = torch.empty_like(o)
        ctx.wait(ctx.submit(vol, view, solo), 60000)
        direct = ctx.render(vol, view)
        torch.cuda.synchronize()
        assert torch.equal(o, solo), f"request {k}: served in the mix differs from served alone"
        assert torch.equal(o, direct), f"request {k}: served differs from the direct render"
    s = ctx.serve_stats()
    assert s["completed"] == 81 and 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["waves"] >= 45


def test_arrivals_overlap_on_the_device(served):
    """Small waves and requests arriving while earlier ones run: the
    scheduler keeps several waves on the GPU at once."""
    ctx, vols = served
    ctx.serve_start(max_waves=3, max_requests_per_wave=2)
    rng = np.random.default_rng(6)
    reqs = _requests(rng, vols, 60)
    tickets, outs = [], []
    for k, (vol, view) in enumerate(reqs):
        o = torch.empty((view.height, view.width), device="cuda:0")
        outs.append(o)
        tickets.append(ctx.submit(vol, view, o))
        if k % 10 == 9:
            time.sleep(0.001)   # arrivals spread in time
    for t in tickets:
        ctx.wait(t, 60000)
    s = ctx.serve_stats(reset=True)
    assert s["completed"] == 60
    assert s["max_waves_in_flight"] >= 2
    assert ctx.serve_stats()["completed"] == 0


def test_memory_admission_and_budget(served):
    """Host-output requests hold their image on the device while they run: a
    budget for two of them admits the rest as memory frees; one larger than
    the whole budget is refused at submission."""
    import paper_2609_09322_gb300 as g
    ctx, vols = served
    grid, vol = vols[0]
    view = gen.view_from_angles(grid, 30.0, 10.0, size=64, c=1.0, t_obs=4.0)
    img_bytes = 64 * 64 * 4
    ctx.serve_start(max_waves=3, request_budget_bytes=2 * img_bytes + 4096)
    hosts = [torch.empty((64, 64), dtype=torch.float32, pin_memory=True) for _ in range(8)]
    tickets = [ctx.submit(vol, view, h) for h in hosts]
    for t in tickets:
        ctx.wait(t, 60000)
    ref = ctx.render(vol, view)
    torch.cuda.synchronize()
    for h in hosts:
        assert torch.equal(h, ref.cpu())
    big = gen.view_from_angles(grid, 30.0, 10.0, size=512, c=1.0, t_obs=4.0)
    with pytest.raises(g.GbdError) as e:
        ctx.submit(vol, big, torch.empty((512, 512), dtype=torch.float32, pin_memory=True))
    assert e.value.code == g.gbdart.ERR_BUDGET
    with pytest.raises(g.GbdError) as e:   # pageable host memory cannot be served
        ctx.submit(vol, view, np.empty((64, 64), dtype=np.float32))
    assert e.value.code == g.gbdart.ERR_INVALID


def test_device_output_is_admitted_by_its_bytes(served):
    """Device-output requests are charged their image at admission: a budget
    of two images keeps at most two of them running at once, and all finish
    with the direct render's image."""
    ctx, vols = served
    grid, vol = vols[2]
    view = gen.view_from_angles(grid, 40.0, 20.0, size=64, c=1.0, t_obs=5.0)
    ctx.serve_start(max_waves=3, max_requests_per_wave=8, request_budget_bytes=2 * 64 * 64 * 4)
    outs = [torch.empty((64, 64), device="cuda:0") for _ in range(12)]
    tickets = [ctx.submit(vol, view, o) for o in outs]
    for t in tickets:
        ctx.wait(t, 60000)
    s = ctx.serve_stats()
    assert s["completed"] == 12 and s["waves"] >= 6 and s["mean_requests_per_wave"] <= 2.0
    ref = ctx.render(vol, view)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)


def test_wait_times_out_and_the_request_still_completes(served):
    """gbd_wait on a request queued behind many one-request waves returns
    GBD_ERR_TIMEOUT after its 1 ms limit; the request stays valid and is
    served afterwards with the direct render's image."""
    import paper_2609_09322_gb300 as g
    ctx, vols = served
    grid, vol = vols[1]
    ctx.serve_start(max_waves=1, max_requests_per_wave=1)
    view = gen.view_from_angles(grid, 25.0, 5.0, size=256, c=1.0, t_obs=3.0)
    outs = [torch.empty((256, 256), device="cuda:0") for _ in range(120)]
    tickets = [ctx.submit(vol, view, o) for o in outs]
    t0 = time.perf_counter()
    with pytest.raises(g.GbdError) as e:
        ctx.wait(tickets[-1], 1)
    waited = time.perf_counter() - t0
    assert e.value.code == g.gbdart.ERR_TIMEOUT and waited < 0.5
    done, _ = ctx.poll(tickets[-1])
    assert not done
    for t in tickets:
        st = ctx.wait(t, 60000)
        assert st["status"] == 0
    ref = ctx.render(vol, view)
    torch.cuda.synchronize()
    assert torch.equal(outs[-1], ref)


def test_cancel_timeout_busy_and_injected_failure(served, monkeypatch):
    import paper_2609_09322_gb300 as g
    ctx, vols = served
    grid, vol = vols[1]
    ctx.serve_start(max_waves=1, max_requests_per_wave=1)
    view = gen.view_from_angles(grid, 20.0, 5.0, size=96, c=1.0, t_obs=3.0)
    outs = [torch.empty((96, 96), device="cuda:0") for _ in range(40)]
    tickets = [ctx.submit(vol, view, o) for o in outs]
    # a volume with queued work cannot go away
    with pytest.raises(g.GbdError) as e:
        ctx.unload(vol)
    assert e.value.code == g.gbdart.ERR_BUSY
    # the last request is still queued behind one-request waves
    ctx.cancel(tickets[-1])
    with pytest.raises(g.GbdError) as e:
        ctx.wait(tickets[-1], 1000)
    assert e.value.code == g.gbdart.ERR_CANCELLED
    for t in tickets[:-1]:
        ctx.wait(t, 60000)
    outs = outs[:3]
    with pytest.raises(g.GbdError) as e:
        ctx.poll(tickets[0])                # a finished request is reported once
    assert e.value.code == g.gbdart.ERR_NOTFOUND
    # an injected admission failure fails exactly that request
    g.gbdart.load_library()  # same library
    monkeypatch.setenv("GBD_FAULT", "admit:2")
    t2 = [ctx.submit(vol, view, o) for o in outs[:3]]
    codes = []
    for t in t2:
        try:
            ctx.wait(t, 60000)
            codes.append(0)
        except g.GbdError as err:
            codes.append(err.code)
    assert codes.count(g.gbdart.ERR_NOMEM) == 1 and codes.count(0) == 2
    ctx.unload(vol)
