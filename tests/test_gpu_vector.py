"""Vector line-of-sight integration (Sec. 2.1: the traced field may be a
vector): a volume carries extra emissivity channels that share its velocity,
and one march sums every channel with the same weights and Doppler factors
as j' (Eq. 19 per channel).

Eq. 19 is linear in j', so channel c must equal the oracle's render with j'
replaced by that channel; a channel 2 j' must give twice component 0 and a
channel -j' its negative; component 0 must equal the scalar render.
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


def _case(seed, n=(21, 17, 26), M=5):
    rng = np.random.default_rng(seed)
    grid = gen.Grid(n=n, origin=(-1.0, 0.5, 2.0), dx=(1.0, 0.9, 1.1), n_epochs=M, t0=0.0, dt=2.2)
    nx, ny, nz = n
    j = (rng.random((M, nz, ny, nx)) + 0.05).astype(np.float32)
    d = rng.normal(size=(M, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    beta = (d * rng.uniform(0.0, 0.9, size=(M, nz, ny, nx, 1))).astype(np.float32)
    views = [gen.view_from_angles(grid, th, ph, size=36, c=1.3, t_obs=4.4)
             for th, ph in [(40.0, 15.0), (95.0, 220.0), (0.0, 0.0)]]
    return grid, j, beta, views


def test_three_channels_against_the_oracle_and_scaling(ctx):
    grid, j, beta, views = _case(1)
    chans = np.stack([2.0 * j, j * j, -j]).astype(np.float32)
    vol = ctx.load_snapshots(grid, j, beta)
    ctx.load_channels(vol, chans)
    assert ctx.volume_info(vol)["channels"] == 3
    out = ctx.render_vector(vol, views)
    scalar = ctx.render_batch(vol, views, launch={"packet": (8, 4), "cta_warps": 8, "depth": 2, "regcap": 0})
    torch.cuda.synchronize()
    out, scalar = out.cpu().numpy(), scalar.cpu().numpy()
    assert out.shape == (3, 4, 36, 36)
    for k, v in enumerate(views):
        assert_parity(out[k, 0], scalar[k], rel=2e-6, what=f"view {k} component 0 vs scalar render")
        assert_parity(out[k, 1], 2.0 * out[k, 0], rel=1e-6, what=f"view {k} channel 2j'")
        assert_parity(-out[k, 3], out[k, 0], rel=1e-6, what=f"view {k} channel -j'")
        for c, field in enumerate([j, chans[0], chans[1]]):
            assert_parity(out[k, c], oracle.render(grid, field, beta, v), what=f"view {k} component {c} vs oracle")
    neg = oracle.render(grid, chans[2], beta, views[0])
    assert_parity(-out[0, 3], -neg, what="signed channel vs oracle")
    # a re-layout carries the channels along
    ctx.relayout(vol, 4, 2, True, False)
    again = ctx.render_vector(vol, views).cpu().numpy()
    for k in range(len(views)):
        for c in range(4):
            assert_parity(again[k, c], out[k, c], rel=2e-5, what=f"relayout view {k} component {c}")
    ctx.unload(vol)


def test_one_channel_bf16_volume(ctx):
    grid, j, beta, views = _case(2, n=(18, 22, 15), M=4)
    chan = (np.sqrt(j) + 0.1).astype(np.float32)[None]
    vol = ctx.load_snapshots(grid, j, beta, store="bf16")
    ctx.load_channels(vol, chan)
    out = ctx.render_vector(vol, views).cpu().numpy()
    torch.cuda.synchronize()
    # the oracle reads the stored velocity (float16 four-velocity) and the float32 channel
    b_st = beta_from_u(four_velocity_f16(beta))
    for k, v in enumerate(views):
        assert_parity(out[k, 0], oracle.render(grid, bf16_round(j), b_st, v), rel=1e-4, what=f"view {k} bf16 j'")
        assert_parity(out[k, 1], oracle.render(grid, chan[0], b_st, v), rel=1e-4, what=f"view {k} channel")
    ctx.unload(vol)


def test_channel_errors(ctx):
    import paper_2609_09322_gb300 as g
    grid, j, beta, views = _case(3, n=(8, 8, 8), M=2)
    vol = ctx.load_snapshots(grid, j, beta)
    with pytest.raises(g.GbdError):
        ctx.render_vector(vol, views)          # no channels yet
    with pytest.raises(g.GbdError):
        ctx.load_channels(vol, np.stack([j, j]))  # two channels: 1 or 3 only
    bad = np.stack([j]).copy()
    bad[0, 1, 2, 3, 4] = np.nan
    with pytest.raises(g.GbdError):
        ctx.load_channels(vol, bad)
    ctx.unload(vol)
