"""gh_detect_batch: many frames of uneven size in one sequence of batched
launches. Small frames against the FP64 oracle's BOMP frame by frame; larger
batches against the single-frame gh_detect (the same kernels on the same
data, so bit for bit), for every scorer configuration, under graph replay,
and on the uneven 256-frame workload (sampled frames)."""
import numpy as np
import pytest

from oracle import bomp
from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu


def _device_frames(torch, frames, synth_ctx=None):
    """(frames for gh_detect_batch, measurements as complex128)."""
    out, Ys = [], []
    for sc in frames:
        if synth_ctx is None:
            Y32, Y = measurement64(sc)
            Yd = to_dev(torch, Y32)
        else:
            noise = torch.from_numpy(sc.noise.astype(np.complex64)).to("cuda:0")
            Yd = synth_ctx.synth(sc.radar, sc.tx, sc.rx, sc.targets, sc.alpha, noise)
            Y = None
        out.append((sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, sc.K))
        Ys.append(Y)
    return out, Ys


def _single(ctx, f):
    radar, tx, rx, Q, Yd, grid, K = f
    return ctx.gh_detect(gh.GH_HOP, radar, tx, rx, Q, Yd, grid, K)


def _same(a, b):
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])


def test_small_uneven_batch_matches_oracle(ctx, torch_cuda):
    frames = scenes.batch_scenes(2, 6, small=True)
    dev, Ys = _device_frames(torch_cuda, frames)
    res = ctx.gh_detect_batch(dev)
    for sc, Y, (cells, scores, alpha) in zip(frames, Ys, res):
        rc, rs, ra, _ = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, sc.K, "hop")
        np.testing.assert_array_equal(cells, rc)
        np.testing.assert_allclose(scores, rs, rtol=1e-4)
        np.testing.assert_allclose(alpha, ra, rtol=0, atol=1e-4 * np.abs(ra).max())


@pytest.mark.parametrize("tuning", [(0, 0), (8, 2), (16, 4), (32, 4)])
def test_batch_equals_single_frame_detect(ctx, torch_cuda, tuning):
    frames = scenes.batch_scenes(3, 10, small=True) + [scenes.tiny_scene(4), scenes.paper_frame(2)]
    dev, _ = _device_frames(torch_cuda, frames)
    ctx.gh_set_batch_tuning(*tuning)
    try:
        res = ctx.gh_detect_batch(dev)
        used = ctx.gh_batch_tuning()
    finally:
        ctx.gh_set_batch_tuning(0, 0)
    if tuning != (0, 0):
        assert used == tuning
    else:
        assert used[0] in (3, 5, 6, 8, 10, 16, 32) and used[1] in (2, 4, 8)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


@pytest.mark.parametrize("tile", [4, 16, 32])
def test_item_sizes_give_single_frame_results(ctx, torch_cuda, tile):
    """Work items of 4, 16 and 32 (x, y) cells (the tuned default is tried
    among them): the same results as gh_detect, bit for bit."""
    frames = scenes.batch_scenes(5, 8, small=True) + [scenes.tiny_scene(2)]
    dev, _ = _device_frames(torch_cuda, frames)
    ctx.gh_set_batch_tile(tile)
    try:
        res = ctx.gh_detect_batch(dev)
        assert ctx.gh_batch_tile() == tile
    finally:
        ctx.gh_set_batch_tile(0)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


@pytest.mark.parametrize("row_mode", [0, 1, 2])
def test_power_row_modes_give_single_frame_results(ctx, torch_cuda, row_mode):
    """The batched scorer kept to one power-row mode (all receivers' rows, one
    receiver's row at a time where a lane's cells form one run, or all rows
    shared by two warps per (x, y) cell in the 8 x 4 layout's classes): the
    same results as gh_detect, bit for bit, on frames with 16..40 velocities
    per axis."""
    frames = scenes.batch_scenes(7, 12) + [scenes.tiny_scene(3)]
    dev, _ = _device_frames(torch_cuda, frames, synth_ctx=ctx)
    ctx.gh_set_batch_row_mode(row_mode)
    try:
        res = ctx.gh_detect_batch(dev)
        if row_mode == 0:
            assert ctx.gh_batch_row_mode() == 0
        if row_mode == 2:
            assert ctx.gh_batch_row_mode() == 2
    finally:
        ctx.gh_set_batch_row_mode(-1)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


@pytest.mark.parametrize("row_mode", [-1, 0, 1, 2])
def test_uneven_velocity_axes_give_single_frame_results(ctx, torch_cuda, row_mode):
    """Velocity grids with unequal and odd axes (partial runs in the 8 x 4
    lane layout, a lane's vy rows over several one-row passes, runs past the
    vx edge): the same results as gh_detect, bit for bit, in every row mode."""
    shapes = [(22, 24), (40, 37), (24, 7), (37, 40), (13, 40), (40, 9), (6, 24), (31, 17)]
    frames = []
    for i, (nvx, nvy) in enumerate(shapes):
        radar = scenes.Radar(24e9, 250e6, 128e-6, 64 << (i % 3), 32 << (i % 2), 4)
        grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (12 + i, 10 + 2 * i, nvx, nvy))
        frames.append(scenes.custom_scene(60 + i, radar, grid, Q=3 + i % 6, T=1 + i % 3, snr_db=10.0))
    dev, _ = _device_frames(torch_cuda, frames, synth_ctx=ctx)
    ctx.gh_set_batch_row_mode(row_mode)
    try:
        res = ctx.gh_detect_batch(dev)
    finally:
        ctx.gh_set_batch_row_mode(-1)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


def test_paired_scorer_gives_single_frame_results(ctx, torch_cuda):
    """Two warps per (x, y) cell sharing one set of power rows (the 8 x 4
    layout's 24 x 24 and 40 x 40 velocity grids and the standard layout's
    16 x 16, 32 x 32 and 12 x 20, odd and even Q, several Nd, K up to 3 so
    that masked cells are skipped): the same results as gh_detect, bit for
    bit, and the paired scorer is the one that ran."""
    frames = []
    for i, nv in enumerate((24, 40, 40, 24, 40, 16, 32, (12, 20))):
        nv = nv if isinstance(nv, tuple) else (nv, nv)
        radar = scenes.Radar(24e9, 250e6, 128e-6, 64 << (i % 3), 64 << (i % 2), 4)
        grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (10 + 2 * i, 12 + i) + nv)
        frames.append(scenes.custom_scene(90 + i, radar, grid, Q=3 + i % 6, T=1 + i % 3, snr_db=12.0))
    dev, _ = _device_frames(torch_cuda, frames, synth_ctx=ctx)
    ctx.gh_set_batch_row_mode(2)
    try:
        res = ctx.gh_detect_batch(dev)
        assert ctx.gh_batch_row_mode() == 2
        assert ctx.gh_batch_tuning() in ((3, 2), (5, 2), (8, 2), (16, 2))
    finally:
        ctx.gh_set_batch_row_mode(-1)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


def test_batch_graph_replay_follows_data(ctx, torch_cuda):
    frames = scenes.batch_scenes(4, 5, small=True)
    dev, _ = _device_frames(torch_cuda, frames)
    first = ctx.gh_detect_batch(dev)
    for _ in range(3):  # eager, recorded, replayed
        for a, b in zip(ctx.gh_detect_batch(dev), first):
            _same(a, b)
    # new measurements in the same buffers: the replay follows them
    for (radar, tx, rx, Q, Yd, grid, K), sc in zip(dev, frames):
        s2 = scenes.custom_scene(sc.seed + 77, sc.radar, sc.grid, Q=sc.Q, T=sc.K, snr_db=10.0)
        s2.rx[:] = sc.rx
        Y32, _ = measurement64(s2)
        Yd.copy_(to_dev(torch_cuda, Y32))
    res = ctx.gh_detect_batch(dev)
    for f, r in zip(dev, res):
        _same(r, _single(ctx, f))


def test_batch_rejects_bad_frames(ctx, torch_cuda):
    sc = scenes.tiny_scene(1)
    Y32, _ = measurement64(sc)
    with pytest.raises(gh.GhError) as e:
        ctx.gh_detect_batch([(sc.radar, sc.tx, sc.rx, sc.Q, Y32, sc.grid, 1)])  # host measurement
    assert e.value.status == gh.GH_EINVAL
    with pytest.raises(gh.GhError):
        ctx.gh_detect_batch([(sc.radar, sc.tx, sc.rx, sc.Q, to_dev(torch_cuda, Y32), sc.grid, 0)])
    with pytest.raises(gh.GhError):
        ctx.gh_set_batch_tuning(12, 4)
    with pytest.raises(gh.GhError) as e:
        ctx.gh_set_batch_tile(12)
    assert e.value.status == gh.GH_EINVAL
    with pytest.raises(gh.GhError):
        ctx.gh_set_batch_row_mode(3)


def test_uneven_256_frame_workload_sampled(ctx, torch_cuda):
    """The batching workload: 256 frames, Q 3..8, Ms 128..512, Mc 64..256,
    grids 64^2 x 16^2 .. 160^2 x 40^2, 1..5 targets at SNR 0..20 dB. Sampled
    frames against the single-frame path (bit for bit) and the smallest frame
    against the FP64 oracle."""
    torch = torch_cuda
    frames = scenes.batch_scenes(1, 256)
    dev, _ = _device_frames(torch, frames, synth_ctx=ctx)
    res = ctx.gh_detect_batch(dev)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.integers(0, 256, 6).tolist()))
    for i in sample:
        _same(res[i], _single(ctx, dev[i]))
    small = int(np.argmin([f.grid.ncells * f.Q * f.K for f in frames]))
    sc = frames[small]
    Y = dev[small][4].cpu().numpy().astype(np.complex128)
    rc, rs, ra, _ = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, sc.K, "hop")
    np.testing.assert_array_equal(res[small][0], rc)
    np.testing.assert_allclose(res[small][1], rs, rtol=1e-4)
    del dev
    torch.cuda.empty_cache()
