"""GPU parity of the grid-hopping scorer (gh_score_grid) and its coordinate
mapping (gh_coord_table) against the FP64 oracle, from oracle-made maps and
through the GPU's own maps, on full small grids, ragged grids and sampled
rows of the paper-shaped frame."""
import numpy as np
import pytest

from oracle import hopping, maps as omaps
from paper_2307_16550_gb300 import scenes
from tests.helpers import measurement64, rel_err, to_dev, top2_margin

pytestmark = pytest.mark.gpu

TOL = 1e-4  # max |S_gpu - S_oracle| / max S_oracle, float32 scores


def _ragged():
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((-3, 1, -12, -9), (37, 29, 14, 11), (41, 29, 13, 11))
    return scenes.custom_scene(11, radar, grid, Q=5, T=2, snr_db=5.0, rx_box=((-5, 30), (-4, 2)))


def _oracle_maps_dev(torch, Y, pad):
    return to_dev(torch, omaps.centred_maps(Y, pad).astype(np.complex64))


@pytest.mark.parametrize("make", [lambda: scenes.tiny_scene(1), lambda: scenes.paper_frame(2), _ragged])
def test_coord_table_bit_exact(ctx, make):
    sc = make()
    ib, tau, coef, w = ctx.gh_coord_table(sc.radar, sc.tx, sc.rx, sc.Q, sc.grid)
    ref = hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)
    np.testing.assert_array_equal(ib, ref["i"])
    np.testing.assert_array_equal(tau, ref["tau"])
    np.testing.assert_array_equal(w[..., 0], ref["wx"])
    np.testing.assert_array_equal(w[..., 1], ref["wy"])
    np.testing.assert_allclose(coef, ref["c"], atol=1e-6)  # stored in float32


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_full_grid_from_oracle_maps(ctx, torch_cuda, seed):
    sc = scenes.tiny_scene(seed)
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, score = ctx.scores(sc.radar, sc.tx, sc.rx, _oracle_maps_dev(torch_cuda, Y, 4), sc.grid)
    got = got.cpu().numpy()
    assert rel_err(got, ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)
    assert score == pytest.approx(got.reshape(-1)[cell])


def test_ragged_grid_through_gpu_maps(ctx, torch_cuda):
    sc = _ragged()
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
    got, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, maps, sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_paper_frame_full_grid_bench_launch(ctx, torch_cuda):
    """The paper-shaped frame (128 x 128 x 32 x 32 cells, Q = 4, Ms = 256,
    Mc = 128) in the benchmark's launch configuration: every score and the
    argmax against the oracle's full grid."""
    sc = scenes.paper_frame(1)
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
    got, cell, score = ctx.scores(sc.radar, sc.tx, sc.rx, maps, sc.grid)
    got = got.cpu().numpy()
    assert rel_err(got, ref) < TOL
    assert top2_margin(ref) > 10 * TOL
    assert cell == hopping.argmax_cell(ref)
    assert score == pytest.approx(ref.max(), rel=TOL)


def test_argmax_without_scores_matches(ctx, torch_cuda):
    sc = scenes.tiny_scene(5)
    Y32, _ = measurement64(sc)
    maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
    _, c1, s1 = ctx.scores(sc.radar, sc.tx, sc.rx, maps, sc.grid)
    c2, s2 = ctx.gh_score_grid(sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, None)
    assert (c1, s1) == (c2, s2)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_noiseless_on_grid_target_peaks_on_true_cell(ctx, torch_cuda, seed):
    sc = scenes.tiny_scene(seed, snr_db=None, on_grid=True)
    Y32, _ = measurement64(sc)
    maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
    cell, _ = ctx.gh_score_grid(sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, None)
    assert cell == sc.target_cells[0]


def test_aliased_ranges_wrap_with_centring_sign(ctx, torch_cuda):
    """Ms = 8 makes r exceed one cycle per sample for d > 9.6 m, so range rows
    wrap around the map (several times); the wrapped reads carry the sign of
    the centring phase. Pad 2 and an odd-sized velocity grid."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 8, 16, 2)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (30, 30, 10, 10), (24, 24, 5, 7))
    sc = scenes.custom_scene(4, radar, grid, Q=3, T=2, snr_db=10.0)
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 2), sc.radar, sc.tx, sc.rx, sc.grid)
    table = hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)
    assert table["i"].max() > 2 * 16  # really wraps
    got, _, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL


def _rows_scene(nv):
    """Q = 8, Nd = 1024: the power rows of all receivers take 32 KiB per warp.
    With 16 x 16 velocity cells a lane's cells form one run and the scorer
    builds one receiver's row at a time; with 16 x 40 (nvy > 32) it builds
    all of them."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, 256, 4)
    grid = scenes.Grid((0.0, 0.0, -15.0, -15.0), (5.0, 4.4, 1.875, 1.875), (8, 9) + nv)
    return scenes.custom_scene(31, radar, grid, Q=8, T=2, snr_db=10.0)


def test_one_receiver_row_at_a_time_matches_oracle(ctx, torch_cuda):
    sc = _rows_scene((16, 16))
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_one_row_at_a_time_and_all_rows_agree_bit_for_bit(ctx, torch_cuda):
    """The 16 x 16 velocity cells are the first cells of the 16 x 40 grid with
    the same origin and steps (same bins): the scores of the two row modes
    are equal bit for bit."""
    small, big = _rows_scene((16, 16)), _rows_scene((16, 40))
    Y32, _ = measurement64(small)
    maps = ctx.maps(small.radar, to_dev(torch_cuda, Y32))
    s_small, _, _ = ctx.scores(small.radar, small.tx, small.rx, maps, small.grid)
    s_big, _, _ = ctx.scores(big.radar, big.tx, big.rx, maps, big.grid)
    np.testing.assert_array_equal(s_small.cpu().numpy(), s_big.cpu().numpy()[:, :, :, :16])


@pytest.mark.parametrize("Q,Mc,nv", [(4, 64, (40, 37)), (3, 64, (24, 24)), (8, 256, (40, 40)), (8, 256, (22, 24))])
def test_wide_velocity_axes_match_oracle(ctx, torch_cuda, Q, Mc, nv):
    """Velocity axes of 22..40 cells take the 8 x 4 lane layout (6 or 10 cells
    per run); with Q = 8, Nd = 1024 the scorer also builds one receiver's row
    at a time. Every score against the oracle."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, Mc, 4)
    grid = scenes.Grid.from_bounds((2, 3, -15, -15), (38, 36, 15, 15), (5, 4) + nv)
    sc = scenes.custom_scene(41 + Q, radar, grid, Q=Q, T=2, snr_db=10.0)
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_lane_layouts_agree_bit_for_bit(ctx, torch_cuda):
    """A 24 x 24 velocity grid (8 x 4 lane layout, 6 cells per run) and the
    24 x 32 grid with the same origin and steps (standard layout): equal
    scores on the shared cells, bit for bit."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, 64, 4)
    mk = lambda nvy: scenes.Grid((0.0, 0.0, -15.0, -15.0), (5.0, 4.0, 1.25, 1.25), (6, 7, 24, nvy))
    small = scenes.custom_scene(51, radar, mk(24), Q=4, T=2, snr_db=10.0)
    big = scenes.custom_scene(51, radar, mk(32), Q=4, T=2, snr_db=10.0)
    Y32, _ = measurement64(small)
    maps = ctx.maps(radar, to_dev(torch_cuda, Y32))
    s_small, _, _ = ctx.scores(radar, small.tx, small.rx, maps, small.grid)
    s_big, _, _ = ctx.scores(radar, big.tx, big.rx, maps, big.grid)
    np.testing.assert_array_equal(s_small.cpu().numpy(), s_big.cpu().numpy()[:, :, :, :24])


@pytest.mark.parametrize("nv", [(64, 64), (44, 40), (76, 40), (20, 24)])
def test_paired_scorer_matches_oracle(ctx, torch_cuda, nv):
    """Q = 8, Nd = 1024 with velocity grids whose cells do not fit one
    register run per lane (64 x 64 standard layout, 44 x 40 and 76 x 40 in
    the 8 x 4 layout): all receivers' rows would leave 6 warps per SM, so two
    warps score each (x, y) cell together. 20 x 24 (one run per lane: one
    receiver's row at a time) for contrast. Every score against the oracle."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, 256, 4)
    grid = scenes.Grid.from_bounds((2, 3, -15, -15), (38, 36, 15, 15), (3, 2) + nv)
    sc = scenes.custom_scene(71, radar, grid, Q=8, T=2, snr_db=10.0)
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_paired_and_single_warp_scores_agree_bit_for_bit(ctx, torch_cuda):
    """The 32 x 32 velocity cells of a Q = 8, Nd = 1024 frame are scored by
    two warps per (x, y) cell in gh_score_grid and by one warp per cell in the
    batched scorer kept to all receivers' rows (the batch's argmax at that
    frame's best cell): the single-frame scores' argmax cell and score equal
    the batch's bit for bit."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 256, 4)
    grid = scenes.Grid.from_bounds((2, 3, -15, -15), (38, 36, 15, 15), (6, 5, 32, 32))
    sc = scenes.custom_scene(72, radar, grid, Q=8, T=1, snr_db=15.0)
    Y32, _ = measurement64(sc)
    Yd = to_dev(torch_cuda, Y32)
    got, cell, best = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, Yd), sc.grid)
    ctx.gh_set_batch_row_mode(0)
    try:
        (bcells, bscores, _), = ctx.gh_detect_batch([(sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, 1)])
    finally:
        ctx.gh_set_batch_row_mode(-1)
    assert int(bcells[0]) == cell
    assert np.float32(bscores[0]) == np.float32(best)
    assert np.float32(got.cpu().numpy().reshape(-1)[cell]) == np.float32(best)

