"""Edge cases of the CUDA path: argument errors with a live context,
degenerate grids (one cell, one receiver, long velocity axes), the TX on a
grid point, K equal to the number of cells, and the instrumentation calls."""
import ctypes

import numpy as np
import pytest

from oracle import direct, hopping, maps as omaps
from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _scene(Q, n, Ms=32, Mc=16, pad=4, seed=3, lo=(0, 0, -10, -10), hi=(20, 20, 10, 10)):
    radar = scenes.Radar(24e9, 250e6, 128e-6, Ms, Mc, pad)
    grid = scenes.Grid.from_bounds(lo, hi, n)
    return scenes.custom_scene(seed, radar, grid, Q=Q, T=1, snr_db=10.0)


def test_invalid_arguments_with_live_context(ctx, torch_cuda):
    sc = _scene(2, (4, 4, 2, 2))
    Y32, _ = measurement64(sc)
    Yd = to_dev(torch_cuda, Y32)
    maps = ctx.maps(sc.radar, Yd)
    bad_radars = [scenes.Radar(24e9, 250e6, 1e-4, 48, 16, 4), scenes.Radar(24e9, 250e6, 1e-4, 32, 16, 3),
                  scenes.Radar(-1.0, 250e6, 1e-4, 32, 16, 4), scenes.Radar(24e9, 250e6, 1e-4, 2, 16, 4),
                  scenes.Radar(24e9, 250e6, 1e-4, 4096, 16, 4)]
    for r in bad_radars:
        with pytest.raises(gh.GhError) as e:
            ctx.gh_make_maps(r, 2, Yd, maps)
        assert e.value.status == gh.GH_EINVAL
    bad_grid = scenes.Grid((0, 0, 0, 0), (1, 1, 1, 1), (4, 0, 2, 2))
    with pytest.raises(gh.GhError) as e:
        ctx.gh_score_grid(sc.radar, sc.tx, sc.rx, 2, maps, bad_grid)
    assert e.value.status == gh.GH_EINVAL
    neg_step = scenes.Grid((0, 0, 0, 0), (1, -1, 1, 1), (4, 4, 2, 2))
    with pytest.raises(gh.GhError):
        ctx.gh_score_grid(sc.radar, sc.tx, sc.rx, 2, maps, neg_step)
    with pytest.raises(gh.GhError) as e:
        ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, 2, Yd, sc.grid, 0)
    assert e.value.status == gh.GH_EINVAL
    with pytest.raises(gh.GhError):
        ctx.gh_detect(7, sc.radar, sc.tx, sc.rx, 2, Yd, sc.grid, 1)
    with pytest.raises(gh.GhError):
        ctx.gh_score_grid(sc.radar, sc.tx, [np.nan, 0, 1, 1], 2, maps, sc.grid)
    with pytest.raises(gh.GhError):  # host array where device memory is required
        ctx.gh_make_maps(sc.radar, 2, Y32, maps)
    with pytest.raises(gh.GhError):
        ctx.gh_make_maps(sc.radar, 2, Yd, maps, map_dtype=9)
    # the context still works after the errors
    ctx.gh_make_maps(sc.radar, 2, Yd, maps)


@pytest.mark.parametrize("n", [(1, 1, 1, 1), (3, 1, 1, 5), (2, 3, 300, 1), (1, 2, 3, 300), (5, 4, 70, 3)])
def test_degenerate_and_long_axes(ctx, torch_cuda, n):
    sc = _scene(1, n, lo=(2, 3, -14, -14), hi=(25, 22, 14, 14))
    Y32, Y = measurement64(sc)
    ref = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    assert cell == hopping.argmax_cell(ref) or np.isclose(ref.reshape(-1)[cell], ref.max(), rtol=TOL)
    ex = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    got_e, _, _ = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sc.grid)
    assert rel_err(got_e.cpu().numpy(), ex) < TOL


def test_tx_on_a_grid_point(ctx, torch_cuda):
    """The TX sits exactly on a cell centre: its unit vector is taken as zero
    on both sides (the bistatic gradient keeps only the RX term)."""
    sc = _scene(2, (8, 8, 4, 4), lo=(-2.5, -2.5, -10, -10), hi=(2.5, 2.5, 10, 10))
    # cell centres are -2.5 + (i + 1/2) * 0.625: i = 3.5 is not a centre, so move the TX
    sc.tx[:] = [-2.5 + 4.5 * 0.625, -2.5 + 4.5 * 0.625]
    Y32, Y = measurement64(sc)
    ib, tau, coef, w = ctx.gh_coord_table(sc.radar, sc.tx, sc.rx, sc.Q, sc.grid)
    ref = hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)
    np.testing.assert_array_equal(w[..., 0], ref["wx"])
    ref_s = hopping.hop_scores(omaps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    got, _, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, to_dev(torch_cuda, Y32)), sc.grid)
    assert rel_err(got.cpu().numpy(), ref_s) < TOL


def test_k_equals_number_of_cells(ctx, torch_cuda):
    sc = _scene(2, (2, 1, 1, 2))
    Y32, _ = measurement64(sc)
    cells, _, _ = ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, 2, to_dev(torch_cuda, Y32), sc.grid, 4)
    assert sorted(cells.tolist()) == [0, 1, 2, 3]
    with pytest.raises(gh.GhError):
        ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, 2, to_dev(torch_cuda, Y32), sc.grid, 5)


def test_timing_and_launch_counts(ctx, torch_cuda):
    sc = scenes.tiny_scene(1)
    Y32, _ = measurement64(sc)
    Yd = to_dev(torch_cuda, Y32)
    ctx.gh_reset_stats()
    ctx.gh_set_timing(True)
    n0 = ctx.gh_launch_count()
    ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, 2)
    n1 = ctx.gh_launch_count()
    ms, launches = ctx.gh_kernel_stats("hop_score")
    ctx.gh_set_timing(False)
    assert launches == 2 and ms > 0
    # the table once; iteration 0: range FFT, Doppler FFT, scorer, BOMP step
    # (selection, new atom, correlation, least squares); later iterations:
    # the residual's maps by linearity, scorer, BOMP step
    assert n1 - n0 == 1 + 4 + 3
    ms_d, launches_d = ctx.gh_kernel_stats("deflate")
    assert launches_d == 1 and ms_d > 0


@pytest.mark.parametrize("Q,Ms,Mc,pad,n", [
    (64, 16, 8, 4, (3, 4, 2, 3)),      # GH_MAX_Q receivers
    (2, 2048, 8, 4, (3, 2, 2, 2)),     # Nr = 8192 = GH_MAX_NFFT
    (2, 8, 2048, 4, (2, 2, 3, 2)),     # Nd = 8192
    (1, 4, 4, 1, (2, 2, 2, 2)),        # smallest transforms, no padding
    (3, 4096, 4, 2, (2, 2, 2, 2)),     # Ms = GH_MAX_M
])
def test_maximum_and_minimum_sizes(ctx, torch_cuda, Q, Ms, Mc, pad, n):
    radar = scenes.Radar(24e9, 250e6, 128e-6, Ms, Mc, pad)
    grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), n)
    sc = scenes.custom_scene(5, radar, grid, Q=Q, T=1, snr_db=10.0)
    Y32, Y = measurement64(sc)
    Yd = to_dev(torch_cuda, Y32)
    ref = hopping.hop_scores(omaps.rd_maps(Y, pad), sc.radar, sc.tx, sc.rx, sc.grid)
    got, _, _ = ctx.scores(sc.radar, sc.tx, sc.rx, ctx.maps(sc.radar, Yd), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    ex = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    got_e, _, _ = ctx.exact_scores(sc.radar, sc.tx, sc.rx, Yd, sc.grid)
    assert rel_err(got_e.cpu().numpy(), ex) < TOL


def test_sizes_beyond_the_limits_are_rejected(ctx, torch_cuda):
    grid = scenes.Grid.from_bounds((0, 0, -1, -1), (1, 1, 1, 1), (2, 2, 2, 2))
    Y = torch_cuda.zeros((1, 8, 8), dtype=torch_cuda.complex64, device="cuda:0")
    for radar, Q in [(scenes.Radar(24e9, 250e6, 1e-4, 4096, 8, 4), 1),   # Nr = 16384 > GH_MAX_NFFT
                     (scenes.Radar(24e9, 250e6, 1e-4, 8192, 8, 1), 1),   # Ms > GH_MAX_M
                     (scenes.Radar(24e9, 250e6, 1e-4, 2, 8, 4), 1),      # Ms < GH_MIN_M
                     (scenes.Radar(24e9, 250e6, 1e-4, 8, 8, 4), 65)]:    # Q > GH_MAX_Q
        with pytest.raises(gh.GhError) as e:
            ctx.gh_detect(gh.GH_HOP, radar, np.zeros(2), np.zeros((Q, 2)) + 1.0, Q, Y, grid, 1)
        assert e.value.status == gh.GH_EINVAL
