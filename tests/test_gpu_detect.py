"""GPU parity of the BOMP detect-and-deflate loop (gh_detect) against the FP64
oracle: identical selected cells, amplitudes and residual scores."""
import numpy as np
import pytest

from oracle import bomp
from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu


def _check(ctx, torch, sc, Y32, Y, K, method, host=False):
    cells, scores, alpha = ctx.gh_detect(gh.GH_HOP if method == "hop" else gh.GH_EXACT, sc.radar, sc.tx, sc.rx,
                                         sc.Q, Y32 if host else to_dev(torch, Y32), sc.grid, K)
    rc, rs, ra, _ = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, K, method)
    np.testing.assert_array_equal(cells, rc)
    np.testing.assert_allclose(scores, rs, rtol=1e-4)
    np.testing.assert_allclose(alpha, ra, rtol=0, atol=1e-4 * np.abs(ra).max())
    return cells


@pytest.mark.parametrize("method", ["hop", "exact"])
@pytest.mark.parametrize("seed", [1, 2])
def test_tiny_k2(ctx, torch_cuda, method, seed):
    sc = scenes.tiny_scene(seed)
    Y32, Y = measurement64(sc)
    _check(ctx, torch_cuda, sc, Y32, Y, 2, method)


def test_multi_target_noiseless_recovery(ctx, torch_cuda):
    radar = scenes.Radar(24e9, 250e6, 100e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (32, 32, 8, 8))
    sc = scenes.custom_scene(3, radar, grid, Q=3, T=3, snr_db=None, on_grid=True)
    Y32, Y = measurement64(sc)
    for method in ("hop", "exact"):
        cells, _, alpha = ctx.gh_detect(gh.GH_HOP if method == "hop" else gh.GH_EXACT, sc.radar, sc.tx, sc.rx,
                                        sc.Q, to_dev(torch_cuda, Y32), sc.grid, 3)
        assert sorted(cells.tolist()) == sorted(sc.target_cells.tolist())
        order = [list(sc.target_cells).index(c) for c in cells]
        np.testing.assert_allclose(alpha, sc.alpha[order], atol=2e-4)


def test_paper_frame_hop_k3_host_input(ctx, torch_cuda):
    """The benchmark's workload: paper-shaped frame, grid hopping, K = 3,
    measurement passed from host memory."""
    sc = scenes.paper_frame(1)
    Y32, Y = measurement64(sc)
    _check(ctx, torch_cuda, sc, Y32, Y, 3, "hop", host=True)


def test_mid_frame_exact_k3(ctx, torch_cuda):
    radar = scenes.Radar(24e9, 250e6, 128e-6, 128, 64, 4)
    grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (40, 40, 12, 12))
    sc = scenes.custom_scene(5, radar, grid, Q=4, T=3, snr_db=10.0)
    Y32, Y = measurement64(sc)
    _check(ctx, torch_cuda, sc, Y32, Y, 3, "exact")


def _many_targets(seed, Q, T):
    radar = scenes.Radar(24e9, 250e6, 100e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (32, 32, 8, 8))
    return scenes.custom_scene(seed, radar, grid, Q=Q, T=T, snr_db=None, on_grid=True)


@pytest.mark.parametrize("method", ["hop", "exact"])
@pytest.mark.parametrize("seed", [11, 12])
def test_six_targets_least_squares_past_four_atoms(ctx, torch_cuda, method, seed):
    """K = 6 noiseless on-grid targets, 3 receivers: the least squares of 5
    and 6 atoms (the general solve, not the 4-atom register one), staged in
    shared memory. Same cells, scores and amplitudes as the oracle, and the
    true cells and amplitudes."""
    sc = _many_targets(seed, 3, 6)
    Y32, Y = measurement64(sc)
    cells = _check(ctx, torch_cuda, sc, Y32, Y, 6, method)
    assert sorted(cells.tolist()) == sorted(sc.target_cells.tolist())


@pytest.mark.parametrize("seed", [21, 22])
def test_ten_targets_eight_receivers_unstaged_solve(ctx, torch_cuda, seed):
    """K = 10, Q = 8: the Gram matrices no longer fit the staging buffer
    (Q (K^2 + 4K) > 1024 doubles), so the solve reads global memory."""
    sc = _many_targets(seed, 8, 10)
    Y32, Y = measurement64(sc)
    cells = _check(ctx, torch_cuda, sc, Y32, Y, 10, "hop")
    assert sorted(cells.tolist()) == sorted(sc.target_cells.tolist())
    _, _, alpha = ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, to_dev(torch_cuda, Y32), sc.grid, 10)
    order = [list(sc.target_cells).index(c) for c in cells]
    np.testing.assert_allclose(alpha, sc.alpha[order], atol=2e-4)


def test_paper_frame_exact_k3(ctx, torch_cuda):
    """The benchmark's exact workload: paper-shaped frame, exact direct
    decision function (tensor-core stages, stage-1 correlations of the
    residual by linearity), K = 3, measurement in device memory."""
    sc = scenes.paper_frame(1)
    Y32, Y = measurement64(sc)
    cells = _check(ctx, torch_cuda, sc, Y32, Y, 3, "exact")
    assert len(set(cells.tolist())) == 3
