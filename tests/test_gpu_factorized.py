"""GPU parity of the paper's factorised estimators (Eq. 3 then Eq. 4, grid
hopping and direct) and of the indirect method (map peaks, multilateration
as in Eq. 2) against the FP64 oracle: identical 4D cells, location and
velocity values within the float32 tolerance (float64 costs for the indirect
method), and the location scores of the whole (x, y) grid."""
import numpy as np
import pytest

from oracle import factorized as fz
from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _scenes():
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (16, 16, 8, 8))
    return {"tiny": scenes.tiny_scene(2), "paper": scenes.paper_frame(3),
            "ongrid": scenes.custom_scene(2, radar, grid, Q=3, T=1, snr_db=None, on_grid=True),
            "ragged": scenes.custom_scene(7, scenes.Radar(24e9, 250e6, 128e-6, 64, 32, 4),
                                          scenes.Grid.from_bounds((1, 2, -9, -7), (19, 15, 8, 9), (13, 9, 5, 7)),
                                          Q=5, T=1, snr_db=15.0)}


@pytest.mark.parametrize("name", ["tiny", "paper", "ongrid", "ragged"])
@pytest.mark.parametrize("method", ["hop", "exact"])
def test_factorized_matches_oracle(ctx, torch_cuda, name, method):
    sc = _scenes()[name]
    Y32, Y = measurement64(sc)
    L = torch_cuda.empty((sc.grid.n[0], sc.grid.n[1]), dtype=torch_cuda.float32, device="cuda:0")
    cell, (sl, sv) = ctx.gh_factorized(gh.GH_HOP if method == "hop" else gh.GH_EXACT, sc.radar, sc.tx, sc.rx,
                                       sc.Q, to_dev(torch_cuda, Y32), sc.grid, loc_scores=L)
    rcell, rsl, rsv = fz.factorized(Y, sc.radar, sc.tx, sc.rx, sc.grid, method)
    ref_L = (fz.location_scores_hop if method == "hop" else fz.location_scores_direct)(Y, sc.radar, sc.tx, sc.rx,
                                                                                          sc.grid)
    assert np.abs(L.cpu().numpy() - ref_L).max() < TOL * ref_L.max()
    assert cell == rcell
    assert sl == pytest.approx(rsl, rel=TOL)
    assert sv == pytest.approx(rsv, rel=TOL)
    if name == "ongrid":
        assert cell == sc.target_cells[0]


@pytest.mark.parametrize("name", ["tiny", "paper", "ongrid", "ragged"])
def test_indirect_matches_oracle(ctx, torch_cuda, name):
    sc = _scenes()[name]
    Y32, Y = measurement64(sc)
    cell, (lc, vc) = ctx.gh_factorized(gh.GH_INDIRECT, sc.radar, sc.tx, sc.rx, sc.Q, Y32, sc.grid)  # host input
    rcell, rlc, rvc = fz.indirect(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    assert cell == rcell
    assert lc == pytest.approx(rlc, rel=1e-9, abs=1e-15)
    assert vc == pytest.approx(rvc, rel=1e-9, abs=1e-15)
