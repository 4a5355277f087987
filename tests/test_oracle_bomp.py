"""Pins of the oracle's BOMP loop: exact recovery of noiseless on-grid targets
(cells, amplitudes, zero residual), the least-squares orthogonality of the
residual, and agreement of the hopping and exact variants."""
import numpy as np
import pytest

from oracle import bomp, model
from paper_2307_16550_gb300 import scenes


def _multi_target_tiny(seed, T):
    radar = scenes.Radar(24e9, 250e6, 100e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (32, 32, 8, 8))
    return scenes.custom_scene(seed, radar, grid, Q=3, T=T, snr_db=None, on_grid=True)


@pytest.mark.parametrize("method", ["exact", "hop"])
@pytest.mark.parametrize("seed", [1, 2])
def test_noiseless_on_grid_recovery(method, seed):
    sc = _multi_target_tiny(seed, 2)
    Y = model.measurement(sc)
    cells, scores, alpha, R = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, 2, method)
    assert sorted(cells.tolist()) == sorted(sc.target_cells.tolist())
    order = [list(sc.target_cells).index(c) for c in cells]
    np.testing.assert_allclose(alpha, sc.alpha[order], atol=1e-9)
    assert np.sqrt(np.sum(np.abs(R) ** 2)) < 1e-8 * np.sqrt(np.sum(np.abs(Y) ** 2))


def test_residual_orthogonal_to_support_atoms():
    sc = scenes.tiny_scene(3)
    Y = model.measurement(sc)
    cells, _, _, R = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, 3, "exact")
    for q in range(sc.Q):
        A = bomp.atom_matrix(sc.radar, sc.tx, sc.rx[q], sc.grid, cells)
        g = A.conj().T @ R[q].reshape(-1)
        assert np.abs(g).max() < 1e-9 * np.linalg.norm(Y[q]) * np.sqrt(A.shape[0])


def test_selected_cells_are_distinct_and_scores_decrease_for_noise():
    sc = scenes.tiny_scene(5)
    Y = model.measurement(sc)
    cells, scores, _, _ = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, 3, "hop")
    assert len(set(cells.tolist())) == 3
    assert scores[0] > scores[1]
