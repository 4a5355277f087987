"""Pins of the oracle's exact direct decision function (Sec. III): brute force
against the factored form, the Cauchy-Schwarz bound and its equality case for
noiseless on-grid targets, and phase invariance."""
import numpy as np
import pytest

from oracle import direct, model
from paper_2307_16550_gb300 import scenes


@pytest.mark.parametrize("seed", [1, 7])
def test_brute_equals_factored(seed):
    sc = scenes.tiny_scene(seed)
    Y = model.measurement(sc)
    S = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid).reshape(-1)
    cells = scenes.splitmix64(seed, 50, 24) % np.uint64(sc.grid.ncells)
    cells = np.concatenate([cells.astype(np.int64), [0, sc.grid.ncells - 1, int(np.argmax(S))]])
    B = direct.brute(Y, sc.radar, sc.tx, sc.rx, sc.grid, cells)
    np.testing.assert_allclose(S[cells], B, rtol=0, atol=1e-11 * S.max())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_noiseless_on_grid_peak_value_and_location(seed):
    """Cauchy-Schwarz: |<alpha atom, atom'>| <= |alpha| Ms Mc, with equality at
    the true cell, so S(true) = (Ms Mc)^2 sum_q |alpha_q|^2 is the maximum."""
    sc = scenes.tiny_scene(seed, snr_db=None, on_grid=True)
    Y = model.measurement(sc)
    S = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid).reshape(-1)
    peak = (sc.radar.Ms * sc.radar.Mc) ** 2 * np.sum(np.abs(sc.alpha[0]) ** 2)
    cell = sc.target_cells[0]
    assert S[cell] == pytest.approx(peak, rel=1e-12)
    assert int(np.argmax(S)) == cell
    assert S.max() <= peak * (1 + 1e-12)


def test_cauchy_schwarz_bound_with_noise():
    sc = scenes.tiny_scene(9)
    Y = model.measurement(sc)
    S = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    bound = sum(np.sum(np.abs(Y[q]) ** 2) for q in range(3)) * sc.radar.Ms * sc.radar.Mc
    assert S.max() <= bound


def test_invariant_under_per_rx_phase_rotation():
    sc = scenes.tiny_scene(10)
    Y = model.measurement(sc)
    rot = np.exp(2j * np.pi * np.array([0.3, -0.2, 0.9]))[:, None, None]
    xy = [(0, 0), (13, 21), (31, 31)]
    S0 = direct.factored(Y, sc.radar, sc.tx, sc.rx, sc.grid, xy)
    S1 = direct.factored(Y * rot, sc.radar, sc.tx, sc.rx, sc.grid, xy)
    np.testing.assert_allclose(S1, S0, rtol=1e-10, atol=1e-10 * S0.max())
