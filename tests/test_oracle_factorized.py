"""Pins of the oracle's factorised estimators (Eqs. 2-4): closed-form peak
values of a noiseless on-grid target, recovery of its cell by all three
methods, the Doppler DFT of g_q against numpy's FFT, grid hopping close to
the direct location score, and the multilateration recovering a cell from
its own exact range and speed values."""
import numpy as np

from oracle import factorized as fz
from oracle import maps, model
from paper_2307_16550_gb300 import scenes


def _scene(seed=2, snr=None):
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (16, 16, 8, 8))
    return scenes.custom_scene(seed, radar, grid, Q=3, T=1, snr_db=snr, on_grid=True)


def test_noiseless_on_grid_target_closed_forms_and_recovery():
    sc = _scene()
    Y = model.measurement(sc)
    al2 = np.sum(np.abs(sc.alpha[0]) ** 2)
    Ms, Mc = sc.radar.Ms, sc.radar.Mc
    cell, sl, sv = fz.factorized(Y, sc.radar, sc.tx, sc.rx, sc.grid, "exact")
    assert cell == sc.target_cells[0]
    # Eq. 3 at the true location: every chirp correlates fully, |<Y[mc], a>| = |alpha| Ms
    assert abs(sl - Mc * Ms ** 2 * al2) < 1e-9 * sl
    # Eq. 4 at the true velocity: g = alpha Ms b(u), |<g, b(u)>| = |alpha| Ms Mc
    assert abs(sv - (Ms * Mc) ** 2 * al2) < 1e-9 * sv
    cell_h, _, _ = fz.factorized(Y, sc.radar, sc.tx, sc.rx, sc.grid, "hop")
    assert cell_h == sc.target_cells[0]
    cell_i, lc, vc = fz.indirect(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    # the map peaks sit on the FFT grid: the indirect cell is the true one or a neighbour
    t = np.array(sc.grid.unravel(sc.target_cells[0]))
    assert np.abs(np.array(sc.grid.unravel(cell_i)) - t).max() <= 1
    assert lc >= 0 and vc >= 0


def test_cauchy_schwarz_bound_of_the_location_score():
    sc = _scene(seed=4, snr=5.0)
    Y = model.measurement(sc)
    L = fz.location_scores_direct(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    assert L.max() <= sc.radar.Ms * np.sum(np.abs(Y) ** 2) * (1 + 1e-12)


def test_hop_location_close_to_direct():
    sc = _scene(seed=6, snr=10.0)
    Y = model.measurement(sc)
    Ld = fz.location_scores_direct(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    Lh = fz.location_scores_hop(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    assert np.abs(Lh - Ld).max() < 1e-3 * Ld.max()


def test_doppler_dft_of_g_matches_numpy_fft():
    sc = _scene(seed=8, snr=10.0)
    Y = model.measurement(sc)
    t = sc.targets[0]
    g = fz.g_vectors(Y, sc.radar, sc.tx, sc.rx, t[0], t[1])
    Nd = sc.radar.pad * sc.radar.Mc
    G = g @ maps.dft_matrix(Nd, sc.radar.Mc).T
    np.testing.assert_allclose(G, np.fft.fft(g, Nd, axis=1), rtol=0, atol=1e-9 * np.abs(G).max())


def test_rd_peaks_match_numpy_fft2():
    sc = _scene(seed=9, snr=10.0)
    Y = model.measurement(sc)
    pk = fz.rd_peaks(Y, 4)
    for q in range(sc.Q):
        A = np.abs(np.fft.fft2(Y[q], s=(4 * sc.radar.Mc, 4 * sc.radar.Ms)))  # (Nd, Nr)
        j, i = np.unravel_index(np.argmax(A), A.shape)
        assert pk[q] == (i, j)


def test_multilateration_recovers_a_cell_from_its_exact_values(monkeypatch):
    sc = _scene(seed=3)
    X, Yg, VX, VY = model.grid_axes(sc.grid)
    ix, iy, ivx, ivy = 5, 11, 2, 6
    Nr, Nd = 4 * sc.radar.Ms, 4 * sc.radar.Mc
    r = [model.range_sense(X[ix], Yg[iy], sc.tx, sc.rx[q], sc.radar) for q in range(sc.Q)]
    u = [model.speed_sense(X[ix], Yg[iy], VX[ivx], VY[ivy], sc.tx, sc.rx[q], sc.radar) for q in range(sc.Q)]
    # peaks that encode the exact values when Nr r and Nd u are read back (no rounding: big N)
    monkeypatch.setattr(fz, "rd_peaks", lambda Y, pad: [(r[q] * Nr, (u[q] % 1.0) * Nd) for q in range(sc.Q)])
    cell, lc, vc = fz.indirect(None, sc.radar, sc.tx, sc.rx, sc.grid)
    assert cell == sc.grid.cell_index(ix, iy, ivx, ivy)
    assert lc < 1e-20 and vc < 1e-20


def _loc_brute(Y, radar, table, ix, iy, coeffs=None):
    """sum_q sum_mc |sum_k c_k <Y_q[mc], a~(n_k / Nr)>|^2 at (ix, iy), with the
    centred atom a~_m(f) = exp(j 2 pi f (m - (Ms-1)/2)) taken at the unwrapped
    bin n_k = i_q + k (no FFT, no folding of n into [0, Nr))."""
    Q = Y.shape[0]
    Ms = radar.Ms
    Nr = radar.pad * Ms
    m = np.arange(Ms) - (Ms - 1) / 2.0
    c_all = table["c"] if coeffs is None else coeffs
    tot = 0.0
    for q in range(Q):
        s = np.zeros(Y.shape[1], np.complex128)
        for kk, k in enumerate((-1, 0, 1)):
            n = int(table["i"][ix, iy, q]) + k
            s += c_all[ix, iy, q, kk] * (Y[q] @ np.conj(np.exp(2j * np.pi * (n / Nr) * m)))
        tot += np.sum(np.abs(s) ** 2)
    return tot


def test_hop_location_wrapped_reads_forced_bins():
    """Bins forced to i = 0 and i = Nr - 1 make the stencil read n = -1 and
    n = Nr; with unit coefficients each read, and with pairs of unit
    coefficients the sum of a wrapped and an unwrapped read (where the
    centring sign of the wrap shows in |.|^2), must equal the chirps'
    correlations with the centred atoms at the unwrapped bins."""
    from oracle import hopping
    sc = _scene(seed=5, snr=10.0)
    Y = model.measurement(sc)
    table = hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)
    Nr = sc.radar.pad * sc.radar.Ms
    table["i"][0, 0, :] = 0
    table["i"][0, 1, :] = Nr - 1
    table["i"][3, 2, 1] = 2 * Nr - 1  # two periods up
    for pick in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (0, 1, 1), (1, -0.5, 1)):
        coeffs = np.zeros_like(table["c"])
        coeffs[...] = pick
        t = dict(table, c=coeffs)
        L = fz.location_scores_hop(Y, sc.radar, sc.tx, sc.rx, sc.grid, table=t)
        for ix, iy in [(0, 0), (0, 1), (3, 2), (7, 9)]:
            ref = _loc_brute(Y, sc.radar, t, ix, iy)
            assert abs(L[ix, iy] - ref) < 1e-9 * ref


def test_hop_location_aliased_ranges_against_brute_force():
    """Ms = 8 makes every bistatic range wrap around the map several times:
    the whole location grid with the polar coefficients against the brute
    force at the unwrapped bins."""
    from oracle import hopping
    for Ms in (8, 16):
        radar = scenes.Radar(24e9, 250e6, 128e-6, Ms, 16, 2)
        grid = scenes.Grid.from_bounds((0, 0, -10, -10), (30, 30, 10, 10), (12, 10, 4, 4))
        sc = scenes.custom_scene(4, radar, grid, Q=3, T=2, snr_db=10.0)
        Y = model.measurement(sc)
        table = hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)
        assert table["i"].max() > 2 * radar.pad * Ms  # really wraps
        L = fz.location_scores_hop(Y, sc.radar, sc.tx, sc.rx, sc.grid)
        ref = np.array([[_loc_brute(Y, radar, table, ix, iy) for iy in range(10)] for ix in range(12)])
        np.testing.assert_allclose(L, ref, rtol=1e-10)
