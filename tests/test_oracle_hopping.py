"""Pins of the oracle's hopping scorer (Sec. IV, Eq. 5): closed-form Dirichlet
kernels, exactness at integer offsets, brute-force correlations at bins
(including wrapped range indices), phase invariance and on-grid recovery."""
import numpy as np
import pytest

from oracle import direct, hopping, maps, model
from paper_2307_16550_gb300 import scenes


def test_dirichlet_closed_form():
    f = np.array([1e-3, 0.01, 0.123, 0.37, 0.5])
    for M in (16, 64, 257):
        np.testing.assert_allclose(hopping.dirichlet(f, M),
                                   np.sin(np.pi * M * f) / np.sin(np.pi * f), rtol=1e-11, atol=1e-10)
    assert hopping.dirichlet(0.0, 64) == pytest.approx(64.0)


def test_polar_coefficients_special_points():
    th = hopping.polar_angle(256, 1024)
    np.testing.assert_allclose(hopping.polar_coeffs(0.0, th), [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(hopping.polar_coeffs(1.0, th), [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(hopping.polar_coeffs(-1.0, th), [1, 0, 0], atol=1e-15)
    taus = np.linspace(-0.5, 0.5, 101)
    c = hopping.polar_coeffs(taus, th)
    np.testing.assert_allclose(c.sum(axis=1), 1.0, atol=1e-14)
    # mirror symmetry: c_k(-tau) = c_{-k}(tau)
    np.testing.assert_allclose(hopping.polar_coeffs(-taus, th), c[:, ::-1], atol=1e-15)


@pytest.mark.parametrize("Ms", [64, 256])
def test_polar_angle_from_atom_geometry(Ms):
    """2 cos(theta/2) = |p(+1) - p(-1)| / |p(+1) - p(0)| for the explicit
    centred atom vectors of bins -1, 0, +1."""
    Nr = 4 * Ms
    m = np.arange(Ms) - (Ms - 1) / 2
    p = {k: np.exp(2j * np.pi * (k / Nr) * m) for k in (-1, 0, 1)}
    ratio = np.linalg.norm(p[1] - p[-1]) / np.linalg.norm(p[1] - p[0])
    assert 2 * np.cos(hopping.polar_angle(Ms, Nr) / 2) == pytest.approx(ratio, rel=1e-12)


@pytest.mark.parametrize("Ms", [64, 256, 512])
def test_polar_interpolation_error_vs_closed_form(Ms):
    """A pure centred tone at r1 correlated with a~(r) is exactly D(r1 - r).

    * On the tone (r = r1, tau swept over [-1/2, 1/2]) the polar estimate of
      |<y, a~(r)>| is within 2e-5 Ms of Ms; linear interpolation misses by
      more than 1e-2 Ms.
    * Off the tone (r1 up to 3 bins away) the error never exceeds the
      Cauchy-Schwarz bound ||y|| ||a~(r) - sum_k c_k a~(r_k)||, and the atom
      error itself stays below 5e-3 ||a~|| (linear: above 3e-2)."""
    Nr = 4 * Ms
    th = hopping.polar_angle(Ms, Nr)
    m = np.arange(Ms) - (Ms - 1) / 2
    taus = np.linspace(-0.5, 0.5, 41)
    on_p = np.abs(np.abs((hopping.polar_coeffs(taus, th) *
                          hopping.dirichlet((taus[:, None] - np.array([-1, 0, 1])) / Nr, Ms)).sum(1)) - Ms)
    on_l = np.abs(np.abs((hopping.linear_coeffs(taus) *
                          hopping.dirichlet((taus[:, None] - np.array([-1, 0, 1])) / Nr, Ms)).sum(1)) - Ms)
    assert on_p.max() < 2e-5 * Ms
    assert on_l.max() > 1e-2 * Ms
    atom_p = atom_l = 0.0
    for tau in taus:
        exact_atom = np.exp(2j * np.pi * (tau / Nr) * m)
        bins_atoms = [np.exp(2j * np.pi * (k / Nr) * m) for k in (-1, 0, 1)]
        ep = np.linalg.norm(exact_atom - sum(c * a for c, a in zip(hopping.polar_coeffs(tau, th), bins_atoms)))
        el = np.linalg.norm(exact_atom - sum(c * a for c, a in zip(hopping.linear_coeffs(tau), bins_atoms)))
        atom_p, atom_l = max(atom_p, ep), max(atom_l, el)
        for off in np.linspace(-3, 3, 13):
            exact = hopping.dirichlet((off - tau) / Nr, Ms)
            bins = hopping.dirichlet((off - np.array([-1, 0, 1])) / Nr, Ms)
            est = (hopping.polar_coeffs(tau, th) * bins).sum()
            assert abs(est - exact) <= ep * np.sqrt(Ms) * (1 + 1e-9) + 1e-9
    assert atom_p < 5e-3 * np.sqrt(Ms)
    assert atom_l > 3e-2 * np.sqrt(Ms)


def _table_for(sc):
    return hopping.coord_table(sc.radar, sc.tx, sc.rx, sc.grid)


def test_hop_at_integer_offset_is_bin_correlation():
    """With coefficients (0,1,0), (1,0,0), (0,0,1) the hopping value is the
    exact correlation <Y, b(j/Nd) (x) a~(n/Nr)> at the unwrapped bin n,
    including n = -1 and n = Nr (wrapped range reads)."""
    sc = scenes.tiny_scene(2)
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, 4)
    table = _table_for(sc)
    Nr, Nd, Ms, Mc = 4 * 64, 4 * 32, 64, 32
    table["i"][0, 0, :] = 0          # force a read of bin -1
    table["i"][0, 1, :] = Nr - 1     # force a read of bin Nr
    _, _, VX, VY = model.grid_axes(sc.grid)
    m = np.arange(Ms) - (Ms - 1) / 2
    for kk, k in enumerate((-1, 0, 1)):
        coeffs = np.zeros_like(table["c"])
        coeffs[..., kk] = 1.0
        s = hopping.hop_correlations(Z, sc.radar, sc.tx, sc.rx, sc.grid,
                                     np.array([0, 0, 5]), np.array([0, 1, 7]), table, coeffs)
        for n_xy, (ix, iy) in enumerate([(0, 0), (0, 1), (5, 7)]):
            for q in range(3):
                for ivx, ivy in [(0, 0), (3, 6), (7, 7)]:
                    j = hopping.doppler_bin(table["wx"][ix, iy, q], table["wy"][ix, iy, q],
                                            VX[ivx], VY[ivy], sc.radar)
                    n = table["i"][ix, iy, q] + k
                    atom = np.outer(np.exp(2j * np.pi * (j / Nd) * np.arange(Mc)),
                                    np.exp(2j * np.pi * (n / Nr) * m))
                    ref = np.vdot(atom, Y[q])
                    assert abs(s[n_xy, q, ivx, ivy] - ref) < 1e-9 * max(1.0, abs(ref))


def test_hop_scores_invariant_under_rx_phase_rotation():
    sc = scenes.tiny_scene(4)
    Y = model.measurement(sc)
    rot = np.exp(2j * np.pi * np.array([0.1, 0.77, 0.4]))[:, None, None]
    H0 = hopping.hop_scores(maps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid, xy_rows=[3, 17])
    H1 = hopping.hop_scores(maps.rd_maps(Y * rot, 4), sc.radar, sc.tx, sc.rx, sc.grid, xy_rows=[3, 17])
    np.testing.assert_allclose(H1, H0, rtol=1e-10, atol=1e-9 * H0.max())


@pytest.mark.parametrize("seed", [1, 2, 3, 5])
def test_hop_noiseless_on_grid_target_peaks_on_true_cell(seed):
    sc = scenes.tiny_scene(seed, snr_db=None, on_grid=True)
    Y = model.measurement(sc)
    H = hopping.hop_scores(maps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    assert hopping.argmax_cell(H) == sc.target_cells[0]


def test_hop_approximates_exact_score():
    """Hopping tracks the exact decision function: at most the nearest-bin
    Doppler loss (4x padding: sinc^2(1/8) ~ 0.95) below it, never above it by
    more than the polar error."""
    sc = scenes.tiny_scene(6, snr_db=None, on_grid=True)
    Y = model.measurement(sc)
    H = hopping.hop_scores(maps.rd_maps(Y, 4), sc.radar, sc.tx, sc.rx, sc.grid)
    S = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    cell = sc.target_cells[0]
    ratio = H.reshape(-1)[cell] / S.reshape(-1)[cell]
    assert 0.9 < ratio <= 1.0 + 1e-4
    assert np.abs(H - S).max() < 0.15 * S.max()


def test_argmax_ties_take_smallest_index():
    s = np.zeros((2, 2, 2, 2))
    s.reshape(-1)[[5, 9, 3]] = 7.0
    assert hopping.argmax_cell(s) == 3


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_quantization_bound_covers_stored_maps(kind):
    """Hopping scores from maps stored in a reduced-precision format stay
    within the per-cell bound, which is not vacuous."""
    sc = scenes.tiny_scene(4)
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, sc.radar.pad)
    s = maps.map_scale_log2(sc.radar.Ms, sc.radar.Mc)
    # the stored maps are the centred ones; quantize those, then undo the centring
    Nr = Z.shape[2]
    ph = maps.centring_phase(np.arange(Nr), Nr, sc.radar.Ms)
    Zq = maps.quantize_maps(Z * ph[None, None, :], kind, s) / ph[None, None, :]
    ref = hopping.hop_scores(Z, sc.radar, sc.tx, sc.rx, sc.grid)
    got = hopping.hop_scores(Zq, sc.radar, sc.tx, sc.rx, sc.grid)
    bound = hopping.hop_quantization_bound(Z, sc.radar, sc.tx, sc.rx, sc.grid, kind)
    slack = 1e-9 * ref.max()  # float64 rounding of the centring round trip
    assert np.all(np.abs(got - ref) <= bound + slack)
    ratio = np.abs(got - ref).max() / bound.max()
    assert 1e-3 < ratio <= 1.0
    u = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}[kind]
    assert bound.max() / ref.max() < 8 * u  # a few units of the format's rounding
