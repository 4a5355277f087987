"""Pins of the oracle's differentiable hopping score (polar interpolation on
both axes) and its analytic gradients: FP64 central differences (step 1e-4 m
and 1e-4 m/s), the exact score of a noiseless target, and the map gradient
as a directional derivative."""
import numpy as np
import pytest

from oracle import hopping, maps, model, smooth
from paper_2307_16550_gb300 import scenes

H = 1e-4


def _scene(seed=3, snr=20.0):
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 32, 4)
    grid = scenes.Grid.from_bounds((0, 0, -10, -10), (20, 20, 10, 10), (8, 8, 4, 4))
    return scenes.custom_scene(seed, radar, grid, Q=3, T=1, snr_db=snr)


def _interior_points(Z, sc, n, seed, margin=0.4):
    """Random points near the target whose tau and sigma stay inside
    (-margin, margin) at every receiver (no bin switch within a few steps)."""
    rng = np.random.default_rng(seed)
    t = sc.targets[0]
    pts = []
    while len(pts) < n:
        p = t + rng.uniform(-1, 1, 4) * np.array([0.5, 0.5, 1.0, 1.0])
        terms = smooth.point_terms(Z, sc.radar, sc.tx, sc.rx, p)
        if all(abs(tt["tau"]) < margin and abs(tt["sigma"]) < margin for tt in terms):
            pts.append(p)
    return np.array(pts)


def test_coefficient_derivatives_by_central_differences():
    th = hopping.polar_angle(256, 1024)
    tau = np.linspace(-0.5, 0.5, 11)
    fd = (hopping.polar_coeffs(tau + 1e-6, th) - hopping.polar_coeffs(tau - 1e-6, th)) / 2e-6
    np.testing.assert_allclose(smooth.polar_coeffs_deriv(tau, th), fd, atol=1e-8)


def test_point_gradient_matches_central_differences():
    sc = _scene()
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, sc.radar.pad)
    pts = _interior_points(Z, sc, 6, seed=1)
    dpt, drx = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, pts)
    for a in range(4):
        e = np.zeros(4)
        e[a] = H
        fd = (smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts + e)[0]
              - smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts - e)[0]) / (2 * H)
        np.testing.assert_allclose(dpt[:, a], fd, rtol=1e-5, atol=1e-6 * np.abs(dpt).max())
    for q in range(sc.Q):
        for a in range(2):
            rp, rm = sc.rx.copy(), sc.rx.copy()
            rp[q, a] += H
            rm[q, a] -= H
            fd = (smooth.smooth_scores(Z, sc.radar, sc.tx, rp, pts)[0]
                  - smooth.smooth_scores(Z, sc.radar, sc.tx, rm, pts)[0]) / (2 * H)
            np.testing.assert_allclose(drx[:, q, a], fd, rtol=1e-5, atol=1e-6 * np.abs(drx).max())


def test_noiseless_target_value_and_stationarity():
    """At a noiseless target the two-axis interpolation reproduces the exact
    score Ms^2 Mc^2 sum|alpha|^2 to the polar model's accuracy, and the score
    is nearly stationary there compared with a point 5 cm / 0.1 m/s away."""
    sc = _scene(seed=5, snr=None)
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, sc.radar.pad)
    t = sc.targets[0]
    S, _ = smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, t[None])
    exact = (sc.radar.Ms * sc.radar.Mc) ** 2 * np.sum(np.abs(sc.alpha[0]) ** 2)
    assert abs(S[0] - exact) < 1e-4 * exact
    off = t + np.array([0.05, 0.05, 0.1, 0.1])
    g_t, _ = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, t[None])
    g_o, _ = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, off[None])
    assert np.linalg.norm(g_t) < 1e-3 * np.linalg.norm(g_o)


def test_two_axis_interpolation_beats_nearest_doppler_bin():
    """Against the exact decision function at random off-grid points, the
    Doppler-interpolated score errs less than the nearest-bin hopping score."""
    sc = _scene(seed=7)
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, sc.radar.pad)
    pts = _interior_points(Z, sc, 8, seed=2, margin=0.5)
    S, _ = smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts)
    ex = np.zeros(len(pts))
    hop = np.zeros(len(pts))
    for p, pt in enumerate(pts):
        for q in range(sc.Q):
            r = model.range_sense(pt[0], pt[1], sc.tx, sc.rx[q], sc.radar)
            u = model.speed_sense(pt[0], pt[1], pt[2], pt[3], sc.tx, sc.rx[q], sc.radar)
            atom = np.outer(model.atom_b(u, sc.radar.Mc), model.atom_a(r, sc.radar.Ms))
            ex[p] += abs(np.sum(Y[q] * np.conj(atom))) ** 2
        terms = smooth.point_terms(Z, sc.radar, sc.tx, sc.rx, pt)
        th = hopping.polar_angle(sc.radar.Ms, Z.shape[2])
        for q, t in enumerate(terms):  # nearest Doppler bin, polar range
            hop[p] += abs(hopping.polar_coeffs(t["tau"], th) @ t["V"][:, 1]) ** 2
    assert np.abs(S - ex).mean() < 0.5 * np.abs(hop - ex).mean()
    assert np.abs(S - ex).max() < 2e-3 * ex.max()


def test_map_gradient_is_the_directional_derivative():
    sc = _scene(seed=9)
    Y = model.measurement(sc)
    Z = maps.rd_maps(Y, sc.radar.pad)
    pts = _interior_points(Z, sc, 3, seed=4)
    g = np.array([1.0, -0.5, 2.0])
    G = smooth.smooth_map_grad(Z, sc.radar, sc.tx, sc.rx, pts, g)
    Q, Nd, Nr = Z.shape
    rng = np.random.default_rng(0)
    E = rng.standard_normal((Q, Nr, Nd)) + 1j * rng.standard_normal((Q, Nr, Nd))  # centred-map direction
    ph = maps.centring_phase(np.arange(Nr), Nr, sc.radar.Ms)
    E_raw = np.transpose(E / ph[None, :, None], (0, 2, 1))  # the same change of the raw maps
    eps = 1e-3
    Lp = g @ smooth.smooth_scores(Z + eps * E_raw, sc.radar, sc.tx, sc.rx, pts)[0]
    Lm = g @ smooth.smooth_scores(Z - eps * E_raw, sc.radar, sc.tx, sc.rx, pts)[0]
    fd = (Lp - Lm) / (2 * eps)
    assert fd == pytest.approx(np.real(np.sum(np.conj(G) * E)), rel=1e-8)
