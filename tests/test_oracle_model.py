"""Pins of the oracle's signal model (Sec. II, Eq. 1, Eq. general-model)
against physics and closed forms that do not reuse the oracle's formulas."""
import json
import os

import numpy as np
import pytest

from oracle import model
from paper_2307_16550_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C = 299_792_458.0


def _wrap(cycles):
    return (np.asarray(cycles) + 0.5) % 1.0 - 0.5


def _dechirped(radar, tx, rxq, x0, v, n_chirps=2, n_samp=4):
    """IQ output of a dechirp receiver from the chirp's definition.

    The TX sends phi(t') = 2 pi (f0 t' + B/(2 Tc) t'^2) in every chirp; the
    echo reaching RX q is delayed by tau(t) = d(t)/c where d is the bistatic
    path of the moving target at absolute time t; the mixer output is
    exp(j (phi(t') - phi(t' - tau))). Sampled at t = mc Tc + m Tc/Ms."""
    S = radar.B / radar.Tc
    out = np.zeros((n_chirps, n_samp), complex)
    for mc in range(n_chirps):
        for m in range(n_samp):
            tp = m * radar.Tc / radar.Ms
            t = mc * radar.Tc + tp
            p = np.asarray(x0) + np.asarray(v) * t
            d = np.hypot(*(p - tx)) + np.hypot(*(p - rxq))
            tau = d / C
            phase = 2 * np.pi * (radar.f0 * tau + S * tau * tp - 0.5 * S * tau * tau)
            out[mc, m] = np.exp(1j * phase)
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sensing_functions_match_dechirp_physics(seed):
    """Phase step per sample is 2 pi r_q and per chirp 2 pi u_q (mod 2 pi), up
    to the range-Doppler coupling terms that the model of Sec. II neglects."""
    sc = scenes.paper_frame(seed)
    radar = sc.radar
    for q in range(sc.Q):
        for (x, y, vx, vy) in sc.targets:
            s = _dechirped(radar, sc.tx, sc.rx[q], (x, y), (vx, vy))
            per_sample = np.angle(s[0, 1] / s[0, 0]) / (2 * np.pi)
            per_chirp = np.angle(s[1, 0] / s[0, 0]) / (2 * np.pi)
            r = model.range_sense(x, y, sc.tx, sc.rx[q], radar)
            u = model.speed_sense(x, y, vx, vy, sc.tx, sc.rx[q], radar)
            assert abs(_wrap(per_sample - r)) < 5e-3
            assert abs(_wrap(per_chirp - u)) < 1e-2
            # a factor-2 slip in either scale would be far outside the tolerance
            assert abs(_wrap(per_chirp - 2 * u)) > 2e-2 or abs(u) < 2e-2


def test_monostatic_special_case():
    """RX at the TX: d = 2R, so r is the textbook beat frequency 2 R B/(c Tc)
    in cycles per sample and u the textbook Doppler 2 v_r f0 / c per chirp."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, 128, 128)
    tx = np.array([1.0, -2.0])
    x, y, vx, vy = 7.0, 9.0, 3.0, -4.0
    R = np.hypot(x - 1.0, y + 2.0)
    v_r = (vx * (x - 1.0) + vy * (y + 2.0)) / R
    r = model.range_sense(x, y, tx, tx, radar)
    u = model.speed_sense(x, y, vx, vy, tx, tx, radar)
    f_beat = 2 * R / C * (radar.B / radar.Tc)
    assert r == pytest.approx(f_beat * radar.Tc / radar.Ms, rel=1e-13)
    assert u == pytest.approx(2 * v_r * radar.f0 / C * radar.Tc, rel=1e-13)


def test_range_resolution_is_papers_60cm():
    """One unpadded range bin (1/Ms cycle per sample) spans c/B of bistatic
    path, i.e. half of it, 60 cm, of range (Fig. 3 caption)."""
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    radar = scenes.Radar(g["f0_hz"]["value"], g["B_hz"]["value"], g["Tc_s"]["value"],
                         g["Ms"]["value"], g["Mc"]["value"])
    tx = np.zeros(2)
    # monostatic target at range R and R + 0.6 m: bistatic paths differ by 1.2 m
    r0 = model.range_sense(10.0, 0.0, tx, tx, radar)
    r1 = model.range_sense(10.0 + g["range_resolution_m"]["value"], 0.0, tx, tx, radar)
    assert (r1 - r0) * radar.Ms == pytest.approx(1.0, rel=2e-3)


def test_degenerate_unit_vector_is_zero():
    radar = scenes.Radar(24e9, 250e6, 128e-6, 64, 32)
    tx = np.array([2.0, 3.0])
    rxq = np.array([5.0, 7.0])
    u = model.speed_sense(2.0, 3.0, 1.0, 1.0, tx, rxq, radar)
    # only the RX unit vector (0.6, 0.8) contributes
    assert u == pytest.approx(radar.f0 * radar.Tc / C * (-0.6 - 0.8), rel=1e-13)


def test_measurement_energy_and_superposition():
    """Noiseless single target: ||Y_q||^2 = |alpha_q|^2 Ms Mc (unit-modulus
    atoms); two targets superpose linearly."""
    sc = scenes.paper_frame(4, snr_db=None, T=2)
    Y = model.measurement(sc)
    a = sc.noiseless()
    a1 = scenes.Scene(**{**a.__dict__, "targets": sc.targets[:1], "alpha": sc.alpha[:1]})
    a2 = scenes.Scene(**{**a.__dict__, "targets": sc.targets[1:], "alpha": sc.alpha[1:]})
    Y1, Y2 = model.measurement(a1), model.measurement(a2)
    np.testing.assert_allclose(Y, Y1 + Y2, atol=1e-12)
    for q in range(sc.Q):
        assert np.sum(np.abs(Y1[q]) ** 2) == pytest.approx(
            abs(sc.alpha[0, q]) ** 2 * sc.radar.Ms * sc.radar.Mc, rel=1e-12)
    # entries are alpha exp(j 2 pi (u mc + r m)): ratio along a row is constant
    row = Y1[0, 3]
    ratios = row[1:] / row[:-1]
    np.testing.assert_allclose(ratios, ratios[0], atol=1e-12)
    assert abs(np.angle(ratios[0]) / (2 * np.pi) - _wrap(
        model.range_sense(*sc.targets[0][:2], sc.tx, sc.rx[0], sc.radar))) < 1e-12


def test_noise_statistics():
    sc = scenes.paper_frame(5)
    var = np.mean(np.abs(sc.noise) ** 2)
    assert var == pytest.approx(10 ** (-10 / 10), rel=0.02)
    assert abs(np.mean(sc.noise)) < 5e-3
