"""Pins of the oracle's range-Doppler maps against the FFT library, closed-form
Dirichlet kernels, Parseval's identity and brute-force correlations."""
import numpy as np
import pytest

from oracle import maps
from paper_2307_16550_gb300 import scenes


def _draw_Y(seed, Q, Mc, Ms):
    return scenes.complex_normal(seed, 99, (Q, Mc, Ms))


def _raw_dirichlet(f, M):
    """e^{j pi f (M-1)} sin(pi M f) / sin(pi f), with its limit M at f = 0."""
    f = np.asarray(f, dtype=np.float64)
    s = np.sin(np.pi * f)
    ratio = np.where(np.abs(s) < 1e-300, M, np.sin(np.pi * M * f) / np.where(s == 0, 1, s))
    return np.exp(1j * np.pi * f * (M - 1)) * ratio


@pytest.mark.parametrize("Mc,Ms", [(8, 16), (32, 64), (16, 128)])
def test_rd_map_equals_numpy_fft2(Mc, Ms):
    Y = _draw_Y(1, 1, Mc, Ms)[0]
    Z = maps.rd_map(Y, 4)
    ref = np.fft.fft2(Y, s=(4 * Mc, 4 * Ms))
    np.testing.assert_allclose(Z, ref, atol=1e-9 * np.abs(ref).max())


def test_pure_tone_closed_form():
    """Y = b(u) (x) a(r): Z[j, i] = D_Mc(u - j/Nd) D_Ms(r - i/Nr)."""
    Mc, Ms, pad = 16, 32, 4
    r, u = 0.3171, -0.2213
    Y = np.exp(2j * np.pi * (u * np.arange(Mc)[:, None] + r * np.arange(Ms)[None, :]))
    Z = maps.rd_map(Y, pad)
    j = np.arange(pad * Mc)[:, None]
    i = np.arange(pad * Ms)[None, :]
    ref = _raw_dirichlet(u - j / (pad * Mc), Mc) * _raw_dirichlet(r - i / (pad * Ms), Ms)
    np.testing.assert_allclose(Z, ref, atol=1e-9)


def test_on_bin_peak_is_Ms_Mc():
    Mc, Ms, pad = 16, 32, 4
    i0, j0 = 37, 11
    r, u = i0 / (pad * Ms), j0 / (pad * Mc)
    Y = np.exp(2j * np.pi * (u * np.arange(Mc)[:, None] + r * np.arange(Ms)[None, :]))
    Z = maps.rd_map(Y, pad)
    assert abs(Z[j0, i0] - Ms * Mc) < 1e-9
    assert np.unravel_index(np.argmax(np.abs(Z)), Z.shape) == (j0, i0)


def test_parseval():
    Y = _draw_Y(2, 2, 32, 64)
    Z = maps.rd_maps(Y, 4)
    assert np.sum(np.abs(Z) ** 2) == pytest.approx(4 * 32 * 4 * 64 * np.sum(np.abs(Y) ** 2), rel=1e-12)


def test_centred_map_is_centred_atom_correlation():
    """Z~[q, i, j] = <Y_q, b(j/Nd) (x) a~(i/Nr)> by brute force, a~ centred."""
    Q, Mc, Ms, pad = 2, 8, 16, 4
    Y = _draw_Y(3, Q, Mc, Ms)
    Zc = maps.centred_maps(Y, pad)
    assert Zc.shape == (Q, pad * Ms, pad * Mc)
    m = np.arange(Ms) - (Ms - 1) / 2
    for q, i, j in [(0, 0, 0), (1, 5, 31), (0, 63, 7), (1, 40, 20)]:
        r, u = i / (pad * Ms), j / (pad * Mc)
        atom = np.outer(np.exp(2j * np.pi * u * np.arange(Mc)), np.exp(2j * np.pi * r * m))
        assert abs(Zc[q, i, j] - np.vdot(atom, Y[q])) < 1e-10
