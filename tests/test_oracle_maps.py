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


# --- reduced-precision storage -------------------------------------------------
def _values():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-25, 10, 200000))
    return np.concatenate([x, [0.0, -0.0, 1.0, 65504.0, 2.0 ** -24, 3 * 2.0 ** -25, 1 + 2.0 ** -11]])


def test_round_f16_equals_numpy_half_cast():
    """numpy's float16 cast is an independent IEEE binary16 rounding (incl.
    subnormals and ties to even)."""
    x = _values()
    x = x[np.abs(x) < 65000]
    np.testing.assert_array_equal(maps.round_format(x, "f16"), x.astype(np.float16).astype(np.float64))
    with pytest.raises(OverflowError):
        maps.round_format(np.array([70000.0]), "f16")


def _bf16_by_bits(x32):
    """bfloat16 round-to-nearest-even on the binary32 bit pattern: add
    0x7fff plus the lowest kept bit, clear the low 16 bits."""
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_round_bf16_equals_bit_rounding():
    x32 = _values().astype(np.float32)
    x32 = x32[np.abs(x32) < 3e38]
    np.testing.assert_array_equal(maps.round_format(x32.astype(np.float64), "bf16"), _bf16_by_bits(x32))
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert maps.round_format(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8]), "bf16").tolist() == [1.0, 1 + 2.0 ** -6]


@pytest.mark.parametrize("kind", ["f16", "bf16"])
def test_quantization_error_bound_holds_and_is_attained(kind):
    s = maps.map_scale_log2(256, 128)
    assert s == 15
    x = _values()
    x = x[np.abs(x) < 6e4] * 2.0 ** s
    u, eta = maps.quantization_error_bound(kind, s)
    q = maps.quantize_maps(x + 0j, kind, s).real
    err = np.abs(q - x)
    assert np.all(err <= u * np.abs(x) + eta)
    assert np.max(err / (u * np.abs(x) + eta)) > 0.9  # the bound is tight
