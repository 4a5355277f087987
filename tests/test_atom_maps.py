"""The closed form of an atom's range-Doppler map that the hopping detection
uses to update the maps of a BOMP residual by linearity (Sec. III maps, the
signal model's atoms of Sec. II): the 2D DFT of b(u) (x) a(r), zero-padded,
times the range-centring factor, equals A[i] B[j] with
A[i] = exp(j pi i (Ms-1)/Nr) F_Ms(r - i/Nr), B[j] = F_Mc(u - j/Nd),
F_M(f) = sum_m exp(j 2 pi f m) = exp(j pi f (M-1)) sin(pi M f) / sin(pi f);
and the exact integer reduction of F's arguments from a 64-bit fixed-point
phase (restated here in Python integers) reproduces F to float precision,
including f near integers and near the zeros of sin(pi M f)."""
import numpy as np

from oracle import maps as omaps

TWO64 = 1 << 64


def _f_closed(f, M):
    s = np.sin(np.pi * f)
    if abs(s) < 1e-300:
        return complex(M)
    return np.exp(1j * np.pi * f * (M - 1)) * np.sin(np.pi * M * f) / s


def _f_fixed(ph, M):
    """F_M at f = ph 2^-64: sin(pi f) from the distance to the nearest
    integer, M f mod 2 from ph M/2 mod 2^64, the phase from the 128-bit
    product ph (M-1) halved, each fraction rounded to float32 once."""
    h = min(ph, (TWO64 - ph) % TWO64)
    if h == 0:
        return complex(M)
    sf = np.sin(np.pi * float(np.float32(h * 2.0 ** -64)))
    x = (ph * (M // 2)) % TWO64
    w = x & ((1 << 63) - 1)
    v = w if w < (1 << 62) else (1 << 63) - w
    sm = np.sin(np.pi * float(np.float32(v * 2.0 ** -63))) * (-1 if x >> 63 else 1)
    half = ((ph * (M - 1)) >> 1) % TWO64
    t = float(np.float32((half >> 32) * 2.0 ** -31))
    return np.exp(1j * np.pi * t) * (sm / sf)


def test_atom_map_is_separable_closed_form():
    Ms, Mc, pad = 64, 32, 4
    Nr, Nd = pad * Ms, pad * Mc
    for r, u in ((0.3137, -0.211), (1.75, 0.49), (0.0, 0.0), (2.0 / Nr, -5.0 / Nd)):
        y = np.exp(2j * np.pi * (u * np.arange(Mc)[:, None] + r * np.arange(Ms)[None, :]))
        Z = omaps.centred_maps(y[None], pad)[0]  # [Nr][Nd], range-centred
        i, j = np.arange(Nr), np.arange(Nd)
        A = np.exp(1j * np.pi * i * (Ms - 1) / Nr) * np.array([_f_closed(r - k / Nr, Ms) for k in i])
        B = np.array([_f_closed(u - k / Nd, Mc) for k in j])
        np.testing.assert_allclose(Z, np.outer(A, B), rtol=0, atol=1e-9 * Ms * Mc)


def test_fixed_point_reduction_matches_the_sum():
    rng = np.random.default_rng(3)
    worst = 0.0
    for trial in range(3000):
        M = int(rng.choice([4, 8, 64, 256, 512, 4096]))
        kind = trial % 4
        if kind == 0:
            f = rng.uniform(-3, 3)
        elif kind == 1:  # near an integer: F close to M
            f = int(rng.integers(-2, 3)) + rng.uniform(-1e-6, 1e-6)
        elif kind == 2:  # near a zero of sin(pi M f)
            f = int(rng.integers(-4, 5)) / M + rng.uniform(-1e-7, 1e-7)
        else:  # near half-integers
            f = int(rng.integers(-4, 4)) * 0.5 + rng.uniform(-1e-8, 1e-8)
        ph = int(round((f % 1.0) * 2.0 ** 64)) % TWO64
        fq = ph / 2.0 ** 64
        ref = np.exp(2j * np.pi * fq * np.arange(M)).sum()
        worst = max(worst, abs(_f_fixed(ph, M) - ref) / M)
    assert worst < 1e-6
