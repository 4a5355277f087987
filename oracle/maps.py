"""Range-Doppler maps: zero-padded 2D DFTs of the measurements, FP64.

Test infrastructure only (see the package docstring).

The i-th bin of the range DFT of a chirp is its correlation with the atom
a(i / Nr) on the DFT's implicit frequency grid (Sec. IV, first paragraph); the
Doppler DFT does the same along chirps with b(j / Nd). Readings:

* The inner product is <y, a> = sum_m y_m conj(a_m), so the forward DFT uses
  exp(-j 2 pi ...).
* Both axes are zero padded by the factor ``pad`` (Nr = pad * Ms,
  Nd = pad * Mc); no window is applied, so every bin is an exact correlation.
* The centred map multiplies range bin i by exp(j pi (i/Nr) (Ms - 1)), which
  turns the bin into the correlation with the centred atom
  a~_m(r) = exp(j 2 pi r (m - (Ms - 1)/2)); the polar interpolation of the
  hopping score works on centred atoms (see ``hopping``).
"""
from __future__ import annotations

import numpy as np


def dft_matrix(N, M):
    """F[k, n] = exp(-j 2 pi k n / N), k < N, n < M (phase reduced exactly)."""
    k = np.arange(N)[:, None]
    n = np.arange(M)[None, :]
    return np.exp(-2j * np.pi * ((k * n) % N) / N)


def rd_map(Yq, pad):
    """Z[j, i] = sum_mc sum_m Y[mc, m] exp(-j 2 pi (j mc / Nd + i m / Nr)),
    shape (Nd, Nr): Doppler bin j, range bin i."""
    Mc, Ms = Yq.shape
    return dft_matrix(pad * Mc, Mc) @ Yq @ dft_matrix(pad * Ms, Ms).T


def rd_maps(Y, pad):
    """Raw (uncentred) maps of all receivers, complex128 (Q, Nd, Nr)."""
    return np.stack([rd_map(Yq, pad) for Yq in Y])


def centring_phase(n, Nr, Ms):
    """exp(j pi (n / Nr) (Ms - 1)) for any integer range index n."""
    return np.exp(1j * np.pi * (n / Nr) * (Ms - 1))


def centred_maps(Y, pad):
    """Centred maps Z~[q, i, j] = Z_q[j, i] * exp(j pi (i/Nr)(Ms-1)), laid out
    range-major, Doppler-contiguous: complex128 (Q, Nr, Nd)."""
    Q, Mc, Ms = Y.shape
    Nr = pad * Ms
    Z = rd_maps(Y, pad)  # (Q, Nd, Nr)
    ph = centring_phase(np.arange(Nr), Nr, Ms)
    return np.ascontiguousarray(np.transpose(Z * ph[None, None, :], (0, 2, 1)))


# ---------------------------------------------------------------------------
# Reduced-precision map storage (the precision mode of the CUDA path; no
# counterpart in the paper). A stored bin is 2^-s times the centred map value,
# s = log2(Ms) + log2(Mc), with its real and imaginary parts each rounded to
# nearest, ties to even, in IEEE binary16 ("f16": 11 significant bits,
# exponents -14..15, subnormal spacing 2^-24) or bfloat16 ("bf16": 8
# significant bits, the binary32 exponent range).
# ---------------------------------------------------------------------------
FORMATS = {"f16": (11, -14, 15), "bf16": (8, -126, 127)}  # significant bits, min / max exponent


def map_scale_log2(Ms, Mc):
    """s with 2^s = Ms * Mc (both powers of two)."""
    return int(round(np.log2(Ms))) + int(round(np.log2(Mc)))


def round_format(x, kind):
    """Round float64 values to the nearest value of the format, ties to even.

    A finite value x = m 2^e (1 <= |m| < 2) keeps p significant bits for
    e >= emin, i.e. x is rounded to a multiple of 2^(max(e, emin) - p + 1);
    below 2^emin the spacing stays 2^(emin - p + 1) (subnormals). Values
    beyond the largest finite value are an error here (the storage scale is
    chosen so that maps never reach it)."""
    p, emin, emax = FORMATS[kind]
    x = np.asarray(x, dtype=np.float64)
    mant, ex = np.frexp(x)                 # x = mant * 2^ex, 0.5 <= |mant| < 1
    e = np.maximum(ex - 1, emin)           # exponent of the leading bit, clamped
    quantum = np.ldexp(1.0, e - p + 1)
    y = np.rint(x / quantum) * quantum     # np.rint rounds half to even; x / quantum is exact
    big = np.ldexp(2.0 - 2.0 ** (1 - p), emax)
    if np.any(np.abs(y) > big):
        raise OverflowError(f"value beyond the {kind} range")
    return y


def quantize_maps(Zc, kind, s):
    """Centred maps as stored and read back: 2^s * round(2^-s Zc), parts rounded separately."""
    scale = np.ldexp(1.0, -s)
    re = round_format(Zc.real * scale, kind)
    im = round_format(Zc.imag * scale, kind)
    return (re + 1j * im) / scale


def quantization_error_bound(kind, s):
    """(u, eta) with |q(x) - x| <= u |x| + eta for every stored part x (before
    the 2^s scale-back): u = 2^-p (half an ulp relative), eta = half the
    subnormal spacing, times 2^s."""
    p, emin, _ = FORMATS[kind]
    return 2.0 ** -p, np.ldexp(1.0, emin - p) * np.ldexp(1.0, s)
