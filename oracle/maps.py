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
