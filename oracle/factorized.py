"""The paper's factorised estimators, FP64: location first (Eq. 3), then
velocity at that location (Eq. 4), for the direct method and for grid
hopping (Sec. IV), and the indirect method (per-receiver map peaks and
multilateration, Eq. 2).

Test infrastructure only (see the package docstring).

Readings:

* The location grid is the (x, y) part of the 4D grid and the velocity grid
  its (vx, vy) part; an estimate is returned as the 4D cell (ix, iy, ivx, ivy)
  with its linear index.
* Eq. 3 (direct location): S_loc(x) = sum_q sum_mc |<Y_q[mc], a(r_q(x))>|^2,
  Y_q[mc] the mc-th chirp (row); ties -> smallest (ix, iy) index.
* Eq. 4 (direct velocity): g_q[mc] = <Y_q[mc], a(r_q(x^))> (the eq.'s
  Y^* a, one value per chirp), S_vel(v) = sum_q |<g_q, b(u_q(x^, v))>|^2.
* Grid hopping (Sec. IV): the location scalar products are the polar
  interpolation of the zero-padded range FFT of each chirp over the three
  bins around Nr r_q(x) (centred bins, as in the 4D scorer); for the velocity
  a single index: the Doppler FFT of g_q, zero-padded to Nd, read at the
  nearest bin floor(Nd u_q + 1/2) mod Nd. g_q is computed exactly at x^ (one
  location: its cost is negligible).
* Eq. 2 (indirect) prints argmax of a squared error; it is an argmin. Per
  receiver the peak (i_q, j_q) of |RD map| gives r^_q = i_q / Nr and
  u^_q = j_q / Nd taken in [-1/2, 1/2); x^ = argmin_x sum_q (r_q(x) - r^_q)^2
  over the location grid, then v^ = argmin_v sum_q (u_q(x^, v) - u^_q)^2 over
  the velocity grid (ties -> smallest index).
"""
from __future__ import annotations

import numpy as np

from .hopping import coord_table, polar_angle, polar_coeffs
from .maps import centring_phase, dft_matrix, rd_maps
from .model import atom_a, atom_b, grid_axes, range_sense, speed_sense


def _cell(grid, ix, iy, ivx, ivy):
    nx, ny, nvx, nvy = grid.n
    return ((ix * ny + iy) * nvx + ivx) * nvy + ivy


def location_scores_direct(Y, radar, tx, rx, grid):
    """Eq. 3 over the (x, y) grid, float64 (nx, ny)."""
    X, Yg, _, _ = grid_axes(grid)
    out = np.zeros((X.size, Yg.size))
    for ix, x in enumerate(X):
        for iy, y in enumerate(Yg):
            for q in range(len(rx)):
                a = atom_a(range_sense(x, y, tx, rx[q], radar), radar.Ms)
                out[ix, iy] += np.sum(np.abs(Y[q] @ np.conj(a)) ** 2)
    return out


def range_rows(Y, pad):
    """Zero-padded range DFT of every chirp with the range-centring factor:
    R[q, mc, i] = exp(j pi (i/Nr)(Ms-1)) sum_m Y[q, mc, m] exp(-j 2 pi i m / Nr)."""
    Q, Mc, Ms = Y.shape
    Nr = pad * Ms
    F = dft_matrix(Nr, Ms)
    R = np.einsum("qcm,im->qci", Y, F)
    return R * centring_phase(np.arange(Nr), Nr, Ms)[None, None, :]


def location_scores_hop(Y, radar, tx, rx, grid, table=None):
    """Grid-hopping Eq. 3: sum_q sum_mc |sum_k c_k R~_q,mc[i_q + k]|^2 with
    the polar coefficients and wrapped reads of the 4D scorer. ``table``
    (a ``hopping.coord_table`` dict, default: the grid's own) supplies the
    bins i_q and coefficients c_k."""
    R = range_rows(Y, radar.pad)
    Q, Mc, Nr = R.shape
    t = coord_table(radar, tx, rx, grid) if table is None else table
    nx, ny = grid.n[0], grid.n[1]
    out = np.zeros((nx, ny))
    for q in range(Q):
        i0 = t["i"][:, :, q]
        c = t["c"][:, :, q]
        s = np.zeros((nx, ny, Mc), dtype=np.complex128)
        for kk, k in enumerate((-1, 0, 1)):
            n = i0 + k
            # the centring phase of the unwrapped index n (Eq. 5 reading)
            val = R[q][:, np.mod(n, Nr)] * (centring_phase(n, Nr, radar.Ms)
                                            / centring_phase(np.mod(n, Nr), Nr, radar.Ms))[None]
            s += c[:, :, kk][:, :, None] * np.moveaxis(val, 0, -1)
        out += (np.abs(s) ** 2).sum(axis=-1)
    return out


def _argmax2(S):
    flat = int(np.argmax(S))
    return divmod(flat, S.shape[1])


def g_vectors(Y, radar, tx, rx, x, y):
    """g_q[mc] = <Y_q[mc], a(r_q(x))> (Eq. 4), complex (Q, Mc)."""
    return np.stack([Y[q] @ np.conj(atom_a(range_sense(x, y, tx, rx[q], radar), radar.Ms))
                     for q in range(len(rx))])


def velocity_scores_direct(Y, radar, tx, rx, grid, x, y):
    """Eq. 4 over the (vx, vy) grid at (x, y), float64 (nvx, nvy)."""
    _, _, VX, VY = grid_axes(grid)
    g = g_vectors(Y, radar, tx, rx, x, y)
    out = np.zeros((VX.size, VY.size))
    for a, vx in enumerate(VX):
        for b, vy in enumerate(VY):
            for q in range(len(rx)):
                u = speed_sense(x, y, vx, vy, tx, rx[q], radar)
                out[a, b] += abs(np.sum(g[q] * np.conj(atom_b(u, radar.Mc)))) ** 2
    return out


def velocity_scores_hop(Y, radar, tx, rx, grid, x, y):
    """Grid-hopping Eq. 4: |G_q[j_q(v)]|^2 summed over q, G_q the Doppler DFT
    of g_q zero-padded to Nd, j_q the nearest bin of Nd u_q (mod Nd)."""
    _, _, VX, VY = grid_axes(grid)
    g = g_vectors(Y, radar, tx, rx, x, y)
    Nd = radar.pad * radar.Mc
    G = g @ dft_matrix(Nd, radar.Mc).T  # (Q, Nd)
    out = np.zeros((VX.size, VY.size))
    for q in range(len(rx)):
        u = speed_sense(x, y, VX[:, None], VY[None, :], tx, rx[q], radar)
        j = np.mod(np.floor(Nd * u + 0.5).astype(np.int64), Nd)
        out += np.abs(G[q][j]) ** 2
    return out


def factorized(Y, radar, tx, rx, grid, method):
    """(cell, S_loc at x^, S_vel at v^) of the factorised estimator; method
    "hop" or "exact"."""
    X, Yg, VX, VY = grid_axes(grid)
    L = (location_scores_hop if method == "hop" else location_scores_direct)(Y, radar, tx, rx, grid)
    ix, iy = _argmax2(L)
    V = (velocity_scores_hop if method == "hop" else velocity_scores_direct)(Y, radar, tx, rx, grid, X[ix], Yg[iy])
    ivx, ivy = _argmax2(V)
    return _cell(grid, ix, iy, ivx, ivy), L[ix, iy], V[ivx, ivy]


def rd_peaks(Y, pad):
    """Per receiver the (i, j) of the largest |RD map| bin (ties -> smallest
    linear index i * Nd + j of the [Nr][Nd] map)."""
    Z = rd_maps(Y, pad)  # (Q, Nd, Nr)
    out = []
    for q in range(Z.shape[0]):
        A = np.abs(Z[q]).T  # (Nr, Nd)
        out.append(divmod(int(np.argmax(A)), A.shape[1]))
    return out


def indirect(Y, radar, tx, rx, grid):
    """(cell, location cost at x^, velocity cost at v^) of the indirect
    method (Eq. 2 as an argmin, then the same for the velocity)."""
    X, Yg, VX, VY = grid_axes(grid)
    Nr, Nd = radar.pad * radar.Ms, radar.pad * radar.Mc
    pk = rd_peaks(Y, radar.pad)
    r_hat = np.array([i / Nr for i, _ in pk])
    u_hat = np.array([(j / Nd) if j < Nd // 2 else (j / Nd - 1.0) for _, j in pk])
    L = np.zeros((X.size, Yg.size))
    for q in range(len(rx)):
        L += (range_sense(X[:, None], Yg[None, :], tx, rx[q], radar) - r_hat[q]) ** 2
    ix, iy = divmod(int(np.argmin(L)), Yg.size)
    V = np.zeros((VX.size, VY.size))
    for q in range(len(rx)):
        V += (speed_sense(X[ix], Yg[iy], VX[:, None], VY[None, :], tx, rx[q], radar) - u_hat[q]) ** 2
    ivx, ivy = divmod(int(np.argmin(V)), VY.size)
    return _cell(grid, ix, iy, ivx, ivy), L[ix, iy], V[ivx, ivy]
