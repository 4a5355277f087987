"""Grid hopping: interpolated evaluation of the direct decision function from
the range-Doppler maps (Sec. IV, Eq. 5), FP64.

Test infrastructure only (see the package docstring).

For every grid cell (x, v) and receiver q the correlation <Y_q, b(u_q) (x) a(r_q)>
of the direct method is replaced by a short linear combination of map bins:

* range axis: polar interpolation over the three bins i-1, i, i+1 around the
  cell's range (Sec. IV cites Fourier-atom polar interpolation; the paper gives
  no formula). Reading: the centred atoms a~(r) all have norm sqrt(Ms) and the
  real Gram <a~(r1), a~(r2)> = D(r1 - r2), D(f) = sum_m exp(j 2 pi f (m - (Ms-1)/2)).
  The three bin atoms are taken as points at angles -theta, 0, +theta of one
  circular arc, and the atom at fractional offset tau (in bins) as the arc point
  at angle theta * tau. The arc through three equally spaced points has
  2 cos(theta/2) = |p(+1) - p(-1)| / |p(+1) - p(0)|, which with the Gram gives
  cos(theta/2) = 1/2 sqrt((Ms - D(2 delta)) / (Ms - D(delta))), delta = 1/Nr.
  Writing the arc point through the three points gives real coefficients
  c_0 = 1 - kappa, c_{+1} = (kappa + sigma)/2, c_{-1} = (kappa - sigma)/2 with
  kappa = (1 - cos(theta tau)) / (1 - cos theta), sigma = sin(theta tau) / sin(theta).
* Doppler axis: a single index, the nearest Doppler bin (Sec. IV, second
  paragraph).
* Bins are found in FP64: rho = Nr * r_q, i = floor(rho + 1/2), tau = rho - i;
  eta = Nd * u_q, j = floor(eta + 1/2) mod Nd. Range indices i + k outside
  [0, Nr) read bin (i + k) mod Nr with the centring phase of the unwrapped
  index.
* The score is S(x, v) = sum_q |s_q|^2 (the sum over receivers of Eq. 3); the
  argmax takes the smallest linear cell index among equal scores.
"""
from __future__ import annotations

import numpy as np

from .model import C_LIGHT, bistatic, grid_axes
from .maps import centring_phase


def dirichlet(f, M):
    """D(f) = sum_{m<M} exp(j 2 pi f (m - (M-1)/2)); real, returned as float."""
    m = np.arange(M) - (M - 1) / 2.0
    f = np.asarray(f, dtype=np.float64)
    return np.real(np.exp(2j * np.pi * f[..., None] * m).sum(axis=-1))


def polar_angle(Ms, Nr):
    """Half-arc angle theta of the three-bin polar model (FP64)."""
    delta = 1.0 / Nr
    D1 = dirichlet(delta, Ms)
    D2 = dirichlet(2.0 * delta, Ms)
    return 2.0 * np.arccos(0.5 * np.sqrt((Ms - D2) / (Ms - D1)))


def polar_coeffs(tau, theta):
    """(c_{-1}, c_0, c_{+1}) for fractional offsets tau, stacked on the last axis."""
    tau = np.asarray(tau, dtype=np.float64)
    kap = (1.0 - np.cos(theta * tau)) / (1.0 - np.cos(theta))
    sig = np.sin(theta * tau) / np.sin(theta)
    return np.stack([(kap - sig) / 2.0, 1.0 - kap, (kap + sig) / 2.0], axis=-1)


def linear_coeffs(tau):
    """Linear interpolation between the two nearest bins (comparison only)."""
    tau = np.asarray(tau, dtype=np.float64)
    return np.stack([np.maximum(-tau, 0.0), 1.0 - np.abs(tau), np.maximum(tau, 0.0)], axis=-1)


def coord_table(radar, tx, rx, grid):
    """Per (ix, iy, q): the coordinate mapping of the hopping scorer.

    Returns a dict of arrays of shape (nx, ny, Q): rho (range in padded bins),
    i (nearest bin, int64), tau, c (..., 3), wx, wy (bistatic gradient, Eq. 1)
    and d (bistatic path)."""
    X, Yg, _, _ = grid_axes(grid)
    x = X[:, None]
    y = Yg[None, :]
    Nr = radar.pad * radar.Ms
    theta = polar_angle(radar.Ms, Nr)
    out = {k: [] for k in ("rho", "i", "tau", "c", "wx", "wy", "d")}
    for q in range(rx.shape[0]):
        d, wx, wy = bistatic(x, y, tx, rx[q])
        r = radar.B * d / (C_LIGHT * radar.Ms)
        rho = Nr * r
        i = np.floor(rho + 0.5)
        tau = rho - i
        out["rho"].append(rho)
        out["i"].append(i.astype(np.int64))
        out["tau"].append(tau)
        out["c"].append(polar_coeffs(tau, theta))
        out["wx"].append(wx)
        out["wy"].append(wy)
        out["d"].append(d)
    return {k: np.stack(v, axis=2) for k, v in out.items()}


def doppler_bin(wx, wy, vx, vy, radar):
    """Nearest Doppler bin j = floor(Nd * u + 1/2) mod Nd (FP64 decision)."""
    Nd = radar.pad * radar.Mc
    u = (radar.f0 * radar.Tc / C_LIGHT) * (wx * vx + wy * vy)
    return np.mod(np.floor(Nd * u + 0.5).astype(np.int64), Nd)


def hop_correlations(Z, radar, tx, rx, grid, ix, iy, table=None, coeffs=None):
    """s_q(x, v) for all velocity cells of the (x, y) cells (ix[n], iy[n]).

    Z are the raw maps (Q, Nd, Nr) of ``maps.rd_maps``. ``coeffs`` replaces the
    polar coefficients (same shape as table['c']) when given. Returns
    complex128 (len(ix), Q, nvx, nvy)."""
    if table is None:
        table = coord_table(radar, tx, rx, grid)
    _, _, VX, VY = grid_axes(grid)
    Q, Nd, Nr = Z.shape
    Ms = radar.Ms
    ix = np.atleast_1d(ix)
    iy = np.atleast_1d(iy)
    out = np.zeros((ix.size, Q, VX.size, VY.size), dtype=np.complex128)
    c_all = table["c"] if coeffs is None else coeffs
    for q in range(Q):
        i0 = table["i"][ix, iy, q]
        c = c_all[ix, iy, q]
        j = doppler_bin(table["wx"][ix, iy, q][:, None, None], table["wy"][ix, iy, q][:, None, None],
                        VX[None, :, None], VY[None, None, :], radar)
        for kk, k in enumerate((-1, 0, 1)):
            n = i0 + k
            val = Z[q][j, np.mod(n, Nr)[:, None, None]] * centring_phase(n, Nr, Ms)[:, None, None]
            out[:, q] += c[:, kk][:, None, None] * val
    return out


def hop_scores(Z, radar, tx, rx, grid, xy_rows=None):
    """Hopping score S(x, v) = sum_q |s_q|^2 over the grid.

    Returns float64 (nx, ny, nvx, nvy), or only the x rows listed in xy_rows
    (shape (len(xy_rows), ny, nvx, nvy))."""
    table = coord_table(radar, tx, rx, grid)
    nx, ny, nvx, nvy = grid.n
    rows = range(nx) if xy_rows is None else xy_rows
    out = np.zeros((len(rows), ny, nvx, nvy))
    iy = np.arange(ny)
    for r, ixv in enumerate(rows):
        s = hop_correlations(Z, radar, tx, rx, grid, np.full(ny, ixv), iy, table)
        out[r] = (np.abs(s) ** 2).sum(axis=1)
    return out


def argmax_cell(scores):
    """Linear index of the largest score; ties go to the smallest index."""
    flat = np.asarray(scores).reshape(-1)
    return int(np.argmax(flat))


def hop_quantization_bound(Z, radar, tx, rx, grid, kind, xy_rows=None):
    """Bound on |S_q - S| per cell when every map part is stored in the
    reduced-precision format ``kind`` (``maps.quantize_maps``) instead of exactly.

    Each stored part is within u |x| + eta of its exact value
    (``maps.quantization_error_bound``), so a complex bin moves by at most
    e_bin = u |Z| + sqrt(2) eta (Minkowski) and the interpolated correlation by
    e_q = sum_k |c_k| e_bin(k); then | |s + d|^2 - |s|^2 | <= (2|s| + e_q) e_q,
    summed over the receivers. Returns float64 of the shape of ``hop_scores``."""
    from .maps import map_scale_log2, quantization_error_bound
    u, eta = quantization_error_bound(kind, map_scale_log2(radar.Ms, radar.Mc))
    table = coord_table(radar, tx, rx, grid)
    _, _, VX, VY = grid_axes(grid)
    Q, Nd, Nr = Z.shape
    nx, ny, nvx, nvy = grid.n
    rows = range(nx) if xy_rows is None else xy_rows
    out = np.zeros((len(rows), ny, nvx, nvy))
    A = np.abs(Z)
    iy = np.arange(ny)
    for r, ixv in enumerate(rows):
        ix = np.full(ny, ixv)
        s = hop_correlations(Z, radar, tx, rx, grid, ix, iy, table)
        for q in range(Q):
            i0 = table["i"][ix, iy, q]
            c = np.abs(table["c"][ix, iy, q])
            j = doppler_bin(table["wx"][ix, iy, q][:, None, None], table["wy"][ix, iy, q][:, None, None],
                            VX[None, :, None], VY[None, None, :], radar)
            e = np.zeros((ny, nvx, nvy))
            for kk, k in enumerate((-1, 0, 1)):
                e += c[:, kk][:, None, None] * (u * A[q][j, np.mod(i0 + k, Nr)[:, None, None]] + np.sqrt(2.0) * eta)
            out[r] += (2.0 * np.abs(s[:, q]) + e) * e
    return out
