"""Exact direct decision function, FP64 (Sec. III, Eqs. 3-4).

Test infrastructure only (see the package docstring).

The direct method scores a cell (x, v) of the 4D grid by

    S(x, v) = sum_q |<Y_q, b(u_q) (x) a(r_q)>|^2,  r_q = S^r_q(x), u_q = S^u_q(x, v).

Reading: Eq. 3 is called the factorised form of the direct method and scores
locations only; the joint 4D function above is the unfactorised decision
function it comes from (Sec. I calls the 4D location-velocity grid the heavy
part of the direct method). Two evaluations are given:

* ``brute``: the definition, one full Mc x Ms correlation per cell and RX.
* ``factored``: the same sum in two contractions. Stage 1 correlates each chirp
  with the range atom, P_q[x, mc] = <Y_q[mc], a(r_q(x))> (the g_q of Eq. 4).
  Stage 2 correlates P_q with the Doppler atom, written separably over the two
  velocity axes: b_mc(u_q) = exp(j 2 pi kappa wx vx mc) exp(j 2 pi kappa wy vy mc),
  kappa = f0 Tc / c.
"""
from __future__ import annotations

import numpy as np

from .model import C_LIGHT, atom_a, atom_b, bistatic, grid_axes, range_sense, speed_sense


def brute(Y, radar, tx, rx, grid, cells):
    """S at the listed linear cell indices, by the definition (slow)."""
    X, Yg, VX, VY = grid_axes(grid)
    nx, ny, nvx, nvy = grid.n
    out = np.zeros(len(cells))
    for n, cell in enumerate(cells):
        cell = int(cell)
        ivy = cell % nvy
        ivx = (cell // nvy) % nvx
        iy = (cell // (nvy * nvx)) % ny
        ix = cell // (nvy * nvx * ny)
        x, y, vx, vy = X[ix], Yg[iy], VX[ivx], VY[ivy]
        for q in range(rx.shape[0]):
            r = range_sense(x, y, tx, rx[q], radar)
            u = speed_sense(x, y, vx, vy, tx, rx[q], radar)
            atom = np.outer(atom_b(u, radar.Mc), atom_a(r, radar.Ms))
            out[n] += abs(np.vdot(atom, Y[q])) ** 2
    return out


def stage1(Yq, r, Ms):
    """P[x, mc] = sum_m Y[mc, m] conj(a_m(r_x)) for a vector of ranges r."""
    A = np.exp(2j * np.pi * np.asarray(r)[:, None] * np.arange(Ms)[None, :])
    return np.conj(A) @ Yq.T


def factored(Y, radar, tx, rx, grid, xy=None, chunk=512):
    """S over all velocity cells of the (x, y) cells ``xy`` (list of (ix, iy);
    default: the whole grid). Returns float64 (len(xy), nvx, nvy)."""
    X, Yg, VX, VY = grid_axes(grid)
    nx, ny, nvx, nvy = grid.n
    if xy is None:
        ixs, iys = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
        xy = np.stack([ixs.ravel(), iys.ravel()], axis=1)
    xy = np.asarray(xy, dtype=np.int64).reshape(-1, 2)
    kappa = radar.f0 * radar.Tc / C_LIGHT
    mc = np.arange(radar.Mc)
    out = np.zeros((len(xy), nvx, nvy))
    for s in range(0, len(xy), chunk):
        blk = xy[s:s + chunk]
        x = X[blk[:, 0]]
        y = Yg[blk[:, 1]]
        for q in range(rx.shape[0]):
            d, wx, wy = bistatic(x, y, tx, rx[q])
            r = radar.B * d / (C_LIGHT * radar.Ms)
            P = stage1(Y[q], r, radar.Ms)                                   # (n, Mc)
            Ex = np.exp(2j * np.pi * kappa * (wx[:, None, None] * VX[None, :, None]) * mc)
            Ey = np.exp(2j * np.pi * kappa * (wy[:, None, None] * VY[None, :, None]) * mc)
            F = (np.conj(Ex) * P[:, None, :]) @ np.conj(Ey).transpose(0, 2, 1)
            out[s:s + chunk] += np.abs(F) ** 2
    return out


def scores_full(Y, radar, tx, rx, grid):
    """Exact S over the whole grid, float64 (nx, ny, nvx, nvy)."""
    nx, ny, nvx, nvy = grid.n
    return factored(Y, radar, tx, rx, grid).reshape(nx, ny, nvx, nvy)


def correlation(Yq, r, u, radar):
    """<Y_q, b(u) (x) a(r)> for one (r, u)."""
    return np.vdot(np.outer(atom_b(u, radar.Mc), atom_a(r, radar.Ms)), Yq)
