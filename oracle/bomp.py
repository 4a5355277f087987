"""Block orthogonal matching pursuit over the grid, FP64.

Test infrastructure only (see the package docstring).

The paper declares BOMP (Block Orthogonal Matching Pursuit) and names
iterative direct algorithms for several targets as future work (Sec. VI); it
gives no algorithm. Reading used here:

* A block is the set of Q per-receiver atoms b(u_q) (x) a(r_q) of one grid
  cell, each with its own amplitude alpha_q.
* Iteration k: (1) score the current residual over the whole grid, by grid
  hopping on its maps or by the exact direct function; (2) add the argmax cell
  to the support, cells already in the support excluded; (3) for each q, solve
  the least-squares problem min ||Y_q - A_q alpha_q|| over all support atoms at
  their exact (r, u), against the original measurement; (4) set the residual
  R_q = Y_q - A_q alpha_q. The loop stops after K iterations.
* alpha multiplies the atoms as written in the signal model (Sec. II).
"""
from __future__ import annotations

import numpy as np

from . import direct, hopping, maps
from .model import atom_a, atom_b, grid_axes, range_sense, speed_sense


def cell_point(grid, cell):
    X, Yg, VX, VY = grid_axes(grid)
    nx, ny, nvx, nvy = grid.n
    cell = int(cell)
    ivy = cell % nvy
    ivx = (cell // nvy) % nvx
    iy = (cell // (nvy * nvx)) % ny
    ix = cell // (nvy * nvx * ny)
    return X[ix], Yg[iy], VX[ivx], VY[ivy]


def atom_matrix(radar, tx, rxq, grid, cells):
    """Columns vec(b(u_q) (x) a(r_q)) of the listed cells, shape (Mc*Ms, k)."""
    cols = []
    for cell in cells:
        x, y, vx, vy = cell_point(grid, cell)
        r = range_sense(x, y, tx, rxq, radar)
        u = speed_sense(x, y, vx, vy, tx, rxq, radar)
        cols.append(np.outer(atom_b(u, radar.Mc), atom_a(r, radar.Ms)).reshape(-1))
    return np.stack(cols, axis=1)


def grid_scores(R, radar, tx, rx, grid, method):
    if method == "hop":
        Z = maps.rd_maps(R, radar.pad)
        return hopping.hop_scores(Z, radar, tx, rx, grid)
    if method == "exact":
        return direct.scores_full(R, radar, tx, rx, grid)
    raise ValueError(method)


def bomp(Y, radar, tx, rx, grid, K, method="hop"):
    """Returns (cells int64 (K,), scores float64 (K,), alpha complex128 (K, Q),
    residual complex128 (Q, Mc, Ms)). scores[k] is the residual's score at the
    cell picked in iteration k."""
    Q = Y.shape[0]
    R = np.array(Y, dtype=np.complex128, copy=True)
    cells, scores = [], []
    alpha = np.zeros((0, Q), np.complex128)
    for _ in range(K):
        S = grid_scores(R, radar, tx, rx, grid, method).reshape(-1).copy()
        S[np.asarray(cells, dtype=np.int64)] = -np.inf
        best = hopping.argmax_cell(S)
        cells.append(best)
        scores.append(S[best])
        alpha = np.zeros((len(cells), Q), np.complex128)
        for q in range(Q):
            A = atom_matrix(radar, tx, rx[q], grid, cells)
            sol, *_ = np.linalg.lstsq(A, Y[q].reshape(-1), rcond=None)
            alpha[:, q] = sol
            R[q] = Y[q] - (A @ sol).reshape(Y[q].shape)
    return np.array(cells, np.int64), np.array(scores), alpha, R
