"""Signal model of a multistatic FMCW radar (Sec. II), FP64.

Test infrastructure only (see the package docstring).

Readings of the paper used here:

* Range scale (Eq. 1, top). The printed factor 2B/c applied to the bistatic
  path gives cycles per chirp and counts the round trip twice. We use the
  dechirped beat frequency (B/Tc) * d/c times the sample period Tc/Ms:
  r_q = B * d_q / (c * Ms) in cycles per sample, with
  d_q = |x - x_TX| + |x - x_RX,q|. One unpadded bin is c/B = 1.2 m of bistatic
  path, i.e. the 60 cm range resolution quoted in Sec. V.
* Speed scale (Eq. 1, bottom). Likewise u_q = (f0 * Tc / c) * <w_q, v> in
  cycles per chirp, where w_q is the sum of the unit vectors from the TX and
  from RX q to the target, so <w_q, v> is the rate of change of d_q. u > 0 for
  a receding target.
* A unit vector whose length is below 1e-9 m is taken as zero.
* Atoms (Sec. II): a_m(r) = exp(j 2 pi r m), b_mc(u) = exp(j 2 pi u mc), with
  0-based m and mc; Y_q[mc, m] is chirp mc's m-th sample (a row, as in the
  notation paragraph of Sec. I).

FP64 expression order (the GPU coordinate kernel evaluates the same
expressions, so that bin decisions agree bit for bit): dx = x - x_TX,
n = sqrt(dx*dx + dy*dy), d = n_TX + n_RX, r = (B*d) / (c*Ms),
w = dx_TX/n_TX + dx_RX/n_RX per axis, u = ((f0*Tc)/c) * (wx*vx + wy*vy).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0  # m/s


def grid_axes(grid):
    """Cell-centred grid points (x, y, vx, vy): lo + (i + 1/2) * step."""
    return [grid.lo[a] + (np.arange(grid.n[a]) + 0.5) * grid.step[a] for a in range(4)]


def _unit(dx, dy):
    n = np.sqrt(dx * dx + dy * dy)
    small = n < 1e-9
    safe = np.where(small, 1.0, n)
    ux = np.where(small, 0.0, dx / safe)
    uy = np.where(small, 0.0, dy / safe)
    return n, ux, uy


def bistatic(x, y, tx, rxq):
    """Bistatic path d_q(x) = |x - x_TX| + |x - x_RX,q| and the gradient
    w_q(x) = (x - x_TX)/|x - x_TX| + (x - x_RX,q)/|x - x_RX,q| (Eq. 1)."""
    n1, ux1, uy1 = _unit(x - tx[0], y - tx[1])
    n2, ux2, uy2 = _unit(x - rxq[0], y - rxq[1])
    return n1 + n2, ux1 + ux2, uy1 + uy2


def range_sense(x, y, tx, rxq, radar):
    """S^r_q(x): normalised range in cycles per sample (Eq. 1, top)."""
    d, _, _ = bistatic(x, y, tx, rxq)
    return radar.B * d / (C_LIGHT * radar.Ms)


def speed_sense(x, y, vx, vy, tx, rxq, radar):
    """S^u_q(x, v): normalised speed in cycles per chirp (Eq. 1, bottom)."""
    _, wx, wy = bistatic(x, y, tx, rxq)
    return (radar.f0 * radar.Tc / C_LIGHT) * (wx * vx + wy * vy)


def atom_a(r, Ms):
    """Range atom a(r), length Ms (Sec. II)."""
    return np.exp(2j * np.pi * r * np.arange(Ms))


def atom_b(u, Mc):
    """Doppler atom b(u), length Mc (Sec. II)."""
    return np.exp(2j * np.pi * u * np.arange(Mc))


def measurement(scene):
    """Y_q = sum_t alpha_{t,q} b(u_{t,q}) (x) a(r_{t,q}) + W_q for every RX q
    (Eq. general-model, one term per target). Returns complex128 (Q, Mc, Ms)."""
    radar = scene.radar
    Q = scene.rx.shape[0]
    Y = np.array(scene.noise, dtype=np.complex128, copy=True)
    for q in range(Q):
        for t, (x, y, vx, vy) in enumerate(scene.targets):
            r = range_sense(x, y, scene.tx, scene.rx[q], radar)
            u = speed_sense(x, y, vx, vy, scene.tx, scene.rx[q], radar)
            Y[q] += scene.alpha[t, q] * np.outer(atom_b(u, radar.Mc), atom_a(r, radar.Ms))
    return Y
