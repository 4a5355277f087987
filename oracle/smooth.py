"""Differentiable hopping score at continuous points and its analytic
gradient, FP64 (the refinement and calibration use of the scorer; the paper's
future work, Sec. VI, asks for off-grid estimates).

Test infrastructure only (see the package docstring).

Reading. The paper's hopping reads the nearest Doppler bin (Sec. IV), which
makes the score piecewise constant in the velocity. For gradients the Doppler
axis is interpolated exactly like the range axis: centred Doppler atoms
b~_mc(u) = exp(j 2 pi u (mc - (Mc-1)/2)), the three bins j-1, j, j+1 on one
polar arc whose half-angle comes from (Mc, Nd), coefficients d_l(sigma) of the
same form as the range coefficients c_k(tau). For a point (x, y, vx, vy):

    rho_q = Nr r_q(x),  i = floor(rho_q + 1/2),  tau = rho_q - i
    eta_q = Nd u_q(x, v), j = floor(eta_q + 1/2), sigma = eta_q - j
    s_q   = sum_{k,l in -1,0,1} c_k(tau) d_l(sigma) V_q(i + k, j + l)
    S     = sum_q |s_q|^2

where V_q(n, m) = <Y_q, b~(m/Nd) (x) a~(n/Nr)> is the raw map bin
(m mod Nd, n mod Nr) times exp(j pi (n (Ms-1)/Nr + m (Mc-1)/Nd)) at the
unwrapped indices (n, m). At tau = sigma = 0 the value is the bin itself.

Gradient (i and j held fixed: the score is smooth between bin switches at
tau, sigma = +-1/2):
    dS/drho_q = 2 Re(conj(s_q) sum c_k'(tau) d_l(sigma) V),  likewise eta with d_l'
    drho/dx = Nr B/(c Ms) w_q,      drho/drx_q = -Nr B/(c Ms) u_rx
    deta/dv = Nd kappa w_q,          deta/dx = Nd kappa (J_tx + J_rx) v,
    deta/drx_q = -Nd kappa J_rx v,  J_p = (I - u_p u_p^T) / |x - p|
with u_p the unit vector from p to x (zero, with J_p = 0, below 1e-9 m),
kappa = f0 Tc / c, and for the polar coefficients
    kappa'(t) = theta sin(theta t) / (1 - cos theta), sigma'(t) = theta cos(theta t) / sin theta,
    c_{-1}' = (kappa' - sigma')/2, c_0' = -kappa', c_{+1}' = (kappa' + sigma')/2.
"""
from __future__ import annotations

import numpy as np

from .hopping import polar_angle, polar_coeffs
from .model import C_LIGHT


def polar_coeffs_deriv(tau, theta):
    """d/dtau of (c_{-1}, c_0, c_{+1})."""
    tau = np.asarray(tau, dtype=np.float64)
    dkap = theta * np.sin(theta * tau) / (1.0 - np.cos(theta))
    dsig = theta * np.cos(theta * tau) / np.sin(theta)
    return np.stack([(dkap - dsig) / 2.0, -dkap, (dkap + dsig) / 2.0], axis=-1)


def _unit_jac(px, py, x, y):
    """Distance n, unit vector u = (x - p)/n and J = (I - u u^T)/n (zero below 1e-9 m)."""
    dx, dy = x - px, y - py
    n = np.sqrt(dx * dx + dy * dy)
    if n < 1e-9:
        return n, np.zeros(2), np.zeros((2, 2))
    u = np.array([dx / n, dy / n])
    return n, u, (np.eye(2) - np.outer(u, u)) / n


def _stencil(Z, q, i, j, Ms, Mc):
    """V_q(i + k, j + l), k, l in -1, 0, 1, from the raw maps Z (Q, Nd, Nr)."""
    _, Nd, Nr = Z.shape
    V = np.zeros((3, 3), dtype=np.complex128)
    for a, k in enumerate((-1, 0, 1)):
        for b, l in enumerate((-1, 0, 1)):
            n, m = i + k, j + l
            ph = np.exp(1j * np.pi * ((n * (Ms - 1)) / Nr + (m * (Mc - 1)) / Nd))
            V[a, b] = Z[q, m % Nd, n % Nr] * ph
    return V


def point_terms(Z, radar, tx, rx, point):
    """Per receiver: (rho, eta, i, j, tau, sigma, V, geometry) of one point."""
    x, y, vx, vy = point
    Q, Nd, Nr = Z.shape
    v = np.array([vx, vy])
    kap = radar.f0 * radar.Tc / C_LIGHT
    out = []
    for q in range(Q):
        n1, u1, J1 = _unit_jac(tx[0], tx[1], x, y)
        n2, u2, J2 = _unit_jac(rx[q][0], rx[q][1], x, y)
        d = n1 + n2
        w = u1 + u2
        rho = Nr * (radar.B * d / (C_LIGHT * radar.Ms))
        eta = Nd * (kap * (w[0] * vx + w[1] * vy))
        i = int(np.floor(rho + 0.5))
        j = int(np.floor(eta + 0.5))
        out.append(dict(rho=rho, eta=eta, i=i, j=j, tau=rho - i, sigma=eta - j,
                        V=_stencil(Z, q, i, j, radar.Ms, radar.Mc), w=w, u_rx=u2, J_tx=J1, J_rx=J2, v=v))
    return out


def smooth_scores(Z, radar, tx, rx, points):
    """S and s_q of every point: float64 (P,), complex128 (P, Q)."""
    Q, Nd, Nr = Z.shape
    thr = polar_angle(radar.Ms, Nr)
    thd = polar_angle(radar.Mc, Nd)
    points = np.asarray(points, dtype=np.float64).reshape(-1, 4)
    s = np.zeros((len(points), Q), dtype=np.complex128)
    for p, pt in enumerate(points):
        for q, t in enumerate(point_terms(Z, radar, tx, rx, pt)):
            c = polar_coeffs(t["tau"], thr)
            dd = polar_coeffs(t["sigma"], thd)
            s[p, q] = c @ t["V"] @ dd
    return (np.abs(s) ** 2).sum(axis=1), s


def smooth_grad(Z, radar, tx, rx, points):
    """Analytic gradient of S: dS/dpoint (P, 4) and dS/drx (P, Q, 2)."""
    Q, Nd, Nr = Z.shape
    thr = polar_angle(radar.Ms, Nr)
    thd = polar_angle(radar.Mc, Nd)
    kap = radar.f0 * radar.Tc / C_LIGHT
    gr = Nr * radar.B / (C_LIGHT * radar.Ms)  # drho / dd
    ge = Nd * kap                              # deta / d<w, v>
    points = np.asarray(points, dtype=np.float64).reshape(-1, 4)
    dpt = np.zeros((len(points), 4))
    drx = np.zeros((len(points), Q, 2))
    for p, pt in enumerate(points):
        for q, t in enumerate(point_terms(Z, radar, tx, rx, pt)):
            c = polar_coeffs(t["tau"], thr)
            dc = polar_coeffs_deriv(t["tau"], thr)
            dd = polar_coeffs(t["sigma"], thd)
            ddd = polar_coeffs_deriv(t["sigma"], thd)
            V = t["V"]
            s = c @ V @ dd
            dS_drho = 2.0 * np.real(np.conj(s) * (dc @ V @ dd))
            dS_deta = 2.0 * np.real(np.conj(s) * (c @ V @ ddd))
            w, v = t["w"], t["v"]
            dpt[p, :2] += dS_drho * gr * w + dS_deta * ge * ((t["J_tx"] + t["J_rx"]) @ v)
            dpt[p, 2:] += dS_deta * ge * w
            drx[p, q] = dS_drho * gr * (-t["u_rx"]) + dS_deta * ge * (-(t["J_rx"] @ v))
    return dpt, drx


def smooth_map_grad(Z, radar, tx, rx, points, g):
    """Gradient of L = sum_p g_p S_p with respect to the range-centred maps
    (Q, Nr, Nd) (bin i carries exp(j pi (i/Nr)(Ms-1)), i in [0, Nr)), as
    dL/dRe + j dL/dIm. A read of stored bin (n mod Nr, m mod Nd) enters s_q with
    weight c_k d_l times (-1)^((Ms-1) floor(n/Nr)) exp(j pi m (Mc-1)/Nd), and
    d|s|^2 / d(bin) in this convention is 2 s conj(weight)."""
    Q, Nd, Nr = Z.shape
    thr = polar_angle(radar.Ms, Nr)
    thd = polar_angle(radar.Mc, Nd)
    G = np.zeros((Q, Nr, Nd), dtype=np.complex128)
    points = np.asarray(points, dtype=np.float64).reshape(-1, 4)
    for p, pt in enumerate(points):
        for q, t in enumerate(point_terms(Z, radar, tx, rx, pt)):
            c = polar_coeffs(t["tau"], thr)
            dd = polar_coeffs(t["sigma"], thd)
            s = c @ t["V"] @ dd
            for a, k in enumerate((-1, 0, 1)):
                for b, l in enumerate((-1, 0, 1)):
                    n, m = t["i"] + k, t["j"] + l
                    wrap = (-1.0) ** (((radar.Ms - 1) * (n // Nr)) % 2)
                    wgt = c[a] * dd[b] * wrap * np.exp(1j * np.pi * (m * (radar.Mc - 1)) / Nd)
                    G[q, n % Nr, m % Nd] += g[p] * 2.0 * s * np.conj(wgt)
    return G
