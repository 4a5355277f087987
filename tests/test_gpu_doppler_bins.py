"""Bit-exact check of the scorer's Doppler-bin decisions (Sec. IV: a single
Doppler index, the nearest bin j_q = floor(Nd u_q + 1/2) mod Nd, decided in
float64) against the oracle's `doppler_bin`.

The maps of one receiver p hold sqrt(j + 1) in every range row of Doppler bin
j, the other receivers' maps are zero. A cell's score is then
|sum_k c_k s_k|^2 (j_p + 1), with s_k the centring sign of the k-th range read
(Sec. IV reading of wrapped reads), so each score reveals the bin the kernel
chose for receiver p. Every receiver of every cell is decoded on the
paper-shaped grid in the benchmark's launch configuration, on a grid whose
Doppler span wraps around Nd several times, and on grids built so that every
cell of one (x, y, q) lies within 2^-34 .. 2^-14 bin of a rounding boundary
(or on it, up to float64 rounding), where the kernel's fixed-point position
hands the decision to its float64 path."""
import numpy as np
import pytest

from oracle import hopping, model
from paper_2307_16550_gb300 import scenes

pytestmark = pytest.mark.gpu


def _bin_maps(torch, radar, Q, p):
    Nr, Nd = radar.pad * radar.Ms, radar.pad * radar.Mc
    Z = np.zeros((Q, Nr, Nd), np.complex64)
    Z[p] = np.sqrt(np.arange(Nd, dtype=np.float64) + 1.0)[None, :].astype(np.float32)
    return torch.from_numpy(Z).to("cuda:0")


def _signed_coeff_sum(radar, table, q):
    """sum_k c_k s_k per (ix, iy) for receiver q, float64 (oracle table)."""
    Nr, Ms = radar.pad * radar.Ms, radar.Ms
    tot = np.zeros(table["i"].shape[:2])
    for kk, k in enumerate((-1, 0, 1)):
        n = table["i"][:, :, q] + k
        sign = 1.0 if (Ms - 1) % 2 == 0 else np.where(np.floor_divide(n, Nr) % 2 == 0, 1.0, -1.0)
        tot += table["c"][:, :, q, kk] * sign
    return tot


def _check_bins(ctx, torch, radar, tx, rx, grid):
    """Decodes every (cell, receiver) bin of the kernel and compares it with
    the oracle's; returns the number of decisions compared."""
    Q = rx.shape[0]
    table = hopping.coord_table(radar, tx, rx, grid)
    _, _, VX, VY = model.grid_axes(grid)
    Nd = radar.pad * radar.Mc
    n = 0
    for p in range(Q):
        S, _, _ = ctx.scores(radar, tx, rx, _bin_maps(torch, radar, Q, p), grid)
        S = S.cpu().numpy().astype(np.float64)
        C2 = _signed_coeff_sum(radar, table, p) ** 2
        assert C2.min() > 0.2
        dec = S / C2[:, :, None, None] - 1.0
        j_gpu = np.rint(dec).astype(np.int64)
        assert np.abs(dec - j_gpu).max() < 0.05, "score does not decode to a single bin"
        j_ref = hopping.doppler_bin(table["wx"][:, :, p, None, None], table["wy"][:, :, p, None, None],
                                    VX[None, None, :, None], VY[None, None, None, :], radar)
        bad = np.argwhere(j_gpu != j_ref)
        assert bad.size == 0, f"receiver {p}: {len(bad)} Doppler bins differ, first at {bad[0].tolist()}"
        assert j_ref.min() >= 0 and j_ref.max() < Nd
        n += j_ref.size
    return n


def test_paper_frame_every_doppler_bin(ctx, torch_cuda):
    sc = scenes.paper_frame(1)
    assert _check_bins(ctx, torch_cuda, sc.radar, sc.tx, sc.rx, sc.grid) == 4 * sc.grid.ncells


def test_wrapping_doppler_span(ctx, torch_cuda):
    """Velocities up to 60 m/s: |Nd u| reaches about 900 bins, so the bins of
    one (x, y) cell wrap around Nd = 512 (the kernel's wrap flag) and
    negative positions fold to Nd + j."""
    sc = scenes.paper_frame(3)
    grid = scenes.Grid.from_bounds((0, 0, -60, -60), (40, 40, 60, 60), (24, 20, 37, 29))
    table = hopping.coord_table(sc.radar, sc.tx, sc.rx, grid)
    _, _, VX, VY = model.grid_axes(grid)
    Nd = sc.radar.pad * sc.radar.Mc
    eta = Nd * (sc.radar.f0 * sc.radar.Tc / model.C_LIGHT) * (
        table["wx"][..., None, None] * VX[:, None] + table["wy"][..., None, None] * VY[None, :])
    assert (eta.max(axis=(-2, -1)) - eta.min(axis=(-2, -1))).max() > Nd  # spans more than Nd bins
    assert eta.min() < -Nd / 2
    _check_bins(ctx, torch_cuda, sc.radar, sc.tx, sc.rx, grid)


def _boundary_grid(radar, tx, rxq, xy, delta):
    """A 3 x 3 x 32 x 32 grid whose centre (x, y) cell is `xy` and whose
    velocity steps move receiver q's Doppler position by one bin each, with
    the first velocity cell at m + 1/2 + delta bins: every velocity cell of
    that (x, y, q) lies delta (up to float64 rounding) from a boundary."""
    x, y = xy
    _, wx, wy = model.bistatic(np.array(x), np.array(y), tx, rxq)
    wx, wy = float(wx), float(wy)
    k = radar.pad * radar.Mc * radar.f0 * radar.Tc / model.C_LIGHT  # bins per (m/s) per unit w
    sx, sy = 1.0 / (k * wx), 1.0 / (k * wy)
    vx0 = -3.1
    eta0 = 37.5 + delta  # target position of cell (0, 0) in bins
    vy0 = (eta0 / k - wx * vx0) / wy
    lo = (x - 1.5 * 0.25, y - 1.5 * 0.25, vx0 - 0.5 * sx, vy0 - 0.5 * sy)
    return scenes.Grid(lo, (0.25, 0.25, sx, sy), (3, 3, 32, 32))


@pytest.mark.parametrize("delta", [0.0, 2.0**-34, -2.0**-34, 2.0**-30, -2.0**-30, 2.0**-26, -2.0**-26,
                                   2.0**-22, -2.0**-22, 2.0**-20, -2.0**-20, 2.0**-18, -2.0**-18,
                                   2.0**-14, -2.0**-14])
def test_cells_at_rounding_boundaries(ctx, torch_cuda, delta):
    sc = scenes.paper_frame(1)
    for q, xy in ((0, (13.3, 21.7)), (2, (31.9, 4.4))):
        grid = _boundary_grid(sc.radar, sc.tx, sc.rx[q], xy, delta)
        table = hopping.coord_table(sc.radar, sc.tx, sc.rx, grid)
        _, _, VX, VY = model.grid_axes(grid)
        Nd = sc.radar.pad * sc.radar.Mc
        eta = Nd * (sc.radar.f0 * sc.radar.Tc / model.C_LIGHT) * (
            table["wx"][1, 1, q] * VX[:, None] + table["wy"][1, 1, q] * VY[None, :])
        frac = eta - np.floor(eta)
        assert np.abs(frac - 0.5).max() < abs(delta) + 1e-9  # really at the boundary
        _check_bins(ctx, torch_cuda, sc.radar, sc.tx, sc.rx, grid)
