"""GPU parity of the differentiable hopping score (gh_score_points), its
adjoint (gh_score_points_adjoint, through torch.autograd) and the on-device
refinement (gh_refine_points) against the FP64 oracle: scores, analytic
gradients, FP64 central differences (step 1e-4 m, 1e-4 m/s), the map
scatter-add, and the refinement workload (64 seeded candidates around the
detections of the paper-shaped frame)."""
import numpy as np
import pytest

from oracle import maps as omaps
from oracle import model, smooth
from paper_2307_16550_gb300 import autograd, gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4
H = 1e-4


def _interior(Z, sc, n, seed, spread=(0.5, 0.5, 1.0, 1.0), margin=0.45, anywhere=False):
    rng = np.random.default_rng(seed)
    pts = []
    lo = np.array(sc.grid.lo, dtype=np.float64)
    hi = lo + np.array(sc.grid.step) * np.array(sc.grid.n)
    while len(pts) < n:
        if anywhere:
            p = lo + rng.uniform(0, 1, 4) * (hi - lo)
        else:
            t = sc.targets[rng.integers(0, len(sc.targets))]
            p = t + rng.uniform(-1, 1, 4) * np.array(spread)
        terms = smooth.point_terms(Z, sc.radar, sc.tx, sc.rx, p)
        if all(abs(tt["tau"]) < margin and abs(tt["sigma"]) < margin for tt in terms):
            pts.append(p)
    return np.array(pts)


def _setup(torch, sc):
    Y32, Y = measurement64(sc)
    Z = omaps.rd_maps(Y, sc.radar.pad)
    return Y32, Y, Z


@pytest.mark.parametrize("name", ["tiny", "paper"])
def test_point_scores_match_oracle(ctx, torch_cuda, name):
    torch = torch_cuda
    sc = scenes.tiny_scene(3) if name == "tiny" else scenes.paper_frame(2)
    Y32, Y, Z = _setup(torch, sc)
    pts = np.concatenate([_interior(Z, sc, 40, 1), _interior(Z, sc, 40, 2, anywhere=True, margin=0.5)])
    maps = ctx.maps(sc.radar, to_dev(torch, Y32))
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda:0")
    S = autograd.score_points(ctx, sc.radar, sc.tx, rx, maps, torch.tensor(pts, device="cuda:0")).cpu().numpy()
    ref, _ = smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts)
    assert np.abs(S - ref).max() < TOL * ref.max()


@pytest.mark.parametrize("name", ["tiny", "paper"])
def test_adjoint_matches_oracle_gradients_and_central_differences(ctx, torch_cuda, name):
    torch = torch_cuda
    sc = scenes.tiny_scene(4) if name == "tiny" else scenes.paper_frame(3)
    Y32, Y, Z = _setup(torch, sc)
    pts = _interior(Z, sc, 24, 5, margin=0.4)
    maps = ctx.maps(sc.radar, to_dev(torch, Y32))
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda:0", requires_grad=True)
    p = torch.tensor(pts, device="cuda:0", requires_grad=True)
    g = torch.linspace(0.5, 1.5, len(pts), dtype=torch.float32, device="cuda:0")
    S = autograd.score_points(ctx, sc.radar, sc.tx, rx, maps, p)
    (S * g).sum().backward()
    dp = p.grad.cpu().numpy()
    drx = rx.grad.cpu().numpy()
    ref_p, ref_rx = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, pts)
    gw = g.cpu().numpy().astype(np.float64)
    ref_p = ref_p * gw[:, None]
    ref_rx = (ref_rx * gw[:, None, None]).sum(axis=0)
    # position and velocity columns have their own scales
    for cols in ((0, 1), (2, 3)):
        c = list(cols)
        assert np.abs(dp[:, c] - ref_p[:, c]).max() < 1e-3 * np.abs(ref_p[:, c]).max()
    assert np.abs(drx - ref_rx).max() < 1e-3 * np.abs(ref_rx).max()
    # FP64 central differences of the oracle score
    for a in range(4):
        e = np.zeros(4)
        e[a] = H
        fd = (smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts + e)[0]
              - smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, pts - e)[0]) / (2 * H) * gw
        assert np.abs(dp[:, a] - fd).max() < 2e-3 * np.abs(fd).max()


def test_map_scatter_add_matches_oracle(ctx, torch_cuda):
    torch = torch_cuda
    sc = scenes.tiny_scene(5)
    Y32, Y, Z = _setup(torch, sc)
    pts = _interior(Z, sc, 8, 6)
    maps = ctx.maps(sc.radar, to_dev(torch, Y32)).requires_grad_(True)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda:0")
    g = np.linspace(1.0, 2.0, len(pts))
    S = autograd.score_points(ctx, sc.radar, sc.tx, rx, maps, torch.tensor(pts, device="cuda:0"))
    (S * torch.tensor(g, dtype=torch.float32, device="cuda:0")).sum().backward()
    got = maps.grad.cpu().numpy()
    ref = smooth.smooth_map_grad(Z, sc.radar, sc.tx, sc.rx, pts, g)
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()
    assert np.count_nonzero(np.abs(ref) > 0) == np.count_nonzero(np.abs(got) > 0)


def test_refinement_workload_paper_frame(ctx, torch_cuda):
    """64 seeded candidates (+-1/2 grid step around the three detections of
    the paper-shaped frame) refined by gradient ascent in one launch: every
    score rises, the FP64 gradient at the refined points is small, and the
    candidates of each detection end near its target."""
    torch = torch_cuda
    sc = scenes.paper_frame(1)
    Y32, Y, Z = _setup(torch, sc)
    Yd = to_dev(torch, Y32)
    cells, _, _ = ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, 3)
    axes = model.grid_axes(sc.grid)
    centres = np.array([[axes[a][i] for a, i in enumerate(np.unravel_index(c, sc.grid.n))] for c in cells])
    rng = np.random.default_rng(11)
    step = np.array(sc.grid.step)
    cand = centres[np.arange(64) % 3] + rng.uniform(-0.5, 0.5, (64, 4)) * step
    maps = ctx.maps(sc.radar, Yd)
    rx = torch.tensor(sc.rx, dtype=torch.float64, device="cuda:0")
    p0 = torch.tensor(cand, device="cuda:0")
    S0 = autograd.score_points(ctx, sc.radar, sc.tx, rx, maps, p0).cpu().numpy()
    p1, S1 = autograd.refine(ctx, sc.radar, sc.tx, rx, maps, p0, iters=20, scale_xy=step[0], scale_v=step[2])
    p1 = p1.cpu().numpy()
    S1 = S1.cpu().numpy()
    assert np.all(S1 >= S0)
    ref1, _ = smooth.smooth_scores(Z, sc.radar, sc.tx, sc.rx, p1)
    assert np.abs(S1 - ref1).max() < TOL * ref1.max()
    # stationary: the FP64 gradient (in scale units) fell by orders of magnitude
    sc4 = np.array([step[0], step[0], step[2], step[2]])
    g0, _ = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, cand)
    g1, _ = smooth.smooth_grad(Z, sc.radar, sc.tx, sc.rx, p1)
    n0 = np.linalg.norm(g0 * sc4, axis=1)
    n1 = np.linalg.norm(g1 * sc4, axis=1)
    assert np.median(n1 / n0) < 1e-2
    # the best candidate of each detection sits on its target (well inside a grid step)
    for k in range(3):
        t = sc.targets[np.argmin(np.linalg.norm(sc.targets[:, :2] - centres[k, :2], axis=1))]
        mine = p1[np.arange(64) % 3 == k]
        best = mine[np.argmax(S1[np.arange(64) % 3 == k])]
        assert np.all(np.abs(best[:2] - t[:2]) < 0.25 * step[0])
        assert np.all(np.abs(best[2:] - t[2:]) < 0.25 * step[2])


def test_rx_calibration_by_gradient_ascent(ctx, torch_cuda):
    """Noiseless frame, targets known: receivers displaced by a few cm move
    back toward their true positions under gradient ascent of the summed
    score (autograd through the adjoint)."""
    torch = torch_cuda
    radar = scenes.Radar(24e9, 250e6, 128e-6, 256, 128, 4)
    grid = scenes.Grid.from_bounds((0, 0, -15, -15), (40, 40, 15, 15), (8, 8, 4, 4))
    sc = scenes.custom_scene(21, radar, grid, Q=4, T=3, snr_db=None)
    Y32, _ = measurement64(sc)
    maps = ctx.maps(sc.radar, to_dev(torch, Y32))
    pts = torch.tensor(sc.targets, device="cuda:0")
    rng = np.random.default_rng(3)
    ang = rng.uniform(0, 2 * np.pi, sc.Q)
    rx0 = sc.rx + 0.03 * np.stack([np.cos(ang), np.sin(ang)], axis=1)  # 3 cm off
    rx = torch.tensor(rx0, device="cuda:0", requires_grad=True)
    opt = torch.optim.Adam([rx], lr=2e-3)
    for _ in range(150):
        opt.zero_grad()
        loss = -autograd.score_points(ctx, sc.radar, sc.tx, rx, maps, pts).sum()
        loss.backward()
        opt.step()
    err0 = np.linalg.norm(rx0 - sc.rx, axis=1)
    err1 = np.linalg.norm(rx.detach().cpu().numpy() - sc.rx, axis=1)
    assert np.all(err1 < 0.25 * err0)
