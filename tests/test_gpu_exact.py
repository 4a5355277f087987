"""GPU parity of the exact direct decision function (gh_direct_exact) against
the FP64 oracle: full small and ragged grids, sampled (x, y) cells of the
paper-shaped frame, host and device inputs."""
import numpy as np
import pytest

from oracle import direct, hopping
from paper_2307_16550_gb300 import scenes
from tests.helpers import measurement64, rel_err, to_dev, top2_margin

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.mark.parametrize("seed", [1, 4])
def test_tiny_full_grid(ctx, torch_cuda, seed):
    sc = scenes.tiny_scene(seed)
    Y32, Y = measurement64(sc)
    ref = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, score = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sc.grid)
    got = got.cpu().numpy()
    assert rel_err(got, ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_ragged_grid_host_input(ctx, torch_cuda):
    radar = scenes.Radar(24e9, 250e6, 128e-6, 32, 64, 4)
    grid = scenes.Grid.from_bounds((2, -1, -7, -13), (33, 27, 15, 9), (19, 23, 9, 14))
    sc = scenes.custom_scene(8, radar, grid, Q=3, T=2, snr_db=0.0)
    Y32, Y = measurement64(sc)
    ref = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    out = torch_cuda.empty(tuple(grid.n), dtype=torch_cuda.float32, device="cuda:0")
    cell, _ = ctx.gh_direct_exact(sc.radar, sc.tx, sc.rx, sc.Q, Y32, sc.grid, out)  # host Y
    assert rel_err(out.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)


def test_paper_frame_sampled_xy(ctx, torch_cuda):
    sc = scenes.paper_frame(2)
    Y32, Y = measurement64(sc)
    got, cell, score = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sc.grid)
    got = got.cpu().numpy()
    ix, iy, _, _ = sc.grid.unravel(cell)
    xy = [(0, 0), (127, 127), (5, 90), (64, 3), (ix, iy)]
    ref = direct.factored(Y, sc.radar, sc.tx, sc.rx, sc.grid, xy)
    g = np.stack([got[a, b] for a, b in xy])
    assert np.abs(g - ref).max() / ref.max() < TOL
    # the picked cell is the best of its (x, y) cell in the oracle too
    assert sc.grid.cell_index(ix, iy, *np.unravel_index(np.argmax(ref[-1]), ref[-1].shape)) == cell


def test_exact_on_grid_noiseless_peak_value(ctx, torch_cuda):
    """Cauchy-Schwarz equality at the true cell: S = (Ms Mc)^2 sum_q |alpha_q|^2."""
    sc = scenes.tiny_scene(2, snr_db=None, on_grid=True)
    Y32, _ = measurement64(sc)
    cell, score = ctx.gh_direct_exact(sc.radar, sc.tx, sc.rx, sc.Q, to_dev(torch_cuda, Y32), sc.grid, None)
    assert cell == sc.target_cells[0]
    peak = (sc.radar.Ms * sc.radar.Mc) ** 2 * np.sum(np.abs(sc.alpha[0]) ** 2)
    assert score == pytest.approx(peak, rel=1e-4)


def test_paper_frame_full_grid(ctx, torch_cuda):
    """Every exact score of the paper-shaped frame (128 x 128 (x, y) cells x
    32 x 32 velocities, Q = 4, Ms = 256, Mc = 128: the tensor-core stage 1 and
    stage 2 the benchmark times) against the oracle's factored evaluation,
    element by element, and the argmax."""
    sc = scenes.paper_frame(1)
    Y32, Y = measurement64(sc)
    got, cell, score = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sc.grid)
    got = got.cpu().numpy()
    ref = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    err = rel_err(got, ref)
    print(f"paper-shaped frame, exact: max |S_gpu - S| / max S = {err:.2e}")
    assert err < TOL
    assert top2_margin(ref) > 10 * TOL
    assert cell == hopping.argmax_cell(ref)
    assert score == pytest.approx(ref.max(), rel=TOL)


@pytest.mark.parametrize("Ms,Mc,n", [
    (64, 128, (6, 5, 32, 64)),    # 64 velocity columns: two 32-column halves of B
    (32, 32, (7, 6, 17, 45)),     # ragged velocity grid, one 32-chirp stage
    (32, 256, (5, 4, 32, 33)),    # eight stages, one column past 32
    (64, 16, (4, 5, 9, 3)),       # fewer chirps than a stage
])
def test_tensor_core_shapes(ctx, torch_cuda, Ms, Mc, n):
    """The tensor-core stage 2 over its shape range (velocity rows <= 32,
    columns <= 64, Mc <= 256): every score against the oracle."""
    radar = scenes.Radar(24e9, 250e6, 128e-6, Ms, Mc, 4)
    grid = scenes.Grid.from_bounds((3, 2, -14, -13), (31, 29, 12, 15), n)
    sc = scenes.custom_scene(6, radar, grid, Q=3, T=2, snr_db=5.0)
    Y32, Y = measurement64(sc)
    ref = direct.scores_full(Y, sc.radar, sc.tx, sc.rx, sc.grid)
    got, cell, _ = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sc.grid)
    assert rel_err(got.cpu().numpy(), ref) < TOL
    if top2_margin(ref) > 10 * TOL:
        assert cell == hopping.argmax_cell(ref)
