"""Reduced-precision range-Doppler maps (GH_C16, GH_CBF16) and the
precision-at-scale workload (Q = 8, Ms = 512 x Mc = 256, 268M cells).

Stored maps are 2^-s times the float32 maps rounded to the format; scores
accumulate in float32. The oracle pins every stored value (rounding bound
of the format) and every score: |S_gpu - S_fp64| <= B(cell) + 1e-4 max S,
where B is the oracle's per-cell bound for maps stored in that format and
1e-4 max S the float32 tolerance of the full-precision path. The measured
errors are printed (pytest -s) beside the bound."""
import numpy as np
import pytest

from oracle import bomp, direct, hopping
from oracle import maps as omaps
from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu

KINDS = {gh.GH_C16: "f16", gh.GH_CBF16: "bf16"}
TOL = 1e-4
TOL_MAP = 1e-5


def _as_complex(maps_t, s):
    a = maps_t.float().cpu().numpy().astype(np.float64)
    return (a[..., 0] + 1j * a[..., 1]) * 2.0 ** s


def _scene(name):
    return {"tiny": lambda: scenes.tiny_scene(2), "paper": lambda: scenes.paper_frame(2),
            "precision": lambda: scenes.precision_scene(1)}[name]()


@pytest.mark.parametrize("mt", [gh.GH_C16, gh.GH_CBF16])
@pytest.mark.parametrize("name", ["tiny", "paper", "precision"])
def test_stored_maps_are_rounded_maps(ctx, torch_cuda, name, mt):
    sc = _scene(name)
    Y32, Y = measurement64(sc)
    ref = omaps.centred_maps(Y, sc.radar.pad)
    s = omaps.map_scale_log2(sc.radar.Ms, sc.radar.Mc)
    u, eta = omaps.quantization_error_bound(KINDS[mt], s)
    got = _as_complex(ctx.maps(sc.radar, to_dev(torch_cuda, Y32), mt), s)
    excess = np.abs(got - ref) - (u * np.abs(ref) + np.sqrt(2.0) * eta)
    assert excess.max() <= TOL_MAP * np.abs(ref).max()
    print(f"{name} {KINDS[mt]}: max |map error| / max |map| = {np.abs(got - ref).max() / np.abs(ref).max():.2e}")


@pytest.mark.parametrize("mt", [gh.GH_C16, gh.GH_CBF16])
@pytest.mark.parametrize("name,rows", [("tiny", None), ("paper", [0, 57, 127]), ("precision", [31, 200])])
def test_scores_within_format_bound(ctx, torch_cuda, name, rows, mt):
    sc = _scene(name)
    Y32, Y = measurement64(sc)
    Z = omaps.rd_maps(Y, sc.radar.pad)
    ref = hopping.hop_scores(Z, sc.radar, sc.tx, sc.rx, sc.grid, xy_rows=rows)
    bound = hopping.hop_quantization_bound(Z, sc.radar, sc.tx, sc.rx, sc.grid, KINDS[mt], xy_rows=rows)
    maps_t = ctx.maps(sc.radar, to_dev(torch_cuda, Y32), mt)
    got_full, cell, _ = ctx.scores(sc.radar, sc.tx, sc.rx, maps_t, sc.grid)
    got = (got_full if rows is None else got_full[rows]).cpu().numpy()
    smax = ref.max()
    err = np.abs(got - ref)
    assert np.all(err <= bound + TOL * smax)
    print(f"{name} {KINDS[mt]}: max |score error| / max S = {err.max() / smax:.2e}, "
          f"bound {bound.max() / smax:.2e}")
    # the argmax of the full grid is a cell whose float64 score is within the bound of the best
    if rows is None:
        assert ref.reshape(-1)[cell] >= smax - 2 * (bound.max() + TOL * smax)
    del got_full


@pytest.mark.parametrize("mt", [gh.GH_C16, gh.GH_CBF16])
def test_detect_with_reduced_maps_matches_oracle_cells(ctx, torch_cuda, mt):
    """Paper-shaped frame, K = 3: the same detections as the FP64 oracle."""
    sc = scenes.paper_frame(1)
    Y32, Y = measurement64(sc)
    rc, rs, ra, _ = bomp.bomp(Y, sc.radar, sc.tx, sc.rx, sc.grid, 3, "hop")
    ctx.gh_set_detect_maps(mt)
    try:
        cells, scores, alpha = ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, to_dev(torch_cuda, Y32),
                                             sc.grid, 3)
    finally:
        ctx.gh_set_detect_maps(gh.GH_C64)
    np.testing.assert_array_equal(cells, rc)
    # amplitudes come from exact correlations (not the maps): full precision
    np.testing.assert_allclose(alpha, ra, rtol=0, atol=1e-4 * np.abs(ra).max())
    print(f"paper {KINDS[mt]} detect: score rel. diff at detections "
          f"{np.abs(scores - rs).max() / rs.max():.2e}")


def test_precision_workload_exact_subgrid(ctx, torch_cuda):
    """Exact direct scores on a 64 x 64 x 32 x 32 sub-grid of the
    precision-at-scale frame (split-BF16 tensor-core path), sampled (x, y)
    cells against the factored FP64 oracle."""
    sc = scenes.precision_scene(1)
    Y32, Y = measurement64(sc)
    t = sc.targets[0]
    lo = (t[0] - 6.4, t[1] - 6.4, -15.0, -15.0)
    sub = scenes.Grid.from_bounds(lo, (t[0] + 6.4, t[1] + 6.4, 15.0, 15.0), (64, 64, 32, 32))
    got, cell, score = ctx.exact_scores(sc.radar, sc.tx, sc.rx, to_dev(torch_cuda, Y32), sub)
    got = got.cpu().numpy()
    rng = np.random.default_rng(7)
    xy = [(int(a), int(b)) for a, b in zip(rng.integers(0, 64, 200), rng.integers(0, 64, 200))]
    ci = np.unravel_index(cell, sub.n)
    xy.append((int(ci[0]), int(ci[1])))
    ref = direct.factored(Y, sc.radar, sc.tx, sc.rx, sub, xy)
    g = np.stack([got[a, b] for a, b in xy])
    smax = max(ref.max(), float(score))
    err = np.abs(g - ref).max() / smax
    assert err < TOL, err
    print(f"precision exact sub-grid: max |score error| / max S = {err:.2e}")
