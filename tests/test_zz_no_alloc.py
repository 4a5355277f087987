"""gh_score_grid_noalloc, the allocation-free entry point for callers that
must not allocate device memory (a real-time frame loop with a per-frame
deadline, or a plug-in inside a framework that owns the device memory
budget). It must give the scores and argmax of gh_score_grid, also when a
second call finds the first call's data in the shared fixed scratch array.

Collected last on purpose: it runs after every other GPU test, and it also
passes alone in a fresh process (its first call sets up the scratch address)."""
import numpy as np
import pytest

from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_noalloc_matches_score_grid_on_two_calls_in_a_row(ctx, torch_cuda):
    stream = torch_cuda.cuda.current_stream()
    for sc in (scenes.paper_frame(3), scenes.tiny_scene(2)):
        Y32, _ = measurement64(sc)
        maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
        ref, ref_cell, ref_score = ctx.scores(sc.radar, sc.tx, sc.rx, maps, sc.grid)
        got = torch_cuda.full(tuple(sc.grid.n), -1.0, dtype=torch_cuda.float32, device="cuda:0")
        cell, score = gh.gh_score_grid_noalloc(stream, sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, got)
        assert rel_err(got.cpu().numpy(), ref.cpu().numpy()) < TOL
        assert cell == ref_cell
        assert score == pytest.approx(ref_score, rel=TOL)
        # argmax only (no score output)
        cell2, score2 = gh.gh_score_grid_noalloc(stream, sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, None)
        assert (cell2, score2) == (cell, score)


def test_noalloc_rejects_problems_beyond_its_scratch(ctx, torch_cuda):
    sc = scenes.tiny_scene(1)
    maps = torch_cuda.zeros((3, 256, 128), dtype=torch_cuda.complex64, device="cuda:0")
    big = scenes.Grid((0, 0, -1, -1), (0.1, 0.1, 1, 1), (256, 256, 2, 2))  # 256*256*3 > limit
    with pytest.raises(gh.GhError) as e:
        gh.gh_score_grid_noalloc(None, sc.radar, sc.tx, sc.rx, 3, maps, big, None)
    assert e.value.status == gh.GH_EINVAL


def test_warm_noalloc_call_leaves_free_device_memory_unchanged(ctx, torch_cuda):
    """After a first call (which may load the kernels' code on the device),
    further calls take no device memory: the device's free memory is the same
    before and after them."""
    stream = torch_cuda.cuda.current_stream()
    sc = scenes.paper_frame(2)
    Y32, _ = measurement64(sc)
    maps = ctx.maps(sc.radar, to_dev(torch_cuda, Y32))
    out = torch_cuda.empty(tuple(sc.grid.n), dtype=torch_cuda.float32, device="cuda:0")
    first = gh.gh_score_grid_noalloc(stream, sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, out)
    torch_cuda.cuda.synchronize()
    free0, _ = torch_cuda.cuda.mem_get_info()
    for _ in range(3):
        assert gh.gh_score_grid_noalloc(stream, sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, out) == first
        assert gh.gh_score_grid_noalloc(stream, sc.radar, sc.tx, sc.rx, sc.Q, maps, sc.grid, None) == first
    torch_cuda.cuda.synchronize()
    free1, _ = torch_cuda.cuda.mem_get_info()
    assert free1 == free0
