"""Failure paths of the four entry points, by host-side fault injection
(gh_inject_fault; nothing faults on the GPU): each call returns the injected
status (out of memory at a workspace acquisition, a failed launch check, a
device wait that gave up), and the next call on the same context succeeds
with the results of a clean call."""
import numpy as np
import pytest

from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame(torch_cuda):
    sc = scenes.tiny_scene(3)
    Y32, _ = measurement64(sc)
    return sc, Y32, to_dev(torch_cuda, Y32)


def _calls(ctx, torch, sc, Y32, Yd):
    """Each entry point as a function returning its results as numpy data."""
    def make_maps():
        return ctx.maps(sc.radar, Yd).cpu().numpy()

    maps = ctx.maps(sc.radar, Yd)

    def score_grid():
        S, cell, score = ctx.scores(sc.radar, sc.tx, sc.rx, maps, sc.grid)
        return S.cpu().numpy(), cell, score

    def direct_exact():
        S, cell, score = ctx.exact_scores(sc.radar, sc.tx, sc.rx, Yd, sc.grid)
        return S.cpu().numpy(), cell, score

    def detect_hop():
        return ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, 2)

    def detect_exact_host():
        return ctx.gh_detect(gh.GH_EXACT, sc.radar, sc.tx, sc.rx, sc.Q, Y32, sc.grid, 2)

    return {"make_maps": make_maps, "score_grid": score_grid, "direct_exact": direct_exact,
            "detect_hop": detect_hop, "detect_exact_host": detect_exact_host}


def _same(a, b):
    if isinstance(a, tuple):
        assert len(a) == len(b)
        for x, y in zip(a, b):
            _same(x, y)
    else:
        np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("name", ["make_maps", "score_grid", "direct_exact", "detect_hop", "detect_exact_host"])
@pytest.mark.parametrize("status", [gh.GH_ENOMEM, gh.GH_ECUDA, gh.GH_ETIMEOUT])
@pytest.mark.parametrize("after", [0, 1])
def test_injected_fault_is_reported_and_the_context_recovers(ctx, torch_cuda, frame, name, status, after):
    if name == "make_maps" and status == gh.GH_ETIMEOUT:
        pytest.skip("gh_make_maps reads no device status word")
    sc, Y32, Yd = frame
    call = _calls(ctx, torch_cuda, sc, Y32, Yd)[name]
    ctx.gh_set_graphs(False)  # every call runs its launch sequence (graph replays: next test)
    try:
        ref = call()
        if status == gh.GH_ETIMEOUT and after > 0:
            after = 0  # one status read per call
        ctx.gh_inject_fault(status, after)
        with pytest.raises(gh.GhError) as e:
            call()
        assert e.value.status == status
        assert "injected fault" in str(e.value) or status == gh.GH_ETIMEOUT
        _same(call(), ref)   # the same context works again, same results
        _same(call(), ref)
    finally:
        ctx.gh_inject_fault(gh.GH_OK, 0)
        ctx.gh_set_graphs(True)


def test_fault_during_graph_recording(ctx, torch_cuda, frame):
    """gh_detect records its CUDA graph on the second call with a
    configuration: a fault there discards the recording; the following
    calls record and replay it with unchanged results."""
    sc, Y32, Yd = frame
    for K, status in ((3, gh.GH_ECUDA), (2, gh.GH_ENOMEM), (1, gh.GH_ETIMEOUT)):
        det = lambda: ctx.gh_detect(gh.GH_HOP, sc.radar, sc.tx, sc.rx, sc.Q, Yd, sc.grid, K)
        ctx.gh_set_graphs(False)
        ref = det()
        ctx.gh_set_graphs(True)
        det()                                                      # first sight of the configuration
        ctx.gh_inject_fault(status, 0 if status == gh.GH_ETIMEOUT else 4)  # fires in the recording call
        with pytest.raises(gh.GhError) as e:
            det()
        assert e.value.status == status
        for _ in range(3):                                         # recorded (again) and replayed
            _same(det(), ref)


def test_disarm(ctx, torch_cuda, frame):
    sc, Y32, Yd = frame
    ctx.gh_inject_fault(gh.GH_ECUDA, 0)
    ctx.gh_inject_fault(gh.GH_OK, 0)
    ctx.maps(sc.radar, Yd)
    with pytest.raises(gh.GhError) as e:
        ctx.gh_inject_fault(gh.GH_EINVAL, 0)
    assert e.value.status == gh.GH_EINVAL
