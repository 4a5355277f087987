"""gh_detect through its CUDA graph: the second call with an unchanged
configuration records the launch sequence and later calls replay it. Replays
must give the results of the eager path on whatever the measurement buffer
holds at the time, keep the launch count and the per-kernel timers right,
and survive a workspace reallocation between calls (which drops the graph)."""
import numpy as np
import pytest

from paper_2307_16550_gb300 import gh, scenes
from tests.helpers import measurement64, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture()
def gctx(torch_cuda):
    from paper_2307_16550_gb300 import build
    build.build()
    c = gh.Context(0)
    yield c
    c.close()


def _detect(c, method, sc, Y, K):
    return c.gh_detect(method, sc.radar, sc.tx, sc.rx, sc.Q, Y, sc.grid, K)


def _same(got, ref):
    """Same kernels on the same data: same cells, scores and amplitudes."""
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_allclose(got[1], ref[1], rtol=1e-6)
    np.testing.assert_allclose(got[2], ref[2], rtol=0, atol=1e-6 * np.abs(ref[2]).max())


@pytest.mark.parametrize("method", [gh.GH_HOP, gh.GH_EXACT])
def test_replay_follows_buffer_contents(gctx, ctx, torch_cuda, method):
    sc = scenes.tiny_scene(2)
    frames = []
    for seed in (2, 5, 7, 9):
        s = scenes.tiny_scene(seed)  # same geometry, new targets and noise
        s.tx[:], s.rx[:] = sc.tx, sc.rx
        frames.append(measurement64(s))
    Yd = to_dev(torch_cuda, frames[0][0])
    ctx.gh_set_graphs(False)
    try:
        for i, (Y32, Y) in enumerate(frames):
            Yd.copy_(to_dev(torch_cuda, Y32))  # same address, new frame
            n0 = gctx.gh_launch_count()
            got = _detect(gctx, method, sc, Yd, 2)
            n1 = gctx.gh_launch_count()
            ref = _detect(ctx, method, sc, to_dev(torch_cuda, Y32), 2)
            _same(got, ref)
            if i == 0:
                per_call = n1 - n0
            assert n1 - n0 == per_call  # replays count their kernels too
    finally:
        ctx.gh_set_graphs(True)


def test_pinned_host_measurement_replays(gctx, torch_cuda):
    sc = scenes.tiny_scene(3)
    Y32, Y = measurement64(sc)
    host = torch_cuda.from_numpy(Y32.copy()).pin_memory()
    eager = gh.Context(0)
    eager.gh_set_graphs(False)
    try:
        ref = _detect(eager, gh.GH_HOP, sc, Y32, 3)
        for _ in range(3):
            got = _detect(gctx, gh.GH_HOP, sc, host, 3)
            _same(got, ref)
        # a new frame written into the same pinned buffer
        s2 = scenes.tiny_scene(11)
        s2.tx[:], s2.rx[:] = sc.tx, sc.rx
        Y32b, _ = measurement64(s2)
        host.copy_(torch_cuda.from_numpy(Y32b))
        got = _detect(gctx, gh.GH_HOP, sc, host, 3)
        ref = _detect(eager, gh.GH_HOP, sc, Y32b, 3)
        _same(got, ref)
    finally:
        eager.close()


def test_timers_and_invalidation(gctx, torch_cuda):
    sc = scenes.tiny_scene(4)
    Y32, _ = measurement64(sc)
    Yd = to_dev(torch_cuda, Y32)
    gctx.gh_set_timing(True)
    ref = _detect(gctx, gh.GH_HOP, sc, Yd, 2)  # eager
    _detect(gctx, gh.GH_HOP, sc, Yd, 2)  # recorded
    gctx.gh_reset_stats()
    for _ in range(3):  # replayed
        got = _detect(gctx, gh.GH_HOP, sc, Yd, 2)
        np.testing.assert_array_equal(got[0], ref[0])
    ms, n = gctx.gh_kernel_stats("hop_score")
    assert n == 3 * 2 and ms > 0
    # a larger problem in between grows the workspace and drops the graph
    big = scenes.paper_frame(1)
    Yb32, _ = measurement64(big)
    gctx.gh_set_timing(False)
    _detect(gctx, gh.GH_HOP, big, to_dev(torch_cuda, Yb32), 1)
    for _ in range(3):
        got = _detect(gctx, gh.GH_HOP, sc, Yd, 2)
        _same(got, ref)
    # turning graphs off keeps the results
    gctx.gh_set_graphs(False)
    got = _detect(gctx, gh.GH_HOP, sc, Yd, 2)
    _same(got, ref)
