"""Tensor-core plumbing of the exact direct path (tcgen05.mma, shared-memory
descriptors in both operand layouts, tensor-memory accumulators) against a
float64 matrix product, and the bounded completion wait that gives up."""
import numpy as np
import pytest

from paper_2307_16550_gb300 import gh

pytestmark = pytest.mark.gpu


def _operands(N, K):
    rng = np.random.default_rng(N * 1000 + K)
    # small integers / 8 are exact in BF16; products and sums are exact in FP32
    A = (rng.integers(-16, 17, size=(128, K)) / 8.0).astype(np.float32)
    B = (rng.integers(-16, 17, size=(N, K)) / 8.0).astype(np.float32)
    return A, B, A.astype(np.float64) @ B.astype(np.float64).T


@pytest.mark.parametrize("N,K", [(32, 16), (64, 64), (128, 32), (256, 256), (64, 256)])
def test_tcgen05_gemm_matches_float64(ctx, N, K):
    A, B, ref = _operands(N, K)
    np.testing.assert_array_equal(ctx.gh_selftest_tcgen05(A, B), ref)


@pytest.mark.parametrize("N,K", [(32, 64), (128, 64), (64, 128), (128, 128), (256, 64)])
def test_tcgen05_gemm_swizzled_layout(ctx, N, K):
    """Operands in the 128-byte swizzled K-major layout (the exact path's
    tensor-core kernels): the same exact product."""
    A, B, ref = _operands(N, K)
    np.testing.assert_array_equal(ctx.gh_selftest_tcgen05_ex(A, B, gh.GH_TC_SW128), ref)


def test_bounded_wait_gives_up_and_context_survives(ctx):
    """No MMA is issued, so nothing arrives on the completion barrier: the
    kernel's bounded wait runs out, it frees its tensor memory and the call
    returns GH_ETIMEOUT; the next calls on the same context succeed."""
    A, B, ref = _operands(64, 64)
    for _ in range(2):
        with pytest.raises(gh.GhError) as e:
            ctx.gh_selftest_tcgen05_ex(A, B, gh.GH_TC_SW128, gh.GH_TC_SKIP_MMA, 1000)
        assert e.value.status == gh.GH_ETIMEOUT
        np.testing.assert_array_equal(ctx.gh_selftest_tcgen05_ex(A, B, gh.GH_TC_SW128), ref)
        np.testing.assert_array_equal(ctx.gh_selftest_tcgen05(A, B), ref)
