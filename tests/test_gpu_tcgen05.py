"""Tensor-core plumbing of the exact direct path (tcgen05.mma, shared-memory
descriptors, tensor-memory accumulators) against a float64 matrix product."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K", [(32, 16), (64, 64), (128, 32), (256, 256), (64, 256)])
def test_tcgen05_gemm_matches_float64(ctx, N, K):
    rng = np.random.default_rng(N * 1000 + K)
    # small integers / 8 are exact in BF16; products and sums are exact in FP32
    A = (rng.integers(-16, 17, size=(128, K)) / 8.0).astype(np.float32)
    B = (rng.integers(-16, 17, size=(N, K)) / 8.0).astype(np.float32)
    D = ctx.gh_selftest_tcgen05(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    np.testing.assert_array_equal(D, ref)
