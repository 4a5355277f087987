// Self-test of the tensor-core plumbing used by the exact direct path:
// D = A * B^T for M = 128, one CTA, BF16 operands in shared memory (K-major,
// no-swizzle or 128-byte-swizzled layout), FP32 accumulation in tensor memory,
// mbarrier completion, and the bounded wait that gives up with GH_ETIMEOUT.
#include "gh_internal.cuh"
#include "gh_tc.cuh"

namespace {

constexpr uint32_t kWaitIters = 1u << 22;
constexpr size_t kSw128Margin = 32 << 10;  // zeroed bytes after the swizzled tiles

// layout 0: no swizzle; 1: 128-byte swizzle. skip_mma: no MMA and no commit
// are issued, so nothing ever arrives on the barrier and the bounded wait
// (wait_iters polls) runs out; the kernel then reports GH_ETIMEOUT and frees
// its tensor memory like every tensor-core kernel of the library.
__global__ void __launch_bounds__(128) tc_selftest_kernel(const float* __restrict__ A, const float* __restrict__ B,
                                                          float* __restrict__ D, int N, int K, int layout,
                                                          int skip_mma, uint32_t wait_iters, int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lboA = (128 / 8) * 128, lboB = (uint32_t)(N / 8) * 128, sbo = 128;
    const size_t tileA = (size_t)128 * K * 2, tileB = (size_t)N * K * 2;
    unsigned char* sA = smem;
    unsigned char* sB = smem + tileA;
    auto offA = [&](int r, int k) {
        return layout == 1 ? gh_tc::sw128_off(r, k, 128) : gh_tc::kmajor_off(r, k, lboA, sbo);
    };
    auto offB = [&](int r, int k) {
        return layout == 1 ? gh_tc::sw128_off(r, k, (uint32_t)N) : gh_tc::kmajor_off(r, k, lboB, sbo);
    };
    if (layout == 1)
        for (size_t i = tileA + tileB + tid; i < tileA + tileB + kSw128Margin; i += blockDim.x) smem[i] = 0;
    for (int idx = tid; idx < 128 * K; idx += blockDim.x) {
        const int r = idx / K, k = idx % K;
        *(__nv_bfloat16*)(sA + offA(r, k)) = __float2bfloat16_rn(A[idx]);
    }
    for (int idx = tid; idx < N * K; idx += blockDim.x) {
        const int r = idx / K, k = idx % K;
        *(__nv_bfloat16*)(sB + offB(r, k)) = __float2bfloat16_rn(B[idx]);
    }
    gh_tc::fence_smem_to_async();
    if (tid == 0) {
        gh_tc::mbar_init(&bar, 1);
        gh_tc::mbar_fence_init();
    }
    if (warp == 0) gh_tc::tmem_alloc(&tmem_holder, 256);
    gh_tc::fence_before_sync();
    __syncthreads();
    gh_tc::fence_after_sync();
    const uint32_t tmem = tmem_holder;
    if (tid == 0 && !skip_mma) {
        const uint32_t idesc = gh_tc::idesc_bf16_f32(128, (uint32_t)N);
        const uint32_t a0 = gh_tc::smem_u32(sA), b0 = gh_tc::smem_u32(sB);
        for (int kk = 0; kk < K / 16; ++kk) {
            uint64_t ad, bd;
            if (layout == 1) {
                // K block kk / 4 of the tile, 32 bytes per K = 16 step inside a row
                ad = gh_tc::smem_desc_sw128(a0 + (uint32_t)(kk >> 2) * 128 * 128 + (uint32_t)(kk & 3) * 32);
                bd = gh_tc::smem_desc_sw128(b0 + (uint32_t)(kk >> 2) * (uint32_t)N * 128 + (uint32_t)(kk & 3) * 32);
            } else {
                ad = gh_tc::smem_desc(a0 + 2 * kk * lboA, lboA, sbo);
                bd = gh_tc::smem_desc(b0 + 2 * kk * lboB, lboB, sbo);
            }
            gh_tc::mma_bf16(tmem, ad, bd, idesc, kk > 0);
        }
        gh_tc::mma_commit(&bar);
    }
    const bool ok = gh_tc::mbar_wait_bounded(&bar, 0, wait_iters);
    if (!ok && lane == 0) atomicExch(status, GH_ETIMEOUT);
    gh_tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            gh_tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            const int row = 32 * warp + lane;
            for (int i = 0; i < 32 && c0 + i < N; ++i) D[(size_t)row * N + c0 + i] = v[i];
        }
    }
    gh_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gh_tc::tmem_dealloc(tmem, 256);
}

}  // namespace

extern "C" int gh_selftest_tcgen05_ex(gh_ctx* ctx, const float* A_host, const float* B_host, float* D_host,
                                      int32_t N, int32_t K, int32_t layout, int32_t flags, int32_t wait_polls) {
    if (!ctx) return GH_EINVAL;
    if (!A_host || !B_host || !D_host) return gh_fail(ctx, GH_EINVAL, "NULL argument");
    if (N < 32 || N > 256 || N % 32 != 0 || K < 16 || K > 256 || K % 16 != 0)
        return gh_fail(ctx, GH_EINVAL, "N must be a multiple of 32 in [32, 256], K a multiple of 16 in [16, 256]");
    if (layout != GH_TC_NOSWIZZLE && layout != GH_TC_SW128) return gh_fail(ctx, GH_EINVAL, "unknown layout %d", layout);
    if (layout == GH_TC_SW128 && K % 64 != 0)
        return gh_fail(ctx, GH_EINVAL, "the 128-byte swizzled layout needs K a multiple of 64");
    if ((flags & ~GH_TC_SKIP_MMA) != 0 || wait_polls < 0) return gh_fail(ctx, GH_EINVAL, "bad flags or wait limit");
    cudaSetDevice(ctx->device);
    const size_t a = (size_t)128 * K, b = (size_t)N * K, dsz = (size_t)128 * N;
    const size_t smem = (a + b) * 2 + (layout == GH_TC_SW128 ? kSw128Margin : 0);
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "self-test needs %zu B of shared memory", smem);
    void* buf;
    GH_TRY(gh_ws(ctx, WS_DIAG, (a + b + dsz) * sizeof(float) + 256, &buf));
    float* dA = (float*)buf;
    float* dB = dA + a;
    float* dD = dB + b;
    int* status = (int*)(dD + dsz);
    GH_CUDA(cudaMemcpyAsync(dA, A_host, a * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    GH_CUDA(cudaMemcpyAsync(dB, B_host, b * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    GH_CUDA(cudaMemsetAsync(status, 0, sizeof(int), ctx->stream));
    GH_CUDA(cudaMemsetAsync(dD, 0, dsz * sizeof(float), ctx->stream));
    GH_CUDA(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_EXACT_S2, &ev);
    tc_selftest_kernel<<<1, 128, smem, ctx->stream>>>(dA, dB, dD, N, K, layout, flags & GH_TC_SKIP_MMA,
                                                      wait_polls > 0 ? (uint32_t)wait_polls : kWaitIters, status);
    GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S2, ev, "tc_selftest_kernel"));
    int st = 0;
    GH_CUDA(cudaMemcpyAsync(D_host, dD, dsz * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    if (st != 0) return gh_fail(ctx, GH_ETIMEOUT, "tensor-core self-test: mbarrier wait timed out");
    return GH_OK;
}

extern "C" int gh_selftest_tcgen05(gh_ctx* ctx, const float* A_host, const float* B_host, float* D_host, int32_t N,
                                   int32_t K) {
    return gh_selftest_tcgen05_ex(ctx, A_host, B_host, D_host, N, K, GH_TC_NOSWIZZLE, 0, 0);
}

// ---------------------------------------------------------------------------
// Read-bandwidth probe: every thread streams 16-byte loads over a buffer of
// `bytes` bytes, `reps` times; a buffer much smaller than L2 measures the
// L2-to-SM bandwidth, a buffer much larger measures DRAM read bandwidth.
// ---------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(512) probe_read_kernel(const float4* __restrict__ buf, long long n4, int reps,
                                                         float* __restrict__ sink) {
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long j = i + u * stride;
                v[u] = j < n4 ? __ldcg(buf + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) acc += v[u].x + v[u].y + v[u].z + v[u].w;
        }
    }
    if (acc == 1.234567e-30f) sink[0] = acc;  // keeps the loads alive
}
}  // namespace

extern "C" int gh_probe_read_bandwidth(gh_ctx* ctx, int64_t bytes, int32_t reps, double* gbs) {
    if (!ctx || !gbs) return GH_EINVAL;
    if (bytes < (1 << 20) || bytes > ((int64_t)64 << 30) || reps < 1 || reps > 1000)
        return gh_fail(ctx, GH_EINVAL, "bytes must be in [1 MiB, 64 GiB], reps in [1, 1000]");
    cudaSetDevice(ctx->device);
    void* buf;
    GH_TRY(gh_ws(ctx, WS_DIAG, (size_t)bytes + 256, &buf));
    GH_CUDA(cudaMemsetAsync(buf, 0, (size_t)bytes + 256, ctx->stream));
    const long long n4 = bytes / 16;
    float* sink = (float*)((char*)buf + bytes);
    const unsigned blocks = (unsigned)ctx->num_sms * 4;
    probe_read_kernel<<<blocks, 512, 0, ctx->stream>>>((const float4*)buf, n4, 1, sink);  // warm
    GH_CUDA(cudaGetLastError());
    cudaEvent_t a, b;
    GH_CUDA(cudaEventCreate(&a));
    GH_CUDA(cudaEventCreate(&b));
    GH_CUDA(cudaEventRecord(a, ctx->stream));
    probe_read_kernel<<<blocks, 512, 0, ctx->stream>>>((const float4*)buf, n4, reps, sink);
    GH_CUDA(cudaGetLastError());
    GH_CUDA(cudaEventRecord(b, ctx->stream));
    GH_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    GH_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    *gbs = (double)(n4 * 16) * reps / (ms * 1e-3) / 1e9;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// Shared-memory load bandwidth and instruction issue rate probes (the limits
// of the hopping scorer's power-row reads and of its instruction stream).
// ---------------------------------------------------------------------------
namespace {
// Every warp reads its own 1 KiB of shared memory with conflict-free 16-byte
// loads (512 contiguous bytes per instruction), `iters` times.
__global__ void __launch_bounds__(1024) probe_smem_kernel(int iters, float* __restrict__ sink) {
    __shared__ __align__(16) float4 buf[32 * 64];  // 32 warps x 1 KiB
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* w = buf + warp * 64;
    for (int i = lane; i < 64; i += 32) w[i] = make_float4(i, lane, warp, 1.f);
    __syncwarp();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 v = w[(j * 8 + lane + it) & 63];  // eight distinct blocks per iteration
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    }
    if (acc.x == 1.234567e-30f) sink[0] = acc.x + acc.y + acc.z + acc.w;
}

// Eight independent FMA chains per thread: the instruction stream never
// waits on a result, so the SM issues at its maximum rate.
__global__ void __launch_bounds__(1024) probe_issue_kernel(int iters, float* __restrict__ sink) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 1e-3f + j;
    const float m = 0.999f, c = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], m, c);
    }
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) t += a[j];
    if (t == 1.234567e-30f) sink[0] = t;
}
}  // namespace

static int probe_time(gh_ctx* ctx, void (*launch)(gh_ctx*, int, float*), int iters, float* sink, double* ms_out) {
    launch(ctx, 16, sink);  // warm
    GH_CUDA(cudaGetLastError());
    cudaEvent_t a, b;
    GH_CUDA(cudaEventCreate(&a));
    GH_CUDA(cudaEventCreate(&b));
    GH_CUDA(cudaEventRecord(a, ctx->stream));
    launch(ctx, iters, sink);
    GH_CUDA(cudaGetLastError());
    GH_CUDA(cudaEventRecord(b, ctx->stream));
    GH_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    GH_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    *ms_out = ms;
    return GH_OK;
}

extern "C" int gh_probe_smem_bandwidth(gh_ctx* ctx, double* gbs) {
    if (!ctx || !gbs) return GH_EINVAL;
    DeviceGuard g(ctx->device);
    void* buf;
    GH_TRY(gh_ws(ctx, WS_DIAG, 256, &buf));
    const int iters = 4096;
    auto launch = [](gh_ctx* c, int it, float* sink) {
        probe_smem_kernel<<<(unsigned)c->num_sms * 2, 1024, 0, c->stream>>>(it, sink);
    };
    double ms;
    GH_TRY(probe_time(ctx, launch, iters, (float*)buf, &ms));
    const double bytes = (double)ctx->num_sms * 2 * 1024 * 16.0 * 8 * iters;
    *gbs = bytes / (ms * 1e-3) / 1e9;
    return GH_OK;
}

extern "C" int gh_probe_issue_rate(gh_ctx* ctx, double* warp_inst_per_s) {
    if (!ctx || !warp_inst_per_s) return GH_EINVAL;
    DeviceGuard g(ctx->device);
    void* buf;
    GH_TRY(gh_ws(ctx, WS_DIAG, 256, &buf));
    const int iters = 16384;
    auto launch = [](gh_ctx* c, int it, float* sink) {
        probe_issue_kernel<<<(unsigned)c->num_sms * 2, 1024, 0, c->stream>>>(it, sink);
    };
    double ms;
    GH_TRY(probe_time(ctx, launch, iters, (float*)buf, &ms));
    // FMAs only (the loop's own instructions are a small extra, not counted)
    const double warp_inst = (double)ctx->num_sms * 2 * (1024 / 32) * 8.0 * iters;
    *warp_inst_per_s = warp_inst / (ms * 1e-3);
    return GH_OK;
}
