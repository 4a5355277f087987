// Exact direct decision function (Sec. III; the joint location-velocity form
// behind Eqs. 3-4):
//   S(x, v) = sum_q | sum_mc conj(b_mc(u_q)) P_q[x][mc] |^2,
//   P_q[x][mc] = sum_m Y_q[mc][m] conj(a_m(r_q(x)))          (stage 1, Eq. 4's g_q)
// with the Doppler atom split over the two velocity axes,
//   conj(b_mc(u_q)) = exp(-j 2 pi k wx vx mc) exp(-j 2 pi k wy vy mc), k = f0 Tc / c.
//
// Stage 1 is a complex GEMM per receiver, (nxy x Ms) atoms times Y_q^T
// (Ms x Mc). Stage 2 is, per (x, y, q), the product of an nvx x Mc matrix Ex
// with an Mc x nvy matrix diag(P) Ey^T, squared and summed over q.
// All atoms are generated on the fly from float64 phases reduced to 64-bit
// fixed point (exact modulo one cycle) and a float32 sincos.
#include <math.h>

#include "gh_internal.cuh"
#include "gh_tc.cuh"

namespace {

constexpr int S1_XT = 32;   // xy cells per stage-1 CTA
constexpr int S1_MT = 64;   // chirps per stage-1 CTA
constexpr int S1_KT = 32;   // samples per k-step

__global__ void __launch_bounds__(256) exact_stage1_kernel(const float2* __restrict__ Y, GeoParams g,
                                                           float2* __restrict__ P) {
    __shared__ float2 As[S1_XT][S1_KT + 1];
    __shared__ float2 Bs[S1_MT][S1_KT + 1];
    __shared__ unsigned long long rfix[S1_XT];
    const int q = blockIdx.z;
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long xy0 = (long long)blockIdx.x * S1_XT;
    const int mc0 = blockIdx.y * S1_MT;
    const int tid = threadIdx.x;
    if (tid < S1_XT) {
        const long long xy = xy0 + tid;
        unsigned long long f = 0;
        if (xy < nxy) {
            const int ix = (int)(xy / g.n[1]);
            const int iy = (int)(xy - (long long)ix * g.n[1]);
            double d, wx, wy;
            gh_bistatic(g, q, gh_axis(g.lo[0], g.step[0], ix), gh_axis(g.lo[1], g.step[1], iy), &d, &wx, &wy);
            f = gh_phase_fix(gh_range(g, d));
        }
        rfix[tid] = f;
    }
    // thread tile: 2 xy x 4 chirps
    const int tx = tid & 15;   // chirp group: mc = mc0 + tx + 16*j
    const int ty = tid >> 4;   // xy pair: xy = 2*ty + i
    float2 acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    const float2* Yq = Y + (size_t)q * g.Mc * g.Ms;
    __syncthreads();
    for (int m0 = 0; m0 < g.Ms; m0 += S1_KT) {
        for (int idx = tid; idx < S1_XT * S1_KT; idx += 256) {
            const int xi = idx / S1_KT, k = idx - xi * S1_KT;
            const float2 a = gh_cis_fix(rfix[xi] * (unsigned long long)(m0 + k));
            As[xi][k] = make_float2(a.x, -a.y);  // conj(a_m(r))
        }
        for (int idx = tid; idx < S1_MT * S1_KT; idx += 256) {
            const int mi = idx / S1_KT, k = idx - mi * S1_KT;
            const int mc = mc0 + mi, m = m0 + k;
            Bs[mi][k] = (mc < g.Mc && m < g.Ms) ? Yq[(size_t)mc * g.Ms + m] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < S1_KT; ++k) {
            const float2 a0 = As[2 * ty][k], a1 = As[2 * ty + 1][k];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 b = Bs[tx + 16 * j][k];
                acc[0][j].x += a0.x * b.x - a0.y * b.y;
                acc[0][j].y += a0.x * b.y + a0.y * b.x;
                acc[1][j].x += a1.x * b.x - a1.y * b.y;
                acc[1][j].y += a1.x * b.y + a1.y * b.x;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const long long xy = xy0 + 2 * ty + i;
        if (xy >= nxy) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int mc = mc0 + tx + 16 * j;
            if (mc < g.Mc) P[((size_t)q * nxy + xy) * g.Mc + mc] = acc[i][j];
        }
    }
}

__device__ __forceinline__ void better(float s, long long c, float& bs, long long& bc) {
    if (s > bs || (s == bs && c < bc)) {
        bs = s;
        bc = c;
    }
}

constexpr int S2_MCC = 64;  // chirps per stage-2 chunk

// One CTA per (x, y) cell; CPT velocity cells per thread.
template <int CPT>
__global__ void __launch_bounds__(256) exact_stage2_kernel(const float2* __restrict__ P, GeoParams g,
                                                           float* __restrict__ scores,
                                                           const int64_t* __restrict__ mask, int nmask,
                                                           ArgPartial* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nvx = g.n[2], nvy = g.n[3];
    float2* Ex = (float2*)smem_raw;            // [nvx][S2_MCC]
    float2* Ey = Ex + (size_t)nvx * S2_MCC;    // [nvy][S2_MCC]
    unsigned long long* phx = (unsigned long long*)(Ey + (size_t)nvy * S2_MCC);  // [nvx]
    unsigned long long* phy = phx + nvx;                                          // [nvy]
    __shared__ float s_bs[8];
    __shared__ long long s_bc[8];
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long xy = blockIdx.x;
    const int tid = threadIdx.x;
    const int nv = nvx * nvy;
    const int ix = (int)(xy / g.n[1]);
    const int iy = (int)(xy - (long long)ix * g.n[1]);
    const double x = gh_axis(g.lo[0], g.step[0], ix), y = gh_axis(g.lo[1], g.step[1], iy);

    float acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = 0.f;

    for (int q = 0; q < g.Q; ++q) {
        double d, wx, wy;
        gh_bistatic(g, q, x, y, &d, &wx, &wy);
        __syncthreads();  // previous q's tables are no longer read
        for (int a = tid; a < nvx; a += blockDim.x)
            phx[a] = gh_phase_fix(g.kappa * wx * gh_axis(g.lo[2], g.step[2], a));
        for (int b = tid; b < nvy; b += blockDim.x)
            phy[b] = gh_phase_fix(g.kappa * wy * gh_axis(g.lo[3], g.step[3], b));
        float2 F[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) F[c] = make_float2(0.f, 0.f);
        const float2* Pq = P + ((size_t)q * nxy + xy) * g.Mc;
        for (int mc0 = 0; mc0 < g.Mc; mc0 += S2_MCC) {
            __syncthreads();
            for (int idx = tid; idx < nvx * S2_MCC; idx += blockDim.x) {
                const int a = idx / S2_MCC, k = idx - a * S2_MCC;
                const float2 e = gh_cis_fix(phx[a] * (unsigned long long)(mc0 + k));
                Ex[idx] = make_float2(e.x, -e.y);
            }
            for (int idx = tid; idx < nvy * S2_MCC; idx += blockDim.x) {
                const int b = idx / S2_MCC, k = idx - b * S2_MCC;
                const int mc = mc0 + k;
                const float2 pv = mc < g.Mc ? Pq[mc] : make_float2(0.f, 0.f);
                const float2 e = gh_cis_fix(phy[b] * (unsigned long long)mc);
                Ey[idx] = cmulc(pv, e);  // P[mc] * conj(e)
            }
            __syncthreads();
            const int kmax = min(S2_MCC, g.Mc - mc0);
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const int cell = tid + c * 256;
                if (cell < nv) {
                    const int a = cell / nvy, b = cell - a * nvy;
                    const float2* ex = Ex + (size_t)a * S2_MCC;
                    const float2* ey = Ey + (size_t)b * S2_MCC;
                    float2 f = F[c];
                    for (int k = 0; k < kmax; ++k) {
                        const float2 u = ex[k], w = ey[k];
                        f.x += u.x * w.x - u.y * w.y;
                        f.y += u.x * w.y + u.y * w.x;
                    }
                    F[c] = f;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[c] += F[c].x * F[c].x + F[c].y * F[c].y;
    }

    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    bool hm = false;
    for (int m = 0; m < nmask; ++m) hm |= (mask[m] / nv == xy);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const int cell = tid + c * 256;
        if (cell < nv) {
            const long long gc = xy * nv + cell;
            if (scores) scores[gc] = acc[c];
            bool masked = false;
            if (hm)
                for (int m = 0; m < nmask; ++m) masked |= (mask[m] == gc);
            if (!masked) better(acc[c], gc, best, bestc);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, best, off);
        const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
        better(os, oc, best, bestc);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) {
        s_bs[warp] = best;
        s_bc[warp] = bestc;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < 8; ++w) better(s_bs[w], s_bc[w], best, bestc);
        parts[xy].score = best;
        parts[xy].cell = bestc;
    }
}

template <int CPT>
int launch_s2(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* P, float* scores, const int64_t* mask,
              int nmask, ArgPartial* parts) {
    const size_t smem = (size_t)(d.nvx + d.nvy) * S2_MCC * sizeof(float2) + (size_t)(d.nvx + d.nvy) * 8;
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "exact stage 2 needs %zu B shared memory", smem);
    GH_CUDA(cudaFuncSetAttribute(exact_stage2_kernel<CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_EXACT_S2, &ev);
    exact_stage2_kernel<CPT><<<(unsigned)d.nxy, 256, smem, ctx->stream>>>(P, g, scores, mask, nmask, parts);
    return gh_launch_end(ctx, GH_K_EXACT_S2, ev, "exact_stage2_kernel");
}

// ---------------------------------------------------------------------------
// Stage 2 on the tensor cores (tcgen05).
//
// Per (x, y, q) the Doppler correlation F[a][b] = sum_mc Ex[a][mc] G[b][mc],
// Ex[a][mc] = exp(-j 2 pi phx_a mc), G[b][mc] = P[mc] exp(-j 2 pi phy_b mc), is
// a complex (nvx x Mc) x (Mc x nvy) product. It is written as one real GEMM
// D = A B^T: row 2a of A holds [Re Ex | -Im Ex], row 2a+1 holds [Im Ex | Re Ex],
// row b of B holds [Re G | Im G] (K = 2 Mc), so D[2a][b] = Re F, D[2a+1][b] = Im F.
// Two receivers' problems share one M = 128 MMA (rows 0-63 and 64-127, their B
// rows side by side in N = 2 * nvy_pad; the cross blocks are discarded).
// Operands are split into BF16 high and low parts and three MMAs per K step
// (hi*hi + hi*lo + lo*hi) accumulate in FP32 in tensor memory.
// The K loop runs over stages of 32 chirps (K = 64 per stage): the 128 threads
// write a stage's operands to shared memory while the tensor core consumes the
// previous stage (two buffers, completion through mbarriers, bounded waits).
// ---------------------------------------------------------------------------
struct ExEntry {
    unsigned long long rfix;        // r_q(x): cycles per sample, 2^64 fixed point
    unsigned long long phx0, dphx;  // kappa wx vx_0 and kappa wx step_x (cycles per chirp)
    unsigned long long phy0, dphy;  // kappa wy vy_0 and kappa wy step_y
};

__global__ void exact_coord_kernel(GeoParams g, ExEntry* __restrict__ tab) {
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxy * g.Q) return;
    const int q = (int)(idx % g.Q);
    const long long xy = idx / g.Q;
    const int ix = (int)(xy / g.n[1]);
    const int iy = (int)(xy - (long long)ix * g.n[1]);
    double d, wx, wy;
    gh_bistatic(g, q, gh_axis(g.lo[0], g.step[0], ix), gh_axis(g.lo[1], g.step[1], iy), &d, &wx, &wy);
    ExEntry e;
    e.rfix = gh_phase_fix(gh_range(g, d));
    const double kx = g.kappa * wx, ky = g.kappa * wy;
    e.phx0 = gh_phase_fix(kx * gh_axis(g.lo[2], g.step[2], 0));
    e.dphx = gh_phase_fix(kx * g.step[2]);
    e.phy0 = gh_phase_fix(ky * gh_axis(g.lo[3], g.step[3], 0));
    e.dphy = gh_phase_fix(ky * g.step[3]);
    tab[idx] = e;
}

struct ExactTcParams {
    int Q, Mc, nvx, nvy, nstages;
    long long nxy, nv;
};

constexpr uint32_t kTcWaitIters = 1u << 22;

// z[k] = exp(-j 2 pi ph (m0 + k)), k < 32, reseeded exactly every 8 chirps.
__device__ __forceinline__ void atoms32(unsigned long long ph, int m0, float2* z) {
    const float2 w = gh_cis_fix(0ull - ph);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float2 v = gh_cis_fix(0ull - ph * (unsigned long long)(m0 + 8 * j));
        z[8 * j] = v;
#pragma unroll
        for (int i = 1; i < 8; ++i) {
            v = cmul(v, w);
            z[8 * j + i] = v;
        }
    }
}

__device__ __forceinline__ void store_chunk(unsigned char* hi, unsigned char* lo, uint32_t off, const float* v) {
    uint4 h, l;
    gh_tc::split_bf16x2(v[0], v[1], &h.x, &l.x);
    gh_tc::split_bf16x2(v[2], v[3], &h.y, &l.y);
    gh_tc::split_bf16x2(v[4], v[5], &h.z, &l.z);
    gh_tc::split_bf16x2(v[6], v[7], &h.w, &l.w);
    *(uint4*)(hi + off) = h;
    *(uint4*)(lo + off) = l;
}

template <int NV32>
__global__ void __launch_bounds__(128) exact_tc_kernel(const float2* __restrict__ P, const ExEntry* __restrict__ tab,
                                                       ExactTcParams p, float* __restrict__ scores,
                                                       const int64_t* __restrict__ mask, int nmask,
                                                       ArgPartial* __restrict__ parts, int* __restrict__ status) {
    constexpr int NVP = 32 * NV32;           // padded nvy
    constexpr int N = 2 * NVP;               // MMA N
    constexpr uint32_t SBO = 128, LBO_A = 16 * 128, LBO_B = (N / 8) * 128;
    constexpr uint32_t A_BYTES = 128 * 64 * 2, B_BYTES = N * 64 * 2;
    constexpr uint32_t BUF_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    constexpr uint32_t TM_COLS = 2 * N <= 32 ? 32 : (2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : (2 * N <= 256 ? 256 : 512)));
    extern __shared__ __align__(1024) unsigned char smem[];
    float* xfer = (float*)(smem + 2 * BUF_BYTES);  // [32][NVP]
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_holder;
    __shared__ float s_bs[4];
    __shared__ long long s_bc[4];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int h = tid >> 6, a = (tid & 63) >> 1, part = tid & 1;
    const int kh = tid & 1;
    const int npairs = (p.Q + 1) >> 1;

    if (tid == 0) {
        gh_tc::mbar_init(&bar[0], 1);
        gh_tc::mbar_init(&bar[1], 1);
        gh_tc::mbar_fence_init();
    }
    if (warp == 0) gh_tc::tmem_alloc(&tmem_holder, TM_COLS);
    gh_tc::fence_before_sync();
    __syncthreads();
    gh_tc::fence_after_sync();
    const uint32_t tmem = tmem_holder;
    const uint32_t idesc = gh_tc::idesc_bf16_f32(128, N);

    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    uint32_t gs = 0;
    int pair_ctr = 0;
    bool aborted = false;

    for (long long xy = blockIdx.x; xy < p.nxy && !aborted; xy += gridDim.x) {
        float acc[NVP];
#pragma unroll
        for (int i = 0; i < NVP; ++i) acc[i] = 0.f;
        for (int pp = 0; pp < npairs && !aborted; ++pp) {
            const int qa = 2 * pp + h;
            const bool va = qa < p.Q && a < p.nvx;
            unsigned long long phx = 0;
            if (va) {
                const ExEntry& e = tab[xy * p.Q + qa];
                phx = e.phx0 + (unsigned long long)a * e.dphx;
            }
            const uint32_t dcol = (uint32_t)(pair_ctr & 1) * N;
            for (int s = 0; s < p.nstages; ++s) {
                const int buf = gs & 1;
                if (gs >= 2) {
                    const bool ok = gh_tc::mbar_wait_bounded(&bar[buf], ((gs - 2) >> 1) & 1, kTcWaitIters);
                    if (__syncthreads_or(!ok)) {
                        aborted = true;
                        break;
                    }
                }
                unsigned char* Ah = smem + buf * BUF_BYTES;
                unsigned char* Al = Ah + A_BYTES;
                unsigned char* Bh = Al + A_BYTES;
                unsigned char* Bl = Bh + B_BYTES;
                const int m0 = 32 * s;
                // ---- A: this thread's row ----
                {
                    float2 z[32];
                    if (va) {
                        atoms32(phx, m0, z);
                    } else {
#pragma unroll
                        for (int k = 0; k < 32; ++k) z[k] = make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        float v[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float2 zz = z[(c & 3) * 8 + i];
                            // chunks 0-3: [Re | Im] of the first half; 4-7: [-Im | Re]
                            v[i] = part == 0 ? (c < 4 ? zz.x : -zz.y) : (c < 4 ? zz.y : zz.x);
                        }
                        store_chunk(Ah, Al, gh_tc::kmajor_off((uint32_t)tid, (uint32_t)(8 * c), LBO_A, SBO), v);
                    }
                }
                // ---- B: rows n = tid/2 + 64 g, chirps m0 + 16 kh .. +15 ----
#pragma unroll
                for (int g = 0; g < N / 64; ++g) {
                    const int n = (tid >> 1) + 64 * g;
                    const int hb = n / NVP, b = n - hb * NVP;
                    const int qb = 2 * pp + hb;
                    const bool vb = qb < p.Q && b < p.nvy;
                    float gr[16], gi[16];
                    if (vb) {
                        const ExEntry& e = tab[xy * p.Q + qb];
                        const unsigned long long phy = e.phy0 + (unsigned long long)b * e.dphy;
                        const float2* Pq = P + ((size_t)qb * p.nxy + xy) * p.Mc;
                        const int mb = m0 + 16 * kh;
                        const float2 w = gh_cis_fix(0ull - phy);
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            float2 at = gh_cis_fix(0ull - phy * (unsigned long long)(mb + 8 * j));
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const int mc = mb + 8 * j + i;
                                const float2 pv = mc < p.Mc ? __ldg(Pq + mc) : make_float2(0.f, 0.f);
                                const float2 gv = cmul(pv, at);
                                gr[8 * j + i] = gv.x;
                                gi[8 * j + i] = gv.y;
                                at = cmul(at, w);
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; ++i) gr[i] = gi[i] = 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        store_chunk(Bh, Bl, gh_tc::kmajor_off((uint32_t)n, (uint32_t)(16 * kh + 8 * j), LBO_B, SBO),
                                    gr + 8 * j);
                        store_chunk(Bh, Bl,
                                    gh_tc::kmajor_off((uint32_t)n, (uint32_t)(32 + 16 * kh + 8 * j), LBO_B, SBO),
                                    gi + 8 * j);
                    }
                }
                gh_tc::fence_smem_to_async();
                gh_tc::fence_before_sync();
                __syncthreads();
                if (tid == 0) {
                    gh_tc::fence_after_sync();
                    const uint32_t ah = gh_tc::smem_u32(Ah), al = gh_tc::smem_u32(Al);
                    const uint32_t bh = gh_tc::smem_u32(Bh), bl = gh_tc::smem_u32(Bl);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t dah = gh_tc::smem_desc(ah + 2 * kk * LBO_A, LBO_A, SBO);
                        const uint64_t dal = gh_tc::smem_desc(al + 2 * kk * LBO_A, LBO_A, SBO);
                        const uint64_t dbh = gh_tc::smem_desc(bh + 2 * kk * LBO_B, LBO_B, SBO);
                        const uint64_t dbl = gh_tc::smem_desc(bl + 2 * kk * LBO_B, LBO_B, SBO);
                        gh_tc::mma_bf16(tmem + dcol, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                        gh_tc::mma_bf16(tmem + dcol, dah, dbl, idesc, 1u);
                        gh_tc::mma_bf16(tmem + dcol, dal, dbh, idesc, 1u);
                    }
                    gh_tc::mma_commit(&bar[buf]);
                }
                ++gs;
            }
            if (aborted) break;
            // epilogue of the pair: |F|^2 of this half's block of D
            {
                const uint32_t last = gs - 1;
                const bool ok = gh_tc::mbar_wait_bounded(&bar[last & 1], (last >> 1) & 1, kTcWaitIters);
                if (__syncthreads_or(!ok)) {
                    aborted = true;
                    break;
                }
                gh_tc::fence_after_sync();
#pragma unroll
                for (int c = 0; c < NV32; ++c) {
                    float v[32];
                    gh_tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + dcol + (uint32_t)(h * NVP + 32 * c), v);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float o = __shfl_xor_sync(0xffffffffu, v[i], 1);
                        acc[32 * c + i] += v[i] * v[i] + o * o;
                    }
                }
                gh_tc::fence_before_sync();
            }
            ++pair_ctr;
        }
        if (aborted) break;
        // sum over receivers: rows 64-127 (odd q) hand their sums to rows 0-63
        __syncthreads();
        if (h == 1 && part == 0 && a < p.nvx) {
#pragma unroll
            for (int b = 0; b < NVP; ++b) xfer[a * NVP + b] = acc[b];
        }
        __syncthreads();
        if (h == 0 && part == 0 && a < p.nvx) {
            const long long cbase = xy * p.nv + (long long)a * p.nvy;
            bool hm = false;
            for (int m = 0; m < nmask; ++m) hm |= (__ldg(&mask[m]) / p.nv == xy);
            float rb = -INFINITY;
            int ri = -1;
#pragma unroll
            for (int b = 0; b < NVP; ++b) {
                if (b < p.nvy) {
                    const float sc = acc[b] + xfer[a * NVP + b];
                    if (scores) scores[cbase + b] = sc;
                    bool masked = false;
                    if (hm)
                        for (int m = 0; m < nmask; ++m) masked |= (__ldg(&mask[m]) == cbase + b);
                    if (!masked && sc > rb) {
                        rb = sc;
                        ri = b;
                    }
                }
            }
            if (ri >= 0) better(rb, cbase + ri, best, bestc);
        }
    }

    if (aborted) {
        if (tid == 0) atomicExch(status, GH_ETIMEOUT);
        // give in-flight tensor-core work a bounded chance to drain before freeing TMEM
        if (gs > 0) gh_tc::mbar_wait_bounded(&bar[(gs - 1) & 1], ((gs - 1) >> 1) & 1, kTcWaitIters);
    }
    gh_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gh_tc::tmem_dealloc(tmem, TM_COLS);

    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, best, off);
        const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
        better(os, oc, best, bestc);
    }
    if (lane == 0) {
        s_bs[warp] = best;
        s_bc[warp] = bestc;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < 4; ++w) better(s_bs[w], s_bc[w], best, bestc);
        parts[blockIdx.x].score = best;
        parts[blockIdx.x].cell = bestc;
    }
}

template <int NV32>
int launch_tc(gh_ctx* ctx, const Dims& d, const float2* P, const ExEntry* tab, float* scores, const int64_t* mask,
              int nmask, ArgPartial* parts, int* status, long long* nparts) {
    constexpr int NVP = 32 * NV32, N = 2 * NVP;
    const size_t smem = (size_t)2 * (2 * 128 * 64 * 2 + 2 * N * 64 * 2) + (size_t)32 * NVP * 4;
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "exact tensor-core path needs %zu B", smem);
    GH_CUDA(cudaFuncSetAttribute(exact_tc_kernel<NV32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, exact_tc_kernel<NV32>, 128, smem));
    if (per_sm < 1) per_sm = 1;
    long long ctas = (long long)ctx->num_sms * per_sm;
    if (ctas > d.nxy) ctas = d.nxy;
    ExactTcParams p;
    p.Q = d.Q;
    p.Mc = d.Mc;
    p.nvx = d.nvx;
    p.nvy = d.nvy;
    p.nstages = (d.Mc + 31) / 32;
    p.nxy = d.nxy;
    p.nv = d.nv;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_EXACT_S2, &ev);
    exact_tc_kernel<NV32><<<(unsigned)ctas, 128, smem, ctx->stream>>>(P, tab, p, scores, mask, nmask, parts, status);
    GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S2, ev, "exact_tc_kernel"));
    *nparts = ctas;
    return GH_OK;
}

}  // namespace

int gh_launch_exact(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, float* scores,
                    const int64_t* mask, int nmask, ArgResult* result) {
    if (d.nxy > 0x7fffffffLL) return gh_fail(ctx, GH_ENOTSUP, "exact path supports < 2^31 (x, y) cells");
    if (d.nv > 256 * 16) return gh_fail(ctx, GH_ENOTSUP, "exact path supports at most 4096 velocity cells");
    void* P;
    GH_TRY(gh_ws(ctx, WS_EXACT_P, (size_t)d.Q * d.nxy * d.Mc * sizeof(float2), &P));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
    dim3 grid1((unsigned)((d.nxy + S1_XT - 1) / S1_XT), (unsigned)((d.Mc + S1_MT - 1) / S1_MT), (unsigned)d.Q);
    exact_stage1_kernel<<<grid1, 256, 0, ctx->stream>>>(Y, g, (float2*)P);
    GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S1, ev, "exact_stage1_kernel"));
    void* parts;
    GH_TRY(gh_ws(ctx, WS_PART, (size_t)d.nxy * sizeof(ArgPartial), &parts));
    if (d.nvx <= 32 && d.nvy <= 64) {
        // tensor-core stage 2
        void* tab;
        GH_TRY(gh_ws(ctx, WS_EXACT_TAB, (size_t)d.nxy * d.Q * sizeof(ExEntry), &tab));
        const long long n = d.nxy * d.Q;
        gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
        exact_coord_kernel<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(g, (ExEntry*)tab);
        GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S1, ev, "exact_coord_kernel"));
        long long nparts = 0;
        int* status = gh_status_dev(ctx);
        if (d.nvy <= 32)
            GH_TRY(launch_tc<1>(ctx, d, (const float2*)P, (const ExEntry*)tab, scores, mask, nmask,
                                (ArgPartial*)parts, status, &nparts));
        else
            GH_TRY(launch_tc<2>(ctx, d, (const float2*)P, (const ExEntry*)tab, scores, mask, nmask,
                                (ArgPartial*)parts, status, &nparts));
        return gh_launch_argmax_finalize(ctx, (const ArgPartial*)parts, (int)nparts, result);
    }
    const int cpt = (int)((d.nv + 255) / 256);
    int st;
    if (cpt <= 1)
        st = launch_s2<1>(ctx, d, g, (const float2*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 2)
        st = launch_s2<2>(ctx, d, g, (const float2*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 4)
        st = launch_s2<4>(ctx, d, g, (const float2*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 8)
        st = launch_s2<8>(ctx, d, g, (const float2*)P, scores, mask, nmask, (ArgPartial*)parts);
    else
        st = launch_s2<16>(ctx, d, g, (const float2*)P, scores, mask, nmask, (ArgPartial*)parts);
    GH_TRY(st);
    return gh_launch_argmax_finalize(ctx, (const ArgPartial*)parts, (int)d.nxy, result);
}
