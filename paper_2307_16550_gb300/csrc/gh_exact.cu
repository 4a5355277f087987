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
