// The paper's factorised estimators (Sec. III, Eqs. 3-4, and their grid
// hopping version, Sec. IV) and the indirect method (Eq. 2): one target,
// location first, then velocity at that location.
//
//   GH_HOP      location: S_loc(x) = sum_q sum_mc |sum_k c_k R~_q,mc[i_q + k]|^2,
//               R~ the zero-padded range FFT of each chirp with the range-centring
//               factor (the three-bin polar interpolation of the 4D scorer);
//               velocity: g_q[mc] = <Y_q[mc], a(r_q(x^))> exactly at x^, its
//               Doppler DFT zero-padded to Nd, read at the nearest bin
//   GH_EXACT    location: S_loc(x) = sum_q sum_mc |<Y_q[mc], a(r_q(x))>|^2 (from
//               the exact path's stage 1, P_q[x][mc] = <Y_q[mc], a(r_q(x))>);
//               velocity: sum_q |<g_q, b(u_q(x^, v))>|^2 exactly
//   GH_INDIRECT per receiver the peak (i_q, j_q) of |RD map|, r^_q = i_q / Nr,
//               u^_q = j_q / Nd in [-1/2, 1/2); x^ = argmin sum_q (r_q(x) - r^_q)^2,
//               then v^ = argmin sum_q (u_q(x^, v) - u^_q)^2 (float64, Eq. 2 read as
//               an argmin)
// Ties go to the smallest index everywhere.
#include <math.h>

#include <algorithm>

#include "gh_internal.cuh"

namespace {

// zt[q][i][mc] = zr[q][mc][i] * exp(j pi (i/Nr)(Ms-1)): range rows, chirps contiguous.
__global__ void rows_t_kernel(const float2* __restrict__ zr, float2* __restrict__ zt, int Ms, int Mc, int Nr) {
    __shared__ float2 tile[32][33];
    const int q = blockIdx.z;
    const int i0 = blockIdx.x * 32, m0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int mc = m0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (mc < Mc && i < Nr) ? zr[((size_t)q * Mc + mc) * Nr + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, mc = m0 + threadIdx.x;
        if (i < Nr && mc < Mc) {
            const long long t = ((long long)i * (Ms - 1)) % (2LL * Nr);
            float s, c;
            sincospif((float)t / (float)Nr, &s, &c);
            zt[((size_t)q * Nr + i) * Mc + mc] = cmul(tile[threadIdx.x][r], make_float2(c, s));
        }
    }
}

__device__ __forceinline__ void better(float s, long long c, float& bs, long long& bc) {
    if (s > bs || (s == bs && c < bc)) {
        bs = s;
        bc = c;
    }
}

__device__ __forceinline__ void block_best(float& best, long long& bestc, ArgPartial* out) {
    __shared__ float s_bs[32];
    __shared__ long long s_bc[32];
    for (int off = 16; off > 0; off >>= 1) {
        const float os = __shfl_down_sync(0xffffffffu, best, off);
        const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
        better(os, oc, best, bestc);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_bs[warp] = best;
        s_bc[warp] = bestc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) better(s_bs[w], s_bc[w], best, bestc);
        out->score = best;
        out->cell = bestc;
    }
}

// Hopping location score of every (x, y) cell: one warp per cell, lanes over
// chirps. The coordinate table is the 4D scorer's (rows, signed coefficients).
__global__ void __launch_bounds__(256) loc_hop_kernel(const float2* __restrict__ zt, const HopEntry* __restrict__ tab,
                                                      int Q, int Mc, int Nr, long long nxy, float* __restrict__ S,
                                                      ArgPartial* __restrict__ parts) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    for (long long xy = (long long)blockIdx.x * 8 + warp; xy < nxy; xy += (long long)gridDim.x * 8) {
        float acc = 0.f;
        for (int q = 0; q < Q; ++q) {
            const HopEntry& e = tab[xy * Q + q];
            const float2* r0 = zt + ((size_t)q * Nr + e.row[0]) * Mc;
            const float2* r1 = zt + ((size_t)q * Nr + e.row[1]) * Mc;
            const float2* r2 = zt + ((size_t)q * Nr + e.row[2]) * Mc;
            const float c0 = e.cs[0], c1 = e.cs[1], c2 = e.cs[2];
            for (int mc = lane; mc < Mc; mc += 32) {
                const float2 a = __ldg(r0 + mc), b = __ldg(r1 + mc), c = __ldg(r2 + mc);
                const float re = c0 * a.x + c1 * b.x + c2 * c.x, im = c0 * a.y + c1 * b.y + c2 * c.y;
                acc += re * re + im * im;
            }
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0 && S) S[xy] = acc;
        better(acc, xy, best, bestc);
    }
    block_best(best, bestc, parts + blockIdx.x);
}

// Exact location score from stage 1: S_loc(x) = sum_q sum_mc |P_q[x][mc]|^2.
__global__ void __launch_bounds__(256) loc_exact_kernel(const float* __restrict__ P, int Q, int Mc, long long nxy,
                                                        float* __restrict__ S, ArgPartial* __restrict__ parts) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    for (long long xy = (long long)blockIdx.x * 8 + warp; xy < nxy; xy += (long long)gridDim.x * 8) {
        float acc = 0.f;
        for (int q = 0; q < Q; ++q) {
            const float* row = P + ((size_t)q * nxy + xy) * 2 * Mc;
            for (int k = lane; k < 2 * Mc; k += 32) {
                const float v = __ldg(row + k);
                acc += v * v;
            }
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0 && S) S[xy] = acc;
        better(acc, xy, best, bestc);
    }
    block_best(best, bestc, parts + blockIdx.x);
}

struct FzResult {
    long long cell;
    double loc, vel;
    int valid, pad;
};

// Velocity step (one CTA): g_q at the location of *loc, then the velocity
// score of every (vx, vy) cell (hop: nearest bin of the Doppler DFT of g_q;
// exact: the correlation with b(u_q)), argmax, and the 4D result.
// Shared memory: atoms a(r_q) [Q][Ms], g [Q][Mc], and for hop the Doppler
// DFT [Q][Nd] and its twiddles [Nd].
__global__ void __launch_bounds__(1024) vel_kernel(const float2* __restrict__ Y, GeoParams g, int hop,
                                                   const ArgResult* __restrict__ loc, FzResult* __restrict__ out) {
    extern __shared__ float2 fz_smem[];
    const int Q = g.Q, Ms = g.Ms, Mc = g.Mc, Nd = g.Nd;
    float2* at = fz_smem;             // [Q][Ms]
    float2* gq = at + Q * Ms;         // [Q][Mc]
    float2* G = gq + Q * Mc;          // [Q][Nd]   (hop)
    float2* tw = G + (hop ? Q * Nd : 0);  // [Nd] (hop)
    __shared__ double s_wx[GH_MAX_Q], s_wy[GH_MAX_Q];
    __shared__ unsigned long long s_rf[GH_MAX_Q];
    const long long xy = loc->cell;
    const int ix = (int)(xy / g.n[1]), iy = (int)(xy - (long long)ix * g.n[1]);
    const double x = gh_axis(g.lo[0], g.step[0], ix), y = gh_axis(g.lo[1], g.step[1], iy);
    for (int q = threadIdx.x; q < Q; q += blockDim.x) {
        double d, wx, wy;
        gh_bistatic(g, q, x, y, &d, &wx, &wy);
        s_wx[q] = wx;
        s_wy[q] = wy;
        s_rf[q] = gh_phase_fix(gh_range(g, d));
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < Q * Ms; idx += blockDim.x) {
        const int q = idx / Ms, m = idx - q * Ms;
        at[idx] = gh_cis_fix(s_rf[q] * (unsigned long long)m);
    }
    if (hop)
        for (int t = threadIdx.x; t < Nd; t += blockDim.x) {
            float s, c;
            sincospif(-2.0f * (float)t / (float)Nd, &s, &c);
            tw[t] = make_float2(c, s);
        }
    __syncthreads();
    // g_q[mc] = sum_m Y[q][mc][m] conj(a_m(r_q)): one warp per chirp, lanes
    // over the samples (coalesced rows), then a butterfly sum
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int idx = warp; idx < Q * Mc; idx += nw) {
            const int q = idx / Mc;
            const float2* row = Y + (size_t)idx * Ms;
            float2 s = make_float2(0.f, 0.f);
            for (int m = lane; m < Ms; m += 32) {
                const float2 v = __ldg(row + m), a = at[q * Ms + m];
                s.x += v.x * a.x + v.y * a.y;
                s.y += v.y * a.x - v.x * a.y;
            }
            for (int off = 16; off > 0; off >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
            }
            if (lane == 0) gq[idx] = s;
        }
    }
    __syncthreads();
    if (hop) {
        // G_q[j] = sum_mc g_q[mc] exp(-j 2 pi j mc / Nd)
        for (int idx = threadIdx.x; idx < Q * Nd; idx += blockDim.x) {
            const int q = idx / Nd, j = idx - q * Nd;
            float2 s = make_float2(0.f, 0.f);
            for (int mc = 0; mc < Mc; ++mc) {
                const float2 w = tw[(int)(((long long)j * mc) & (Nd - 1))];
                s = make_float2(s.x + (gq[q * Mc + mc].x * w.x - gq[q * Mc + mc].y * w.y),
                                s.y + (gq[q * Mc + mc].x * w.y + gq[q * Mc + mc].y * w.x));
            }
            G[idx] = s;
        }
        __syncthreads();
    }
    const int nvx = g.n[2], nvy = g.n[3];
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    for (long long v = threadIdx.x; v < (long long)nvx * nvy; v += blockDim.x) {
        const int a = (int)(v / nvy), b = (int)(v - (long long)a * nvy);
        const double vx = gh_axis(g.lo[2], g.step[2], a), vy = gh_axis(g.lo[3], g.step[3], b);
        float acc = 0.f;
        for (int q = 0; q < Q; ++q) {
            const double u = gh_speed(g, s_wx[q], s_wy[q], vx, vy);
            if (hop) {
                long long j = (long long)floor(__dadd_rn(__dmul_rn((double)Nd, u), 0.5));
                j %= Nd;
                if (j < 0) j += Nd;
                const float2 z = G[q * Nd + j];
                acc += z.x * z.x + z.y * z.y;
            } else {
                // b_mc(u) = exp(j 2 pi u mc): an exact value from the fixed-point
                // phase every 32 chirps, the recurrence b_{mc+1} = b_mc w between
                const unsigned long long uf = gh_phase_fix(u);
                const float2 w = gh_cis_fix(uf);
                float2 s = make_float2(0.f, 0.f);
                for (int mc0 = 0; mc0 < Mc; mc0 += 32) {
                    float2 bb = gh_cis_fix(uf * (unsigned long long)mc0);
                    const int m1 = min(mc0 + 32, Mc);
                    for (int mc = mc0; mc < m1; ++mc) {
                        const float2 z = gq[q * Mc + mc];
                        s.x += z.x * bb.x + z.y * bb.y;  // z conj(b)
                        s.y += z.y * bb.x - z.x * bb.y;
                        bb = cmul(bb, w);
                    }
                }
                acc += s.x * s.x + s.y * s.y;
            }
        }
        better(acc, v, best, bestc);
    }
    __shared__ ArgPartial s_best;
    block_best(best, bestc, &s_best);
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long vcell = s_best.cell;
        const int a = (int)(vcell / nvy), b = (int)(vcell - (long long)a * nvy);
        out->cell = (((long long)ix * g.n[1] + iy) * nvx + a) * nvy + b;
        out->loc = (double)loc->score;
        out->vel = (double)s_best.score;
        out->valid = loc->valid && vcell != 0x7fffffffffffffffLL;
    }
}

// Per-receiver peak of |RD map|^2 over [Nr][Nd] (index i * Nd + j): partials
// per (chunk, q).
__global__ void __launch_bounds__(256) rd_peak_kernel(const float2* __restrict__ maps, long long per_q, int chunk,
                                                      ArgPartial* __restrict__ parts) {
    const int q = blockIdx.y;
    const float2* m = maps + (size_t)q * per_q;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    const long long i0 = (long long)blockIdx.x * chunk;
    const long long i1 = i0 + chunk < per_q ? i0 + chunk : per_q;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const float2 z = __ldg(m + i);
        better(z.x * z.x + z.y * z.y, i, best, bestc);
    }
    block_best(best, bestc, parts + (size_t)q * gridDim.x + blockIdx.x);
}

// Per-receiver map peaks from the rd_peak partials: r^_q = i / Nr and
// u^_q = j / Nd in [-1/2, 1/2) (one warp per receiver; ties -> smallest index).
__device__ void peaks_to_values(const GeoParams& g, const ArgPartial* __restrict__ parts, int nchunks, double* r,
                                double* u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < g.Q; q += nw) {
        float best = -INFINITY;
        long long bestc = 0x7fffffffffffffffLL;
        for (int c = lane; c < nchunks; c += 32)
            better(parts[(size_t)q * nchunks + c].score, parts[(size_t)q * nchunks + c].cell, best, bestc);
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_down_sync(0xffffffffu, best, off);
            const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
            better(os, oc, best, bestc);
        }
        if (lane == 0) {
            const long long i = bestc / g.Nd, j = bestc - i * g.Nd;
            r[q] = __ddiv_rn((double)i, (double)g.Nr);
            u[q] = j < g.Nd / 2 ? __ddiv_rn((double)j, (double)g.Nd)
                                : __dsub_rn(__ddiv_rn((double)j, (double)g.Nd), 1.0);
        }
    }
}

struct MinPartial {
    double v;
    long long i;
};

__device__ __forceinline__ void take_min(double v, long long i, double& bv, long long& bi) {
    if (v < bv || (v == bv && i < bi)) {
        bv = v;
        bi = i;
    }
}

// Block-wide argmin (float64, ties -> smallest index); thread 0 gets the result.
__device__ void block_min(double& bv, long long& bi) {
    __shared__ double s_bv[32];
    __shared__ long long s_bi[32];
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, off);
        const long long oi = __shfl_down_sync(0xffffffffu, bi, off);
        take_min(ov, oi, bv, bi);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_bv[warp] = bv;
        s_bi[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) take_min(s_bv[w], s_bi[w], bv, bi);
}

// Eq. 2 location cost sum_q (r_q(x) - r^_q)^2 of the (x, y) cells, float64;
// per-CTA argmin partials.
__global__ void __launch_bounds__(256) multilat_loc_kernel(GeoParams g, const ArgPartial* __restrict__ parts,
                                                           int nchunks, MinPartial* __restrict__ out) {
    __shared__ double s_r[GH_MAX_Q], s_u[GH_MAX_Q];
    peaks_to_values(g, parts, nchunks, s_r, s_u);
    __syncthreads();
    const long long nxy = (long long)g.n[0] * g.n[1];
    double bv = INFINITY;
    long long bi = 0x7fffffffffffffffLL;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nxy;
         c += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(c / g.n[1]), iy = (int)(c - (long long)ix * g.n[1]);
        const double x = gh_axis(g.lo[0], g.step[0], ix), y = gh_axis(g.lo[1], g.step[1], iy);
        double L = 0.0;
        for (int q = 0; q < g.Q; ++q) {
            double d, wx, wy;
            gh_bistatic(g, q, x, y, &d, &wx, &wy);
            const double e = __dsub_rn(gh_range(g, d), s_r[q]);
            L = __dadd_rn(L, __dmul_rn(e, e));
        }
        take_min(L, c, bv, bi);
    }
    block_min(bv, bi);
    if (threadIdx.x == 0) out[blockIdx.x] = MinPartial{bv, bi};
}

// Location from the partials, then the velocity cost sum_q (u_q(x^, v) - u^_q)^2
// over the (vx, vy) cells and its argmin (one CTA).
__global__ void __launch_bounds__(1024) multilat_vel_kernel(GeoParams g, const ArgPartial* __restrict__ parts,
                                                            int nchunks, const MinPartial* __restrict__ loc,
                                                            int nloc, FzResult* __restrict__ out) {
    __shared__ double s_r[GH_MAX_Q], s_u[GH_MAX_Q], s_wx[GH_MAX_Q], s_wy[GH_MAX_Q];
    __shared__ MinPartial s_loc;
    peaks_to_values(g, parts, nchunks, s_r, s_u);
    double bv = INFINITY;
    long long bi = 0x7fffffffffffffffLL;
    for (int c = threadIdx.x; c < nloc; c += blockDim.x) take_min(loc[c].v, loc[c].i, bv, bi);
    block_min(bv, bi);
    if (threadIdx.x == 0) s_loc = MinPartial{bv, bi};
    __syncthreads();
    const long long xy = s_loc.i;
    const int ix = (int)(xy / g.n[1]), iy = (int)(xy - (long long)ix * g.n[1]);
    const double x = gh_axis(g.lo[0], g.step[0], ix), y = gh_axis(g.lo[1], g.step[1], iy);
    for (int q = threadIdx.x; q < g.Q; q += blockDim.x) {
        double d, wx, wy;
        gh_bistatic(g, q, x, y, &d, &wx, &wy);
        s_wx[q] = wx;
        s_wy[q] = wy;
    }
    __syncthreads();
    const int nvy = g.n[3];
    bv = INFINITY;
    bi = 0x7fffffffffffffffLL;
    for (long long c = threadIdx.x; c < (long long)g.n[2] * nvy; c += blockDim.x) {
        const int a = (int)(c / nvy), b = (int)(c - (long long)a * nvy);
        const double vx = gh_axis(g.lo[2], g.step[2], a), vy = gh_axis(g.lo[3], g.step[3], b);
        double V = 0.0;
        for (int q = 0; q < g.Q; ++q) {
            const double e = __dsub_rn(gh_speed(g, s_wx[q], s_wy[q], vx, vy), s_u[q]);
            V = __dadd_rn(V, __dmul_rn(e, e));
        }
        take_min(V, c, bv, bi);
    }
    block_min(bv, bi);
    if (threadIdx.x == 0) {
        const long long a = bi / nvy, b = bi - a * nvy;
        out->cell = ((xy * g.n[2]) + a) * nvy + b;
        out->loc = s_loc.v;
        out->vel = bv;
        out->valid = 1;
    }
}

}  // namespace

extern "C" int gh_factorized(gh_ctx* ctx, int32_t method, const gh_radar* radar, const double* tx_host,
                             const double* rx_host, int32_t Q, const void* Y, const gh_grid* grid,
                             int64_t* cell_host, double* values_host, float* loc_scores_dev) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_grid(ctx, grid, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    if (method != GH_HOP && method != GH_EXACT && method != GH_INDIRECT)
        return gh_fail(ctx, GH_EINVAL, "method %d unknown", method);
    if (!cell_host) return gh_fail(ctx, GH_EINVAL, "cell_host is NULL");
    if (!Y) return gh_fail(ctx, GH_EINVAL, "Y is NULL");
    DeviceGuard dg(ctx->device);
    if (loc_scores_dev) {
        const int dv = gh_is_device_ptr(ctx, loc_scores_dev);
        if (dv < 0) return dv;
        if (!dv) return gh_fail(ctx, GH_EINVAL, "loc_scores_dev must be device memory");
    }
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, grid);
    const int ydev = gh_is_device_ptr(ctx, Y);
    if (ydev < 0) return ydev;
    const float2* Yd = (const float2*)Y;
    if (!ydev) {
        void* p;
        const size_t bytes = (size_t)Q * d.Mc * d.Ms * sizeof(float2);
        GH_TRY(gh_ws(ctx, WS_Y, bytes, &p));
        GH_CUDA(cudaMemcpyAsync(p, Y, bytes, cudaMemcpyHostToDevice, ctx->stream));
        Yd = (const float2*)p;
    }
    void* res;
    GH_TRY(gh_ws(ctx, WS_RESULT, 64 * sizeof(ArgResult), &res));
    ArgResult* locres = (ArgResult*)res;
    FzResult* fres = (FzResult*)((char*)res + 32 * sizeof(ArgResult));
    GH_TRY(gh_status_reset(ctx));
    cudaEvent_t ev;
    const int ctas = ctx->num_sms * 4;
    if (method == GH_INDIRECT) {
        void* maps;
        GH_TRY(gh_ws(ctx, WS_MAPS, (size_t)Q * d.Nr * d.Nd * sizeof(float2), &maps));
        GH_TRY(gh_launch_maps(ctx, d, Yd, nullptr, maps, GH_C64));
        const long long per_q = (long long)d.Nr * d.Nd;
        const int nch = (int)std::min<long long>(256, (per_q + 4095) / 4096);
        const int chunk = (int)((per_q + nch - 1) / nch);
        void* parts;
        GH_TRY(gh_ws(ctx, WS_PART, (size_t)nch * Q * sizeof(ArgPartial), &parts));
        gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
        rd_peak_kernel<<<dim3(nch, Q), 256, 0, ctx->stream>>>((const float2*)maps, per_q, chunk, (ArgPartial*)parts);
        GH_TRY(gh_launch_end(ctx, GH_K_ARGMAX, ev, "rd_peak_kernel"));
        void* mins;
        const int nloc = (int)std::min<long long>(ctas, (d.nxy + 255) / 256);
        GH_TRY(gh_ws(ctx, WS_DIAG, (size_t)nloc * sizeof(MinPartial), &mins));
        gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
        multilat_loc_kernel<<<nloc, 256, 0, ctx->stream>>>(geo, (const ArgPartial*)parts, nch, (MinPartial*)mins);
        GH_TRY(gh_launch_end(ctx, GH_K_ARGMAX, ev, "multilat_loc_kernel"));
        gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
        multilat_vel_kernel<<<1, 1024, 0, ctx->stream>>>(geo, (const ArgPartial*)parts, nch, (const MinPartial*)mins,
                                                          nloc, fres);
        GH_TRY(gh_launch_end(ctx, GH_K_ARGMAX, ev, "multilat_vel_kernel"));
    } else {
        void* parts;
        GH_TRY(gh_ws(ctx, WS_PART, (size_t)ctas * sizeof(ArgPartial), &parts));
        if (method == GH_HOP) {
            void *zr_unused, *zt, *table;
            (void)zr_unused;
            // range FFT of every chirp, transposed with the centring factor
            GH_TRY(gh_launch_range_rows(ctx, d, Yd, &zr_unused));
            GH_TRY(gh_ws(ctx, WS_MAPS, (size_t)Q * d.Nr * d.Mc * sizeof(float2), &zt));
            gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
            rows_t_kernel<<<dim3(d.Nr / 32, (d.Mc + 31) / 32, Q), dim3(32, 8), 0, ctx->stream>>>(
                (const float2*)zr_unused, (float2*)zt, d.Ms, d.Mc, d.Nr);
            GH_TRY(gh_launch_end(ctx, GH_K_RANGE_FFT, ev, "rows_t_kernel"));
            GH_TRY(gh_ws(ctx, WS_TABLE, gh_hop_table_bytes(d), &table));
            GH_TRY(gh_launch_coord(ctx, d, geo, table, nullptr, nullptr, nullptr, nullptr));
            gh_launch_begin(ctx, GH_K_HOP_SCORE, &ev);
            loc_hop_kernel<<<ctas, 256, 0, ctx->stream>>>((const float2*)zt, (const HopEntry*)table, Q, d.Mc, d.Nr,
                                                          d.nxy, loc_scores_dev, (ArgPartial*)parts);
            GH_TRY(gh_launch_end(ctx, GH_K_HOP_SCORE, ev, "loc_hop_kernel"));
        } else {
            const float* P;
            GH_TRY(gh_launch_exact_stage1(ctx, d, geo, Yd, &P));
            gh_launch_begin(ctx, GH_K_EXACT_S2, &ev);
            loc_exact_kernel<<<ctas, 256, 0, ctx->stream>>>(P, Q, d.Mc, d.nxy, loc_scores_dev, (ArgPartial*)parts);
            GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S2, ev, "loc_exact_kernel"));
        }
        GH_TRY(gh_launch_argmax_finalize(ctx, (const ArgPartial*)parts, ctas, locres));
        const int hop = method == GH_HOP;
        const size_t smem = ((size_t)Q * d.Ms + (size_t)Q * d.Mc + (hop ? (size_t)Q * d.Nd + d.Nd : 0)) *
                            sizeof(float2);
        if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "velocity step needs %zu B", smem);
        GH_CUDA(cudaFuncSetAttribute(vel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
        vel_kernel<<<1, 1024, smem, ctx->stream>>>(Yd, geo, hop, locres, fres);
        GH_TRY(gh_launch_end(ctx, GH_K_ARGMAX, ev, "vel_kernel"));
    }
    FzResult hres;
    GH_CUDA(cudaMemcpyAsync(&hres, fres, sizeof(FzResult), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!hres.valid) return gh_fail(ctx, GH_ECUDA, "no estimate (empty scores)");
    *cell_host = hres.cell;
    if (values_host) {
        values_host[0] = hres.loc;
        values_host[1] = hres.vel;
    }
    return GH_OK;
}
