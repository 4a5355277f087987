// Grid-hopping score (Sec. IV, Eq. 5) over the 4D grid, its argmax, and the
// coordinate mapping it needs (Eq. 1).
//
// coord_kernel (two threads per (x, y), each every other receiver, float64):
//   rho = Nr * r_q(x), i = floor(rho + 1/2), tau = rho - i, the three polar
//   coefficients c_k(tau) on rows (i + k) mod Nr (signed by the centring phase
//   of a wrapped index), and the Doppler bin position as 64-bit fixed point:
//   eta(a, b) = Nd * kappa * (wx * vx_a + wy * vy_b) is affine in the cell
//   indices (a, b), so eta * 2^32 = base + a * ax + b * by exactly up to the
//   rounding of three integers (error <= (1 + a + b) * 2^-33 bins).
//
// hop_score_kernel (one warp per (x, y) cell at a time, no block barriers):
//   For a fixed (x, y, q) the hopping value at Doppler bin j is
//   T_q[j] = sum_k c_k Z~_q[i+k][j], and the cell's contribution is |T_q[j_q]|^2.
//   The warp first evaluates P_q[j] = |T_q[j]|^2 into its own shared-memory
//   rows (indexed relative to j_ref) for the bins the velocity grid reaches,
//   reading the three map rows with 16-byte loads (a pair of float32 bins, or
//   four 16-bit bins, per load); then each lane scores its velocity cells in
//   runs of AC, one shared-memory read per cell and receiver. Row modes: the
//   rows of all receivers first, or (large Q Nd, one run per vy row of a
//   lane) one receiver's row at a time added into register sums. Lane
//   layouts: b = lane mod min(nvy, 32), or 8 (vy) x 4 (vx) lanes with 6 or 10
//   cells per run for velocity axes of about 24 or 40 cells.
//   The bin j_q = floor(eta + 1/2) is the high word of the fixed-point value;
//   when its fraction lies within `tol` of a rounding boundary the bin is
//   recomputed with the float64 expression floor(Nd * (kappa * (wx*vx + wy*vy)) + 1/2),
//   so every bin decision equals a plain float64 evaluation.
//   The warps of a CTA work on neighbouring y cells at the same time, so their
//   map rows overlap in L1. Scores (optional) are written coalesced; the best
//   (score, cell) is reduced per lane, then with warp shuffles and once per
//   CTA (ties: smallest cell index).
//
// hop_pair_score_kernel, hop_pair_kernel (batched): where all receivers' rows
//   leave few warps per SM (large Q Nd, cells that do not fit one register
//   run), the two warps of a 64-thread CTA score each (x, y) cell together
//   from one set of rows, with the lanes' velocity cells split between them.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <algorithm>

#include "gh_internal.cuh"

namespace {

// Fixed-point tolerance (2^-32 bin units) of the Doppler bin decision: at least
// 2^-20 of a bin and four times the rounding bound (1 + nvx + nvy) * 2^-33.
inline uint32_t hop_tol(int nvx, int nvy) {
    const long long t = 4LL * (nvx + nvy + 2);
    return (uint32_t)(t > 4096 ? t : 4096);
}

#ifndef GH_HOP_U
#define GH_HOP_U 4  // map-row loads in flight per lane in the power-row build
#endif
#ifndef GH_HOP_MINB
#define GH_HOP_MINB 2  // CTAs per SM the scorer's register budget targets
#endif




// Entry idx = xy * Q + q of the coordinate table (diagnostics optional), at
// the point (x, y) whose transmitter distance and unit vector are given.
__device__ __forceinline__ void coord_entry_at(const GeoParams& g, const CoordParams& cp, long long idx, int q,
                                               double x, double y, double n1, double ux1, double uy1,
                                               HopEntry* __restrict__ table, int32_t* diag_i, double* diag_tau,
                                               float* diag_c, double* diag_w, double* rw) {
    double d, wx, wy;
    gh_bistatic_rx(g, q, x, y, n1, ux1, uy1, &d, &wx, &wy);
    const double r = gh_range(g, d);
    const double rho = __dmul_rn((double)g.Nr, r);
    const double fi = floor(__dadd_rn(rho, 0.5));
    const double tau = __dsub_rn(rho, fi);
    const long long i = (long long)fi;

    // polar coefficients on the arc through bins i-1, i, i+1 (float32: they are
    // stored in float32; 1 - cos(theta tau) = 2 sin^2(theta tau / 2) avoids cancellation)
    float sh, ch, sf, cf;
    sincosf(0.5f * cp.theta_f * (float)tau, &sh, &ch);
    sincosf(cp.theta_f * (float)tau, &sf, &cf);
    const float kap = sh * sh * cp.inv_sin2_half;
    const float sig = sf * cp.inv_sin_t;
    const float c[3] = {0.5f * (kap - sig), 1.0f - kap, 0.5f * (kap + sig)};

    HopEntry e;
    const int lgNr = __ffs(g.Nr) - 1;  // Nr is a power of two
    for (int k = 0; k < 3; ++k) {
        const long long n = i + (k - 1);
        const long long w = n >> lgNr;  // floor(n / Nr)
        e.row[k] = (int)(n & (long long)(g.Nr - 1));
        const bool flip = cp.Ms_odd_sign && (w & 1);
        e.cs[k] = flip ? -c[k] : c[k];
    }

    // Doppler bin position, affine in (ivx, ivy)
    const double Nd = (double)g.Nd;
    const double A = Nd * g.kappa * wx, Bv = Nd * g.kappa * wy;
    const double vx0 = gh_axis(g.lo[2], g.step[2], 0), vy0 = gh_axis(g.lo[3], g.step[3], 0);
    const double eta00 = A * vx0 + Bv * vy0;
    const double ax = A * g.step[2], by = Bv * g.step[3];
    const double ex = ax * (g.n[2] - 1), ey = by * (g.n[3] - 1);
    const double emin = eta00 + fmin(0.0, ex) + fmin(0.0, ey);
    const double emax = eta00 + fmax(0.0, ex) + fmax(0.0, ey);
    const long long j_lo = (long long)floor(emin + 0.5) - 1;
    const long long j_hi = (long long)floor(emax + 0.5) + 1;
    const long long j_ref = j_lo & ~3LL;  // a multiple of 4 (16-bit maps build groups of four bins), <= j_lo
    const long long nu = j_hi - j_ref + 1;
    const bool wrap = nu > g.Nd;
    const double two32 = 4294967296.0;
    e.base = llrint((eta00 - (double)j_ref + 0.5) * two32) + (long long)cp.tol;
    e.ax = llrint(ax * two32);
    e.by = llrint(by * two32);
    e.wx = wx;
    e.wy = wy;
    e.j_ref = (int)j_ref;
    e.npair = wrap ? g.Nd / 2 : (int)((nu + 1) >> 1);  // at most Nd / 2 (nu <= Nd)
    e.wrap = wrap ? 1 : 0;
    table[idx] = e;
    if (rw) {  // float64 (r, wx, wy) of the entry, for the BOMP atoms
        rw[3 * idx] = r;
        rw[3 * idx + 1] = wx;
        rw[3 * idx + 2] = wy;
    }

    if (diag_i) {
        diag_i[idx] = (int32_t)i;
        diag_tau[idx] = tau;
        for (int k = 0; k < 3; ++k) diag_c[3 * idx + k] = c[k];
        diag_w[2 * idx] = wx;
        diag_w[2 * idx + 1] = wy;
    }
}

// Two threads per (x, y), each taking every other receiver: the
// transmitter's distance and unit vector once per thread, then its receivers'
// entries. Float64 latency is the limit: sharing the transmitter half saves
// float64 work, and two threads per cell keep enough of them in flight
// (measured 24 us with one thread per cell, 20 us with two, 22 us with four).
// rowlim (optional, device int[2Q]: Q minima preset large, then Q maxima
// preset to -1): per receiver the smallest and largest map row any entry
// reads (the map rows a detection's scorer can touch). rw (optional, device
// double[3][nxy Q]): every entry's float64 (r, wx, wy).
__global__ void coord_kernel(GeoParams g, CoordParams cp, HopEntry* __restrict__ table, int32_t* diag_i,
                             double* diag_tau, float* diag_c, double* diag_w, int* __restrict__ rowlim,
                             double* __restrict__ rw) {
    __shared__ int s_lim[2 * GH_MAX_Q];
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long xy = t >> 1;
    const int q0 = (int)(t & 1);
    if (rowlim) {
        for (int i = threadIdx.x; i < g.Q; i += blockDim.x) {
            s_lim[i] = 0x7fffffff;
            s_lim[g.Q + i] = -1;
        }
        __syncthreads();
    }
    if (xy < nxy) {
        const int ix = (int)(xy / g.n[1]);
        const int iy = (int)(xy - (long long)ix * g.n[1]);
        const double x = gh_axis(g.lo[0], g.step[0], ix);
        const double y = gh_axis(g.lo[1], g.step[1], iy);
        double n1, ux1, uy1;
        gh_unit(__dsub_rn(x, g.tx[0]), __dsub_rn(y, g.tx[1]), &n1, &ux1, &uy1);
        for (int q = q0; q < g.Q; q += 2) {
            const long long idx = xy * g.Q + q;
            coord_entry_at(g, cp, idx, q, x, y, n1, ux1, uy1, table, diag_i, diag_tau, diag_c, diag_w, rw);
            if (rowlim) {
                const HopEntry& e = table[idx];
                const int lo = min(e.row[0], min(e.row[1], e.row[2]));
                const int hi = max(e.row[0], max(e.row[1], e.row[2]));
                atomicMin(&s_lim[q], lo);
                atomicMax(&s_lim[g.Q + q], hi);
            }
        }
    }
    if (rowlim) {
        __syncthreads();
        for (int i = threadIdx.x; i < g.Q; i += blockDim.x) {
            if (s_lim[g.Q + i] >= 0) {
                atomicMin(&rowlim[i], s_lim[i]);
                atomicMax(&rowlim[g.Q + i], s_lim[g.Q + i]);
            }
        }
    }
}

// Batched tables: item = (frame, first (x, y) cell, count <= 16), one warp;
// two threads per cell, each taking every other receiver after the
// transmitter's distance and unit vector (as coord_kernel); the frame's row
// limits (reset to empty by batch_reset_kernel) take the rows the entries read.
__global__ void coord_batch_kernel(const BatchFrame* __restrict__ frames, const BatchItem* __restrict__ items) {
    __shared__ int s_lim[2 * GH_MAX_Q];
    const BatchItem it = items[blockIdx.x];
    const int c = threadIdx.x >> 1, q0 = threadIdx.x & 1;
    const BatchFrame& F = frames[it.frame];
    const GeoParams& g = F.g;
    for (int i = threadIdx.x; i < g.Q; i += blockDim.x) {
        s_lim[i] = 0x7fffffff;
        s_lim[g.Q + i] = -1;
    }
    __syncwarp();
    if (c < it.count) {
        const long long xy = it.start + c;
        const int ix = (int)(xy / g.n[1]);
        const int iy = (int)(xy - (long long)ix * g.n[1]);
        const double x = gh_axis(g.lo[0], g.step[0], ix);
        const double y = gh_axis(g.lo[1], g.step[1], iy);
        double n1, ux1, uy1;
        gh_unit(__dsub_rn(x, g.tx[0]), __dsub_rn(y, g.tx[1]), &n1, &ux1, &uy1);
        HopEntry* table = (HopEntry*)F.table;
        for (int q = q0; q < g.Q; q += 2) {
            const long long idx = xy * g.Q + q;
            coord_entry_at(g, F.cp, idx, q, x, y, n1, ux1, uy1, table, nullptr, nullptr, nullptr, nullptr, nullptr);
            const HopEntry& e = table[idx];
            atomicMin(&s_lim[q], min(e.row[0], min(e.row[1], e.row[2])));
            atomicMax(&s_lim[g.Q + q], max(e.row[0], max(e.row[1], e.row[2])));
        }
    }
    __syncwarp();
    for (int i = threadIdx.x; i < g.Q; i += blockDim.x) {
        if (s_lim[g.Q + i] >= 0) {
            atomicMin(&F.rowlim[i], s_lim[i]);
            atomicMax(&F.rowlim[g.Q + i], s_lim[g.Q + i]);
        }
    }
}


// Exact float64 Doppler bin of cell (a, b), unwrapped.
__device__ __noinline__ long long slow_bin(double wx, double wy, int a, int b, double lo2, double step2, double lo3,
                                           double step3, double kappa, int Nd) {
    const double vx = gh_axis(lo2, step2, a);
    const double vy = gh_axis(lo3, step3, b);
    const double u = __dmul_rn(kappa, __dadd_rn(__dmul_rn(wx, vx), __dmul_rn(wy, vy)));
    return (long long)floor(__dadd_rn(__dmul_rn((double)Nd, u), 0.5));
}

__device__ __forceinline__ void better(float s, long long c, float& bs, long long& bc) {
    if (s > bs || (s == bs && c < bc)) {
        bs = s;
        bc = c;
    }
}

// Two consecutive map bins (an even bin and the next) of a map row, as float32
// (re0, im0, re1, im1), from storage type MT.
template <int MT>
__device__ __forceinline__ float4 load_pair(const void* row, int jh) {
    if constexpr (MT == GH_C64) {
        return __ldg((const float4*)row + jh);
    } else {
        const uint2 w = __ldg((const uint2*)row + jh);
        float2 a, b;
        if constexpr (MT == GH_C16) {
            a = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
            b = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        } else {
            a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.x));
            b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w.y));
        }
        return make_float4(a.x, a.y, b.x, b.y);
    }
}

// One bin (re, im) of a 16-bit map as float32.
template <int MT>
__device__ __forceinline__ float2 unpack_bin(uint32_t w) {
    if constexpr (MT == GH_C16) {
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    } else {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
}

// Power row P_q[u] = |T_q[u]|^2 (u relative to j_ref) of receiver q, with
// staged entry eq, into Pq: NL lanes (one warp, or the two warps of a pair;
// `lane` in [0, NL)).
template <int MT, int NL = 32>
__device__ __forceinline__ void build_row(const void* __restrict__ maps, const HopParams& p, const HopEntry& eq,
                                          int q, float* Pq, int lane) {
    const int ndm = p.Nd - 1;
    const int j_ref = eq.j_ref, npair = eq.npair;
    const float c0 = eq.cs[0] * p.cscale, c1 = eq.cs[1] * p.cscale, c2 = eq.cs[2] * p.cscale;
    const size_t qb = (size_t)q * p.Nr;
    constexpr size_t BB = MT == GH_C64 ? 8 : 4;  // bytes per bin
    const char* r0 = (const char*)maps + (qb + eq.row[0]) * p.Nd * BB;
    const char* r1 = (const char*)maps + (qb + eq.row[1]) * p.Nd * BB;
    const char* r2 = (const char*)maps + (qb + eq.row[2]) * p.Nd * BB;
    constexpr int U = GH_HOP_U;  // row loads in flight per lane
    if constexpr (MT == GH_C64) {
        // pairs of bins: one 16-byte load per row and pair
        for (int pp0 = 0; pp0 < npair; pp0 += NL * U) {
            float4 z0[U], z1[U], z2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pp = pp0 + lane + NL * u;
                if (pp < npair) {
                    const int jh = ((j_ref + 2 * pp) & ndm) >> 1;  // pair of absolute bins
                    z0[u] = load_pair<MT>(r0, jh);
                    z1[u] = load_pair<MT>(r1, jh);
                    z2[u] = load_pair<MT>(r2, jh);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pp = pp0 + lane + NL * u;
                if (pp < npair) {
                    const float re0 = c0 * z0[u].x + c1 * z1[u].x + c2 * z2[u].x;
                    const float im0 = c0 * z0[u].y + c1 * z1[u].y + c2 * z2[u].y;
                    const float re1 = c0 * z0[u].z + c1 * z1[u].z + c2 * z2[u].z;
                    const float im1 = c0 * z0[u].w + c1 * z1[u].w + c2 * z2[u].w;
                    *(float2*)(Pq + 2 * pp) = make_float2(re0 * re0 + im0 * im0, re1 * re1 + im1 * im1);
                }
            }
        }
    } else {
        // 16-bit maps: groups of four bins (j_ref is a multiple of 4), one
        // 16-byte load per row and group, lanes on consecutive groups; the
        // same registers in flight cover twice the bins of the pair loop
        const int nquad = (npair + 1) >> 1;
        for (int g0 = 0; g0 < nquad; g0 += NL * U) {
            uint4 z0[U], z1[U], z2[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + lane + NL * u;
                if (g < nquad) {
                    const int jq = ((j_ref + 4 * g) & ndm) >> 2;  // group of four absolute bins
                    z0[u] = __ldg((const uint4*)r0 + jq);
                    z1[u] = __ldg((const uint4*)r1 + jq);
                    z2[u] = __ldg((const uint4*)r2 + jq);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int g = g0 + lane + NL * u;
                if (g < nquad) {
                    const uint32_t* w0 = &z0[u].x;
                    const uint32_t* w1 = &z1[u].x;
                    const uint32_t* w2 = &z2[u].x;
                    float pw[4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const float2 a0 = unpack_bin<MT>(w0[b]), a1 = unpack_bin<MT>(w1[b]),
                                     a2 = unpack_bin<MT>(w2[b]);
                        const float re = c0 * a0.x + c1 * a1.x + c2 * a2.x;
                        const float im = c0 * a0.y + c1 * a1.y + c2 * a2.y;
                        pw[b] = re * re + im * im;
                    }
                    *(float4*)(Pq + 4 * g) = make_float4(pw[0], pw[1], pw[2], pw[3]);
                }
            }
        }
    }
}

// Adds receiver q's power-row values at the Doppler bins of the run of AC
// cells (a0 + i SA, b) to acc. Entries of cells on the grid lie in [0, Nd)
// (wrapping mod Nd only when the grid reaches Nd or more bins); cells of a
// partial run past the grid's edge are read and discarded, and the mask keeps
// those reads inside the row as well.
template <int AC>
__device__ __forceinline__ void score_run_q(const HopParams& p, const HopEntry& eq, const float* Pq, int a0, int b,
                                            float (&acc)[AC], float* fix) {
    const int ndm = p.Nd - 1;
    const long long t0 = eq.base + (long long)b * eq.by + (long long)a0 * eq.ax;
    const long long st = (long long)p.SA * eq.ax;
    const int imask = ndm;
    long long t = t0;
    bool amb = false;
    {
#pragma unroll
        for (int i = 0; i < AC; ++i) {
            amb |= (uint32_t)t < p.tol2;
            acc[i] += Pq[(int)(t >> 32) & imask];
            t += st;
        }
    }
    if (amb) {
        // rare: a bin decision within tol of a rounding boundary;
        // replace the fast bin by the float64 one for those cells
        // (corrections go through shared memory so that the
        // float64 path keeps the accumulators in registers)
        t = t0;
#pragma unroll 1
        for (int i = 0; i < AC; ++i) {
            float dlt = 0.f;
            if ((uint32_t)t < p.tol2) {
                const int fast = (int)(t >> 32) & imask;
                const long long j = slow_bin(eq.wx, eq.wy, a0 + i * p.SA, b, p.lo2, p.step2, p.lo3,
                                             p.step3, p.kappa, p.Nd);
                const int exact = (int)(j - eq.j_ref) & imask;
                if (exact != fast) dlt = Pq[exact] - Pq[fast];
            }
            fix[i] = dlt;
            t += st;
        }
#pragma unroll
        for (int i = 0; i < AC; ++i) acc[i] += fix[i];
    }
}

// Best unmasked cell of a run (cells in increasing index order) merged into
// (best, bestc); scores written when asked for.
template <int AC>
__device__ __forceinline__ void finish_run(const HopParams& p, const float (&acc)[AC], long long cbase, int a0, int b,
                                           float* __restrict__ scores, const int64_t* __restrict__ mask, int nmask,
                                           bool hm, float& best, long long& bestc) {
    // best of this run (cells in increasing index order), then merge
    float rb = -INFINITY;
    int ri = -1;
    const bool full = a0 + (AC - 1) * p.SA < p.nvx;
#pragma unroll
    for (int i = 0; i < AC; ++i) {
        if (full || a0 + i * p.SA < p.nvx) {
            const long long cell = cbase + (long long)(a0 + i * p.SA) * p.nvy + b;
            if (scores) scores[cell] = acc[i];
            bool masked = false;
            if (hm)
                for (int m = 0; m < nmask; ++m) masked |= (__ldg(&mask[m]) == cell);
            if (!masked && acc[i] > rb) {
                rb = acc[i];
                ri = i;
            }
        }
    }
    if (ri >= 0) better(rb, cbase + (long long)(a0 + ri * p.SA) * p.nvy + b, best, bestc);
}

// Scores every velocity cell of the (x, y) cell `xy` with one warp: builds the
// Doppler power rows P_q of the receivers in the warp's shared memory, then
// each lane sums the rows at its cells' Doppler bins; merges the best unmasked
// cell into (best, bestc). P, E and fix are the warp's shared-memory areas.
// PR = false: the rows of all Q receivers are built first (P holds Q Nd
// floats), then each run of a lane's cells is scored. PR = true (the lane's
// cells form one run: nvy <= 32 and nvx <= SA AC): one receiver's row at a
// time (P holds Nd floats) added into the run's accumulators, so that frames
// with large Q Nd keep many warps per SM. Same arithmetic in the same order.
template <int AC, int MT, bool PR>
__device__ __forceinline__ void score_xy(const void* __restrict__ maps, const HopEntry* __restrict__ table,
                                         const HopParams& p, float* __restrict__ scores,
                                         const int64_t* __restrict__ mask, int nmask, long long xy, float* P,
                                         HopEntry* E, float* fix, int lane, int tb, int ta, bool active, float& best,
                                         long long& bestc) {
    const int ewords = p.Q * (int)(sizeof(HopEntry) / 8);
    __syncwarp();  // the previous cell's reads of P and E are done
    {
        const long long* src = (const long long*)(table + xy * p.Q);
        long long* dst = (long long*)E;
        for (int w = lane; w < ewords; w += 32) dst[w] = __ldg(src + w);
    }
    __syncwarp();
    // does a masked cell lie in this (x, y) cell's block [xy nv, (xy + 1) nv)?
    auto has_mask = [&]() {
        bool hm = false;
        const long long lo = xy * p.nv, hi = lo + p.nv;
        for (int m = 0; m < nmask; ++m) {
            const long long mc = __ldg(&mask[m]);
            hm |= mc >= lo && mc < hi;
        }
        return hm;
    };
    if constexpr (PR) {
        // the 8 x 4 lane layout (AC = 6, 10) gives a lane one run per vy row
        // it takes; G rows' runs per pass (the rows are rebuilt per pass)
        constexpr int G = (AC == 6 || AC == 10) ? 3 : 1;
        const int nrows = (p.nvy + p.NB - 1) / p.NB;
        const bool hm = has_mask();
        for (int r0 = 0; r0 < nrows; r0 += G) {
            float acc[G][AC];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int i = 0; i < AC; ++i) acc[g][i] = 0.f;
            for (int q = 0; q < p.Q; ++q) {
                build_row<MT>(maps, p, E[q], q, P, lane);
                __syncwarp();  // row q complete
                if (active) {
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int b = tb + p.NB * (r0 + g);
                        if (b < p.nvy) score_run_q<AC>(p, E[q], P, ta, b, acc[g], fix);
                    }
                }
                __syncwarp();  // reads of row q done
            }
            if (active) {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int b = tb + p.NB * (r0 + g);
                    if (b < p.nvy) finish_run<AC>(p, acc[g], xy * p.nv, ta, b, scores, mask, nmask, hm, best, bestc);
                }
            }
        }
    } else {
        for (int q = 0; q < p.Q; ++q) build_row<MT>(maps, p, E[q], q, P + (size_t)q * p.Nd, lane);
        const bool hm = has_mask();
        __syncwarp();  // P rows complete
        if (!active) return;
        const long long cbase = xy * p.nv;
        for (int b = tb; b < p.nvy; b += p.NB) {
            for (int a0 = ta; a0 < p.nvx; a0 += p.SA * AC) {
                float acc[AC];
#pragma unroll
                for (int i = 0; i < AC; ++i) acc[i] = 0.f;
                for (int q = 0; q < p.Q; ++q) score_run_q<AC>(p, E[q], P + (size_t)q * p.Nd, a0, b, acc, fix);
                finish_run<AC>(p, acc, cbase, a0, b, scores, mask, nmask, hm, best, bestc);
            }
        }
    }
}

// Paired scoring: the two warps of a 64-thread CTA score each (x, y) cell
// together, so that one set of power rows (all receivers', Q Nd floats) serves
// 64 lanes and frames with large Q Nd keep twice the warps per SM. The pair's
// lanes v in [0, 64) take b = v % NB (stride NB) and a = v / NB (stride SA)
// with the pair's NB and SA: NB = min(nvy, 32) and SA = 64 / NB, or, in the
// 8 x 4 layout, NB = SA = 8 with runs of 3 or 5 cells (the 6- and 10-cell
// runs split in two). Every cell's sum takes the same terms in the same order
// as score_xy. Both warps pass every __syncthreads below: the loop bounds
// they depend on (cells, Q) are the same for both, and no barrier sits in
// lane- or warp-dependent code.
template <int AC, int MT>
__device__ __forceinline__ void score_xy_pair(const void* __restrict__ maps, const HopEntry* __restrict__ table,
                                              const HopParams& p, float* __restrict__ scores,
                                              const int64_t* __restrict__ mask, int nmask, long long xy, float* P,
                                              HopEntry* E, float* fix, int v, int tb, int ta, bool active,
                                              float& best, long long& bestc) {
    const int ewords = p.Q * (int)(sizeof(HopEntry) / 8);
    __syncthreads();  // the previous cell's reads of P and E are done
    {
        const long long* src = (const long long*)(table + xy * p.Q);
        long long* dst = (long long*)E;
        for (int w = v; w < ewords; w += 64) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    for (int q = 0; q < p.Q; ++q) build_row<MT, 64>(maps, p, E[q], q, P + (size_t)q * p.Nd, v);
    bool hm = false;
    {
        const long long lo = xy * p.nv, hi = lo + p.nv;
        for (int m = 0; m < nmask; ++m) {
            const long long mc = __ldg(&mask[m]);
            hm |= mc >= lo && mc < hi;
        }
    }
    __syncthreads();  // P rows complete
    if (!active) return;
    const long long cbase = xy * p.nv;
    for (int b = tb; b < p.nvy; b += p.NB) {
        for (int a0 = ta; a0 < p.nvx; a0 += p.SA * AC) {
            float acc[AC];
#pragma unroll
            for (int i = 0; i < AC; ++i) acc[i] = 0.f;
            for (int q = 0; q < p.Q; ++q) score_run_q<AC>(p, E[q], P + (size_t)q * p.Nd, a0, b, acc, fix);
            finish_run<AC>(p, acc, cbase, a0, b, scores, mask, nmask, hm, best, bestc);
        }
    }
}

// Paired single-frame scorer: CTA = one pair of warps walking its (x, y)
// cells with score_xy_pair (p.NB, p.SA: the pair's layout), then one argmax
// partial per CTA. Shared memory: all receivers' rows, entries, the 64
// lanes' corrections.
template <int AC, int MT>
__global__ void __launch_bounds__(64, 8) hop_pair_score_kernel(const void* __restrict__ maps,
                                                               const HopEntry* __restrict__ table, HopParams p,
                                                               float* __restrict__ scores,
                                                               const int64_t* __restrict__ mask, int nmask,
                                                               ArgPartial* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char smem_hop[];
    __shared__ float s_bs[2];
    __shared__ long long s_bc[2];
    const int v = threadIdx.x, warp = v >> 5, lane = v & 31;
    float* P = (float*)smem_hop;
    HopEntry* E = (HopEntry*)(P + (size_t)p.Q * p.Nd);
    float* fix = (float*)(E + p.Q) + v * AC;
    const int tb = v % p.NB, ta = v / p.NB;
    const bool active = ta < p.SA;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    const long long xy0 = (long long)blockIdx.x * p.xy_per_cta;
    long long xy1 = xy0 + p.xy_per_cta;
    if (xy1 > p.nxy) xy1 = p.nxy;
    for (long long xy = xy0; xy < xy1; ++xy)
        score_xy_pair<AC, MT>(maps, table, p, scores, mask, nmask, xy, P, E, fix, v, tb, ta, active, best, bestc);
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
    if (v == 0) {
        better(s_bs[1], s_bc[1], best, bestc);
        parts[blockIdx.x].score = best;
        parts[blockIdx.x].cell = bestc;
    }
}

// AC: velocity cells per lane per pass (along vx, stride SA); MT: map storage
// type; PR: one receiver's power row at a time (see score_xy).
template <int AC, int MT, bool PR>
__global__ void __launch_bounds__(256, GH_HOP_MINB) hop_score_kernel(const void* __restrict__ maps,
                                                           const HopEntry* __restrict__ table, HopParams p,
                                                           float* __restrict__ scores,
                                                           const int64_t* __restrict__ mask, int nmask,
                                                           ArgPartial* __restrict__ parts) {
    // [warps] x ([Q][Nd] floats, or [Nd] with PR, + [Q] entries + corrections)
    extern __shared__ __align__(16) unsigned char smem_hop[];
    __shared__ float s_bs[8];
    __shared__ long long s_bc[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const size_t pfloats = PR ? (size_t)p.Nd : (size_t)p.Q * p.Nd;
    const size_t warp_bytes =
        pfloats * sizeof(float) + (size_t)p.Q * sizeof(HopEntry) + (size_t)32 * AC * sizeof(float);
    float* P = (float*)(smem_hop + warp * warp_bytes);
    HopEntry* E = (HopEntry*)(P + pfloats);
    float* fix = (float*)(E + p.Q) + lane * AC;  // per-lane corrections of the float64 path
    const int tb = lane % p.NB, ta = lane / p.NB;
    const bool active = ta < p.SA;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;

    const long long xy0 = (long long)blockIdx.x * p.xy_per_cta;
    long long xy1 = xy0 + p.xy_per_cta;
    if (xy1 > p.nxy) xy1 = p.nxy;
    for (long long xy = xy0 + warp; xy < xy1; xy += W) {
        score_xy<AC, MT, PR>(maps, table, p, scores, mask, nmask, xy, P, E, fix, lane, tb, ta, active, best, bestc);
    }


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
    if (threadIdx.x == 0) {
        for (int w = 1; w < W; ++w) better(s_bs[w], s_bc[w], best, bestc);
        parts[blockIdx.x].score = best;
        parts[blockIdx.x].cell = bestc;
    }
}

__global__ void __launch_bounds__(1024) argmax_finalize_kernel(const ArgPartial* __restrict__ parts, int n,
                                                               ArgResult* __restrict__ out) {
    __shared__ float s_bs[32];
    __shared__ long long s_bc[32];
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    for (int i = threadIdx.x; i < n; i += blockDim.x) better(parts[i].score, parts[i].cell, best, bestc);
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
        out->cell = bestc;
        out->score = best;
        out->valid = bestc != 0x7fffffffffffffffLL;
    }
}

HopParams hop_params(const Dims& d, const GeoParams& g) {
    HopParams hp;
    hp.Q = d.Q;
    hp.Nr = d.Nr;
    hp.Nd = d.Nd;
    hp.nvx = d.nvx;
    hp.nvy = d.nvy;
    hp.cscale = 1.0f;
    hp.NB = d.nvy < 32 ? d.nvy : 32;
    hp.SA = 32 / hp.NB;
    hp.tol2 = 2u * hop_tol(d.nvx, d.nvy);
    hp.nxy = d.nxy;
    hp.nv = d.nv;
    hp.xy_per_cta = 1;
    hp.lo2 = g.lo[2];
    hp.step2 = g.step[2];
    hp.lo3 = g.lo[3];
    hp.step3 = g.step[3];
    hp.kappa = g.kappa;
    return hp;
}

CoordParams coord_params(const Dims& d);

// Shared memory of one scorer warp: power rows (all receivers', or one with
// PR), entries, float64-path corrections.
inline size_t hop_warp_bytes(const Dims& d, int ac, bool pr) {
    return (size_t)(pr ? 1 : d.Q) * d.Nd * sizeof(float) + (size_t)d.Q * sizeof(HopEntry) +
           (size_t)32 * ac * sizeof(float);
}

// Launch of the scorer (shared by the context path and the allocation-free
// entry point). Returns the number of CTAs (partials) in *nparts.
template <int AC, int MT, bool PR>
int hop_launch_t(cudaStream_t stream, const Dims& d, HopParams hp, const void* maps, const HopEntry* table,
                 float* scores, const int64_t* mask, int nmask, ArgPartial* parts, long long max_ctas, int num_sms,
                 size_t smem_optin, long long* nparts) {
    const size_t per_warp = hop_warp_bytes(d, AC, PR);
    if (per_warp > smem_optin) return GH_ENOTSUP;
    int W = (int)((size_t)(100 << 10) / per_warp);
    if (W > 8) W = 8;
    if (W < 1) W = 1;
    const size_t smem = per_warp * W;
    auto kern = hop_score_kernel<AC, MT, PR>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return GH_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W, smem) != cudaSuccess) return GH_ECUDA;
    if (per_sm < 1) per_sm = 1;
    long long ctas = (long long)num_sms * per_sm;
    if (ctas > max_ctas) ctas = max_ctas;
    if (ctas > d.nxy) ctas = d.nxy;
    hp.xy_per_cta = (d.nxy + ctas - 1) / ctas;
    ctas = (d.nxy + hp.xy_per_cta - 1) / hp.xy_per_cta;
    // the launch's own status (cudaLaunchKernelEx returns it), so that an error
    // another caller left pending in the thread is neither reported nor cleared
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(32 * W);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    *nparts = ctas;
    if (cudaLaunchKernelEx(&cfg, kern, maps, table, hp, scores, mask, nmask, parts) != cudaSuccess) {
        (void)cudaGetLastError();  // consume this launch's own error
        return GH_ECUDA;
    }
    return GH_OK;
}

// Shared memory of one paired scorer CTA: all receivers' rows, entries, the
// 64 lanes' corrections.
inline size_t hop_pair_frame_bytes(const Dims& d, int ac) {
    const size_t b = (size_t)d.Q * d.Nd * sizeof(float) + (size_t)d.Q * sizeof(HopEntry) +
                     (size_t)64 * ac * sizeof(float);
    return (b + 15) & ~(size_t)15;
}

// Whether the paired scorer (pair_bytes per 64-thread CTA) keeps more warps
// per SM than one warp per cell (per_warp bytes, W warps per CTA as
// hop_launch_t picks them), from the 128-register budget of both and the
// SM's shared memory (1 KiB reserved per CTA).
inline bool pair_keeps_more_warps(size_t per_warp, size_t pair_bytes, size_t smem_optin) {
    const size_t sm = smem_optin + 1024;
    int W = (int)((size_t)(100 << 10) / per_warp);
    if (W > 8) W = 8;
    if (W < 1) W = 1;
    const size_t by_regs = (size_t)(16 / W), by_smem = sm / (W * per_warp + 1024);
    const size_t one = (size_t)W * std::min(by_regs, by_smem);
    const size_t two = 2 * std::min((size_t)8, sm / (pair_bytes + 1024));
    return two > one;
}

// Launch of the paired scorer; hp carries the pair's NB and SA.
template <int AC, int MT>
int hop_pair_launch_t(cudaStream_t stream, const Dims& d, HopParams hp, const void* maps, const HopEntry* table,
                      float* scores, const int64_t* mask, int nmask, ArgPartial* parts, long long max_ctas,
                      int num_sms, size_t smem_optin, long long* nparts) {
    const size_t smem = hop_pair_frame_bytes(d, AC);
    if (smem > smem_optin) return GH_ENOTSUP;
    auto kern = hop_pair_score_kernel<AC, MT>;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(smem_optin - fa.sharedSizeBytes)) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return GH_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64, smem) != cudaSuccess) return GH_ECUDA;
    if (per_sm < 1) per_sm = 1;
    long long ctas = (long long)num_sms * per_sm;
    if (ctas > max_ctas) ctas = max_ctas;
    if (ctas > d.nxy) ctas = d.nxy;
    hp.xy_per_cta = (d.nxy + ctas - 1) / ctas;
    ctas = (d.nxy + hp.xy_per_cta - 1) / hp.xy_per_cta;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(64);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    *nparts = ctas;
    if (cudaLaunchKernelEx(&cfg, kern, maps, table, hp, scores, mask, nmask, parts) != cudaSuccess) {
        (void)cudaGetLastError();  // consume this launch's own error
        return GH_ECUDA;
    }
    return GH_OK;
}

template <int MT>
int hop_launch_mt(cudaStream_t stream, const Dims& d, const HopParams& hp, const void* maps, const HopEntry* table,
                  float* scores, const int64_t* mask, int nmask, ArgPartial* parts, long long max_ctas, int num_sms,
                  size_t smem_optin, long long* nparts) {
    // cells per lane and run: at most 16 (a lane takes several runs when the
    // velocity axis is longer); measured faster than 32 on the paper-shaped
    // frame (82 against 86 us per launch) at the same occupancy
    // lanes 8 (vy) x 4 (vx) with 6 or 10 cells per run where that fills the
    // runs best (velocity axes of 24 or 40 cells); one receiver's row at a
    // time when the rows of all receivers would leave fewer than eight warps
    // per CTA and each vy row of a lane is one run
    const int lay = lane_layout_ac(d);
    if (lay) {
        HopParams h8 = hp;
        h8.NB = 8;
        h8.SA = 4;
        const bool pr8 = (d.nvx + 3) / 4 <= lay && hop_warp_bytes(d, lay, false) * 8 > (100 << 10);
        // all rows: two warps per (x, y) cell where that keeps more warps per SM
        if (!pr8 && pair_keeps_more_warps(hop_warp_bytes(d, lay, false), hop_pair_frame_bytes(d, lay / 2),
                                          smem_optin)) {
            HopParams h2 = hp;
            h2.NB = 8;
            h2.SA = 8;
            return lay == 6 ? hop_pair_launch_t<3, MT>(stream, d, h2, maps, table, scores, mask, nmask, parts,
                                                       max_ctas, num_sms, smem_optin, nparts)
                            : hop_pair_launch_t<5, MT>(stream, d, h2, maps, table, scores, mask, nmask, parts,
                                                       max_ctas, num_sms, smem_optin, nparts);
        }
#define GH_HOP_LAYOUT(N)                                                                                          \
    return pr8 ? hop_launch_t<N, MT, true>(stream, d, h8, maps, table, scores, mask, nmask, parts, max_ctas,      \
                                           num_sms, smem_optin, nparts)                                          \
               : hop_launch_t<N, MT, false>(stream, d, h8, maps, table, scores, mask, nmask, parts, max_ctas,     \
                                            num_sms, smem_optin, nparts);
        if (lay == 6) GH_HOP_LAYOUT(6)
        GH_HOP_LAYOUT(10)
#undef GH_HOP_LAYOUT
    }
    const int full = (d.nvx + hp.SA - 1) / hp.SA;
    const int need = std::min(full, 16);
    // one receiver's row at a time when the lane's cells form one run and the
    // rows of all receivers would leave fewer than eight warps per CTA
    const int ac = need <= 1 ? 1 : need <= 2 ? 2 : need <= 4 ? 4 : need <= 8 ? 8 : 16;
    const bool pr = d.nvy <= 32 && full <= 16 && hop_warp_bytes(d, ac, false) * 8 > (100 << 10);
    if (!pr) {
        // all rows: two warps per (x, y) cell (SA doubled) where that keeps
        // more warps per SM
        HopParams h2 = hp;
        h2.SA = 64 / hp.NB;
        const int pac = (d.nvx + h2.SA - 1) / h2.SA <= 8 ? 8 : 16;
        if (pair_keeps_more_warps(hop_warp_bytes(d, ac, false), hop_pair_frame_bytes(d, pac), smem_optin))
            return pac == 8 ? hop_pair_launch_t<8, MT>(stream, d, h2, maps, table, scores, mask, nmask, parts,
                                                       max_ctas, num_sms, smem_optin, nparts)
                            : hop_pair_launch_t<16, MT>(stream, d, h2, maps, table, scores, mask, nmask, parts,
                                                        max_ctas, num_sms, smem_optin, nparts);
    }
#define GH_HOP_CASE(N)                                                                                             \
    if (need <= N)                                                                                                 \
        return pr ? hop_launch_t<N, MT, true>(stream, d, hp, maps, table, scores, mask, nmask, parts, max_ctas,  \
                                              num_sms, smem_optin, nparts)                                         \
                  : hop_launch_t<N, MT, false>(stream, d, hp, maps, table, scores, mask, nmask, parts, max_ctas, \
                                               num_sms, smem_optin, nparts);
    GH_HOP_CASE(1)
    GH_HOP_CASE(2)
    GH_HOP_CASE(4)
    GH_HOP_CASE(8)
    GH_HOP_CASE(16)
#undef GH_HOP_CASE
    return GH_ENOTSUP;
}

int hop_launch(cudaStream_t stream, const Dims& d, HopParams hp, const void* maps, int map_dtype,
               const HopEntry* table, float* scores, const int64_t* mask, int nmask, ArgPartial* parts,
               long long max_ctas, int num_sms, size_t smem_optin, long long* nparts) {
    hp.cscale = ldexpf(1.0f, gh_map_scale_log2(d, map_dtype));
    if (map_dtype == GH_C16)
        return hop_launch_mt<GH_C16>(stream, d, hp, maps, table, scores, mask, nmask, parts, max_ctas, num_sms,
                                     smem_optin, nparts);
    if (map_dtype == GH_CBF16)
        return hop_launch_mt<GH_CBF16>(stream, d, hp, maps, table, scores, mask, nmask, parts, max_ctas, num_sms,
                                       smem_optin, nparts);
    return hop_launch_mt<GH_C64>(stream, d, hp, maps, table, scores, mask, nmask, parts, max_ctas, num_sms,
                                 smem_optin, nparts);
}

// Lane layout: b = lane % NB, a = lane / NB with the frame's NB = min(nvy, 32)
// for AC = 8, 16, 32, and NB = 8, SA = 4 for AC = 6 and 10 (a lane's cells
// of a 24 x 24 or 40 x 40 velocity grid then fill its runs exactly).
// Persistent batched scorer (complex float32 maps): each warp takes work items
// (frame, first (x, y) cell, count) from *counter until none is left, scores
// the item's cells with score_xy and folds the item's best unmasked cell into
// the frame's key[k] = score bits << 32 | (2^32 - 1 - cell) (largest key: best
// score, then smallest cell). The warp's shared-memory area holds a copy of
// the frame's scorer parameters, its power rows, entries and corrections.
template <int AC, bool PR>
__global__ void __launch_bounds__(256, GH_HOP_MINB) hop_batch_kernel(const BatchFrame* __restrict__ frames,
                                                          const BatchItem* __restrict__ items, int nitems,
                                                          unsigned* __restrict__ counter, int k,
                                                          int per_warp_bytes) {
    extern __shared__ __align__(16) unsigned char smem_hop[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = smem_hop + (size_t)warp * per_warp_bytes;
    HopParams& p = *(HopParams*)base;
    constexpr int kParamBytes = (int)((sizeof(HopParams) + 15) & ~(size_t)15);
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(counter, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nitems) break;
        const BatchItem item = items[it];
        const BatchFrame& F = frames[item.frame];
        __syncwarp();  // the previous item's reads of p are done
        {
            const int* src = (const int*)&F.hp;
            int* dst = (int*)&p;
            for (int w = lane; w < (int)(sizeof(HopParams) / 4); w += 32) dst[w] = src[w];
        }
        __syncwarp();
        if constexpr (AC == 6 || AC == 10) {  // lanes 8 (vy) x 4 (vx): grids of 24 or 40 velocities per axis
            if (lane == 0) {
                p.NB = 8;
                p.SA = 4;
            }
            __syncwarp();
        }
        float* P = (float*)(base + kParamBytes);
        HopEntry* E = (HopEntry*)(P + (PR ? (size_t)p.Nd : (size_t)p.Q * p.Nd));
        float* fix = (float*)(E + p.Q) + lane * AC;
        const int tb = lane % p.NB, ta = lane / p.NB;
        const bool active = ta < p.SA;
        float best = -INFINITY;
        long long bestc = 0x7fffffffffffffffLL;
        for (long long xy = item.start; xy < item.start + item.count; ++xy)
            score_xy<AC, GH_C64, PR>(F.maps, (const HopEntry*)F.table, p, nullptr, F.mask, k, xy, P, E, fix, lane,
                                     tb, ta, active, best, bestc);
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_down_sync(0xffffffffu, best, off);
            const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
            better(os, oc, best, bestc);
        }
        if (lane == 0 && bestc != 0x7fffffffffffffffLL) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(best) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)bestc);
            atomicMax(&F.key[k], key);
        }
    }
}

// Persistent paired batched scorer (complex float32 maps, all receivers'
// rows): each CTA of two warps takes work items from *counter as
// hop_batch_kernel's warps do and scores their cells with score_xy_pair (the
// loop bounds come from shared memory, so both warps pass the same barriers);
// each warp folds its own best cell into the frame's key. L8: the 8 x 4
// layout's runs split in two (NB = SA = 8, AC = 3 or 5), else the standard
// layout with SA doubled (SA = 64 / NB). Shared memory: the frame's scorer
// parameters (with the pair's NB and SA), power rows, entries and the 64
// lanes' corrections.
template <int AC, bool L8>
__global__ void __launch_bounds__(64, 8) hop_pair_kernel(const BatchFrame* __restrict__ frames,
                                                         const BatchItem* __restrict__ items, int nitems,
                                                         unsigned* __restrict__ counter, int k) {
    extern __shared__ __align__(16) unsigned char smem_hop[];
    __shared__ int s_item;
    const int v = threadIdx.x, lane = v & 31;
    HopParams& p = *(HopParams*)smem_hop;
    constexpr int kParamBytes = (int)((sizeof(HopParams) + 15) & ~(size_t)15);
    for (;;) {
        if (v == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();  // s_item set; the previous item's reads of p are done
        const int it = s_item;
        if (it >= nitems) break;  // the same for both warps
        const BatchItem item = items[it];
        const BatchFrame& F = frames[item.frame];
        {
            const int* src = (const int*)&F.hp;
            int* dst = (int*)&p;
            for (int w = v; w < (int)(sizeof(HopParams) / 4); w += 64) dst[w] = src[w];
        }
        __syncthreads();  // p copied; both warps have read s_item
        if (v == 0) {
            if (L8) {
                p.NB = 8;
                p.SA = 8;
            } else {
                p.SA = 64 / p.NB;  // NB = min(nvy, 32)
            }
        }
        __syncthreads();
        const int tb = v % p.NB, ta = v / p.NB;
        const bool active = ta < p.SA;
        float* P = (float*)(smem_hop + kParamBytes);
        HopEntry* E = (HopEntry*)(P + (size_t)p.Q * p.Nd);
        float* fix = (float*)(E + p.Q) + v * AC;
        float best = -INFINITY;
        long long bestc = 0x7fffffffffffffffLL;
        for (long long xy = item.start; xy < item.start + item.count; ++xy)
            score_xy_pair<AC, GH_C64>(F.maps, (const HopEntry*)F.table, p, nullptr, F.mask, k, xy, P, E, fix, v,
                                      tb, ta, active, best, bestc);
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_down_sync(0xffffffffu, best, off);
            const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
            better(os, oc, best, bestc);
        }
        if (lane == 0 && bestc != 0x7fffffffffffffffLL) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(best) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)bestc);
            atomicMax(&F.key[k], key);
        }
    }
}

// Shared memory of one paired-scorer CTA for frames with Q Nd <= row_floats.
size_t hop_pair_bytes(int ac, int row_floats, int max_q) {
    const size_t b = ((sizeof(HopParams) + 15) & ~(size_t)15) + (size_t)row_floats * sizeof(float) +
                     (size_t)max_q * sizeof(HopEntry) + (size_t)64 * ac * sizeof(float);
    return (b + 15) & ~(size_t)15;
}

template <int AC, bool L8>
int hop_pair_launch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, unsigned* counter, int k,
                    int max_q_nd, int max_q) {
    const size_t smem = hop_pair_bytes(AC, max_q_nd, max_q);
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "paired scorer: %zu bytes of shared memory", smem);
    auto kern = hop_pair_kernel<AC, L8>;
    // the function's limit: the device's largest (see hop_batch_launch)
    cudaFuncAttributes fa;
    GH_CUDA(cudaFuncGetAttributes(&fa, kern));
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ctx->smem_optin - fa.sharedSizeBytes)));
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64, smem));
    if (per_sm < 1) per_sm = 1;
    GH_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_HOP_SCORE, &ev);
    kern<<<ctx->num_sms * per_sm, 64, smem, ctx->stream>>>(frames, items, n, counter, k);
    return gh_launch_end(ctx, GH_K_HOP_SCORE, ev, "hop_pair_kernel");
}

// Shared memory of one batched-scorer warp for frames with power rows of at
// most `row_floats` floats (Q * Nd, or Nd with one receiver's row at a time).
size_t hop_batch_warp_bytes(int ac, int row_floats, int max_q) {
    const size_t b = ((sizeof(HopParams) + 15) & ~(size_t)15) + (size_t)row_floats * sizeof(float) +
                     (size_t)max_q * sizeof(HopEntry) + (size_t)32 * ac * sizeof(float);
    return (b + 15) & ~(size_t)15;
}

template <int AC, bool PR>
int hop_batch_launch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, unsigned* counter, int k,
                     int warps, int max_nd, int max_q_nd, int max_q) {
    const size_t per_warp = hop_batch_warp_bytes(AC, PR ? max_nd : max_q_nd, max_q);
    const size_t smem = per_warp * warps;
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "batched scorer: %zu bytes of shared memory", smem);
    auto kern = hop_batch_kernel<AC, PR>;
    // The classes of one batch launch the same kernel with different shared
    // memory; the function's limit is set to the device's largest, so that
    // every launch (also a graph node launched on its own) stays within it
    // whatever class set it last.
    cudaFuncAttributes fa;
    GH_CUDA(cudaFuncGetAttributes(&fa, kern));
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ctx->smem_optin - fa.sharedSizeBytes)));
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps, smem));
    if (per_sm < 1) per_sm = 1;
    GH_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_HOP_SCORE, &ev);
    kern<<<ctx->num_sms * per_sm, 32 * warps, smem, ctx->stream>>>(frames, items, n, counter, k, (int)per_warp);
    return gh_launch_end(ctx, GH_K_HOP_SCORE, ev, "hop_batch_kernel");
}

double dirichlet_closed(double f, int M) {
    const double pi = 3.14159265358979323846264338327950288;
    return sin(pi * M * f) / sin(pi * f);
}

CoordParams coord_params(const Dims& d) {
    CoordParams cp;
    // Half-arc angle of the three-bin polar model, from the Gram of centred
    // atoms: cos(theta/2) = 1/2 sqrt((Ms - D(2/Nr)) / (Ms - D(1/Nr))).
    const double D1 = dirichlet_closed(1.0 / d.Nr, d.Ms), D2 = dirichlet_closed(2.0 / d.Nr, d.Ms);
    const double theta = 2.0 * acos(0.5 * sqrt((d.Ms - D2) / (d.Ms - D1)));
    const double sh = sin(0.5 * theta);
    cp.theta_f = (float)theta;
    cp.inv_sin2_half = (float)(1.0 / (sh * sh));
    cp.inv_sin_t = (float)(1.0 / sin(theta));
    cp.Ms_odd_sign = ((d.Ms - 1) & 1) ? 1 : 0;
    cp.tol = hop_tol(d.nvx, d.nvy);
    return cp;
}

}  // namespace

size_t gh_hop_table_bytes(const Dims& d) { return (size_t)d.nxy * d.Q * sizeof(HopEntry); }

int gh_launch_coord(gh_ctx* ctx, const Dims& d, const GeoParams& g, void* table, int32_t* diag_i,
                    double* diag_tau, float* diag_c, double* diag_w, int* rowlim, double* rw) {
    const CoordParams cp = coord_params(d);
    if (rowlim) {  // minima 0x7f7f7f7f, maxima -1 (byte patterns)
        GH_CUDA(cudaMemsetAsync(rowlim, 0x7f, (size_t)d.Q * sizeof(int), ctx->stream));
        GH_CUDA(cudaMemsetAsync(rowlim + d.Q, 0xff, (size_t)d.Q * sizeof(int), ctx->stream));
    }
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_COORD, &ev);
    // one warp per CTA: the (x, y) cells spread over every SM's sub-partitions
    coord_kernel<<<(unsigned)((2 * d.nxy + 31) / 32), 32, 0, ctx->stream>>>(g, cp, (HopEntry*)table, diag_i,
                                                                             diag_tau, diag_c, diag_w, rowlim, rw);
    return gh_launch_end(ctx, GH_K_COORD, ev, "coord_kernel");
}

int gh_launch_argmax_finalize(gh_ctx* ctx, const ArgPartial* parts, int nparts, ArgResult* out) {
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
    argmax_finalize_kernel<<<1, 1024, 0, ctx->stream>>>(parts, nparts, out);
    return gh_launch_end(ctx, GH_K_ARGMAX, ev, "argmax_finalize_kernel");
}

int gh_launch_hop_parts(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                        const void* table, float* scores, const int64_t* mask, int nmask, ArgPartial** parts_out,
                        int* nparts_out) {
    const HopParams hp = hop_params(d, g);
    const long long max_ctas = (long long)ctx->num_sms * 32;
    void* parts;
    GH_TRY(gh_ws(ctx, WS_PART, (size_t)max_ctas * sizeof(ArgPartial), &parts));
    cudaEvent_t ev;
    long long nparts = 0;
    gh_launch_begin(ctx, GH_K_HOP_SCORE, &ev);
    const int st = hop_launch(ctx->stream, d, hp, maps, map_dtype, (const HopEntry*)table, scores, mask, nmask,
                              (ArgPartial*)parts, max_ctas, ctx->num_sms, ctx->smem_optin, &nparts);
    if (st == GH_ENOTSUP) return gh_fail(ctx, GH_ENOTSUP, "hop scorer: Q*Nd*4 bytes exceed shared memory");
    GH_TRY(gh_launch_end(ctx, GH_K_HOP_SCORE, ev, "hop_score_kernel"));
    if (st != GH_OK) return gh_fail(ctx, st, "hop scorer launch failed");
    *parts_out = (ArgPartial*)parts;
    *nparts_out = (int)nparts;
    return GH_OK;
}

int gh_launch_hop(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                  const void* table, float* scores, const int64_t* mask, int nmask, ArgResult* result) {
    ArgPartial* parts;
    int nparts;
    GH_TRY(gh_launch_hop_parts(ctx, d, g, maps, map_dtype, table, scores, mask, nmask, &parts, &nparts));
    return gh_launch_argmax_finalize(ctx, parts, nparts, result);
}

// ---------------------------------------------------------------------------
// gh_score_grid_noalloc: the hopping score and argmax of gh_score_grid for
// callers that cannot allocate device memory. The paper has no counterpart.
//
// Its scratch (coordinate table, per-CTA argmax partials, result slot) is the
// file-scope array below, which every GPU that loads the library holds until
// the process exits. Host code only ever passes the array's device address,
// obtained per device with cudaGetSymbolAddress on the first call made with
// that device current (the array's name in host code is a host-side stand-in,
// not a device address). Nothing in the array needs to start at zero: every
// call writes each scratch word it reads. All calls share the array, so calls
// whose GPU work overlaps (two streams, two host threads) race on it.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kNoAllocTableBytes = (size_t)GH_NOALLOC_MAX_XYQ * sizeof(HopEntry);
constexpr int kNoAllocMaxCtas = 4096;
constexpr size_t kNoAllocPartsBytes = (size_t)kNoAllocMaxCtas * sizeof(ArgPartial);
constexpr size_t kNoAllocBytes = kNoAllocTableBytes + kNoAllocPartsBytes + 256;
static_assert(kNoAllocBytes <= ((size_t)8 << 20), "scratch must stay at or below 8 MiB");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};  // device address of the scratch, per device ordinal

int noalloc_scratch(int dev, unsigned char** p) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GH_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess || !addr) return GH_ECUDA;
        g_noalloc_addr[dev] = addr;
    }
    *p = (unsigned char*)g_noalloc_addr[dev];
    return GH_OK;
}

// Launches kernel<<<grid, block, 0, stream>>>(args...) and returns GH_ECUDA
// if that launch itself failed (its error is consumed), GH_OK otherwise.
template <typename... P, typename... A>
int noalloc_launch(void (*kernel)(P...), dim3 grid, dim3 block, cudaStream_t stream, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.stream = stream;
    if (cudaLaunchKernelEx(&cfg, kernel, args...) != cudaSuccess) {
        (void)cudaGetLastError();
        return GH_ECUDA;
    }
    return GH_OK;
}

}  // namespace

extern "C" int gh_score_grid_noalloc(void* stream_ptr, const gh_radar* radar, const double* tx_host,
                                     const double* rx_host, int32_t Q, const void* maps_dev, const gh_grid* grid,
                                     float* scores_dev, int64_t* best_cell, float* best_score) {
    Dims d = {};
    GH_TRY(gh_check_radar(nullptr, radar, Q, &d));
    GH_TRY(gh_check_grid(nullptr, grid, &d));
    GH_TRY(gh_check_positions(nullptr, tx_host, rx_host, Q));
    if (!maps_dev) return GH_EINVAL;
    if (d.nxy * d.Q > (int64_t)GH_NOALLOC_MAX_XYQ) return GH_EINVAL;  // beyond the fixed scratch
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    int dev = 0, num_sms = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GH_ECUDA;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GH_ECUDA;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return GH_ECUDA;
    unsigned char* scratch;
    GH_TRY(noalloc_scratch(dev, &scratch));
    HopEntry* table = (HopEntry*)scratch;
    ArgPartial* parts = (ArgPartial*)(scratch + kNoAllocTableBytes);
    ArgResult* result = (ArgResult*)(scratch + kNoAllocTableBytes + kNoAllocPartsBytes);

    GeoParams g;
    gh_fill_geo(&g, radar, tx_host, rx_host, Q, grid);
    const CoordParams cp = coord_params(d);
    // launches checked by their own return status (noalloc_launch): an error
    // left pending by other code in this thread is neither reported nor cleared
    GH_TRY(noalloc_launch(coord_kernel, dim3((unsigned)((2 * d.nxy + 31) / 32)), dim3(32), stream, g, cp, table,
                          (int32_t*)nullptr, (double*)nullptr, (float*)nullptr, (double*)nullptr, (int*)nullptr,
                          (double*)nullptr));
    const HopParams hp = hop_params(d, g);
    long long nparts = 0;
    int st = hop_launch(stream, d, hp, maps_dev, GH_C64, table, scores_dev, nullptr, 0, parts,
                        kNoAllocMaxCtas, num_sms, (size_t)smem_optin, &nparts);
    if (st != GH_OK) return st;
    GH_TRY(noalloc_launch(argmax_finalize_kernel, dim3(1), dim3(1024), stream, (const ArgPartial*)parts,
                          (int)nparts, result));
    if (best_cell || best_score) {
        ArgResult h;
        if (cudaMemcpyAsync(&h, result, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return GH_ECUDA;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return GH_ECUDA;
        if (best_cell) *best_cell = h.cell;
        if (best_score) *best_score = h.score;
    }
    return GH_OK;
}

void gh_hop_frame_params(const Dims& d, const GeoParams& g, HopParams* hp, CoordParams* cp) {
    *hp = hop_params(d, g);
    *cp = coord_params(d);
}

int gh_launch_coord_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n) {
    if (n == 0) return GH_OK;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_COORD, &ev);
    coord_batch_kernel<<<n, 32, 0, ctx->stream>>>(frames, items);
    return gh_launch_end(ctx, GH_K_COORD, ev, "coord_batch_kernel");
}

int gh_launch_hop_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, unsigned* counter,
                        int k, int ac, int warps, bool per_rx, bool pair, int max_nd, int max_q_nd, int max_q) {
    if (n == 0) return GH_OK;
    if (pair) {  // two warps per (x, y) cell
        if (warps != 2 || per_rx) return gh_fail(ctx, GH_EINVAL, "paired scorer: 2 warps, all rows");
        if (ac == 3) return hop_pair_launch<3, true>(ctx, frames, items, n, counter, k, max_q_nd, max_q);
        if (ac == 5) return hop_pair_launch<5, true>(ctx, frames, items, n, counter, k, max_q_nd, max_q);
        if (ac == 8) return hop_pair_launch<8, false>(ctx, frames, items, n, counter, k, max_q_nd, max_q);
        if (ac == 16) return hop_pair_launch<16, false>(ctx, frames, items, n, counter, k, max_q_nd, max_q);
        return gh_fail(ctx, GH_EINVAL, "paired scorer: cells per lane %d not in {3, 5, 8, 16}", ac);
    }
#define GH_BATCH_CASE(N)                                                                                            \
    if (ac == N)                                                                                                    \
        return per_rx ? hop_batch_launch<N, true>(ctx, frames, items, n, counter, k, warps, max_nd, max_q_nd, max_q) \
                      : hop_batch_launch<N, false>(ctx, frames, items, n, counter, k, warps, max_nd, max_q_nd, max_q);
    GH_BATCH_CASE(8)
    GH_BATCH_CASE(16)
    GH_BATCH_CASE(32)
    GH_BATCH_CASE(6)
    GH_BATCH_CASE(10)
#undef GH_BATCH_CASE
    return gh_fail(ctx, GH_EINVAL, "batched scorer: cells per lane %d not in {6, 8, 10, 16, 32}", ac);
}

size_t gh_hop_batch_warp_bytes(int ac, int row_floats, int max_q) { return hop_batch_warp_bytes(ac, row_floats, max_q); }
size_t gh_hop_pair_bytes(int ac, int row_floats, int max_q) { return hop_pair_bytes(ac, row_floats, max_q); }
