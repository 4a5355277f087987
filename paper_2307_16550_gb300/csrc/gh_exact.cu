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
                                                           float* __restrict__ P) {
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
            if (mc < g.Mc) {
                float* row = P + ((size_t)q * nxy + xy) * 2 * g.Mc;  // planar: Re row, then Im row
                row[mc] = acc[i][j].x;
                row[g.Mc + mc] = acc[i][j].y;
            }
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
__global__ void __launch_bounds__(256) exact_stage2_kernel(const float* __restrict__ P, GeoParams g,
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
        const float* Pq = P + ((size_t)q * nxy + xy) * 2 * g.Mc;  // planar: Re row, then Im row
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
                const float2 pv = mc < g.Mc ? make_float2(Pq[mc], Pq[g.Mc + mc]) : make_float2(0.f, 0.f);
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
int launch_s2(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float* P, float* scores, const int64_t* mask,
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
// a complex (nvx x Mc) x (Mc x nvy) product, written as the four real
// products of its parts (Re Ex Re G, Re Ex Im G, Im Ex Re G, Im Ex Im G) in
// one real GEMM D = A B^T with K = Mc:
//   A rows (M = 128): Re Ex and Im Ex of every velocity row a, each split into
//     BF16 high and low parts (x = hi + lo to about 16 significant bits);
//   B rows (N = 4 nvy_pad): Re G and Im G of every velocity column b, split
//     the same way.
// Every block of D is used: Re F = sum (ReA ReB - ImA ImB), Im F = sum (ReA ImB
// + ImA ReB) over the four (A part, B part) split combinations, so four MMAs
// per 64 chirps give the split-BF16 product of one receiver (FP32 products of
// BF16 values are exact; the accumulation is FP32 in tensor memory).
// Operands are K-major in the 128-byte swizzled layout, one 128-byte row of 64
// chirps per operand row and stage. Row orders are chosen so that a 16x256b
// tensor-memory load hands each epilogue thread all sixteen partial products
// of its cells:
//   A row 32 (a / 8) + 8 s + a % 8, s = (Re hi, Re lo, Im hi, Im lo);
//   B row 32 (b / 8) + 8 t + b % 8, t = (Re hi, Im hi, Re lo, Im lo).
// ---------------------------------------------------------------------------
struct ExEntry {
    unsigned long long rfix;        // r_q(x): cycles per sample, 2^64 fixed point
    unsigned long long phx0, dphx;  // kappa wx vx_0 and kappa wx step_x (cycles per chirp)
    unsigned long long phy0, dphy;  // kappa wy vy_0 and kappa wy step_y
};

// Two threads per (x, y), each taking every other receiver, the
// transmitter's distance and unit vector once per thread (float64
// latency-bound, like coord_kernel).
__global__ void exact_coord_kernel(GeoParams g, ExEntry* __restrict__ tab) {
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long xy = t >> 1;
    const int q0 = (int)(t & 1);
    if (xy >= nxy) return;
    const int ix = (int)(xy / g.n[1]);
    const int iy = (int)(xy - (long long)ix * g.n[1]);
    const double x = gh_axis(g.lo[0], g.step[0], ix), y = gh_axis(g.lo[1], g.step[1], iy);
    double n1, ux1, uy1;
    gh_unit(__dsub_rn(x, g.tx[0]), __dsub_rn(y, g.tx[1]), &n1, &ux1, &uy1);
    for (int q = q0; q < g.Q; q += 2) {
        double d, wx, wy;
        gh_bistatic_rx(g, q, x, y, n1, ux1, uy1, &d, &wx, &wy);
        ExEntry e;
        e.rfix = gh_phase_fix(gh_range(g, d));
        const double kx = g.kappa * wx, ky = g.kappa * wy;
        e.phx0 = gh_phase_fix(kx * gh_axis(g.lo[2], g.step[2], 0));
        e.dphx = gh_phase_fix(kx * g.step[2]);
        e.phy0 = gh_phase_fix(ky * gh_axis(g.lo[3], g.step[3], 0));
        e.dphy = gh_phase_fix(ky * g.step[3]);
        tab[xy * g.Q + q] = e;
    }
}

struct ExactTcParams {
    int Q, Mc, nvx, nvy, nstages;
    long long nxy, nv;
};

constexpr uint32_t kTcWaitIters = 1u << 22;

__device__ __forceinline__ void st16(unsigned char* p, const uint32_t* w, uint32_t flip) {
    *(uint4*)p = make_uint4(w[0] ^ flip, w[1] ^ flip, w[2] ^ flip, w[3] ^ flip);
}

// ---------------------------------------------------------------------------
// Stage 2 kernel, warp-specialised: the warps of a CTA (one per SM,
// persistent over the items (x, y, q), receivers fastest) have fixed roles
// and meet only at mbarriers. Sixteen warps, so that each SM sub-partition
// (warp % 4) runs one epilogue warp, one A and one B producer:
//   warp 0       : TMEM owner; its lane 0 issues the four MMAs of each stage
//                  and the commits that free a stage slot (empty) and publish
//                  an accumulator (accfull); warps 1..3 have no role
//   warps 4..7   : epilogue, one per TMEM lane quarter (8 velocity rows a);
//                  combine the sixteen partial products of each cell into
//                  |F|^2, hand the accumulator back (accempty, count 4) and
//                  keep each cell's sum over receivers; after the last
//                  receiver of a cell (x, y): scores, mask and argmax
//   warps 8..11  : A producers, warps 12..15: B producers; warp j of each
//                  operand makes chirp chunks 2j and 2j + 1 (8 chirps each)
//                  of every stage (64 chirps) into a ring of shared-memory
//                  slots (full, count 8)
// Two accumulators in TMEM let the MMAs of one item run while the epilogue
// reads the previous one. Every wait is bounded; a wait that gives up sets a
// shared abort flag that ends every role's loop, and the kernel reports
// GH_ETIMEOUT through the status word after freeing its tensor memory.
// ---------------------------------------------------------------------------
constexpr int kProdWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreadsWS = 32 * 16;
constexpr int kEpiWarp0 = 4, kProdWarp0 = 8;
constexpr int kStageChirps = 64;  // one 128-byte swizzled row of BF16 per operand row

template <int NV32>
struct S2Cfg {
    static constexpr int NVP = 32 * NV32;  // velocity columns b, padded
    static constexpr int N = 4 * NVP;      // B rows: (Re, Im) x (hi, lo) per column b
    static constexpr int STAGES = NV32 == 1 ? 6 : 4;
    static constexpr uint32_t A_BYTES = 128 * 128, B_BYTES = N * 128;
    static constexpr uint32_t SLOT = A_BYTES + B_BYTES;
    static constexpr uint32_t SMEM = STAGES * SLOT + 1024;  // + alignment of the slots to 1024 B
    static constexpr uint32_t TM_COLS = 2 * N;              // two accumulators: 256 or 512 columns
};

// Bounded wait of one thread, sleeping in the wait instruction (up to 20 us
// per poll, at most kWsPolls polls: a few seconds); gives up when another role
// has aborted.
constexpr uint32_t kWsPolls = 1u << 17;
__device__ __forceinline__ bool ws_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t i = 0; i < kWsPolls; ++i) {
        if (gh_tc::mbar_try_wait_sleep(bar, parity, 20000u)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(gh_tc::smem_u32(bar)) : "memory");
}

// Barrier of the 128 epilogue threads that also ANDs their predicates, so that
// the four warps take the same decision after their bounded waits.
__device__ __forceinline__ bool epi_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// Atoms of one row for the two 8-chirp chunks (2j, 2j + 1) a producer warp
// makes in every stage: z[k] = exp(-j 2 pi ph (m0 + k)), m0 = 64 s + 16 j
// (+ 8 for the second chunk). The step w = exp(-j 2 pi ph) and the first
// chunk's start are exact to float32 rounding (fixed-point phases,
// polynomial sincos); w^8 and w^64 come from w by squaring. Inside a chunk
// the three-term recurrence z[k + 1] = 2 cos(2 pi ph) z[k] - z[k - 1]
// (|w| = 1); the second chunk starts at the first one's start times w^8 and
// the next stage's start is the first one's start times w^64.
struct AtomRow {
    float2 seed, w, w8, w64;
};

__device__ __forceinline__ AtomRow atom_row(unsigned long long ph, int m0) {
    AtomRow r;
    r.w = gh_cis_fix_poly(0ull - ph);
    float2 t = cmul(r.w, r.w);  // w^2
    t = cmul(t, t);             // w^4
    r.w8 = cmul(t, t);
    t = cmul(r.w8, r.w8);  // w^16
    t = cmul(t, t);        // w^32
    r.w64 = cmul(t, t);
    r.seed = gh_cis_fix_poly(0ull - ph * (unsigned long long)m0);
    return r;
}

// z[0..7] from a chunk start z0: z[1] = z0 w, then the three-term recurrence.
__device__ __forceinline__ void atoms8(float2 z0, float2 w, float* zr, float* zi) {
    const float c2 = 2.f * w.x;
    const float2 z1 = cmul(z0, w);
    zr[0] = z0.x;
    zi[0] = z0.y;
    zr[1] = z1.x;
    zi[1] = z1.y;
#pragma unroll
    for (int i = 2; i < 8; ++i) {
        zr[i] = fmaf(c2, zr[i - 1], -zr[i - 2]);
        zi[i] = fmaf(c2, zi[i - 1], -zi[i - 2]);
    }
}

// Splits 8 values into BF16 high and low parts, packed in pairs.
__device__ __forceinline__ void split8v(const float* v, uint32_t* H, uint32_t* L) {
#pragma unroll
    for (int i = 0; i < 4; ++i) gh_tc::split_bf16x2(v[2 * i], v[2 * i + 1], &H[i], &L[i]);
}

// 16 consecutive-chunk TMEM values of the 16x256b shape (x4: four 8-column
// chunks): thread t gets lane (base + t/4) in v[4c + 0, 1] and lane
// (base + t/4 + 8) in v[4c + 2, 3], columns 8c + 2 (t % 4) + {0, 1}.
__device__ __forceinline__ void tmem_ld_16x256b_x4(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NV32>
__global__ void __launch_bounds__(kThreadsWS, 1) exact_s2_tc_kernel(const float* __restrict__ P,
                                                                    const ExEntry* __restrict__ tab, ExactTcParams p,
                                                                    float* __restrict__ scores,
                                                                    const int64_t* __restrict__ mask, int nmask,
                                                                    ArgPartial* __restrict__ parts,
                                                                    int* __restrict__ status) {
    using C = S2Cfg<NV32>;
    constexpr int NVP = C::NVP, N = C::N, S = C::STAGES;
    constexpr int NBLK = NVP / 8;  // 8-column blocks of b
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full[S], empty[S], accfull[2], accempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ int s_abort;
    __shared__ int s_last_slot, s_last_par;  // last stage the MMA thread committed (abort drain)
    __shared__ float s_bs[kEpiWarps];
    __shared__ long long s_bc[kEpiWarps];
    // the swizzled tiles need 1024-byte aligned slots
    unsigned char* smem = smem_raw + ((1024u - (gh_tc::smem_u32(smem_raw) & 1023u)) & 1023u);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long nitems_cta =
        (blockIdx.x < p.nxy ? (p.nxy - 1 - blockIdx.x) / gridDim.x + 1 : 0) * (long long)p.Q;
    volatile int* abort_flag = &s_abort;
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            gh_tc::mbar_init(&full[i], kProdWarps);
            gh_tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            gh_tc::mbar_init(&accfull[i], 1);
            gh_tc::mbar_init(&accempty[i], kEpiWarps);
        }
        s_abort = 0;
        s_last_slot = -1;
        s_last_par = 0;
        gh_tc::mbar_fence_init();
    }
    if (warp == 0) gh_tc::tmem_alloc(&tmem_holder, C::TM_COLS);
    gh_tc::fence_before_sync();
    __syncthreads();
    gh_tc::fence_after_sync();
    const uint32_t tmem = tmem_holder;

    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;

    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = gh_tc::idesc_bf16_f32(128, N);
            const uint32_t base = gh_tc::smem_u32(smem);
            const uint64_t dA0 = gh_tc::smem_desc_sw128(base), dB0 = gh_tc::smem_desc_sw128(base + C::A_BYTES);
            uint32_t g = 0;
            bool ok = true;
            for (long long it = 0; it < nitems_cta && ok; ++it) {
                const uint32_t buf = (uint32_t)it & 1;
                if (!ws_wait(&accempty[buf], ((uint32_t)(it >> 1) & 1) ^ 1, abort_flag)) break;
                gh_tc::fence_after_sync();
                const uint32_t dcol = tmem + buf * N;
                for (int s = 0; s < p.nstages; ++s, ++g) {
                    const uint32_t slot = g % S;
                    if (!ws_wait(&full[slot], (g / S) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    gh_tc::fence_after_sync();
                    const uint64_t so = (uint64_t)((slot * C::SLOT) >> 4);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)  // K = 16 steps: 32 bytes along the swizzled row
                        gh_tc::mma_bf16(dcol, dA0 + so + 2 * kk, dB0 + so + 2 * kk, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    gh_tc::mma_commit(&empty[slot]);  // the slot is free once these MMAs are done
                    s_last_slot = (int)slot;
                    s_last_par = (int)((g / S) & 1);
                }
                if (!ok) break;
                gh_tc::mma_commit(&accfull[buf]);  // the item's accumulator is complete
            }
        }
    } else if (warp >= kProdWarp0) {
        // ---------------- producers ----------------
        // Warp j of an operand makes chirp chunks 2j and 2j + 1 of every stage
        // (chirps 64 s + 16 j .. + 15); lane = operand row (a, or b and
        // b + 32). The inputs of the next item (its phase entry and, for B
        // warps, its row of P) are loaded while the current one is generated.
        // P values depend on the chirp only: lane l of a B warp holds chirps
        // 64 (l / 8) + 16 j + l % 8 and + 8, and a stage takes its 16 values
        // by shuffles.
        const int pw = warp - kProdWarp0;
        const bool a_role = pw < 4;
        const int j = pw & 3;
        // chunk c of row r sits at 16 (c ^ (r % 8)) in the row's 128 bytes
        auto row_off = [&](int r, int c) {
            return (uint32_t)(32 * (r >> 3) + (r & 7)) * 128u + (uint32_t)((c ^ (r & 7)) << 4);
        };
        long long fxy = blockIdx.x;
        int fq = 0;
        auto fetch = [&](long long it, unsigned long long& f0, unsigned long long& f1, float4& fp) {
            f0 = f1 = 0ull;
            fp = make_float4(0.f, 0.f, 0.f, 0.f);
            if (it >= nitems_cta) return;
            const ExEntry& e = tab[fxy * p.Q + fq];
            if (a_role) {
                f0 = e.phx0;
                f1 = e.dphx;
            } else {
                f0 = e.phy0;
                f1 = e.dphy;
                const int mc = 64 * (lane >> 3) + 16 * j + (lane & 7);
                const float* Pq = P + ((size_t)fq * p.nxy + fxy) * 2 * p.Mc;
                if (mc < p.Mc) {
                    fp.x = __ldg(Pq + mc);
                    fp.y = __ldg(Pq + p.Mc + mc);
                }
                if (mc + 8 < p.Mc) {
                    fp.z = __ldg(Pq + mc + 8);
                    fp.w = __ldg(Pq + p.Mc + mc + 8);
                }
            }
        };
        bool ok = true;
        unsigned long long n0, n1;
        float4 np_;
        fetch(0, n0, n1, np_);
        uint32_t g = 0;
        for (long long it = 0; it < nitems_cta && ok; ++it) {
            const unsigned long long c0e = n0, c1e = n1;
            const float4 cp = np_;
            if (++fq == p.Q) {  // the next item's (x, y, q), by counting
                fq = 0;
                fxy += gridDim.x;
            }
            fetch(it + 1, n0, n1, np_);  // in flight during this item
            AtomRow ar[NV32];
            bool vrow[NV32];
#pragma unroll
            for (int gg = 0; gg < NV32; ++gg) {
                const int r = lane + 32 * gg;
                vrow[gg] = a_role ? (gg == 0 && r < p.nvx) : r < p.nvy;
                if (vrow[gg]) ar[gg] = atom_row(c0e + (unsigned long long)r * c1e, 16 * j);
            }
            for (int s = 0; s < p.nstages; ++s, ++g) {
                const uint32_t slot = g % S;
                float pr[16], pi[16];  // P of the stage's 16 chirps of this warp
                if (!a_role) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        pr[k] = __shfl_sync(0xffffffffu, cp.x, 8 * s + k);
                        pi[k] = __shfl_sync(0xffffffffu, cp.y, 8 * s + k);
                        pr[8 + k] = __shfl_sync(0xffffffffu, cp.z, 8 * s + k);
                        pi[8 + k] = __shfl_sync(0xffffffffu, cp.w, 8 * s + k);
                    }
                }
                const bool w_ok = ws_wait(&empty[slot], ((g / S) & 1) ^ 1, abort_flag);
                if (!__all_sync(0xffffffffu, w_ok)) {
                    ok = false;
                    break;
                }
                unsigned char* As = smem + slot * C::SLOT;
#pragma unroll
                for (int gg = 0; gg < (a_role ? 1 : NV32); ++gg) {
                    const int r = lane + 32 * gg;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {  // chunk 2j + h
                        float zr[8], zi[8];
                        if (vrow[gg]) {
                            const float2 z0 = h == 0 ? ar[gg].seed : cmul(ar[gg].seed, ar[gg].w8);
                            atoms8(z0, ar[gg].w, zr, zi);
                            if (!a_role) {
#pragma unroll
                                for (int k = 0; k < 8; ++k) {  // G = P conj(Ey)
                                    const float a = pr[8 * h + k], b = pi[8 * h + k];
                                    const float x = zr[k], y = zi[k];
                                    zr[k] = a * x - b * y;
                                    zi[k] = a * y + b * x;
                                }
                            }
                        } else {
#pragma unroll
                            for (int k = 0; k < 8; ++k) zr[k] = zi[k] = 0.f;
                        }
                        uint32_t reH[4], reL[4], imH[4], imL[4];
                        split8v(zr, reH, reL);
                        split8v(zi, imH, imL);
                        if (a_role) {  // A rows: Re hi, Re lo, Im hi, Im lo
                            unsigned char* d = As + row_off(r, 2 * j + h);
                            st16(d, reH, 0u);
                            st16(d + 8 * 128, reL, 0u);
                            st16(d + 16 * 128, imH, 0u);
                            st16(d + 24 * 128, imL, 0u);
                        } else {  // B rows: Re hi, Im hi, Re lo, Im lo
                            unsigned char* d = As + C::A_BYTES + row_off(r, 2 * j + h);
                            st16(d, reH, 0u);
                            st16(d + 8 * 128, imH, 0u);
                            st16(d + 16 * 128, reL, 0u);
                            st16(d + 24 * 128, imL, 0u);
                        }
                    }
                    if (vrow[gg]) ar[gg].seed = cmul(ar[gg].seed, ar[gg].w64);  // next stage
                }
                gh_tc::fence_smem_to_async();  // generic stores -> tensor core
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[slot]);
            }
        }
    } else if (warp >= kEpiWarp0) {
        // ---------------- epilogue ----------------
        // Warp of TMEM lane quarter e: velocity rows a = 8 e + lane / 4; per
        // 8-column block of b, columns b = 8 blk + 2 (lane % 4) + {0, 1}.
        const int e = warp & 3;
        const int a = 8 * e + (lane >> 2);
        const int bq = 2 * (lane & 3);
        float sacc[2 * NBLK];
#pragma unroll
        for (int i = 0; i < 2 * NBLK; ++i) sacc[i] = 0.f;
        bool ok = true;
        long long xy = blockIdx.x;
        int q = 0;
        for (long long it = 0; it < nitems_cta && ok; ++it) {
            const uint32_t buf = (uint32_t)it & 1;
            const bool w_ok = ws_wait(&accfull[buf], (uint32_t)(it >> 1) & 1, abort_flag);
            if (!epi_all(w_ok)) {  // same decision in all four epilogue warps
                ok = false;
                break;
            }
            gh_tc::fence_after_sync();
            const uint32_t t0 = tmem + ((uint32_t)(32 * e) << 16) + buf * N;
#pragma unroll
            for (int blk = 0; blk < NBLK; ++blk) {
                float re[16], im[16];  // [t][r][c]: B part t, A hi/lo r, column c
                tmem_ld_16x256b_x4(t0 + 32 * blk, re);                 // A rows Re hi, Re lo
                tmem_ld_16x256b_x4(t0 + (16u << 16) + 32 * blk, im);   // A rows Im hi, Im lo
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    // B parts t: 0 Re hi, 1 Im hi, 2 Re lo, 3 Im lo; index 4 t + 2 r + c
                    const float rr = (re[0 + c] + re[2 + c]) + (re[8 + c] + re[10 + c]);   // Re A . Re G
                    const float ri = (re[4 + c] + re[6 + c]) + (re[12 + c] + re[14 + c]);  // Re A . Im G
                    const float ir = (im[0 + c] + im[2 + c]) + (im[8 + c] + im[10 + c]);   // Im A . Re G
                    const float ii = (im[4 + c] + im[6 + c]) + (im[12 + c] + im[14 + c]);  // Im A . Im G
                    const float fr = rr - ii, fi = ri + ir;
                    sacc[2 * blk + c] += fr * fr + fi * fi;
                }
            }
            gh_tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[buf]);
            if (++q < p.Q) continue;
            // cell (x, y) complete: scores, mask, argmax
            q = 0;
            if (a < p.nvx) {
                const long long cbase = xy * p.nv + (long long)a * p.nvy;
                bool hm = false;
                for (int m = 0; m < nmask; ++m) {  // a masked cell in this (x, y) cell's block?
                    const long long mc = __ldg(&mask[m]);
                    hm |= mc >= xy * p.nv && mc < (xy + 1) * p.nv;
                }
#pragma unroll
                for (int i = 0; i < 2 * NBLK; ++i) {
                    const int b = 8 * (i >> 1) + bq + (i & 1);
                    if (b < p.nvy) {
                        if (scores) scores[cbase + b] = sacc[i];
                        bool masked = false;
                        if (hm)
                            for (int m = 0; m < nmask; ++m) masked |= (__ldg(&mask[m]) == cbase + b);
                        if (!masked) better(sacc[i], cbase + b, best, bestc);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 2 * NBLK; ++i) sacc[i] = 0.f;
            xy += gridDim.x;
        }
    }

    __syncthreads();
    if (*abort_flag) {
        if (tid == 0) atomicExch(status, GH_ETIMEOUT);
        // give issued tensor-core work a bounded chance to drain before freeing
        // TMEM (tcgen05 work completes in issue order: the last commit suffices)
        if (tid == 0 && s_last_slot >= 0)
            gh_tc::mbar_wait_bounded(&empty[s_last_slot], (uint32_t)s_last_par, kTcWaitIters);
    }
    gh_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        gh_tc::tmem_dealloc(tmem, C::TM_COLS);
    }

    // argmax over the epilogue warps
    if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
        for (int off = 16; off > 0; off >>= 1) {
            const float os = __shfl_down_sync(0xffffffffu, best, off);
            const long long oc = __shfl_down_sync(0xffffffffu, bestc, off);
            better(os, oc, best, bestc);
        }
        if (lane == 0) {
            s_bs[warp - kEpiWarp0] = best;
            s_bc[warp - kEpiWarp0] = bestc;
        }
    }
    __syncthreads();
    if (tid == 0) {
        float b = s_bs[0];
        long long c = s_bc[0];
        for (int w = 1; w < kEpiWarps; ++w) better(s_bs[w], s_bc[w], b, c);
        parts[blockIdx.x].score = b;
        parts[blockIdx.x].cell = c;
    }
}

// ---------------------------------------------------------------------------
// Stage 1 on the tensor cores: P_q[x][mc] = sum_m Y_q[mc][m] conj(a_m(r_q(x))).
// Real form per receiver: A rows [Re ca | -Im ca] and [Im ca | Re ca] with
// ca_m = exp(-j 2 pi r m) for a tile of 64 (x, y) cells (M = 128), B rows
// [Re Y | Im Y] of the Mc chirps (N = Mc), K = 2 Ms in stages of 32 samples.
// Y is split into BF16 high/low tiles once per call, already in the 128-byte
// swizzled K-major layout the MMAs read (one 128-byte row of 32 samples x
// Re/Im per operand row and stage), and each stage's B tiles arrive with one
// bulk copy (TMA) that completes on an mbarrier. Split-BF16, three MMAs per
// K step.
// ---------------------------------------------------------------------------
// Splits 8 floats into BF16 high/low parts and stores one 16-byte chunk of each.
__device__ __forceinline__ void store_chunk(unsigned char* hi, unsigned char* lo, uint32_t off, const float* v) {
    uint4 a, b;
    gh_tc::split_bf16x2(v[0], v[1], &a.x, &b.x);
    gh_tc::split_bf16x2(v[2], v[3], &a.y, &b.y);
    gh_tc::split_bf16x2(v[4], v[5], &a.z, &b.z);
    gh_tc::split_bf16x2(v[6], v[7], &a.w, &b.w);
    *(uint4*)(hi + off) = a;
    *(uint4*)(lo + off) = b;
}

// Y -> per (q, stage) B tiles [hi | lo], rows mc, K = [Re Y[mc][32s..] | Im Y[mc][32s..]],
// K-major in the 128-byte swizzled layout (one 128-byte row per chirp).
__global__ void y_split_kernel(const float2* __restrict__ Y, int Q, int Ms, int Mc, Deflate df,
                               unsigned char* __restrict__ out) {
    const int nst = Ms / 32;
    const long long total = (long long)Q * nst * Mc * 8;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int c = (int)(idx & 7);
    long long t = idx >> 3;
    const int mc = (int)(t % Mc);
    t /= Mc;
    const int s = (int)(t % nst);
    const int q = (int)(t / nst);
    const uint32_t tile = (uint32_t)Mc * 64 * 2;
    unsigned char* hi = out + ((size_t)(q * nst + s) * 2) * tile;
    unsigned char* lo = hi + tile;
    const int m0 = 32 * s + 8 * (c & 3);
    const float2* row = Y + ((size_t)q * Mc + mc) * Ms + m0;
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 y = row[i];
        if (df.n > 0) y = gh_deflate(df, Q, Ms, Mc, q, mc, m0 + i, y);
        v[i] = c < 4 ? y.x : y.y;
    }
    const uint32_t off = gh_tc::sw128_off((uint32_t)mc, (uint32_t)(8 * c), (uint32_t)Mc);
    store_chunk(hi, lo, off, v);
}

// z[k] = exp(-j 2 pi ph (m0 + k)), k < 8.
__device__ __forceinline__ void atoms8(unsigned long long ph, int m0, float2* z) {
    const float2 w = gh_cis_fix(0ull - ph);
    float2 v = gh_cis_fix(0ull - ph * (unsigned long long)m0);
    z[0] = v;
#pragma unroll
    for (int i = 1; i < 8; ++i) {
        v = cmul(v, w);
        z[i] = v;
    }
}

struct S1Params {
    int Q, Ms, nstages, ntiles_xy;
    long long nxy;
};

template <int NMC>
__global__ void __launch_bounds__(256, 1) exact_s1_tc_kernel(const unsigned char* __restrict__ Bt,
                                                             const ExEntry* __restrict__ tab, S1Params p,
                                                             float* __restrict__ Pout, int* __restrict__ status) {
    constexpr int N = NMC;
    constexpr uint32_t A_BYTES = 128 * 64 * 2, B_BYTES = N * 64 * 2;
    constexpr uint32_t BUF_BYTES = 2 * A_BYTES + 2 * B_BYTES;
    constexpr uint32_t TM_COLS = 2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : (2 * N <= 256 ? 256 : 512));
    constexpr uint32_t FLIP = 0x80008000u;
    constexpr int CH = N / 2;  // columns per epilogue warp
    extern __shared__ unsigned char smem_raw1[];
    __shared__ uint64_t mbar[2], tbar[2];
    __shared__ uint32_t tmem_holder;
    // the swizzled tiles need 1024-byte aligned buffers
    unsigned char* smem = smem_raw1 + ((1024u - (gh_tc::smem_u32(smem_raw1) & 1023u)) & 1023u);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int h = warp >> 2;        // xy half of the tile (generation)
    const int kq = warp & 3;        // 8-sample quarter of a stage (generation)
    const int quarter = warp & 3;   // TMEM lane quarter (epilogue)
    const int chalf = warp >> 2;    // column half (epilogue)
    if (tid == 0) {
        gh_tc::mbar_init(&mbar[0], 1);
        gh_tc::mbar_init(&mbar[1], 1);
        gh_tc::mbar_init(&tbar[0], 1);
        gh_tc::mbar_init(&tbar[1], 1);
        gh_tc::mbar_fence_init();
    }
    if (warp == 0) gh_tc::tmem_alloc(&tmem_holder, TM_COLS);
    gh_tc::fence_before_sync();
    __syncthreads();
    gh_tc::fence_after_sync();
    const uint32_t tmem = tmem_holder;
    const uint32_t idesc = gh_tc::idesc_bf16_f32(128, N);
    // A rows h*64 + lane (Re row: [Re ca | -Im ca]) and h*64 + 32 + lane (Im row:
    // [Im ca | Re ca]), 128-byte swizzled: K chunk c of row r at 16 (c ^ (r % 8))
    const int rre = h * 64 + lane, rim = h * 64 + 32 + lane;
    auto offA = [](int r, int c) { return (uint32_t)r * 128u + (uint32_t)(((c ^ (r & 7)) & 7) << 4); };

    uint32_t gs = 0;
    int tile_ctr = 0;
    bool aborted = false;
    const long long ntiles = (long long)p.Q * p.ntiles_xy;
    for (long long tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
        const int q = (int)(tile / p.ntiles_xy);
        const long long xy0 = (tile - (long long)q * p.ntiles_xy) * 64;
        const long long xy = xy0 + h * 32 + lane;
        const unsigned long long rf = xy < p.nxy ? tab[xy * p.Q + q].rfix : 0ull;
        const bool vx = xy < p.nxy;
        const uint32_t dcol = (uint32_t)(tile_ctr & 1) * N;
        for (int s = 0; s < p.nstages; ++s) {
            const int buf = gs & 1;
            if (gs >= 2) {
                const bool ok = gh_tc::mbar_wait_bounded(&mbar[buf], ((gs - 2) >> 1) & 1, kTcWaitIters);
                if (__syncthreads_or(!ok)) {
                    aborted = true;
                    break;
                }
            }
            unsigned char* Ah = smem + buf * BUF_BYTES;
            unsigned char* Al = Ah + A_BYTES;
            unsigned char* Bh = Al + A_BYTES;
            if (tid == 0) {
                gh_tc::mbar_arrive_expect_tx(&tbar[buf], 2 * B_BYTES);
                gh_tc::bulk_g2s(Bh, Bt + ((size_t)(q * p.nstages + s) * 2) * B_BYTES, 2 * B_BYTES, &tbar[buf]);
            }
            {
                float2 z[8];
                if (vx) {
                    atoms8(rf, 32 * s + 8 * kq, z);
                } else {
#pragma unroll
                    for (int k = 0; k < 8; ++k) z[k] = make_float2(0.f, 0.f);
                }
                uint32_t reH[4], reL[4], imH[4], imL[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    gh_tc::split_bf16x2(z[2 * i].x, z[2 * i + 1].x, &reH[i], &reL[i]);
                    gh_tc::split_bf16x2(z[2 * i].y, z[2 * i + 1].y, &imH[i], &imL[i]);
                }
                // Re row: [Re ca | -Im ca]; Im row: [Im ca | Re ca]
                st16(Ah + offA(rre, kq), reH, 0u);
                st16(Al + offA(rre, kq), reL, 0u);
                st16(Ah + offA(rre, 4 + kq), imH, FLIP);
                st16(Al + offA(rre, 4 + kq), imL, FLIP);
                st16(Ah + offA(rim, kq), imH, 0u);
                st16(Al + offA(rim, kq), imL, 0u);
                st16(Ah + offA(rim, 4 + kq), reH, 0u);
                st16(Al + offA(rim, 4 + kq), reL, 0u);
            }
            gh_tc::fence_smem_to_async();
            const bool tok = gh_tc::mbar_wait_bounded(&tbar[buf], (gs >> 1) & 1, kTcWaitIters);
            gh_tc::fence_before_sync();
            if (__syncthreads_or(!tok)) {
                aborted = true;
                break;
            }
            if (tid == 0) {
                gh_tc::fence_after_sync();
                const uint32_t ah = gh_tc::smem_u32(Ah), al = gh_tc::smem_u32(Al);
                const uint32_t bh = gh_tc::smem_u32(Bh), bl = bh + B_BYTES;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // K = 16 steps: 32 bytes along the swizzled rows
                    const uint64_t dah = gh_tc::smem_desc_sw128(ah + 32 * kk);
                    const uint64_t dal = gh_tc::smem_desc_sw128(al + 32 * kk);
                    const uint64_t dbh = gh_tc::smem_desc_sw128(bh + 32 * kk);
                    const uint64_t dbl = gh_tc::smem_desc_sw128(bl + 32 * kk);
                    gh_tc::mma_bf16(tmem + dcol, dah, dbh, idesc, (s > 0 || kk > 0) ? 1u : 0u);
                    gh_tc::mma_bf16(tmem + dcol, dah, dbl, idesc, 1u);
                    gh_tc::mma_bf16(tmem + dcol, dal, dbh, idesc, 1u);
                }
                gh_tc::mma_commit(&mbar[buf]);
            }
            ++gs;
        }
        if (aborted) break;
        // epilogue: this warp's quarter holds Re P or Im P of 32 cells; write its column half
        {
            const uint32_t last = gs - 1;
            const bool ok = gh_tc::mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, kTcWaitIters);
            if (__syncthreads_or(!ok)) {
                aborted = true;
                break;
            }
            gh_tc::fence_after_sync();
            const int eh = quarter >> 1, part = quarter & 1;
            const long long exy = xy0 + eh * 32 + lane;
            float* dst = Pout + ((size_t)q * p.nxy + exy) * 2 * N + (size_t)part * N + chalf * CH;
#pragma unroll
            for (int c = 0; c < CH / 16; ++c) {
                float v[16];
                gh_tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + dcol + (uint32_t)(chalf * CH + 16 * c), v);
                if (exy < p.nxy) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *(float4*)(dst + 16 * c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                }
            }
            gh_tc::fence_before_sync();
        }
        ++tile_ctr;
    }
    if (aborted) {
        if (tid == 0) atomicExch(status, GH_ETIMEOUT);
        if (gs > 0) gh_tc::mbar_wait_bounded(&mbar[(gs - 1) & 1], ((gs - 1) >> 1) & 1, kTcWaitIters);
    }
    gh_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gh_tc::tmem_dealloc(tmem, TM_COLS);
}

template <int NMC>
int launch_s1_tc(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate& df, const ExEntry* tab, float* P,
                 int* status) {
    constexpr uint32_t B_BYTES = NMC * 64 * 2;
    const size_t smem = (size_t)2 * (2 * 128 * 64 * 2 + 2 * B_BYTES) + 1024;  // + alignment
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "stage-1 tensor-core path needs %zu B", smem);
    const int nst = d.Ms / 32;
    void* bt;
    GH_TRY(gh_ws(ctx, WS_EXACT_B, (size_t)d.Q * nst * 2 * B_BYTES, &bt));
    cudaEvent_t ev;
    const long long nsplit = (long long)d.Q * nst * d.Mc * 8;
    gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
    y_split_kernel<<<(unsigned)((nsplit + 255) / 256), 256, 0, ctx->stream>>>(Y, d.Q, d.Ms, d.Mc, df,
                                                                               (unsigned char*)bt);
    GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S1, ev, "y_split_kernel"));
    GH_CUDA(cudaFuncSetAttribute(exact_s1_tc_kernel<NMC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GH_CUDA(cudaFuncSetAttribute(exact_s1_tc_kernel<NMC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    S1Params p;
    p.Q = d.Q;
    p.Ms = d.Ms;
    p.nstages = nst;
    p.ntiles_xy = (int)((d.nxy + 63) / 64);
    p.nxy = d.nxy;
    long long ctas = (long long)ctx->num_sms;
    const long long ntiles = (long long)d.Q * p.ntiles_xy;
    if (ctas > ntiles) ctas = ntiles;
    gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
    exact_s1_tc_kernel<NMC><<<(unsigned)ctas, 256, smem, ctx->stream>>>((const unsigned char*)bt, tab, p, P, status);
    return gh_launch_end(ctx, GH_K_EXACT_S1, ev, "exact_s1_tc_kernel");
}

template <int NV32>
int launch_tc(gh_ctx* ctx, const Dims& d, const float* P, const ExEntry* tab, float* scores, const int64_t* mask,
              int nmask, ArgPartial* parts, int* status, long long* nparts) {
    using C = S2Cfg<NV32>;
    if (d.Mc > 256) return gh_fail(ctx, GH_ENOTSUP, "exact tensor-core stage 2 supports Mc <= 256");
    const size_t smem = C::SMEM;
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "exact tensor-core path needs %zu B", smem);
    GH_CUDA(cudaFuncSetAttribute(exact_s2_tc_kernel<NV32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    long long ctas = ctx->num_sms;  // one persistent CTA per SM
    if (ctas > d.nxy) ctas = d.nxy;
    ExactTcParams p;
    p.Q = d.Q;
    p.Mc = d.Mc;
    p.nvx = d.nvx;
    p.nvy = d.nvy;
    p.nstages = (d.Mc + kStageChirps - 1) / kStageChirps;
    p.nxy = d.nxy;
    p.nv = d.nv;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_EXACT_S2, &ev);
    exact_s2_tc_kernel<NV32><<<(unsigned)ctas, kThreadsWS, smem, ctx->stream>>>(P, tab, p, scores, mask, nmask, parts,
                                                                                status);
    GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S2, ev, "exact_s2_tc_kernel"));
    *nparts = ctas;
    return GH_OK;
}

}  // namespace

// Stage 1 (and the phase table the tensor-core kernels read): P planar
// [Q][nxy][Re row | Im row][Mc]; *tab_out is NULL when no table was made.
namespace {

// Stage 1 of a BOMP residual by linearity (iterations k >= 1, in place): the
// correlation of atom t with a(r) over the samples is
// <b(u_t) (x) a(r_t), a(r)>_m = b(u_t)[mc] F_Ms(r_t - r) (Eq. 3's inner
// products), so every (x, y, q) row loses
// sum_t (alpha_t - alpha'_t) F_Ms(r_t - r_q(x)) b_t[mc], the part the rows do
// not yet hold. F from fixed-point phases (exact argument reduction). Grid
// (row blocks of kDeflRows, Q): the float64 parts (alpha_t - alpha'_t and the
// fixed-point phase of r_t) depend on (t, q) only and are taken once per CTA
// (float64 issues one warp instruction per 64 cycles per SM sub-partition);
// then one warp per row (row = q nxy + xy), lanes over chirps.
constexpr int kDeflRows = 64;  // (x, y) rows per CTA, 8 per warp

__global__ void __launch_bounds__(256) exact_p_deflate_kernel(float* __restrict__ P,
                                                              const ExEntry* __restrict__ tab, Deflate df, int Q,
                                                              long long nxy, int Ms, int Mc) {
    __shared__ float2 s_da[GH_MAX_K];              // alpha_t - alpha'_t, this CTA's receiver
    __shared__ unsigned long long s_rf[GH_MAX_K];  // fixed-point phase of r_t
    __shared__ float2 s_ct[8][GH_MAX_K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = blockIdx.y;
    if (threadIdx.x < df.n) {
        const int t = threadIdx.x;
        const double2 al = df.alpha[(size_t)t * Q + q], ap = df.alpha_prev[(size_t)t * Q + q];
        s_da[t] = make_float2((float)(al.x - ap.x), (float)(al.y - ap.y));
        s_rf[t] = gh_phase_fix(df.ru[(size_t)t * Q + q].x);
    }
    __syncthreads();
    const long long xy0 = (long long)blockIdx.x * kDeflRows;
    const long long xy1 = xy0 + kDeflRows < nxy ? xy0 + kDeflRows : nxy;
    const int n4 = Mc >> 2;
    for (long long xy = xy0 + warp; xy < xy1; xy += 8) {
        const long long row = (long long)q * nxy + xy;
        // the row's values first (4 chirps per 16-byte access, Mc <= 256), then
        // the coefficients while those loads are in flight
        float4* pr = (float4*)(P + (size_t)row * 2 * Mc);  // Re row, then Im row
        float4 re[2], im[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int v = lane + 32 * u;
            if (v < n4) {
                re[u] = pr[v];
                im[u] = pr[n4 + v];
            }
        }
        if (lane < df.n) {
            const int t = lane;
            const float2 F = gh_dtft_fix(s_rf[t] - tab[xy * Q + q].rfix, Ms);
            s_ct[warp][t] = cmul(s_da[t], F);
        }
        __syncwarp();
        for (int t = 0; t < df.n; ++t) {
            const float2 c = s_ct[warp][t];
            const float4* bt = (const float4*)(df.atoms_b + ((size_t)t * Q + q) * Mc);  // 2 chirps per float4
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int v = lane + 32 * u;
                if (v < n4) {
                    const float4 b0 = __ldg(bt + 2 * v), b1 = __ldg(bt + 2 * v + 1);  // chirps 4v .. 4v + 3
                    re[u].x -= c.x * b0.x - c.y * b0.y;
                    im[u].x -= c.x * b0.y + c.y * b0.x;
                    re[u].y -= c.x * b0.z - c.y * b0.w;
                    im[u].y -= c.x * b0.w + c.y * b0.z;
                    re[u].z -= c.x * b1.x - c.y * b1.y;
                    im[u].z -= c.x * b1.y + c.y * b1.x;
                    re[u].w -= c.x * b1.z - c.y * b1.w;
                    im[u].w -= c.x * b1.w + c.y * b1.z;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int v = lane + 32 * u;
            if (v < n4) {
                pr[v] = re[u];
                pr[n4 + v] = im[u];
            }
        }
        __syncwarp();  // this row's coefficients read before the next row's
    }
}

}  // namespace

// Stage 1 (P and, when needed, the coordinate table). With df.n > 0 and the
// table of this detection already built (k >= 1), P of the residual is
// updated in place by linearity instead of being recomputed.
static int exact_stage1(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, const Deflate& df,
                        bool need_tab, void** P_out, void** tab_out) {
    void* P;  // planar [Q][nxy][Re row | Im row][Mc]
    GH_TRY(gh_ws(ctx, WS_EXACT_P, (size_t)d.Q * d.nxy * 2 * d.Mc * sizeof(float), &P));
    const bool tc1 = d.Ms % 32 == 0 && (d.Mc == 32 || d.Mc == 64 || d.Mc == 128 || d.Mc == 256);
    int* status = gh_status_dev(ctx);
    cudaEvent_t ev;
    void* tab = nullptr;
    if (df.n > 0 && df.n <= GH_MAX_K && (tc1 || need_tab) && d.Mc <= 256) {  // residual of iteration k >= 1
        GH_TRY(gh_ws(ctx, WS_EXACT_TAB, (size_t)d.nxy * d.Q * sizeof(ExEntry), &tab));
        gh_launch_begin(ctx, GH_K_DEFLATE, &ev);
        exact_p_deflate_kernel<<<dim3((unsigned)((d.nxy + kDeflRows - 1) / kDeflRows), d.Q), 256, 0, ctx->stream>>>(
            (float*)P, (const ExEntry*)tab, df, d.Q, d.nxy, d.Ms, d.Mc);
        GH_TRY(gh_launch_end(ctx, GH_K_DEFLATE, ev, "exact_p_deflate_kernel"));
        *P_out = P;
        *tab_out = tab;
        return GH_OK;
    }
    if (tc1 || need_tab) {
        GH_TRY(gh_ws(ctx, WS_EXACT_TAB, (size_t)d.nxy * d.Q * sizeof(ExEntry), &tab));
        gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
        exact_coord_kernel<<<(unsigned)((2 * d.nxy + 31) / 32), 32, 0, ctx->stream>>>(g, (ExEntry*)tab);
        GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S1, ev, "exact_coord_kernel"));
    }
    if (tc1) {
        const ExEntry* t = (const ExEntry*)tab;
        float* Pf = (float*)P;
        if (d.Mc == 32) GH_TRY(launch_s1_tc<32>(ctx, d, Y, df, t, Pf, status));
        else if (d.Mc == 64) GH_TRY(launch_s1_tc<64>(ctx, d, Y, df, t, Pf, status));
        else if (d.Mc == 128) GH_TRY(launch_s1_tc<128>(ctx, d, Y, df, t, Pf, status));
        else GH_TRY(launch_s1_tc<256>(ctx, d, Y, df, t, Pf, status));
    } else {
        const float2* Ys = Y;
        if (df.n > 0) {  // the CUDA-core stage 1 reads a stored residual
            void* R;
            GH_TRY(gh_ws(ctx, WS_R, (size_t)d.Q * d.Mc * d.Ms * sizeof(float2), &R));
            GH_TRY(gh_launch_residual(ctx, d, Y, df, (float2*)R));
            Ys = (const float2*)R;
        }
        gh_launch_begin(ctx, GH_K_EXACT_S1, &ev);
        dim3 grid1((unsigned)((d.nxy + S1_XT - 1) / S1_XT), (unsigned)((d.Mc + S1_MT - 1) / S1_MT), (unsigned)d.Q);
        exact_stage1_kernel<<<grid1, 256, 0, ctx->stream>>>(Ys, g, (float*)P);
        GH_TRY(gh_launch_end(ctx, GH_K_EXACT_S1, ev, "exact_stage1_kernel"));
    }
    *P_out = P;
    *tab_out = tab;
    return GH_OK;
}

int gh_launch_exact_stage1(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, const float** P) {
    if (d.nxy > 0x7fffffffLL) return gh_fail(ctx, GH_ENOTSUP, "exact path supports < 2^31 (x, y) cells");
    void *Pv, *tab;
    GH_TRY(exact_stage1(ctx, d, g, Y, Deflate{nullptr, nullptr, nullptr, 0}, false, &Pv, &tab));
    *P = (const float*)Pv;
    return GH_OK;
}

int gh_launch_exact_parts(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, const Deflate* dfp,
                          float* scores, const int64_t* mask, int nmask, ArgPartial** parts_out, int* nparts_out) {
    if (d.nxy > 0x7fffffffLL) return gh_fail(ctx, GH_ENOTSUP, "exact path supports < 2^31 (x, y) cells");
    if (d.nv > 256 * 16) return gh_fail(ctx, GH_ENOTSUP, "exact path supports at most 4096 velocity cells");
    const Deflate df = dfp ? *dfp : Deflate{nullptr, nullptr, nullptr, 0};
    // the tensor-core stage 2 prefetches P for at most 8 stages of 32 chirps
    const bool tc2 = d.nvx <= 32 && d.nvy <= 64 && d.Mc <= 256;
    int* status = gh_status_dev(ctx);
    void *P, *tab;
    GH_TRY(exact_stage1(ctx, d, g, Y, df, tc2, &P, &tab));
    void* parts;
    GH_TRY(gh_ws(ctx, WS_PART, (size_t)d.nxy * sizeof(ArgPartial), &parts));
    *parts_out = (ArgPartial*)parts;
    if (tc2) {
        long long nparts = 0;
        if (d.nvy <= 32)
            GH_TRY(launch_tc<1>(ctx, d, (const float*)P, (const ExEntry*)tab, scores, mask, nmask,
                                (ArgPartial*)parts, status, &nparts));
        else
            GH_TRY(launch_tc<2>(ctx, d, (const float*)P, (const ExEntry*)tab, scores, mask, nmask,
                                (ArgPartial*)parts, status, &nparts));
        *nparts_out = (int)nparts;
        return GH_OK;
    }
    const int cpt = (int)((d.nv + 255) / 256);
    int st;
    if (cpt <= 1)
        st = launch_s2<1>(ctx, d, g, (const float*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 2)
        st = launch_s2<2>(ctx, d, g, (const float*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 4)
        st = launch_s2<4>(ctx, d, g, (const float*)P, scores, mask, nmask, (ArgPartial*)parts);
    else if (cpt <= 8)
        st = launch_s2<8>(ctx, d, g, (const float*)P, scores, mask, nmask, (ArgPartial*)parts);
    else
        st = launch_s2<16>(ctx, d, g, (const float*)P, scores, mask, nmask, (ArgPartial*)parts);
    GH_TRY(st);
    *nparts_out = (int)d.nxy;
    return GH_OK;
}

int gh_launch_exact(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, float* scores,
                    const int64_t* mask, int nmask, ArgResult* result) {
    ArgPartial* parts;
    int nparts;
    GH_TRY(gh_launch_exact_parts(ctx, d, g, Y, nullptr, scores, mask, nmask, &parts, &nparts));
    return gh_launch_argmax_finalize(ctx, parts, nparts, result);
}
