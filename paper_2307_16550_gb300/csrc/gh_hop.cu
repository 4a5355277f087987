// Grid-hopping score (Sec. IV, Eq. 5) over the 4D grid, its argmax, and the
// coordinate mapping it needs (Eq. 1).
//
// coord_kernel (one thread per (x, y, q), float64):
//   rho = Nr * r_q(x), i = floor(rho + 1/2), tau = rho - i, the three polar
//   coefficients c_k(tau) on rows (i + k) mod Nr (signed by the centring phase
//   of a wrapped index), and the Doppler bin position as 64-bit fixed point:
//   eta(a, b) = Nd * kappa * (wx * vx_a + wy * vy_b) is affine in the cell
//   indices (a, b), so eta * 2^32 = base + a * ax + b * by exactly up to the
//   rounding of three integers (error <= (1 + a + b) * 2^-33 bins).
//
// hop_score_kernel (one CTA per run of (x, y) cells):
//   For a fixed (x, y, q) the hopping value at Doppler bin j is
//   T_q[j] = sum_k c_k Z~_q[i+k][j], and the cell's contribution is |T_q[j_q]|^2.
//   The CTA first evaluates P_q[j] = |T_q[j]|^2 for the Doppler bins that the
//   velocity grid reaches (coalesced reads of three map rows), then every
//   velocity cell sums P_q over q with one shared-memory read per receiver.
//   The bin j_q = floor(eta + 1/2) comes from the fixed-point value; when its
//   fraction lies within 2^-20 of a rounding boundary the bin is recomputed
//   with the float64 expression floor(Nd * (kappa * (wx*vx + wy*vy)) + 1/2),
//   so every bin decision equals a plain float64 evaluation.
//   P rows are double buffered: one barrier per (x, y) cell.
//   Scores (optional) are written coalesced; the CTA's best (score, cell) is
//   reduced with warp shuffles (ties: smallest cell index).
#include <math.h>

#include "gh_internal.cuh"

namespace {

constexpr uint32_t kTol = 4096u;  // 2^-20 of a bin, in 2^-32 units

struct __align__(16) HopEntry {
    long long base;  // (eta(0,0) - j_lo + 1/2) * 2^32 + kTol
    long long ax;    // d eta / d ivx * 2^32
    long long by;    // d eta / d ivy * 2^32
    double wx, wy;   // bistatic gradient (float64 bin decisions)
    int row[3];      // map rows (i + k) mod Nr, k = -1, 0, 1
    float cs[3];     // polar coefficients times the wrap sign
    int j_lo;        // Doppler bin of P[0]
    int nP;          // number of P entries (<= Nd)
};
static_assert(sizeof(HopEntry) == 80, "HopEntry layout");

struct CoordParams {
    double theta, cos_t, sin_t;  // polar half-arc angle
    int Ms_odd_sign;             // 1 if (Ms - 1) is odd (wrap flips the sign)
};

__global__ void coord_kernel(GeoParams g, CoordParams cp, HopEntry* __restrict__ table, int32_t* diag_i,
                             double* diag_tau, float* diag_c, double* diag_w) {
    const long long nxy = (long long)g.n[0] * g.n[1];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nxy * g.Q) return;
    const int q = (int)(idx % g.Q);
    const long long xy = idx / g.Q;
    const int ix = (int)(xy / g.n[1]);
    const int iy = (int)(xy - (long long)ix * g.n[1]);
    const double x = gh_axis(g.lo[0], g.step[0], ix);
    const double y = gh_axis(g.lo[1], g.step[1], iy);
    double d, wx, wy;
    gh_bistatic(g, q, x, y, &d, &wx, &wy);
    const double r = gh_range(g, d);
    const double rho = __dmul_rn((double)g.Nr, r);
    const double fi = floor(__dadd_rn(rho, 0.5));
    const double tau = __dsub_rn(rho, fi);
    const long long i = (long long)fi;

    // polar coefficients on the arc through bins i-1, i, i+1
    const double kap = (1.0 - cos(cp.theta * tau)) / (1.0 - cp.cos_t);
    const double sig = sin(cp.theta * tau) / cp.sin_t;
    const double c[3] = {0.5 * (kap - sig), 1.0 - kap, 0.5 * (kap + sig)};

    HopEntry e;
    for (int k = 0; k < 3; ++k) {
        const long long n = i + (k - 1);
        long long w = n / g.Nr;
        if (n < 0 && w * g.Nr != n) --w;  // floor division
        e.row[k] = (int)(n - w * g.Nr);
        const bool flip = cp.Ms_odd_sign && (w & 1);
        e.cs[k] = (float)(flip ? -c[k] : c[k]);
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
    const long long span = j_hi - j_lo + 1;
    const double two32 = 4294967296.0;
    e.base = llrint((eta00 - (double)j_lo + 0.5) * two32) + (long long)kTol;
    e.ax = llrint(ax * two32);
    e.by = llrint(by * two32);
    e.wx = wx;
    e.wy = wy;
    e.j_lo = (int)j_lo;
    e.nP = (int)(span < g.Nd ? span : g.Nd);
    table[idx] = e;

    if (diag_i) {
        diag_i[idx] = (int32_t)i;
        diag_tau[idx] = tau;
        for (int k = 0; k < 3; ++k) diag_c[3 * idx + k] = (float)c[k];
        diag_w[2 * idx] = wx;
        diag_w[2 * idx + 1] = wy;
    }
}

struct HopParams {
    int Q, Nr, Nd, nvx, nvy;
    int NB, SA;           // thread mapping: b = tid % NB (stride NB), a = tid / NB (stride SA)
    long long nxy, nv;
    long long xy_per_cta;
    double lo2, step2, lo3, step3, kappa;
};

// Exact float64 Doppler bin for cell (a, b), as an index into the P row.
__device__ __noinline__ int slow_bin(const HopParams& p, double wx, double wy, int j_lo, int a, int b) {
    const double vx = gh_axis(p.lo2, p.step2, a);
    const double vy = gh_axis(p.lo3, p.step3, b);
    const double u = __dmul_rn(p.kappa, __dadd_rn(__dmul_rn(wx, vx), __dmul_rn(wy, vy)));
    const long long j = (long long)floor(__dadd_rn(__dmul_rn((double)p.Nd, u), 0.5));
    return (int)((j - j_lo) & (p.Nd - 1));
}

__device__ __forceinline__ void better(float s, long long c, float& bs, long long& bc) {
    if (s > bs || (s == bs && c < bc)) {
        bs = s;
        bc = c;
    }
}

template <int AMAX>
__global__ void __launch_bounds__(256) hop_score_kernel(const float2* __restrict__ maps,
                                                        const HopEntry* __restrict__ table, HopParams p,
                                                        float* __restrict__ scores, const int64_t* __restrict__ mask,
                                                        int nmask, ArgPartial* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* P = (float*)smem_raw;                                        // [2][Q][Nd]
    HopEntry* tab = (HopEntry*)(smem_raw + (size_t)2 * p.Q * p.Nd * 4);  // [2][Q]
    __shared__ int s_mask[2];
    __shared__ float s_bs[8];
    __shared__ long long s_bc[8];

    const int tid = threadIdx.x;
    const long long xy0 = (long long)blockIdx.x * p.xy_per_cta;
    long long xy1 = xy0 + p.xy_per_cta;
    if (xy1 > p.nxy) xy1 = p.nxy;
    const int cnt = (int)(xy1 - xy0);
    const int tb = tid % p.NB;
    const int ta = tid / p.NB;
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;

    auto build = [&](long long xy, int buf) {
        const HopEntry* e = table + xy * p.Q;
        const long long* src = (const long long*)e;
        long long* dst = (long long*)(tab + buf * p.Q);
        const int words = p.Q * (int)(sizeof(HopEntry) / 8);
        for (int t = tid; t < words; t += blockDim.x) dst[t] = __ldg(src + t);
        if (tid == 0) {
            int f = 0;
            for (int m = 0; m < nmask; ++m) f |= (mask[m] / p.nv == xy);
            s_mask[buf] = f;
        }
        for (int q = 0; q < p.Q; ++q) {
            const int nP = __ldg(&e[q].nP);
            const int j_lo = __ldg(&e[q].j_lo);
            const float2* r0 = maps + ((size_t)q * p.Nr + __ldg(&e[q].row[0])) * p.Nd;
            const float2* r1 = maps + ((size_t)q * p.Nr + __ldg(&e[q].row[1])) * p.Nd;
            const float2* r2 = maps + ((size_t)q * p.Nr + __ldg(&e[q].row[2])) * p.Nd;
            const float c0 = __ldg(&e[q].cs[0]), c1 = __ldg(&e[q].cs[1]), c2 = __ldg(&e[q].cs[2]);
            const int js = j_lo & (p.Nd - 1);
            float* Pq = P + ((size_t)buf * p.Q + q) * p.Nd;
            for (int t = tid; t < nP; t += blockDim.x) {
                const int j = (js + t) & (p.Nd - 1);
                const float2 z0 = __ldg(r0 + j), z1 = __ldg(r1 + j), z2 = __ldg(r2 + j);
                const float re = c0 * z0.x + c1 * z1.x + c2 * z2.x;
                const float im = c0 * z0.y + c1 * z1.y + c2 * z2.y;
                Pq[t] = re * re + im * im;
            }
        }
    };

    auto gather = [&](long long xy, int buf) {
        if (ta >= p.SA) return;
        const HopEntry* E = tab + buf * p.Q;
        const bool hm = s_mask[buf] != 0;
        const long long cbase = xy * p.nv;
        const float* Pb = P + (size_t)buf * p.Q * p.Nd;
        for (int b = tb; b < p.nvy; b += p.NB) {
            for (int a0 = 0; a0 < p.nvx; a0 += p.SA * AMAX) {
                float acc[AMAX];
#pragma unroll
                for (int i = 0; i < AMAX; ++i) acc[i] = 0.f;
                for (int q = 0; q < p.Q; ++q) {
                    const long long ax = E[q].ax;
                    long long t = E[q].base + (long long)b * E[q].by + (long long)(a0 + ta) * ax;
                    const long long st = (long long)p.SA * ax;
                    const float* Pq = Pb + (size_t)q * p.Nd;
#pragma unroll
                    for (int i = 0; i < AMAX; ++i) {
                        const int a = a0 + ta + i * p.SA;
                        if (a < p.nvx) {
                            const uint32_t lo = (uint32_t)t;
                            int idx = (int)(t >> 32) & (p.Nd - 1);
                            if (lo < 2u * kTol) idx = slow_bin(p, E[q].wx, E[q].wy, E[q].j_lo, a, b);
                            acc[i] += Pq[idx];
                        }
                        t += st;
                    }
                }
#pragma unroll
                for (int i = 0; i < AMAX; ++i) {
                    const int a = a0 + ta + i * p.SA;
                    if (a < p.nvx) {
                        const long long cell = cbase + (long long)a * p.nvy + b;
                        const float s = acc[i];
                        if (scores) scores[cell] = s;
                        bool masked = false;
                        if (hm)
                            for (int m = 0; m < nmask; ++m) masked |= (mask[m] == cell);
                        if (!masked) better(s, cell, best, bestc);
                    }
                }
            }
        }
    };

    if (cnt > 0) {
        build(xy0, 0);
        for (int n = 0; n < cnt; ++n) {
            __syncthreads();
            if (n + 1 < cnt) build(xy0 + n + 1, (n + 1) & 1);
            gather(xy0 + n, n & 1);
        }
    }

    // block argmax
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
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) better(s_bs[w], s_bc[w], best, bestc);
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

template <int AMAX>
int launch_hop_t(gh_ctx* ctx, const Dims& d, const HopParams& hp0, const float2* maps, const HopEntry* table,
                 float* scores, const int64_t* mask, int nmask, ArgResult* result) {
    HopParams hp = hp0;
    const size_t smem = (size_t)2 * d.Q * d.Nd * sizeof(float) + (size_t)2 * d.Q * sizeof(HopEntry);
    if (smem > ctx->smem_optin) return gh_fail(ctx, GH_ENOTSUP, "hop scorer needs %zu B shared memory", smem);
    GH_CUDA(cudaFuncSetAttribute(hop_score_kernel<AMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hop_score_kernel<AMAX>, 256, smem));
    if (per_sm < 1) per_sm = 1;
    long long ctas = (long long)ctx->num_sms * per_sm;
    if (ctas > d.nxy) ctas = d.nxy;
    hp.xy_per_cta = (d.nxy + ctas - 1) / ctas;
    ctas = (d.nxy + hp.xy_per_cta - 1) / hp.xy_per_cta;
    void* parts;
    GH_TRY(gh_ws(ctx, WS_PART, (size_t)ctas * sizeof(ArgPartial), &parts));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_HOP_SCORE, &ev);
    hop_score_kernel<AMAX><<<(unsigned)ctas, 256, smem, ctx->stream>>>(maps, table, hp, scores, mask, nmask,
                                                                        (ArgPartial*)parts);
    GH_TRY(gh_launch_end(ctx, GH_K_HOP_SCORE, ev, "hop_score_kernel"));
    return gh_launch_argmax_finalize(ctx, (const ArgPartial*)parts, (int)ctas, result);
}

double dirichlet_closed(double f, int M) {
    const double pi = 3.14159265358979323846264338327950288;
    return sin(pi * M * f) / sin(pi * f);
}

}  // namespace

size_t gh_hop_table_bytes(const Dims& d) { return (size_t)d.nxy * d.Q * sizeof(HopEntry); }

int gh_launch_coord(gh_ctx* ctx, const Dims& d, const GeoParams& g, void* table, int32_t* diag_i,
                    double* diag_tau, float* diag_c, double* diag_w) {
    CoordParams cp;
    // Half-arc angle of the three-bin polar model, from the Gram of centred
    // atoms: cos(theta/2) = 1/2 sqrt((Ms - D(2/Nr)) / (Ms - D(1/Nr))).
    const double D1 = dirichlet_closed(1.0 / d.Nr, d.Ms), D2 = dirichlet_closed(2.0 / d.Nr, d.Ms);
    cp.theta = 2.0 * acos(0.5 * sqrt((d.Ms - D2) / (d.Ms - D1)));
    cp.cos_t = cos(cp.theta);
    cp.sin_t = sin(cp.theta);
    cp.Ms_odd_sign = ((d.Ms - 1) & 1) ? 1 : 0;
    const long long n = d.nxy * d.Q;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_COORD, &ev);
    coord_kernel<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(g, cp, (HopEntry*)table, diag_i, diag_tau,
                                                                       diag_c, diag_w);
    return gh_launch_end(ctx, GH_K_COORD, ev, "coord_kernel");
}

int gh_launch_argmax_finalize(gh_ctx* ctx, const ArgPartial* parts, int nparts, ArgResult* out) {
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
    argmax_finalize_kernel<<<1, 1024, 0, ctx->stream>>>(parts, nparts, out);
    return gh_launch_end(ctx, GH_K_ARGMAX, ev, "argmax_finalize_kernel");
}

int gh_launch_hop(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* maps, const void* table,
                  float* scores, const int64_t* mask, int nmask, ArgResult* result) {
    HopParams hp;
    hp.Q = d.Q;
    hp.Nr = d.Nr;
    hp.Nd = d.Nd;
    hp.nvx = d.nvx;
    hp.nvy = d.nvy;
    hp.NB = d.nvy < 256 ? d.nvy : 256;
    hp.SA = 256 / hp.NB;
    hp.nxy = d.nxy;
    hp.nv = d.nv;
    hp.xy_per_cta = 1;
    hp.lo2 = g.lo[2];
    hp.step2 = g.step[2];
    hp.lo3 = g.lo[3];
    hp.step3 = g.step[3];
    hp.kappa = g.kappa;
    const int need = (d.nvx + hp.SA - 1) / hp.SA;
    const HopEntry* t = (const HopEntry*)table;
    if (need <= 1) return launch_hop_t<1>(ctx, d, hp, maps, t, scores, mask, nmask, result);
    if (need <= 2) return launch_hop_t<2>(ctx, d, hp, maps, t, scores, mask, nmask, result);
    if (need <= 4) return launch_hop_t<4>(ctx, d, hp, maps, t, scores, mask, nmask, result);
    if (need <= 8) return launch_hop_t<8>(ctx, d, hp, maps, t, scores, mask, nmask, result);
    if (need <= 16) return launch_hop_t<16>(ctx, d, hp, maps, t, scores, mask, nmask, result);
    return launch_hop_t<32>(ctx, d, hp, maps, t, scores, mask, nmask, result);
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

template <int AMAX>
int noalloc_score(cudaStream_t stream, const Dims& d, const HopParams& hp0, const float2* maps,
                  const HopEntry* table, float* scores, ArgPartial* parts, ArgResult* result, int num_sms,
                  int smem_optin) {
    HopParams hp = hp0;
    const size_t smem = (size_t)2 * d.Q * d.Nd * sizeof(float) + (size_t)2 * d.Q * sizeof(HopEntry);
    if (smem > (size_t)smem_optin) return GH_ENOTSUP;
    if (cudaFuncSetAttribute(hop_score_kernel<AMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return GH_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hop_score_kernel<AMAX>, 256, smem) != cudaSuccess)
        return GH_ECUDA;
    if (per_sm < 1) per_sm = 1;
    long long ctas = (long long)num_sms * per_sm;
    if (ctas > kNoAllocMaxCtas) ctas = kNoAllocMaxCtas;
    if (ctas > d.nxy) ctas = d.nxy;
    hp.xy_per_cta = (d.nxy + ctas - 1) / ctas;
    ctas = (d.nxy + hp.xy_per_cta - 1) / hp.xy_per_cta;
    hop_score_kernel<AMAX><<<(unsigned)ctas, 256, smem, stream>>>(maps, table, hp, scores, nullptr, 0, parts);
    if (cudaGetLastError() != cudaSuccess) return GH_ECUDA;
    argmax_finalize_kernel<<<1, 1024, 0, stream>>>(parts, (int)ctas, result);
    return cudaGetLastError() == cudaSuccess ? GH_OK : GH_ECUDA;
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
    CoordParams cp;
    const double D1 = dirichlet_closed(1.0 / d.Nr, d.Ms), D2 = dirichlet_closed(2.0 / d.Nr, d.Ms);
    cp.theta = 2.0 * acos(0.5 * sqrt((d.Ms - D2) / (d.Ms - D1)));
    cp.cos_t = cos(cp.theta);
    cp.sin_t = sin(cp.theta);
    cp.Ms_odd_sign = ((d.Ms - 1) & 1) ? 1 : 0;
    const long long n = d.nxy * d.Q;
    coord_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(g, cp, table, nullptr, nullptr, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return GH_ECUDA;

    HopParams hp;
    hp.Q = d.Q;
    hp.Nr = d.Nr;
    hp.Nd = d.Nd;
    hp.nvx = d.nvx;
    hp.nvy = d.nvy;
    hp.NB = d.nvy < 256 ? d.nvy : 256;
    hp.SA = 256 / hp.NB;
    hp.nxy = d.nxy;
    hp.nv = d.nv;
    hp.xy_per_cta = 1;
    hp.lo2 = g.lo[2];
    hp.step2 = g.step[2];
    hp.lo3 = g.lo[3];
    hp.step3 = g.step[3];
    hp.kappa = g.kappa;
    const int need = (d.nvx + hp.SA - 1) / hp.SA;
    const float2* maps = (const float2*)maps_dev;
    int st;
    if (need <= 1)
        st = noalloc_score<1>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    else if (need <= 2)
        st = noalloc_score<2>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    else if (need <= 4)
        st = noalloc_score<4>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    else if (need <= 8)
        st = noalloc_score<8>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    else if (need <= 16)
        st = noalloc_score<16>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    else
        st = noalloc_score<32>(stream, d, hp, maps, table, scores_dev, parts, result, num_sms, smem_optin);
    if (st != GH_OK) return st;
    if (best_cell || best_score) {
        ArgResult h;
        if (cudaMemcpyAsync(&h, result, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return GH_ECUDA;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return GH_ECUDA;
        if (best_cell) *best_cell = h.cell;
        if (best_score) *best_score = h.score;
    }
    return GH_OK;
}
