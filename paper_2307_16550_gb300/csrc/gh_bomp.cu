// Block orthogonal matching pursuit (BOMP, the paper's acronym list; several
// targets by iterative direct detection, Sec. VI) and the measurement
// synthesiser of the signal model (Sec. II).
//
// BOMP iteration k, after the scorer has written its per-CTA argmax partials
// (no host round trip):
//   selection   : the partials reduce to the selected cell sel[k] (ties: the
//                 smallest index), appended to the mask; the new atom at every
//                 receiver q: (r, u) in float64, its centring phase
//                 exp(j pi (r (Ms-1) + u (Mc-1))), row k of the real Gram
//                 matrix G[s][t] = D_Ms(r_t - r_s) D_Mc(u_t - u_s) with
//                 D_M(f) = sin(pi M f) / sin(pi f), and the atoms a(r), b(u).
//                 Trigonometric arguments are reduced exactly in float64 before
//                 a float32 sincos.
//   correlation : c_{k,q} = <Y_q, b(u) (x) a(r)> (float32 row sums added in
//                 float64); the last CTA to finish solves, per receiver, the
//                 float64 normal equations of atoms 0..k (closed form for up
//                 to three atoms, else Cholesky; dependent atoms dropped) and
//                 rotates the amplitudes back to the atoms of the signal model
//                 (Sec. II).
// A single frame runs both in one launch (bomp_step_kernel); a batch of frames
// runs them as two (bomp_select_batch_kernel, bomp_corr_batch_kernel). The
// residual Y - sum_t alpha_t atom_t is never stored on the hopping path: the
// next iteration's maps subtract the new atoms' maps (A_t (x) B_t, tabulated
// here) by linearity, or the map-making pass subtracts the atoms while loading
// Y (gh_deflate).
#include <math.h>

#include "gh_internal.cuh"

namespace {

constexpr int kCorrRows = 8;  // chirps per correlation CTA (one per warp)
constexpr int kStepThreads = 32 * (kCorrRows + 1);  // BOMP step CTA: the correlation warps and a Gram warp

struct BompLayout {
    size_t alpha, corr, ru, phase, gram, corrp, atoms_a, atoms_b, alpha_prev, tab_a, tab_b, counter, total;
    int chunks;
};

BompLayout bomp_layout(const Dims& d, int K) {
    BompLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o += (bytes + 255) & ~(size_t)255;
        return at;
    };
    L.chunks = (d.Mc + kCorrRows - 1) / kCorrRows;
    L.alpha = take((size_t)K * d.Q * 2 * sizeof(double));    // double2 [K][Q]  (must stay at offset 0)
    L.corr = take((size_t)K * d.Q * 2 * sizeof(double));     // double2 [K][Q]  <Y_q, atom>
    L.ru = take((size_t)K * d.Q * 2 * sizeof(double));       // (r, u) [K][Q]
    L.phase = take((size_t)K * d.Q * 2 * sizeof(double));    // (cos, sin)(pi (r (Ms-1) + u (Mc-1))) [K][Q]
    L.gram = take((size_t)d.Q * K * K * sizeof(double));      // [Q][K][K]
    L.corrp = take((size_t)K * d.Q * L.chunks * 2 * sizeof(double));  // double2 [K][Q][chunks]
    L.atoms_a = take((size_t)K * d.Q * d.Ms * sizeof(float2));
    L.atoms_b = take((size_t)K * d.Q * d.Mc * sizeof(float2));
    L.alpha_prev = take((size_t)K * d.Q * 2 * sizeof(double));  // double2 [K][Q]
    L.tab_a = take((size_t)K * d.Q * d.Nr * sizeof(float2));      // [K][Q][Nr]
    L.tab_b = take((size_t)K * d.Q * d.Nd * sizeof(float2));      // [K][Q][Nd]
    L.counter = take((size_t)(1 + K * d.Q) * sizeof(unsigned int));  // completion counter, then [K][Q] table counters
    L.total = o;
    return L;
}


BompPtrs bomp_ptrs(void* ws, const Dims& d, int K) {
    const BompLayout L = bomp_layout(d, K);
    char* b = (char*)ws;
    BompPtrs w;
    w.alpha = (double2*)(b + L.alpha);
    w.corr = (double2*)(b + L.corr);
    w.ru = (double2*)(b + L.ru);
    w.phase = (double2*)(b + L.phase);
    w.gram = (double*)(b + L.gram);
    w.corrp = (double2*)(b + L.corrp);
    w.atoms_a = (float2*)(b + L.atoms_a);
    w.atoms_b = (float2*)(b + L.atoms_b);
    w.alpha_prev = (double2*)(b + L.alpha_prev);
    w.tab_a = (float2*)(b + L.tab_a);
    w.tab_b = (float2*)(b + L.tab_b);
    w.counter = (unsigned int*)(b + L.counter);
    w.tab_counter = w.counter + 1;
    w.chunks = L.chunks;
    return w;
}

// x mod 2, exactly, as a float (argument of sinpif / cospif).
__device__ __forceinline__ float mod2f(double x) { return (float)(x - 2.0 * floor(0.5 * x)); }

// D_M(f) = sin(pi M f) / sin(pi f) (M a power of two, so M f is exact).
__device__ double dirichlet(double f, int M) {
    const float s = sinpif(mod2f(f));
    if (fabsf(s) < 1e-6f) {
        // f is (numerically) an integer n: D_M(n) = M (-1)^(n (M - 1))
        const long long n = llrint(f);
        return ((n * (long long)(M - 1)) & 1) ? -(double)M : (double)M;
    }
    return (double)(sinpif(mod2f((double)M * f)) / s);
}

// Maps of the signal-model atom b(u) (x) a(r) as the map maker computes them
// (Sec. III; its bins are the inner products of Sec. IV): the 2D DFT of the
// atom, times the range-centring factor, is A[i] B[j] with
//   A[i] = exp(j pi i (Ms-1) / Nr) F_Ms(r - i/Nr),   B[j] = F_Mc(u - j/Nd),
// from the fixed-point phases rf, uf of r and u (Nr, Nd powers of two, so
// i/Nr and j/Nd are exact phase steps). Written by threads t0, t0 + nt, ...
// of the calling group.
// Entry e of the tables: A[e] for e < Nr, else B[e - Nr] (e < Nr + Nd).
__device__ __forceinline__ void atom_map_entry(uint64_t rf, uint64_t uf, int Ms, int Mc, int Nr, int Nd,
                                               float2* __restrict__ A, float2* __restrict__ B, int e) {
    if (e < Nr) {
        const uint64_t sr = 0ull - (~0ull / (uint64_t)Nr + 1ull);  // -2^64 / Nr (mod 2^64)
        const float2 f = gh_dtft_fix(rf + (uint64_t)e * sr, Ms);
        // exp(j pi i (Ms-1) / Nr), the angle reduced exactly (as the Doppler FFT does)
        const int t = (int)(((unsigned)e * (unsigned)(Ms - 1)) & (unsigned)(2 * Nr - 1));
        float s, c;
        sincospif((float)t / (float)Nr, &s, &c);
        A[e] = make_float2(c * f.x - s * f.y, c * f.y + s * f.x);
    } else {
        const int j = e - Nr;
        const uint64_t sd = 0ull - (~0ull / (uint64_t)Nd + 1ull);  // -2^64 / Nd
        B[j] = gh_dtft_fix(uf + (uint64_t)j * sd, Mc);
    }
}

__device__ void atom_map_tables(uint64_t rf, uint64_t uf, int Ms, int Mc, int Nr, int Nd, float2* __restrict__ A,
                                float2* __restrict__ B, int t0, int nt) {
    for (int e = t0; e < Nr + Nd; e += nt) atom_map_entry(rf, uf, Ms, Mc, Nr, Nd, A, B, e);
}

// The tables of one atom and receiver, shared out in slices of blockDim.x
// entries through a counter (zeroed before the detection) among the CTAs that
// call this; every CTA of the group calls it, so every slice gets taken.
__device__ void atom_map_tables_shared(uint64_t rf, uint64_t uf, int Ms, int Mc, int Nr, int Nd,
                                       float2* __restrict__ A, float2* __restrict__ B, unsigned* counter) {
    __shared__ unsigned s_base;
    for (;;) {
        if (threadIdx.x == 0) s_base = atomicAdd(counter, blockDim.x);
        __syncthreads();
        const unsigned base = s_base;
        __syncthreads();
        if (base >= (unsigned)(Nr + Nd)) break;
        const unsigned e = base + threadIdx.x;
        if (e < (unsigned)(Nr + Nd)) atom_map_entry(rf, uf, Ms, Mc, Nr, Nd, A, B, (int)e);
    }
}

// The same slices taken by one warp (32 entries at a time).
__device__ void atom_map_tables_warp(uint64_t rf, uint64_t uf, int Ms, int Mc, int Nr, int Nd,
                                     float2* __restrict__ A, float2* __restrict__ B, unsigned* counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned base = 0u;
        if (lane == 0) base = atomicAdd(counter, 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned)(Nr + Nd)) break;
        const unsigned e = base + lane;
        if (e < (unsigned)(Nr + Nd)) atom_map_entry(rf, uf, Ms, Mc, Nr, Nd, A, B, (int)e);
    }
}

__device__ __forceinline__ void better(float s, long long c, float& bs, long long& bc) {
    if (s > bs || (s == bs && c < bc)) {
        bs = s;
        bc = c;
    }
}

// Second half of a selection (one CTA of 1024 threads): thread 0 holds the
// best (score, cell) of iteration k; writes sel[k] and mask[k] and prepares
// the new atom at every receiver: (r, u) in float64, its centring phase, row
// k of the Gram matrices and the atom tables.
// (r, u) of receiver q at a 4D cell (Eq. 1), float64. With rw (the
// coordinate kernel's float64 (r, wx, wy) per (x, y, q)) the geometry is read
// instead of recomputed: the same operations on the same values, so the same
// (r, u).
// Grid indices (ix, iy, ivx, ivy) of a 4D cell.
__device__ __forceinline__ void cell_decode(const GeoParams& g, long long cell, int* ix, int* iy, int* ivx,
                                            int* ivy) {
    const int nvy = g.n[3], nvx = g.n[2], ny = g.n[1];
    if (cell < (1ll << 32)) {  // 32-bit division: a shorter chain than the 64-bit one
        unsigned c = (unsigned)cell;
        *ivy = (int)(c % (unsigned)nvy);
        c /= (unsigned)nvy;
        *ivx = (int)(c % (unsigned)nvx);
        c /= (unsigned)nvx;
        *iy = (int)(c % (unsigned)ny);
        *ix = (int)(c / (unsigned)ny);
    } else {
        *ivy = (int)(cell % nvy);
        cell /= nvy;
        *ivx = (int)(cell % nvx);
        cell /= nvx;
        *iy = (int)(cell % ny);
        *ix = (int)(cell / ny);
    }
}

__device__ __forceinline__ void cell_ru(const GeoParams& g, long long cell, int q, const double* rw, double* r,
                                        double* u) {
    int ix, iy, ivx, ivy;
    cell_decode(g, cell, &ix, &iy, &ivx, &ivy);
    double d, wx, wy;
    if (rw) {
        const double* e = rw + (((long long)ix * g.n[1] + iy) * g.Q + q) * 3;
        *r = e[0];
        wx = e[1];
        wy = e[2];
    } else {
        gh_bistatic(g, q, gh_axis(g.lo[0], g.step[0], ix), gh_axis(g.lo[1], g.step[1], iy), &d, &wx, &wy);
        *r = gh_range(g, d);
    }
    *u = gh_speed(g, wx, wy, gh_axis(g.lo[2], g.step[2], ivx), gh_axis(g.lo[3], g.step[3], ivy));
}

__device__ void bomp_select_body(float best, long long bestc, ArgResult* __restrict__ sel,
                                 int64_t* __restrict__ mask, int k, int K, const GeoParams& g, const BompPtrs& w) {
    __shared__ long long s_cell;
    __shared__ unsigned long long s_rf[GH_MAX_Q], s_uf[GH_MAX_Q];
    __shared__ double s_r[GH_MAX_Q], s_u[GH_MAX_Q];
    if (threadIdx.x == 0) {
        const bool valid = bestc != 0x7fffffffffffffffLL;
        sel[k].cell = bestc;
        sel[k].score = best;
        sel[k].valid = valid;
        mask[k] = bestc;
        s_cell = valid ? bestc : 0;
    }
    __syncthreads();
    const int q = threadIdx.x;
    if (q < g.Q) {
        long long cell = s_cell;
        const int nvy = g.n[3], nvx = g.n[2], ny = g.n[1];
        const int ivy = (int)(cell % nvy);
        cell /= nvy;
        const int ivx = (int)(cell % nvx);
        cell /= nvx;
        const int iy = (int)(cell % ny);
        const int ix = (int)(cell / ny);
        double d, wx, wy;
        gh_bistatic(g, q, gh_axis(g.lo[0], g.step[0], ix), gh_axis(g.lo[1], g.step[1], iy), &d, &wx, &wy);
        const double r = gh_range(g, d);
        const double u = gh_speed(g, wx, wy, gh_axis(g.lo[2], g.step[2], ivx), gh_axis(g.lo[3], g.step[3], ivy));
        w.ru[(size_t)k * g.Q + q] = make_double2(r, u);
        float sn, cs;
        sincospif(mod2f(r * (g.Ms - 1) + u * (g.Mc - 1)), &sn, &cs);
        w.phase[(size_t)k * g.Q + q] = make_double2(cs, sn);
        s_r[q] = r;
        s_u[q] = u;
        s_rf[q] = gh_phase_fix(r);
        s_uf[q] = gh_phase_fix(u);
    }
    __syncthreads();
    // row k of the Gram matrix of every receiver
    for (int idx = threadIdx.x; idx < g.Q * (k + 1); idx += blockDim.x) {
        const int qq = idx / (k + 1), t = idx - qq * (k + 1);
        const double2 rut = t == k ? make_double2(s_r[qq], s_u[qq]) : w.ru[(size_t)t * g.Q + qq];
        const double v = dirichlet(s_r[qq] - rut.x, g.Ms) * dirichlet(s_u[qq] - rut.y, g.Mc);
        double* G = w.gram + (size_t)qq * K * K;
        G[k * K + t] = v;
        G[t * K + k] = v;
    }
    for (int idx = threadIdx.x; idx < g.Q * g.Ms; idx += blockDim.x) {
        const int qq = idx / g.Ms, m = idx - qq * g.Ms;
        w.atoms_a[((size_t)k * g.Q + qq) * g.Ms + m] = gh_cis_fix(s_rf[qq] * (unsigned long long)m);
    }
    for (int idx = threadIdx.x; idx < g.Q * g.Mc; idx += blockDim.x) {
        const int qq = idx / g.Mc, m = idx - qq * g.Mc;
        w.atoms_b[((size_t)k * g.Q + qq) * g.Mc + m] = gh_cis_fix(s_uf[qq] * (unsigned long long)m);
    }
    for (int qq = 0; qq < g.Q; ++qq)
        atom_map_tables(s_rf[qq], s_uf[qq], g.Ms, g.Mc, g.Nr, g.Nd, w.tab_a + ((size_t)k * g.Q + qq) * g.Nr,
                        w.tab_b + ((size_t)k * g.Q + qq) * g.Nd, threadIdx.x, blockDim.x);
}


// One CTA of 1024 threads.
// Batched selection: one CTA per listed frame, best cell from the frame's key.
__global__ void __launch_bounds__(1024) bomp_select_batch_kernel(const BatchFrame* __restrict__ frames,
                                                                 const int* __restrict__ active, int k) {
    const BatchFrame& F = frames[active[blockIdx.x]];
    const unsigned long long key = F.key[k];
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    if (key != 0ull) {
        best = __uint_as_float((unsigned)(key >> 32));
        bestc = (long long)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
    }
    bomp_select_body(best, bestc, F.sel, F.mask, k, F.K, F.g, F.bw);
}

// 1 / sqrt(v) for a positive normal float64 v inside the float32 range:
// Newton's iteration y <- y (3 - v y^2) / 2 from the float32 reciprocal
// square root, whose relative error (about 2^-23) squares at every step:
// two steps reach float64 rounding. (A Gram pivot lies between the
// dependence floor 1e-9 Ms Mc and Ms Mc <= 2^26.)
__device__ __forceinline__ double rsqrt_newton(double v) {
    double y = (double)rsqrtf((float)v);
    y = y * (1.5 - 0.5 * v * y * y);
    y = y * (1.5 - 0.5 * v * y * y);
    return y;
}

// Float64 normal equations of atoms 0..N-1 of one receiver (Cholesky,
// dependent atoms dropped), amplitudes rotated back to the atoms of the signal
// model. G: the receiver's Gram matrix (row stride ldg); z: exp(+j pi ph_t)
// <Y, atom_t> (stride sz); ph: the centring phases (stride sp); alpha: output
// (stride sa). The factor is kept as rows scaled by the reciprocal square
// roots of the pivots, so the solve has no division; the loops unroll for the
// exact size N (the float64 dependency chain is as long as N needs) and the
// factor stays in registers.
template <int N>
__device__ __forceinline__ void bomp_solve_n(int Ms, int Mc, const double* G, int ldg, const double2* z, int sz,
                                             const double2* ph, int sp, double2* alpha, int sa) {
    constexpr int NM = N;
    const int n = N;
    double L[NM][NM];
    double zr[NM], zi[NM], rs[NM];  // rs[j] = 1 / L[j][j] (0 for a dependent atom)
#pragma unroll
    for (int t = 0; t < NM; ++t) {
        if (t < n) {
            const double2 v = z[(size_t)t * sz];
            zr[t] = v.x;
            zi[t] = v.y;
        }
    }
    const double floor_v = 1e-9 * (double)Ms * (double)Mc;
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        if (j < n) {
            double v = G[j * ldg + j];
#pragma unroll
            for (int t = 0; t < j; ++t) v -= L[j][t] * L[j][t];
            rs[j] = v > floor_v ? rsqrt_newton(v) : 0.0;
#pragma unroll
            for (int i = j + 1; i < NM; ++i) {
                if (i < n) {
                    double e = G[i * ldg + j];
#pragma unroll
                    for (int t = 0; t < j; ++t) e -= L[i][t] * L[j][t];
                    L[i][j] = e * rs[j];
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {  // L z' = z
        if (i < n) {
#pragma unroll
            for (int t = 0; t < i; ++t) {
                zr[i] -= L[i][t] * zr[t];
                zi[i] -= L[i][t] * zi[t];
            }
            zr[i] *= rs[i];
            zi[i] *= rs[i];
        }
    }
#pragma unroll
    for (int i = NM - 1; i >= 0; --i) {  // L^T alpha~ = z'
        if (i < n) {
#pragma unroll
            for (int t = i + 1; t < NM; ++t) {
                if (t < n) {
                    zr[i] -= L[t][i] * zr[t];
                    zi[i] -= L[t][i] * zi[t];
                }
            }
            zr[i] *= rs[i];
            zi[i] *= rs[i];
        }
    }
#pragma unroll
    for (int t = 0; t < NM; ++t) {
        if (t < n) {
            const double2 p = ph[(size_t)t * sp];  // alpha = alpha~ exp(-j pi ph)
            alpha[(size_t)t * sa] = make_double2(p.x * zr[t] + p.y * zi[t], p.x * zi[t] - p.y * zr[t]);
        }
    }
}

// The same solve for any n <= GH_MAX_K, loops not unrolled (the factor in
// local memory).
__device__ __noinline__ void bomp_solve_big(int Ms, int Mc, int n, const double* G, int ldg, const double2* z,
                                            int sz, const double2* ph, int sp, double2* alpha, int sa) {
    double L[GH_MAX_K][GH_MAX_K];
    double zr[GH_MAX_K], zi[GH_MAX_K], rs[GH_MAX_K];
    for (int t = 0; t < n; ++t) {
        const double2 v = z[(size_t)t * sz];
        zr[t] = v.x;
        zi[t] = v.y;
    }
    const double floor_v = 1e-9 * (double)Ms * (double)Mc;
    for (int j = 0; j < n; ++j) {
        double v = G[j * ldg + j];
        for (int t = 0; t < j; ++t) v -= L[j][t] * L[j][t];
        rs[j] = v > floor_v ? rsqrt_newton(v) : 0.0;
        for (int i = j + 1; i < n; ++i) {
            double e = G[i * ldg + j];
            for (int t = 0; t < j; ++t) e -= L[i][t] * L[j][t];
            L[i][j] = e * rs[j];
        }
    }
    for (int i = 0; i < n; ++i) {
        for (int t = 0; t < i; ++t) {
            zr[i] -= L[i][t] * zr[t];
            zi[i] -= L[i][t] * zi[t];
        }
        zr[i] *= rs[i];
        zi[i] *= rs[i];
    }
    for (int i = n - 1; i >= 0; --i) {
        for (int t = i + 1; t < n; ++t) {
            zr[i] -= L[t][i] * zr[t];
            zi[i] -= L[t][i] * zi[t];
        }
        zr[i] *= rs[i];
        zi[i] *= rs[i];
    }
    for (int t = 0; t < n; ++t) {
        const double2 p = ph[(size_t)t * sp];
        alpha[(size_t)t * sa] = make_double2(p.x * zr[t] + p.y * zi[t], p.x * zi[t] - p.y * zr[t]);
    }
}

// 1 / d for a positive normal float64 d inside the float32 range: one
// third-order Newton step y <- y (1 + e + e^2), e = 1 - d y, from the float32
// reciprocal (relative error about 2^-23, cubed by the step).
__device__ __forceinline__ double rcp_newton(double d) {
    const double y = (double)__frcp_rn((float)d);
    const double e = fma(-d, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// The same normal equations for N <= 3 atoms in closed form (cofactors over
// the determinant, Cramer's rule): a float64 dependency chain about a third
// as long as the factorisation's. Used when every Cholesky pivot clears twice
// the dependence floor (pivot j = det G_{0..j} / det G_{0..j-1}); otherwise
// the factorisation decides which atoms to drop.
template <int N>
__device__ __forceinline__ void bomp_solve_cramer(int Ms, int Mc, const double* G, int ldg, const double2* z, int sz,
                                                  const double2* ph, int sp, double2* alpha, int sa) {
    const double floor2 = 2e-9 * (double)Ms * (double)Mc;
    double C[N][N], det;
    bool ok;
    if constexpr (N == 1) {
        det = G[0];
        C[0][0] = 1.0;
        ok = det > floor2;
    } else if constexpr (N == 2) {
        const double g00 = G[0], g01 = G[1], g11 = G[ldg + 1];
        det = fma(g00, g11, -g01 * g01);
        C[0][0] = g11;
        C[0][1] = C[1][0] = -g01;
        C[1][1] = g00;
        ok = g00 > floor2 && det > floor2 * g00;
    } else {
        const double g00 = G[0], g01 = G[1], g02 = G[2];
        const double g11 = G[ldg + 1], g12 = G[ldg + 2], g22 = G[2 * ldg + 2];
        C[0][0] = fma(g11, g22, -g12 * g12);
        C[0][1] = C[1][0] = fma(g02, g12, -g01 * g22);
        C[0][2] = C[2][0] = fma(g01, g12, -g02 * g11);
        C[1][1] = fma(g00, g22, -g02 * g02);
        C[1][2] = C[2][1] = fma(g01, g02, -g00 * g12);
        C[2][2] = fma(g00, g11, -g01 * g01);
        det = fma(g02, C[0][2], fma(g01, C[0][1], g00 * C[0][0]));
        ok = g00 > floor2 && C[2][2] > floor2 * g00 && det > floor2 * C[2][2];
    }
    if (!ok) {
        bomp_solve_n<N>(Ms, Mc, G, ldg, z, sz, ph, sp, alpha, sa);
        return;
    }
    const double inv = rcp_newton(det);
    double zr[N], zi[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        const double2 v = z[(size_t)t * sz];
        zr[t] = v.x;
        zi[t] = v.y;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double ar = C[i][0] * zr[0], ai = C[i][0] * zi[0];
#pragma unroll
        for (int t = 1; t < N; ++t) {
            ar = fma(C[i][t], zr[t], ar);
            ai = fma(C[i][t], zi[t], ai);
        }
        ar *= inv;
        ai *= inv;
        const double2 p = ph[(size_t)i * sp];  // alpha = alpha~ exp(-j pi ph)
        alpha[(size_t)i * sa] = make_double2(p.x * ar + p.y * ai, p.x * ai - p.y * ar);
    }
}

// The solve in closed form for n <= 3, with the factor in registers for
// n = 4, else in local memory.
__device__ __forceinline__ void bomp_solve_any(int Ms, int Mc, int n, const double* G, int ldg, const double2* z,
                                               int sz, const double2* ph, int sp, double2* alpha, int sa) {
    switch (n) {
        case 1: bomp_solve_cramer<1>(Ms, Mc, G, ldg, z, sz, ph, sp, alpha, sa); break;
        case 2: bomp_solve_cramer<2>(Ms, Mc, G, ldg, z, sz, ph, sp, alpha, sa); break;
        case 3: bomp_solve_cramer<3>(Ms, Mc, G, ldg, z, sz, ph, sp, alpha, sa); break;
        case 4: bomp_solve_n<4>(Ms, Mc, G, ldg, z, sz, ph, sp, alpha, sa); break;
        default: bomp_solve_big(Ms, Mc, n, G, ldg, z, sz, ph, sp, alpha, sa);
    }
}

constexpr int kSolveStage = 1024;  // doubles of shared memory for the staged solve

// The smallest power of two >= min(n, 32).
__device__ __forceinline__ int lane_span(int n) {
    const int m = n < 32 ? n : 32;
    return m <= 1 ? 1 : 1 << (32 - __clz(m - 1));
}

// Last CTA of a BOMP iteration (its first nthr threads, a multiple of 32;
// they synchronise on named barrier 1): c_{k,q} = the sum of the
// chunks' partial correlations (one warp per receiver, lanes over chunks,
// then a fixed butterfly order), then every receiver's least squares. When
// they fit, the Gram matrices, rotated correlations and phases are staged in
// shared memory by the whole CTA in the same round of loads as the partial
// correlations, so that the solves wait for one round of loads in all.
__device__ void bomp_sum_solve(const GeoParams& g, int k, int K, const BompPtrs& w, int nthr) {
    __shared__ double2 s_stage[kSolveStage / 2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nthr >> 5;
    const int n = k + 1, Q = g.Q;
    // the amplitudes the maps of this iteration's residual hold (atom k: none),
    // kept before the solve replaces them
    for (int i = threadIdx.x; i < n * Q; i += nthr)
        w.alpha_prev[i] = i < k * Q ? w.alpha[i] : make_double2(0.0, 0.0);
    const int gsz = (Q * n * n + 1) & ~1;  // doubles of the Gram part, even: the double2 parts stay 16-byte aligned
    const bool staged = (size_t)gsz + (size_t)4 * Q * n <= (size_t)kSolveStage;
    double* sG = (double*)s_stage;    // [Q][n][n]
    double2* sz = s_stage + gsz / 2;  // [Q][n]
    double2* sp = sz + Q * n;         // [Q][n]
    if (staged) {
        for (int i = threadIdx.x; i < Q * n * n; i += nthr) {
            const int qq = i / (n * n), e = i - qq * n * n, r = e / n, c = e - r * n;
            sG[i] = __ldcg(w.gram + ((size_t)qq * K + r) * K + c);
        }
        for (int i = threadIdx.x; i < Q * n; i += nthr) {
            const int qq = i / n, t = i - qq * n;
            const double2 p = __ldcg(w.phase + (size_t)t * Q + qq);
            sp[i] = p;
            if (t < k) {
                const double2 c = w.corr[(size_t)t * Q + qq];
                sz[i] = make_double2(p.x * c.x - p.y * c.y, p.x * c.y + p.y * c.x);  // exp(+j pi ph) <Y, atom>
            }
        }
    }
    for (int qq = warp; qq < Q; qq += nw) {
        const double2* pp = w.corrp + ((size_t)k * Q + qq) * w.chunks;
        double2 p = make_double2(0.0, 0.0);
        if (staged && lane == 0) p = __ldcg(w.phase + (size_t)k * Q + qq);
        double cx = 0.0, cy = 0.0;
        // lanes at or above min(chunks, 32) hold zeros: the butterfly starts
        // at half the next power of two
        if (w.chunks <= 16) {
            // real parts on lanes 0-15, imaginary parts on lanes 16-31: one
            // butterfly (within each half) for both, the same additions
            double a = 0.0;
            const int c = lane & 15;
            if (c < w.chunks) {
                const double2 v = __ldcg(pp + c);
                a += lane < 16 ? v.x : v.y;
            }
            for (int off = lane_span(w.chunks) >> 1; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            cx = __shfl_sync(0xffffffffu, a, 0);
            cy = __shfl_sync(0xffffffffu, a, 16);
        } else {
            for (int c = lane; c < w.chunks; c += 32) {
                const double2 v = __ldcg(pp + c);
                cx += v.x;
                cy += v.y;
            }
            for (int off = lane_span(w.chunks) >> 1; off > 0; off >>= 1) {
                cx += __shfl_xor_sync(0xffffffffu, cx, off);
                cy += __shfl_xor_sync(0xffffffffu, cy, off);
            }
        }
        if (lane == 0) {
            w.corr[(size_t)k * Q + qq] = make_double2(cx, cy);
            if (staged) sz[qq * n + k] = make_double2(p.x * cx - p.y * cy, p.x * cy + p.y * cx);
        }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
    if (staged) {
        for (int qq = threadIdx.x; qq < Q; qq += nthr)
            bomp_solve_any(g.Ms, g.Mc, n, sG + qq * n * n, n, sz + qq * n, 1, sp + qq * n, 1, w.alpha + qq, Q);
    } else {
        for (int qq = threadIdx.x; qq < Q; qq += nthr) {
            double2 z[GH_MAX_K];
            for (int t = 0; t < n; ++t) {
                const double2 p = w.phase[(size_t)t * Q + qq];
                const double2 c = w.corr[(size_t)t * Q + qq];
                z[t] = make_double2(p.x * c.x - p.y * c.y, p.x * c.y + p.y * c.x);
            }
            bomp_solve_any(g.Ms, g.Mc, n, w.gram + (size_t)qq * K * K, K, z, 1, w.phase + qq, Q, w.alpha + qq, Q);
        }
    }
}

// Sum of the kCorrRows chirp correlations of a CTA, in a pairwise tree (a
// float64 dependency chain of log2(kCorrRows) additions).
__device__ __forceinline__ double sum_rows(const double* r) {
    static_assert(kCorrRows == 8, "pairwise tree of eight");
    return ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
}

// Both sums (real parts rx, imaginary parts ry) by one warp, lanes 0 and 1
// side by side (float64 issues per warp instruction, so two lanes cost what
// one does); every lane of the warp gets the pair.
__device__ __forceinline__ double2 sum_rows_xy(const double* rx, const double* ry, int lane) {
    const double s = lane < 2 ? sum_rows(lane == 0 ? rx : ry) : 0.0;
    return make_double2(__shfl_sync(0xffffffffu, s, 0), __shfl_sync(0xffffffffu, s, 1));
}

// CTA (chunk, q): partial <Y_q, b(u) (x) a(r)> over kCorrRows chirps. The last
// of the frame's `total` CTAs to finish sums the partials and solves every
// receiver's least squares.
__device__ void bomp_corr_body(const float2* __restrict__ Y, const GeoParams& g, int k, int K, const BompPtrs& w,
                               int ch, int q, unsigned total) {
    const float2* a = w.atoms_a + ((size_t)k * g.Q + q) * g.Ms;
    const float2* b = w.atoms_b + ((size_t)k * g.Q + q) * g.Mc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mc = ch * kCorrRows + warp;
    __shared__ double rx[kCorrRows], ry[kCorrRows];
    __shared__ bool s_last;
    double sx = 0.0, sy = 0.0;
    if (warp < kCorrRows && mc < g.Mc) {
        const float2* row = Y + ((size_t)q * g.Mc + mc) * g.Ms;
        float2 s = make_float2(0.f, 0.f);
        for (int m = lane; m < g.Ms; m += 32) {
            const float2 y = row[m];
            const float2 v = a[m];
            s.x += y.x * v.x + y.y * v.y;  // y * conj(a)
            s.y += y.y * v.x - y.x * v.y;
        }
        for (int off = 16; off > 0; off >>= 1) {
            s.x += __shfl_down_sync(0xffffffffu, s.x, off);
            s.y += __shfl_down_sync(0xffffffffu, s.y, off);
        }
        const double bx = b[mc].x, by = b[mc].y;  // s * conj(b)
        sx = (double)s.x * bx + (double)s.y * by;
        sy = (double)s.y * bx - (double)s.x * by;
    }
    if (lane == 0 && warp < kCorrRows) {
        rx[warp] = sx;
        ry[warp] = sy;
    }
    __syncthreads();
    if (warp == 0) {
        const double2 t = sum_rows_xy(rx, ry, lane);
        if (lane == 0) {
            w.corrp[((size_t)k * g.Q + q) * w.chunks + ch] = t;
            __threadfence();
            s_last = atomicAdd(w.counter, 1u) == total - 1;
        }
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bomp_sum_solve(g, k, K, w, blockDim.x);
    if (threadIdx.x == 0) *w.counter = 0u;  // ready for the next iteration
}


// One BOMP iteration in one launch, grid (chunks, Q), kStepThreads threads:
// every CTA reduces the scorer's partials to the selected cell (all CTAs get
// the same cell) and takes the new atom's (r, u) at its receiver; then its
// first kCorrRows warps make the atom a(r_q) in shared memory (the CTAs of
// chunk 0 also store it for the next maps' residual) and correlate kCorrRows
// chirps with the atom (storing their b(u_q) values), while its last warp
// writes the CTA's share of row k of the receiver's Gram matrix (entries
// t = chunk, chunk + chunks, ...). The last CTA to finish writes the
// selection, sums the correlations and solves every receiver's least
// squares. Same arithmetic as a selection followed by bomp_corr_body.
__global__ void __launch_bounds__(kStepThreads) bomp_step_kernel(const ArgPartial* __restrict__ parts, int nparts,
                                                        const float2* __restrict__ Y, ArgResult* __restrict__ sel,
                                                        int64_t* __restrict__ mask, int k, int K, GeoParams g,
                                                        BompPtrs w, const double* __restrict__ rw) {
    extern __shared__ float2 s_at[];  // a(r_q), Ms values
    __shared__ float s_bs[kStepThreads / 32];
    __shared__ long long s_bc[kStepThreads / 32];
    __shared__ long long s_best_cell;
    __shared__ float s_best;
    __shared__ unsigned long long s_rf, s_uf;
    __shared__ double rx[kCorrRows], ry[kCorrRows];
    __shared__ bool s_last;
    __shared__ double s_rk, s_uk;  // the new atom at this CTA's receiver
    const int ch = blockIdx.x, q = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this warp's chirp of Y, loaded now (Ms <= 256: eight samples per lane)
    // so that the loads overlap the selection and the new atom's geometry
    const int mc = ch * kCorrRows + warp;
    const bool has_row = warp < kCorrRows && mc < g.Mc;
    const float2* row = Y + ((size_t)q * g.Mc + (has_row ? mc : 0)) * g.Ms;
    constexpr int kPre = 8;
    const bool pre = g.Ms <= 32 * kPre;
    float2 yv[kPre];
#pragma unroll
    for (int j = 0; j < kPre; ++j) {
        const int m = lane + 32 * j;
        yv[j] = (pre && has_row && m < g.Ms) ? row[m] : make_float2(0.f, 0.f);
    }
    // selection (the same reduction in every CTA)
    float best = -INFINITY;
    long long bestc = 0x7fffffffffffffffLL;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) better(parts[i].score, parts[i].cell, best, bestc);
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
    if (warp == 0) {
        if (lane == 0) {
            for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) better(s_bs[ww], s_bc[ww], best, bestc);
            s_best = best;
            s_best_cell = bestc;
        }
        long long cell = __shfl_sync(0xffffffffu, bestc, 0);
        if (cell == 0x7fffffffffffffffLL) cell = 0;
        double r = 0.0, u = 0.0;
        if (rw) {
            // the new atom's (r, u) and fixed-point phases, lanes 0 and 1 side
            // by side (vx | vy, then r | u): float64 issues per warp
            // instruction, so the second lane comes free; the same operations
            // on the same values as cell_ru
            if (lane < 2) {
                int ix, iy, ivx, ivy;
                cell_decode(g, cell, &ix, &iy, &ivx, &ivy);
                const double* e = rw + (((long long)ix * g.n[1] + iy) * g.Q + q) * 3;
                r = e[0];
                const double wx = e[1], wy = e[2];
                const double v = lane == 0 ? gh_axis(g.lo[2], g.step[2], ivx) : gh_axis(g.lo[3], g.step[3], ivy);
                const double vo = __shfl_sync(0x3u, v, lane ^ 1);
                u = gh_speed(g, wx, wy, lane == 0 ? v : vo, lane == 0 ? vo : v);
                const uint64_t f = gh_phase_fix(lane == 0 ? r : u);
                if (lane == 0) {
                    s_rf = f;
                    s_rk = r;
                } else {
                    s_uf = f;
                    s_uk = u;
                }
            }
        } else if (lane == 0) {
            cell_ru(g, cell, q, rw, &r, &u);
            s_rf = gh_phase_fix(r);
            s_uf = gh_phase_fix(u);
            s_rk = r;
            s_uk = u;
        }
        if (ch == 0 && lane == 0) {  // the new atom's parameters at this receiver, for the last CTA
            w.ru[(size_t)k * g.Q + q] = make_double2(r, u);
            float sn, cs;
            sincospif(mod2f(r * (g.Ms - 1) + u * (g.Mc - 1)), &sn, &cs);
            w.phase[(size_t)k * g.Q + q] = make_double2(cs, sn);
        }
    }
    __syncthreads();
    double sx = 0.0, sy = 0.0;
    if (warp == kCorrRows) {
        // this CTA's entries of row k of the receiver's Gram matrix
        double* G = w.gram + (size_t)q * K * K;
        for (int t = ch + lane * (int)gridDim.x; t <= k; t += 32 * (int)gridDim.x) {
            const double2 rut = t == k ? make_double2(s_rk, s_uk) : __ldcg(w.ru + (size_t)t * g.Q + q);
            const double v = dirichlet(s_rk - rut.x, g.Ms) * dirichlet(s_uk - rut.y, g.Mc);
            G[k * K + t] = v;
            G[t * K + k] = v;
        }
        __threadfence();
    } else {
        float2* a_glob = w.atoms_a + ((size_t)k * g.Q + q) * g.Ms;
        for (int m = threadIdx.x; m < g.Ms; m += 32 * kCorrRows) {
            const float2 a = gh_cis_fix(s_rf * (unsigned long long)m);
            s_at[m] = a;
            if (ch == 0) a_glob[m] = a;
        }
        // the correlation warps only (the Gram warp does not wait for the atom)
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kCorrRows) : "memory");
        // correlation of kCorrRows chirps with b(u) (x) a(r)
        if (has_row) {
            float2 sm = make_float2(0.f, 0.f);
            if (pre) {
#pragma unroll
                for (int j = 0; j < kPre; ++j) {
                    const int m = lane + 32 * j;
                    if (m < g.Ms) {
                        const float2 y = yv[j];
                        const float2 v = s_at[m];
                        sm.x += y.x * v.x + y.y * v.y;  // y * conj(a)
                        sm.y += y.y * v.x - y.x * v.y;
                    }
                }
            } else {
                for (int m = lane; m < g.Ms; m += 32) {
                    const float2 y = row[m];
                    const float2 v = s_at[m];
                    sm.x += y.x * v.x + y.y * v.y;  // y * conj(a)
                    sm.y += y.y * v.x - y.x * v.y;
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                sm.x += __shfl_down_sync(0xffffffffu, sm.x, off);
                sm.y += __shfl_down_sync(0xffffffffu, sm.y, off);
            }
            const float2 b = gh_cis_fix(s_uf * (unsigned long long)mc);
            if (lane == 0) w.atoms_b[((size_t)k * g.Q + q) * g.Mc + mc] = b;
            const double bx = b.x, by = b.y;  // s * conj(b)
            sx = (double)sm.x * bx + (double)sm.y * by;
            sy = (double)sm.y * bx - (double)sm.x * by;
        }
    }
    if (lane == 0 && warp < kCorrRows) {
        rx[warp] = sx;
        ry[warp] = sy;
    }
    __syncthreads();
    if (warp == 0) {
        const double2 t = sum_rows_xy(rx, ry, lane);
        if (lane == 0) {
            w.corrp[((size_t)k * g.Q + q) * w.chunks + ch] = t;
            __threadfence();
            s_last = atomicAdd(w.counter, 1u) == gridDim.x * gridDim.y - 1;
        }
    }
    __syncthreads();
    // the new atom's maps at this receiver (for the next iteration's residual
    // maps), shared out among this receiver's CTAs that are done, so that the
    // last CTA's work does not wait for them; the last CTA takes what is left
    float2* tab_a = w.tab_a + ((size_t)k * g.Q + q) * g.Nr;
    float2* tab_b = w.tab_b + ((size_t)k * g.Q + q) * g.Nd;
    unsigned* tab_cnt = w.tab_counter + (size_t)k * g.Q + q;
    if (!s_last) {
        atom_map_tables_shared(s_rf, s_uf, g.Ms, g.Mc, g.Nr, g.Nd, tab_a, tab_b, tab_cnt);
        return;
    }
    __threadfence();
    if (warp == kCorrRows) {
        // the Gram warp takes what is left of the tables while the others solve
        atom_map_tables_warp(s_rf, s_uf, g.Ms, g.Mc, g.Nr, g.Nd, tab_a, tab_b, tab_cnt);
        return;
    }
    if (threadIdx.x == 0) {
        const bool valid = s_best_cell != 0x7fffffffffffffffLL;
        sel[k].cell = s_best_cell;
        sel[k].score = s_best;
        sel[k].valid = valid;
        mask[k] = s_best_cell;
    }
    bomp_sum_solve(g, k, K, w, 32 * kCorrRows);
    if (threadIdx.x == 0) *w.counter = 0u;  // ready for the next iteration
}

// Batched correlations: grid (max chunks, max Q, listed frames).
__global__ void __launch_bounds__(256) bomp_corr_batch_kernel(const BatchFrame* __restrict__ frames,
                                                              const int* __restrict__ active, int k) {
    const BatchFrame& F = frames[active[blockIdx.z]];
    if ((int)blockIdx.x >= F.bw.chunks || (int)blockIdx.y >= F.g.Q) return;
    bomp_corr_body(F.Y, F.g, k, F.K, F.bw, blockIdx.x, blockIdx.y, (unsigned)F.bw.chunks * (unsigned)F.g.Q);
}

__global__ void batch_reset_kernel(const BatchFrame* __restrict__ frames) {
    const BatchFrame& F = frames[blockIdx.x];
    if (threadIdx.x == 0) *F.bw.counter = 0u;
    for (int i = threadIdx.x; i < F.d.Q; i += blockDim.x) {  // row limits, filled by the coordinate tables
        F.rowlim[i] = 0x7fffffff;
        F.rowlim[F.d.Q + i] = -1;
    }
}

// Packs frame f's selections (ArgResult [K]) and amplitudes (double2 [K][Q])
// at byte offset offsets[f] of out; one CTA per frame.
__global__ void batch_gather_kernel(const BatchFrame* __restrict__ frames, const long long* __restrict__ offsets,
                                    unsigned char* __restrict__ out) {
    const BatchFrame& F = frames[blockIdx.x];
    ArgResult* s = (ArgResult*)(out + offsets[blockIdx.x]);
    double2* a = (double2*)(s + F.K);
    for (int i = threadIdx.x; i < F.K; i += blockDim.x) s[i] = F.sel[i];
    for (int i = threadIdx.x; i < F.K * F.g.Q; i += blockDim.x) a[i] = F.bw.alpha[i];
}

__global__ void __launch_bounds__(256) residual_kernel(const float2* __restrict__ Y, int Q, int Ms, int Mc,
                                                       Deflate df, float2* __restrict__ R) {
    const size_t per_q = (size_t)Mc * Ms;
    const size_t total = per_q * Q;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(idx / per_q);
        const size_t e = idx - (size_t)q * per_q;
        const int mc = (int)(e / Ms), m = (int)(e - (size_t)mc * Ms);
        R[idx] = gh_deflate(df, Q, Ms, Mc, q, mc, m, Y[idx]);
    }
}

// Measurement of the signal model; T targets, tgt = [T][4] then alpha [T][Q][2].
__global__ void __launch_bounds__(256) synth_kernel(GeoParams g, int T, const double* __restrict__ tgt,
                                                    const float2* __restrict__ noise, float2* __restrict__ Y) {
    __shared__ unsigned long long rf[64], uf[64];
    __shared__ float2 al[64];
    const int q = blockIdx.y;
    if (threadIdx.x < T) {
        const int t = threadIdx.x;
        const double x = tgt[4 * t], y = tgt[4 * t + 1], vx = tgt[4 * t + 2], vy = tgt[4 * t + 3];
        double d, wx, wy;
        gh_bistatic(g, q, x, y, &d, &wx, &wy);
        rf[t] = gh_phase_fix(gh_range(g, d));
        uf[t] = gh_phase_fix(gh_speed(g, wx, wy, vx, vy));
        const double* a = tgt + 4 * T + 2 * ((size_t)t * g.Q + q);
        al[t] = make_float2((float)a[0], (float)a[1]);
    }
    __syncthreads();
    const size_t per_q = (size_t)g.Mc * g.Ms;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_q; e += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long mc = e / g.Ms, m = e - mc * g.Ms;
        float2 v = noise ? noise[(size_t)q * per_q + e] : make_float2(0.f, 0.f);
        for (int t = 0; t < T; ++t) {
            const float2 c = cmul(al[t], gh_cis_fix(rf[t] * m + uf[t] * mc));
            v.x += c.x;
            v.y += c.y;
        }
        Y[(size_t)q * per_q + e] = v;
    }
}

}  // namespace

size_t gh_bomp_ws_bytes(const Dims& d, int K) { return bomp_layout(d, K).total; }

Deflate gh_bomp_deflate(void* ws, const Dims& d, int K, int n) {
    const BompPtrs w = bomp_ptrs(ws, d, K);
    Deflate f;
    f.alpha = w.alpha;
    f.atoms_a = w.atoms_a;
    f.atoms_b = w.atoms_b;
    f.n = n;
    f.alpha_prev = w.alpha_prev;
    f.tab_a = w.tab_a;
    f.tab_b = w.tab_b;
    f.ru = w.ru;
    return f;
}

int gh_bomp_reset(gh_ctx* ctx, const Dims& d, int K, void* ws) {
    const BompPtrs w = bomp_ptrs(ws, d, K);
    GH_CUDA(cudaMemsetAsync(w.counter, 0, (size_t)(1 + K * d.Q) * sizeof(unsigned int), ctx->stream));
    return GH_OK;
}

int gh_launch_bomp_step(gh_ctx* ctx, const Dims& d, const GeoParams& g, const ArgPartial* parts, int nparts,
                        const float2* Y, ArgResult* sel, int64_t* mask, int k, int K, void* ws, const double* rw) {
    const BompPtrs w = bomp_ptrs(ws, d, K);
    const size_t smem = (size_t)d.Ms * sizeof(float2);
    GH_CUDA(cudaFuncSetAttribute(bomp_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_step_kernel<<<dim3(w.chunks, d.Q), kStepThreads, smem, ctx->stream>>>(parts, nparts, Y, sel, mask, k, K,
                                                                                  g, w, rw);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_step_kernel");
}

int gh_launch_residual(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate& df, float2* R) {
    const size_t total = (size_t)d.Q * d.Mc * d.Ms;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (blocks > (unsigned)ctx->num_sms * 8) blocks = (unsigned)ctx->num_sms * 8;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    residual_kernel<<<blocks, 256, 0, ctx->stream>>>(Y, d.Q, d.Ms, d.Mc, df, R);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "residual_kernel");
}

int gh_launch_synth(gh_ctx* ctx, const Dims& d, const GeoParams& g, int T, const double* tgt, const float2* noise,
                    float2* Y) {
    const size_t per_q = (size_t)d.Mc * d.Ms;
    unsigned bx = (unsigned)((per_q + 255) / 256);
    if (bx > 1024) bx = 1024;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_SYNTH, &ev);
    synth_kernel<<<dim3(bx, d.Q), 256, 0, ctx->stream>>>(g, T, tgt, noise, Y);
    return gh_launch_end(ctx, GH_K_SYNTH, ev, "synth_kernel");
}

int gh_launch_bomp_select_batch(gh_ctx* ctx, const BatchFrame* frames, const int* active, int n, int k) {
    if (n == 0) return GH_OK;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_ARGMAX, &ev);
    bomp_select_batch_kernel<<<n, 1024, 0, ctx->stream>>>(frames, active, k);
    return gh_launch_end(ctx, GH_K_ARGMAX, ev, "bomp_select_batch_kernel");
}

int gh_launch_bomp_corr_batch(gh_ctx* ctx, const BatchFrame* frames, const int* active, int n, int k, int max_chunks,
                              int max_q) {
    if (n == 0) return GH_OK;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_corr_batch_kernel<<<dim3(max_chunks, max_q, n), 32 * kCorrRows, 0, ctx->stream>>>(frames, active, k);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_corr_batch_kernel");
}

int gh_launch_batch_gather(gh_ctx* ctx, const BatchFrame* frames, int nframes, const long long* offsets, void* out) {
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    batch_gather_kernel<<<nframes, 128, 0, ctx->stream>>>(frames, offsets, (unsigned char*)out);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "batch_gather_kernel");
}

BompPtrs gh_bomp_ptrs(void* ws, const Dims& d, int K) { return bomp_ptrs(ws, d, K); }
int gh_bomp_chunks(const Dims& d) { return (d.Mc + kCorrRows - 1) / kCorrRows; }

int gh_launch_batch_reset(gh_ctx* ctx, const BatchFrame* frames, int nframes) {
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    batch_reset_kernel<<<nframes, 32, 0, ctx->stream>>>(frames);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "batch_reset_kernel");
}
