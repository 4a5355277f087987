// Range-Doppler maps (Sec. III: the 2D FFT of each Y_q; Sec. IV: the FFT bins
// are correlations with the atoms on the FFT's frequency grid).
//
// Two FFT kernels, both Stockham (radix-16 register passes, a last radix-2,
// -4, -8 or -16 pass; the first pass reads global memory, the last writes it,
// the others work in place in shared memory) with float32 data and a twiddle
// table rounded from float64 and staged in shared memory:
//   range_fft   : per (q, mc) row, the Ms samples zero-padded to Nr = pad*Ms,
//                 written [Q][Mc][Nr]; a BOMP residual can be subtracted from
//                 the samples as they are loaded;
//   doppler_fft : per (q, block of IB range bins), the Mc chirps zero-padded to
//                 Nd = pad*Mc, times the range-centring factor
//                 exp(j pi (i/Nr)(Ms-1)), written [Q][Nr][Nd] so that one
//                 range bin's Doppler row is contiguous for the scorer.
// and maps_deflate, which takes complex float32 maps to those of a BOMP
// residual by linearity (the atoms' maps in closed form, see Deflate).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <vector>

#include "gh_internal.cuh"

namespace {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Position of element i of a column in shared memory: one float2 of padding
// after every 16, so that the strided stores of the first pass (runs of R
// outputs every R) fall into different banks.
__device__ __forceinline__ int p16(int i) { return i + (i >> 4); }

// exp(-j 2 pi t / 16) for t = 0 .. 9 (the in-register twiddles of a 16-point
// DFT split 4 x 4): cos(pi/8), sin(pi/8) and sqrt(1/2).
constexpr float kC8 = 0.92387953251128675613f, kS8 = 0.38268343236508977173f, kR2 = 0.70710678118654752440f;
__host__ __device__ constexpr float cos16(int t) {
    return t == 0 ? 1.f : t == 1 ? kC8 : t == 2 ? kR2 : t == 3 ? kS8 : t == 4 ? 0.f : t == 5 ? -kS8
         : t == 6 ? -kR2 : t == 7 ? -kC8 : t == 8 ? -1.f : -kC8;
}
__host__ __device__ constexpr float sin16(int t) {
    return t == 0 ? 0.f : t == 1 ? kS8 : t == 2 ? kR2 : t == 3 ? kC8 : t == 4 ? 1.f : t == 5 ? kC8
         : t == 6 ? kR2 : t == 7 ? kS8 : t == 8 ? 0.f : -kS8;
}

// v * exp(-j 2 pi t / R), t and R compile-time after unrolling.
template <int R>
__device__ __forceinline__ float2 rot(float2 v, int t) {
    const int u = t * (16 / R);
    if (u == 0) return v;
    if (u == 4) return make_float2(v.y, -v.x);
    const float c = cos16(u), s = sin16(u);
    return make_float2(v.x * c + v.y * s, v.y * c - v.x * s);
}

// In-register forward DFTs, natural order in and out.
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = f2add(t, b);
    b = f2sub(t, b);
}
__device__ __forceinline__ void dft4(float2& a, float2& b, float2& c, float2& d) {
    const float2 s0 = f2add(a, c), s1 = f2sub(a, c), s2 = f2add(b, d), t = f2sub(b, d);
    const float2 s3 = make_float2(t.y, -t.x);  // (b - d) * (-j)
    a = f2add(s0, s2);
    b = f2add(s1, s3);
    c = f2sub(s0, s2);
    d = f2sub(s1, s3);
}
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
    if constexpr (R == 2) {
        dft2(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4(v[0], v[1], v[2], v[3]);
    } else {
        // R = 4 x R2: n = R2 n1 + n2, k = k1 + 4 k2; 4-point DFTs over n1, the
        // twiddles exp(-j 2 pi n2 k1 / R), then R2-point DFTs over n2
        constexpr int R2 = R / 4;
        float2 a[R];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) {
            float2 c0 = v[n2], c1 = v[R2 + n2], c2 = v[2 * R2 + n2], c3 = v[3 * R2 + n2];
            dft4(c0, c1, c2, c3);
            a[n2 * 4 + 0] = c0;
            a[n2 * 4 + 1] = rot<R>(c1, n2);
            a[n2 * 4 + 2] = rot<R>(c2, 2 * n2);
            a[n2 * 4 + 3] = rot<R>(c3, 3 * n2);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            if constexpr (R2 == 2) {
                float2 b0 = a[k1], b1 = a[4 + k1];
                dft2(b0, b1);
                v[k1] = b0;
                v[k1 + 4] = b1;
            } else {
                float2 b0 = a[k1], b1 = a[4 + k1], b2 = a[8 + k1], b3 = a[12 + k1];
                dft4(b0, b1, b2, b3);
                v[k1] = b0;
                v[k1 + 4] = b1;
                v[k1 + 8] = b2;
                v[k1 + 12] = b3;
            }
        }
    }
}

// Where a Stockham pass reads its inputs and writes its outputs.
enum { kGlobal = 0, kShared = 1 };

// One radix-R Stockham pass over `ncol` columns of length N = 2^logN whose
// sub-transforms of length Ns are done: item (c, j), k = j mod Ns, takes
// x[j + m N/R] (m < R), multiplies it by exp(-j 2 pi m k / (R Ns)), takes the
// R-point DFT and writes y[(j - k) R + k + r Ns] (r < R).
//  * SRC kGlobal: the first pass (Ns = 1, no twiddles); the item's inputs
//    n = j + m N/R come from load.load_item, only those with n < nz (the
//    rest is the zero padding).
//  * SRC kShared: inputs from buf[c * ld + p16(n)]; the twiddles come from
//    tw[t] = exp(-j 2 pi t / N), t < N/2: the powers 1, 2, 4, 8 of
//    exp(-j 2 pi k / (R Ns)) are read and the others are their products.
//  * DST kShared: outputs to buf; with SRC kShared the pass is in place (one
//    item per thread, all reads before a barrier, then all writes), which
//    needs ncol N / R <= blockDim.x.
//  * DST kGlobal: outputs to store(c, n, value).
// CF: items numbered column-fastest (c = idx mod ncol), for loads that are
// contiguous across columns; otherwise j-fastest.
template <int R, int LR, int SRC, int DST, bool CF, class Load, class Store>
__device__ __forceinline__ void fft_pass(float2* buf, int logN, int Ns, int ncol, int ld, const float2* tw, int nz,
                                         const Load& load, const Store& store) {
    const int lq = logN - LR, q = 1 << lq;
    const int total = ncol << lq;
    const int tstep = q / Ns;
    auto item = [&](int idx, int& c, int& j, int& k, float2 (&v)[R]) {
        if (CF) {
            j = idx / ncol;
            c = idx - j * ncol;
        } else {
            c = idx >> lq;
            j = idx & (q - 1);
        }
        k = j & (Ns - 1);
        if constexpr (SRC == kGlobal) {
#pragma unroll
            load.template load_item<R>(c, j, q, nz, v);
        } else {
            const float2* xc = buf + c * ld;
#pragma unroll
            for (int m = 0; m < R; ++m) v[m] = xc[p16(j + m * q)];
            if (Ns > 1) {
                const int s = k * tstep;
                float2 w[R];
                w[1] = tw[s];
                if constexpr (R >= 4) {
                    w[2] = tw[2 * s];
                    w[3] = cmul(w[1], w[2]);
                }
                if constexpr (R >= 8) {
                    w[4] = tw[4 * s];
#pragma unroll
                    for (int m = 5; m < 8; ++m) w[m] = cmul(w[4], w[m - 4]);
                }
                if constexpr (R >= 16) {
                    w[8] = tw[8 * s];
#pragma unroll
                    for (int m = 9; m < 16; ++m) w[m] = cmul(w[8], w[m - 8]);
                }
#pragma unroll
                for (int m = 1; m < R; ++m) v[m] = cmul(v[m], w[m]);
            }
        }
        dft<R>(v);
    };
    auto emit = [&](int c, int j, int k, const float2 (&v)[R]) {
        const int o = ((j - k) << LR) + k;
        if constexpr (DST == kShared) {
            float2* yc = buf + c * ld;
#pragma unroll
            for (int r = 0; r < R; ++r) yc[p16(o + r * Ns)] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) store(c, o + r * Ns, v[r]);
        }
    };
    if constexpr (SRC == kShared && DST == kShared) {
        const bool has = (int)threadIdx.x < total;
        int c = 0, j = 0, k = 0;
        float2 v[R];
        if (has) item(threadIdx.x, c, j, k, v);
        __syncthreads();
        if (has) emit(c, j, k, v);
    } else {
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int c, j, k;
            float2 v[R];
            item(idx, c, j, k, v);
            emit(c, j, k, v);
        }
    }
}

// Last pass of an FFT: radix 2^LR with LR in [1, 4], shared memory to global.
template <class Load, class Store>
__device__ __forceinline__ void fft_last(float2* buf, int logN, int LR, int Ns, int ncol, int ld, const float2* tw,
                                         int nz, const Load& load, const Store& store) {
    switch (LR) {
        case 1: fft_pass<2, 1, kShared, kGlobal, false>(buf, logN, Ns, ncol, ld, tw, nz, load, store); break;
        case 2: fft_pass<4, 2, kShared, kGlobal, false>(buf, logN, Ns, ncol, ld, tw, nz, load, store); break;
        case 3: fft_pass<8, 3, kShared, kGlobal, false>(buf, logN, Ns, ncol, ld, tw, nz, load, store); break;
        default: fft_pass<16, 4, kShared, kGlobal, false>(buf, logN, Ns, ncol, ld, tw, nz, load, store); break;
    }
}

// Stockham FFT of `ncol` columns of length N = 2^logN (N >= 4) from global
// memory to global memory: load.load_item<R>(c, j, s, nz, v) reads the
// inputs n = j + m s (m < R) of column c, only those with n < nz (the rest is
// the zero padding); output bin n is passed to store(c, n, value). Radix-16 passes and one last radix-2, -4, -8 or -16
// pass; the first pass reads global memory, the last writes it, the others
// work in place in buf (element n of column c at buf[c * ld + p16(n)],
// ld >= N + N/16). tw: exp(-j 2 pi t / N), t < N/2, in shared memory and
// complete before the first barrier. blockDim.x >= ncol N / 16 when N > 256.
template <bool CF, class Load, class Store>
__device__ __forceinline__ void fft_columns(float2* buf, int logN, int ncol, int ld, const float2* tw, int nz,
                                            const Load& load, const Store& store) {
    const int P = (logN + 3) >> 2;          // passes
    const int LR = logN - 4 * (P - 1);      // log2 of the last pass's radix
    if (P == 1) {
        if (LR == 2) fft_pass<4, 2, kGlobal, kGlobal, CF>(buf, logN, 1, ncol, ld, tw, nz, load, store);
        else if (LR == 3) fft_pass<8, 3, kGlobal, kGlobal, CF>(buf, logN, 1, ncol, ld, tw, nz, load, store);
        else fft_pass<16, 4, kGlobal, kGlobal, CF>(buf, logN, 1, ncol, ld, tw, nz, load, store);
        return;
    }
    fft_pass<16, 4, kGlobal, kShared, CF>(buf, logN, 1, ncol, ld, tw, nz, load, store);
    __syncthreads();
    int Ns = 16;
    for (int p = 1; p < P - 1; ++p) {
        fft_pass<16, 4, kShared, kShared, false>(buf, logN, Ns, ncol, ld, tw, nz, load, store);
        __syncthreads();
        Ns <<= 4;
    }
    fft_last(buf, logN, LR, Ns, ncol, ld, tw, nz, load, store);
}

__device__ void load_twiddles(float2* dst, const float2* __restrict__ src, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = __ldg(src + t);
}

// Range FFT input: samples n = j + m s (m < R, n < nz) of row r0 + c
// (row = q * Mc + mc), minus the BOMP residual sum_t alpha_t b_t[mc] a_t[n]
// (gh_deflate's arithmetic; the row's amplitude and b value are loaded once
// per item); output: bin n of that row, [Q][Mc][Nr].
struct RangeIO {
    const float2* __restrict__ Y;
    float2* __restrict__ out;
    Deflate df;
    int Q, Ms, Mc, r0, logNr;
    template <int R>
    __device__ __forceinline__ void load_item(int c, int j, int s, int nz, float2 (&v)[R]) const {
        const int row = r0 + c;
        const float2* y = Y + (size_t)row * Ms;
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = j + m * s < nz ? y[j + m * s] : make_float2(0.f, 0.f);
        if (df.n > 0) {
            const int qq = row / Mc, mc = row - qq * Mc;
            for (int t = 0; t < df.n; ++t) {
                const double2 al = df.alpha[(size_t)t * Q + qq];
                const float2 b = df.atoms_b[((size_t)t * Q + qq) * Mc + mc];
                const float2* a = df.atoms_a + ((size_t)t * Q + qq) * Ms;
                const float ax = (float)al.x, ay = (float)al.y;
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    if (j + m * s < nz) {
                        const float2 av = a[j + m * s];
                        const float2 ab = make_float2(av.x * b.x - av.y * b.y, av.x * b.y + av.y * b.x);
                        v[m].x -= ax * ab.x - ay * ab.y;
                        v[m].y -= ax * ab.y + ay * ab.x;
                    }
                }
            }
        }
    }
    __device__ void operator()(int c, int n, float2 v) const { out[((size_t)(r0 + c) << logNr) + n] = v; }
};

// Range FFTs of rows r0 .. r0 + nrow - 1 (row = q * Mc + mc) of one frame;
// shared memory: gh_fft_smem_range(nrow, Nr) bytes.
__device__ __forceinline__ void range_rows(const float2* __restrict__ Y, float2* __restrict__ out, int Q, int Ms,
                                           int Mc, int logNr, int r0, int nrow, const Deflate& df,
                                           const float2* __restrict__ tw, float2* smem) {
    const int Nr = 1 << logNr;
    const int ld = gh_fft_ld(Nr);
    float2* twS = smem + nrow * ld;
    load_twiddles(twS, tw, Nr / 2);
    const RangeIO io{Y, out, df, Q, Ms, Mc, r0, logNr};
    fft_columns<false>(smem, logNr, nrow, ld, twS, Ms, io, io);
}

__global__ void __launch_bounds__(512) range_fft_kernel(const float2* __restrict__ Y, float2* __restrict__ out,
                                                        int Q, int Ms, int Mc, int logNr, int rows,
                                                        int rows_per_cta, Deflate df,
                                                        const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int r0 = blockIdx.x * rows_per_cta;
    range_rows(Y, out, Q, Ms, Mc, logNr, r0, min(rows_per_cta, rows - r0), df, tw, smem);
}

// One map bin in storage type MT (float32 pair, or 2^-s times the value
// rounded to nearest-even float16 / bfloat16).
template <int MT>
__device__ __forceinline__ void store_bin(void* maps, size_t idx, float2 v, float oscale) {
    if constexpr (MT == GH_C64) {
        ((float2*)maps)[idx] = v;
    } else if constexpr (MT == GH_C16) {
        ((__half2*)maps)[idx] = __floats2half2_rn(v.x * oscale, v.y * oscale);
    } else {
        ((__nv_bfloat162*)maps)[idx] = __floats2bfloat162_rn(v.x * oscale, v.y * oscale);
    }
}

// Doppler FFT input: chirp n of range bin i0 + c of receiver q ([Q][Mc][Nr]);
// output: Doppler bin n of that range bin times the range-centring factor,
// [Q][Nr][Nd] in storage type MT.
template <int MT>
struct DopplerIO {
    const float2* __restrict__ src;  // Zr + q Mc Nr + i0
    void* __restrict__ maps;
    size_t dst;  // (q Nr + i0) Nd
    const float2* ramp;
    float oscale;
    int Nr, logNd;
    template <int R>
    __device__ __forceinline__ void load_item(int c, int j, int s, int nz, float2 (&v)[R]) const {
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = j + m * s < nz ? src[(size_t)(j + m * s) * Nr + c] : make_float2(0.f, 0.f);
    }
    __device__ void operator()(int c, int n, float2 v) const {
        store_bin<MT>(maps, dst + ((size_t)c << logNd) + n, cmul(v, ramp[c]), oscale);
    }
};

// Doppler FFTs of range bins i0 .. i0 + IB - 1 of receiver q of one frame,
// times the range-centring factor, stored in type MT. Shared memory:
// gh_fft_smem_dop(IB, Nd) bytes.
template <int MT>
__device__ __forceinline__ void doppler_cols(const float2* __restrict__ Zr, void* __restrict__ maps, int Ms, int Mc,
                                             int logNr, int logNd, int IB, int q, int i0,
                                             const float2* __restrict__ tw, float oscale, float2* smem) {
    const int Nr = 1 << logNr;
    const int Nd = 1 << logNd;
    // column stride = 2 mod 16 float2: the column-fastest first pass stores
    // (8 columns x 2 items per half-warp) spread over the banks
    const int ld = gh_fft_ld(Nd) + 2;
    float2* ramp = smem + IB * ld;
    float2* twS = ramp + IB;
    load_twiddles(twS, tw, Nd / 2);
    if (threadIdx.x < IB) {
        // exp(j pi (i/Nr)(Ms-1)) with the angle reduced exactly modulo 2 pi
        const long long t = ((long long)(i0 + threadIdx.x) * (Ms - 1)) % (2LL * Nr);
        float s, c;
        sincospif((float)t / (float)Nr, &s, &c);
        ramp[threadIdx.x] = make_float2(c, s);
    }
    if (logNd <= 4) __syncthreads();  // one pass, no barrier before the stores read ramp
    const DopplerIO<MT> io{Zr + (size_t)q * Mc * Nr + i0, maps, ((size_t)q * Nr + i0) * Nd, ramp, oscale, Nr, logNd};
    fft_columns<true>(smem, logNd, IB, ld, twS, Mc, io, io);
}

template <int MT>
__global__ void __launch_bounds__(512, 2) doppler_fft_kernel(const float2* __restrict__ Zr, void* __restrict__ maps,
                                                          int Ms, int Mc, int logNr, int logNd, int IB,
                                                          const float2* __restrict__ tw, float oscale,
                                                          const int* __restrict__ rowlim, int Q) {
    extern __shared__ float2 smem[];
    const int i0 = blockIdx.x * IB;
    if (rowlim && (i0 + IB - 1 < rowlim[blockIdx.y] || i0 > rowlim[Q + blockIdx.y])) return;  // whole CTA
    doppler_cols<MT>(Zr, maps, Ms, Mc, logNr, logNd, IB, blockIdx.y, i0, tw, oscale, smem);
}

// Maps of the residual by linearity (complex float32 maps, in place): range
// bins i0 .. i0 + IB - 1 of receiver q lose
//   sum_{t < df.n} (alpha_t - alpha_prev_t) tab_a_t[i] tab_b_t[j],
// the part of the atoms' maps (Sec. III) the maps do not yet hold; IB <= 16.
__device__ __forceinline__ void deflate_rows(float2* __restrict__ maps, const Deflate& df, int Q, int Nr, int Nd,
                                             int logNd, int q, int i0, int IB) {
    __shared__ float2 s_c[GH_MAX_K * 16];  // (alpha_t - alpha_prev_t) tab_a_t[i], per atom and row
    const int n = df.n;
    // two bins per 16-byte access, eight accesses in flight per thread (the
    // whole share of a CTA of eight 512-bin rows); the first eight are issued
    // before the coefficients are staged, so that the two rounds of loads
    // overlap
    constexpr int U = 8;
    float4* row = (float4*)(maps + ((size_t)q * Nr + i0) * Nd);
    const int hp = Nd >> 1, lp = logNd - 1, npair = IB * hp;
    float4 v[U];
    auto load_u = [&](int base) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int pidx = base + u * blockDim.x;
            if (pidx < npair) v[u] = row[pidx];
        }
    };
    load_u(threadIdx.x);
    for (int idx = threadIdx.x; idx < n * IB; idx += blockDim.x) {
        const int t = idx / IB, ii = idx - t * IB;
        const double2 al = df.alpha[(size_t)t * Q + q], ap = df.alpha_prev[(size_t)t * Q + q];
        const float2 da = make_float2((float)(al.x - ap.x), (float)(al.y - ap.y));
        s_c[idx] = cmul(da, df.tab_a[((size_t)t * Q + q) * Nr + i0 + ii]);
    }
    __syncthreads();
    for (int base = threadIdx.x; base < npair; base += U * blockDim.x) {
        if (base != (int)threadIdx.x) load_u(base);
        for (int t = 0; t < n; ++t) {
            const float4* tb = (const float4*)(df.tab_b + ((size_t)t * Q + q) * Nd);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int pidx = base + u * blockDim.x;
                if (pidx < npair) {
                    const float4 b = __ldg(tb + (pidx & (hp - 1)));
                    const float2 c = s_c[t * IB + (pidx >> lp)];
                    v[u].x -= c.x * b.x - c.y * b.y;
                    v[u].y -= c.x * b.y + c.y * b.x;
                    v[u].z -= c.x * b.z - c.y * b.w;
                    v[u].w -= c.x * b.w + c.y * b.z;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (base + u * blockDim.x < npair) row[base + u * blockDim.x] = v[u];
    }
}

__global__ void __launch_bounds__(256) maps_deflate_kernel(float2* __restrict__ maps, Deflate df, int Q, int Nr,
                                                           int Nd, int logNd, int IB, const int* __restrict__ rowlim) {
    const int i0 = blockIdx.x * IB;
    if (rowlim && (i0 + IB - 1 < rowlim[blockIdx.y] || i0 > rowlim[Q + blockIdx.y])) return;  // whole CTA
    deflate_rows(maps, df, Q, Nr, Nd, logNd, blockIdx.y, i0, IB);
}

// Batched maps of several frames: one work item (frame, first row / range
// bin, count) per CTA; the residual of iteration k is applied on load.
__global__ void __launch_bounds__(512) range_fft_batch_kernel(const BatchFrame* __restrict__ frames,
                                                              const BatchItem* __restrict__ items, int k) {
    extern __shared__ float2 smem[];
    const BatchItem it = items[blockIdx.x];
    const BatchFrame& F = frames[it.frame];
    Deflate df = F.df;
    df.n = k;
    int logNr = 0;
    while ((1 << logNr) < F.d.Nr) ++logNr;
    range_rows(F.Y, F.zr, F.d.Q, F.d.Ms, F.d.Mc, logNr, (int)it.start, (int)it.count, df, F.twr, smem);
}

// Batched residual maps by linearity: one item (frame, receiver, first range
// bin, count) per CTA, iteration k (atoms 0 .. k-1); items outside the frame's
// row limits (rows no coordinate entry reads) do nothing, as in gh_detect.
__global__ void __launch_bounds__(256) maps_deflate_batch_kernel(const BatchFrame* __restrict__ frames,
                                                                 const BatchItem* __restrict__ items, int k) {
    const BatchItem it = items[blockIdx.x];
    const BatchFrame& F = frames[it.frame];
    const int i0 = (int)it.start, q = it.aux;
    if (i0 + (int)it.count - 1 < F.rowlim[q] || i0 > F.rowlim[F.d.Q + q]) return;  // rows the scorer never reads
    Deflate df = F.df;
    df.n = k;
    int logNd = 0;
    while ((1 << logNd) < F.d.Nd) ++logNd;
    deflate_rows(F.maps, df, F.d.Q, F.d.Nr, F.d.Nd, logNd, q, i0, (int)it.count);
}

__global__ void __launch_bounds__(512, 2) doppler_fft_batch_kernel(const BatchFrame* __restrict__ frames,
                                                                const BatchItem* __restrict__ items) {
    extern __shared__ float2 smem[];
    const BatchItem it = items[blockIdx.x];
    const BatchFrame& F = frames[it.frame];
    const int i0 = (int)it.start, q = it.aux;
    if (i0 + (int)it.count - 1 < F.rowlim[q] || i0 > F.rowlim[F.d.Q + q]) return;  // rows the scorer never reads
    int logNr = 0, logNd = 0;
    while ((1 << logNr) < F.d.Nr) ++logNr;
    while ((1 << logNd) < F.d.Nd) ++logNd;
    doppler_cols<GH_C64>(F.zr, F.maps, F.d.Ms, F.d.Mc, logNr, logNd, (int)it.count, q, i0, F.twd, 1.0f, smem);
}

}  // namespace

void gh_twiddles(int N, float2* out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < N / 2; ++t) {
        const double a = -two_pi * (double)t / (double)N;
        out[t] = make_float2((float)cos(a), (float)sin(a));
    }
}

namespace {

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Uploads exp(-j 2 pi t / N), t < N/2, for N = Nr then N = Nd (float64 -> float32).
int ensure_twiddles(gh_ctx* ctx, int Nr, int Nd, const float2** twr, const float2** twd) {
    const int nr = Nr / 2, nd = Nd / 2;
    size_t bytes = (size_t)(nr + nd) * sizeof(float2);
    void* p;
    GH_TRY(gh_ws(ctx, WS_TWIDDLE, bytes, &p));
    if (ctx->tw_n[0] != Nr || ctx->tw_n[1] != Nd) {
        if (ctx->capturing) return gh_fail(ctx, GH_ECUDA, "twiddle upload during graph capture");
        gh_graph_invalidate(ctx);  // cached graphs read the old tables
        std::vector<float2> h(nr + nd);
        gh_twiddles(Nr, h.data());
        gh_twiddles(Nd, h.data() + nr);
        GH_CUDA(cudaMemcpyAsync(p, h.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
        GH_CUDA(cudaStreamSynchronize(ctx->stream));  // h goes out of scope
        ctx->tw_n[0] = Nr;
        ctx->tw_n[1] = Nd;
    }
    *twr = (const float2*)p;
    *twd = (const float2*)p + nr;
    return GH_OK;
}

}  // namespace

static int range_fft(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate* df, const float2* twr,
                     void** zr_out) {
    Deflate none = {nullptr, nullptr, nullptr, 0};
    void* zr;
    GH_TRY(gh_ws(ctx, WS_RANGE, (size_t)d.Q * d.Mc * d.Nr * sizeof(float2), &zr));
    // rows of Nr points, 2048 points per CTA (one row when Nr > 2048), one
    // thread per radix-16 butterfly
    const int logNr = ilog2(d.Nr);
    const int rpc = gh_fft_rows_per_cta(d.Nr);
    const int rows = d.Q * d.Mc;
    const size_t smem1 = gh_fft_smem_range(rpc, d.Nr);
    const int threads = gh_fft_threads(rpc * d.Nr);
    GH_CUDA(cudaFuncSetAttribute(range_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
    range_fft_kernel<<<(rows + rpc - 1) / rpc, threads, smem1, ctx->stream>>>(
        Y, (float2*)zr, d.Q, d.Ms, d.Mc, logNr, rows, rpc, df ? *df : none, twr);
    GH_TRY(gh_launch_end(ctx, GH_K_RANGE_FFT, ev, "range_fft_kernel"));
    *zr_out = zr;
    return GH_OK;
}

int gh_launch_range_rows(gh_ctx* ctx, const Dims& d, const float2* Y, void** zr) {
    const float2 *twr, *twd;
    GH_TRY(ensure_twiddles(ctx, d.Nr, d.Nd, &twr, &twd));
    return range_fft(ctx, d, Y, nullptr, twr, zr);
}

int gh_launch_maps(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate* df, void* maps, int map_dtype,
                   const int* rowlim) {
    const float2 *twr, *twd;
    GH_TRY(ensure_twiddles(ctx, d.Nr, d.Nd, &twr, &twd));
    void* zr;
    GH_TRY(range_fft(ctx, d, Y, df, twr, &zr));
    const int logNr = ilog2(d.Nr), logNd = ilog2(d.Nd);
    cudaEvent_t ev;
    // Doppler FFT: IB range bins per CTA
    const int IB = gh_fft_bins_per_cta(d.Nr, d.Nd);
    const size_t smem2 = gh_fft_smem_dop(IB, d.Nd);
    const int threads = gh_fft_threads(IB * d.Nd);
    const float oscale = ldexpf(1.0f, -gh_map_scale_log2(d, map_dtype));
    auto kern = map_dtype == GH_C16 ? doppler_fft_kernel<GH_C16>
              : map_dtype == GH_CBF16 ? doppler_fft_kernel<GH_CBF16> : doppler_fft_kernel<GH_C64>;
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    gh_launch_begin(ctx, GH_K_DOPPLER_FFT, &ev);
    kern<<<dim3(d.Nr / IB, d.Q), threads, smem2, ctx->stream>>>((const float2*)zr, maps, d.Ms, d.Mc, logNr, logNd, IB,
                                                            twd, oscale, rowlim, d.Q);
    return gh_launch_end(ctx, GH_K_DOPPLER_FFT, ev, "doppler_fft_kernel");
}

int gh_launch_maps_deflate(gh_ctx* ctx, const Dims& d, const Deflate& df, void* maps, const int* rowlim) {
    if (df.n == 0) return GH_OK;
    if (df.n > GH_MAX_K) return gh_fail(ctx, GH_EINVAL, "maps deflation of %d atoms", df.n);
    const int IB = gh_fft_bins_per_cta(d.Nr, d.Nd);
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_DEFLATE, &ev);
    maps_deflate_kernel<<<dim3(d.Nr / IB, d.Q), 256, 0, ctx->stream>>>((float2*)maps, df, d.Q, d.Nr, d.Nd,
                                                                      ilog2(d.Nd), IB, rowlim);
    return gh_launch_end(ctx, GH_K_DEFLATE, ev, "maps_deflate_kernel");
}

int gh_launch_maps_deflate_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, int k) {
    if (n == 0 || k == 0) return GH_OK;
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_DEFLATE, &ev);
    maps_deflate_batch_kernel<<<n, 256, 0, ctx->stream>>>(frames, items, k);
    return gh_launch_end(ctx, GH_K_DEFLATE, ev, "maps_deflate_batch_kernel");
}

int gh_launch_maps_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* range_items, int n_range,
                         int thr_range, size_t smem_range, const BatchItem* dop_items, int n_dop, int thr_dop,
                         size_t smem_dop, int k) {
    if (n_range > 0) {
        GH_CUDA(cudaFuncSetAttribute(range_fft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_range));
        cudaEvent_t ev;
        gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
        range_fft_batch_kernel<<<n_range, thr_range, smem_range, ctx->stream>>>(frames, range_items, k);
        GH_TRY(gh_launch_end(ctx, GH_K_RANGE_FFT, ev, "range_fft_batch_kernel"));
    }
    if (n_dop > 0) {
        GH_CUDA(cudaFuncSetAttribute(doppler_fft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_dop));
        cudaEvent_t ev;
        gh_launch_begin(ctx, GH_K_DOPPLER_FFT, &ev);
        doppler_fft_batch_kernel<<<n_dop, thr_dop, smem_dop, ctx->stream>>>(frames, dop_items);
        GH_TRY(gh_launch_end(ctx, GH_K_DOPPLER_FFT, ev, "doppler_fft_batch_kernel"));
    }
    return GH_OK;
}
