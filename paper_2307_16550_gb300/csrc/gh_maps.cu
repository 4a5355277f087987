// Range-Doppler maps (Sec. III: the 2D FFT of each Y_q; Sec. IV: the FFT bins
// are correlations with the atoms on the FFT's frequency grid).
//
// Two kernels, both Stockham FFTs in shared memory (radix-4 passes, one
// radix-2 pass for odd log2 sizes) with float32 data and a twiddle table
// rounded from float64 and staged in shared memory:
//   range_fft   : per (q, mc) row, the Ms samples zero-padded to Nr = pad*Ms,
//                 written [Q][Mc][Nr]; a BOMP residual is subtracted from the
//                 samples as they are loaded;
//   doppler_fft : per (q, block of IB range bins), the Mc chirps zero-padded to
//                 Nd = pad*Mc, times the range-centring factor
//                 exp(j pi (i/Nr)(Ms-1)), written [Q][Nr][Nd] so that one
//                 range bin's Doppler row is contiguous for the scorer.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include <vector>

#include "gh_internal.cuh"

namespace {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Position of element i of a column in shared memory: one float2 of padding
// after every 16, so that the strided stores of the early passes (runs of 4
// consecutive outputs every 16) fall into different banks.
__device__ __forceinline__ int p16(int i) { return i + (i >> 4); }

// Ping-pong Stockham FFT of `ncol` columns of length N = 2^logN, element i of
// column c at x[c * ld + p16(i)]: radix-4 passes, then one radix-2 pass when
// logN is odd. When only the first nz <= N/4 inputs are nonzero (zero padding
// by 4 or more), the first radix-4 pass reduces to replicating each input to
// its four outputs and the other inputs are neither stored nor read.
// tw[t] = exp(-j 2 pi t / N), t < 3N/4 (in shared memory). Returns the buffer
// holding the transform (x or y).
__device__ float2* fft_columns(float2* x, float2* y, int logN, int ncol, int ld, const float2* tw, int nz) {
    const int N = 1 << logN;
    int Ns = 1, rem = logN;
    while (rem >= 2) {
        const int lq = logN - 2, q4 = 1 << lq;
        const int total = ncol << lq;
        const int tstep = N / (4 * Ns);
        const bool replicate = Ns == 1 && nz <= q4;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx >> lq;
            const int j = idx & (q4 - 1);
            const int k = j & (Ns - 1);
            const float2* xc = x + c * ld;
            float2* yc = y + c * ld;
            const int o = ((j - k) << 2) + k;
            if (replicate) {
                const float2 v0 = j < nz ? xc[p16(j)] : make_float2(0.f, 0.f);
                yc[p16(o)] = v0;
                yc[p16(o + 1)] = v0;
                yc[p16(o + 2)] = v0;
                yc[p16(o + 3)] = v0;
                continue;
            }
            float2 v0 = xc[p16(j)], v1 = xc[p16(j + q4)], v2 = xc[p16(j + 2 * q4)], v3 = xc[p16(j + 3 * q4)];
            if (Ns > 1) {
                const int s = tstep * k;
                v1 = cmul(v1, tw[s]);
                v2 = cmul(v2, tw[2 * s]);
                v3 = cmul(v3, tw[3 * s]);
            }
            const float2 a = f2add(v0, v2), b = f2sub(v0, v2), cc = f2add(v1, v3);
            const float2 dd = f2sub(v1, v3);
            const float2 d = make_float2(dd.y, -dd.x);  // (v1 - v3) * (-j)
            yc[p16(o)] = f2add(a, cc);
            yc[p16(o + Ns)] = f2add(b, d);
            yc[p16(o + 2 * Ns)] = f2sub(a, cc);
            yc[p16(o + 3 * Ns)] = f2sub(b, d);
        }
        __syncthreads();
        float2* t = x;
        x = y;
        y = t;
        Ns <<= 2;
        rem -= 2;
    }
    if (rem == 1) {
        const int lh = logN - 1, half = 1 << lh;
        const int total = ncol << lh;
        const int tstep = N / (2 * Ns);
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx >> lh;
            const int j = idx & (half - 1);
            const int k = j & (Ns - 1);
            const float2* xc = x + c * ld;
            float2* yc = y + c * ld;
            float2 a, b;
            if (Ns == 1 && nz <= half) {  // N = 2: inputs beyond nz are zero
                a = j < nz ? xc[p16(j)] : make_float2(0.f, 0.f);
                b = make_float2(0.f, 0.f);
            } else {
                a = xc[p16(j)];
                b = cmul(xc[p16(j + half)], tw[tstep * k]);
            }
            const int o = ((j - k) << 1) + k;
            yc[p16(o)] = f2add(a, b);
            yc[p16(o + Ns)] = f2sub(a, b);
        }
        __syncthreads();
        float2* t = x;
        x = y;
        y = t;
    }
    return x;
}

__device__ void load_twiddles(float2* dst, const float2* __restrict__ src, int n) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = __ldg(src + t);
}

// Range FFTs of rows r0 .. r0 + nrow - 1 (row = q * Mc + mc) of one frame;
// shared memory: 2 * rows_alloc * gh_fft_ld(Nr) + 3 Nr / 4 float2.
__device__ __forceinline__ void range_rows(const float2* __restrict__ Y, float2* __restrict__ out, int Q, int Ms,
                                           int Mc, int logNr, int r0, int nrow, int rows_alloc, const Deflate& df,
                                           const float2* __restrict__ tw, float2* smem) {
    const int Nr = 1 << logNr;
    const int ld = gh_fft_ld(Nr);
    float2* x = smem;
    float2* y = smem + rows_alloc * ld;
    float2* twS = y + rows_alloc * ld;
    load_twiddles(twS, tw, 3 * Nr / 4);
    // only the Ms samples are stored when the first pass can skip the zero padding
    const int nstore = Ms <= Nr / 4 ? Ms : Nr;
    const int lst = Ms <= Nr / 4 ? 31 - __clz(Ms) : logNr;  // log2(nstore)
    for (int idx = threadIdx.x; idx < nrow * nstore; idx += blockDim.x) {
        const int c = idx >> lst;
        const int n = idx & (nstore - 1);
        float2 v = make_float2(0.f, 0.f);
        if (n < Ms) {
            const int row = r0 + c;  // q * Mc + mc
            v = Y[(size_t)row * Ms + n];
            if (df.n > 0) v = gh_deflate(df, Q, Ms, Mc, row / Mc, row % Mc, n, v);
        }
        x[c * ld + p16(n)] = v;
    }
    __syncthreads();
    float2* res = fft_columns(x, y, logNr, nrow, ld, twS, Ms);
    for (int idx = threadIdx.x; idx < nrow * Nr; idx += blockDim.x) {
        const int c = idx >> logNr, n = idx & (Nr - 1);
        out[(size_t)r0 * Nr + idx] = res[c * ld + p16(n)];
    }
}

__global__ void __launch_bounds__(256) range_fft_kernel(const float2* __restrict__ Y, float2* __restrict__ out,
                                                        int Q, int Ms, int Mc, int logNr, int rows,
                                                        int rows_per_cta, Deflate df,
                                                        const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int r0 = blockIdx.x * rows_per_cta;
    range_rows(Y, out, Q, Ms, Mc, logNr, r0, min(rows_per_cta, rows - r0), rows_per_cta, df, tw, smem);
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

// Doppler FFTs of range bins i0 .. i0 + IB - 1 of receiver q of one frame,
// times the range-centring factor, stored in type MT. Shared memory:
// 2 * IB * (gh_fft_ld(Nd) + 1) + IB + 3 Nd / 4 float2.
template <int MT>
__device__ __forceinline__ void doppler_cols(const float2* __restrict__ Zr, void* __restrict__ maps, int Ms, int Mc,
                                             int logNr, int logNd, int IB, int q, int i0,
                                             const float2* __restrict__ tw, float oscale, float2* smem) {
    const int Nr = 1 << logNr;
    const int Nd = 1 << logNd;
    const int ld = gh_fft_ld(Nd) + 1;  // odd column stride: the transposing loads spread over the banks
    float2* x = smem;
    float2* y = smem + IB * ld;
    float2* ramp = y + IB * ld;
    float2* twS = ramp + IB;
    load_twiddles(twS, tw, 3 * Nd / 4);
    const float2* src = Zr + (size_t)q * Mc * Nr + i0;
    for (int idx = threadIdx.x; idx < Mc * IB; idx += blockDim.x) {
        const int mc = idx / IB;
        const int c = idx - mc * IB;
        x[c * ld + p16(mc)] = src[(size_t)mc * Nr + c];
    }
    if (Mc > Nd / 4)  // the first pass reads the zero padding
        for (int idx = threadIdx.x; idx < (Nd - Mc) * IB; idx += blockDim.x) {
            const int c = idx / (Nd - Mc);
            const int n = Mc + (idx - c * (Nd - Mc));
            x[c * ld + p16(n)] = make_float2(0.f, 0.f);
        }
    if (threadIdx.x < IB) {
        // exp(j pi (i/Nr)(Ms-1)) with the angle reduced exactly modulo 2 pi
        const long long t = ((long long)(i0 + threadIdx.x) * (Ms - 1)) % (2LL * Nr);
        float s, c;
        sincospif((float)t / (float)Nr, &s, &c);
        ramp[threadIdx.x] = make_float2(c, s);
    }
    __syncthreads();
    float2* res = fft_columns(x, y, logNd, IB, ld, twS, Mc);
    const size_t dst = ((size_t)q * Nr + i0) * Nd;
    for (int idx = threadIdx.x; idx < IB * Nd; idx += blockDim.x) {
        const int c = idx >> logNd;
        const int j = idx & (Nd - 1);
        store_bin<MT>(maps, dst + idx, cmul(res[c * ld + p16(j)], ramp[c]), oscale);
    }
}

template <int MT>
__global__ void __launch_bounds__(256) doppler_fft_kernel(const float2* __restrict__ Zr, void* __restrict__ maps,
                                                          int Ms, int Mc, int logNr, int logNd, int IB,
                                                          const float2* __restrict__ tw, float oscale,
                                                          const int* __restrict__ rowlim, int Q) {
    extern __shared__ float2 smem[];
    const int i0 = blockIdx.x * IB;
    if (rowlim && (i0 + IB - 1 < rowlim[blockIdx.y] || i0 > rowlim[Q + blockIdx.y])) return;  // whole CTA
    doppler_cols<MT>(Zr, maps, Ms, Mc, logNr, logNd, IB, blockIdx.y, i0, tw, oscale, smem);
}

// Batched maps of several frames: one work item (frame, first row / range
// bin, count) per CTA; the residual of iteration k is applied on load.
__global__ void __launch_bounds__(256) range_fft_batch_kernel(const BatchFrame* __restrict__ frames,
                                                              const BatchItem* __restrict__ items, int k,
                                                              int rows_alloc) {
    extern __shared__ float2 smem[];
    const BatchItem it = items[blockIdx.x];
    const BatchFrame& F = frames[it.frame];
    Deflate df = F.df;
    df.n = k;
    int logNr = 0;
    while ((1 << logNr) < F.d.Nr) ++logNr;
    (void)rows_alloc;
    range_rows(F.Y, F.zr, F.d.Q, F.d.Ms, F.d.Mc, logNr, (int)it.start, (int)it.count, (int)it.count, df, F.twr,
               smem);
}

__global__ void __launch_bounds__(256) doppler_fft_batch_kernel(const BatchFrame* __restrict__ frames,
                                                                const BatchItem* __restrict__ items) {
    extern __shared__ float2 smem[];
    const BatchItem it = items[blockIdx.x];
    const BatchFrame& F = frames[it.frame];
    int logNr = 0, logNd = 0;
    while ((1 << logNr) < F.d.Nr) ++logNr;
    while ((1 << logNd) < F.d.Nd) ++logNd;
    doppler_cols<GH_C64>(F.zr, F.maps, F.d.Ms, F.d.Mc, logNr, logNd, (int)it.count, it.aux, (int)it.start, F.twd,
                         1.0f, smem);
}

}  // namespace

void gh_twiddles(int N, float2* out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < 3 * N / 4; ++t) {
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

// Uploads exp(-j 2 pi t / N), t < 3N/4, for N = Nr then N = Nd (float64 -> float32).
int ensure_twiddles(gh_ctx* ctx, int Nr, int Nd, const float2** twr, const float2** twd) {
    const int nr = 3 * Nr / 4, nd = 3 * Nd / 4;
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
    // rows of Nr points, as many rows per CTA as fit in ~32 KB
    const int logNr = ilog2(d.Nr);
    int rpc = 2048 / d.Nr;
    if (rpc < 1) rpc = 1;
    const int rows = d.Q * d.Mc;
    size_t smem1 = ((size_t)2 * rpc * gh_fft_ld(d.Nr) + 3 * d.Nr / 4) * sizeof(float2);
    GH_CUDA(cudaFuncSetAttribute(range_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
    range_fft_kernel<<<(rows + rpc - 1) / rpc, 256, smem1, ctx->stream>>>(Y, (float2*)zr, d.Q, d.Ms, d.Mc, logNr,
                                                                          rows, rpc, df ? *df : none, twr);
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
    int IB = 4096 / d.Nd;
    if (IB < 1) IB = 1;
    if (IB > 16) IB = 16;
    if (IB > d.Nr) IB = d.Nr;
    size_t smem2 = ((size_t)2 * IB * (gh_fft_ld(d.Nd) + 1) + IB + 3 * d.Nd / 4) * sizeof(float2);
    const float oscale = ldexpf(1.0f, -gh_map_scale_log2(d, map_dtype));
    auto kern = map_dtype == GH_C16 ? doppler_fft_kernel<GH_C16>
              : map_dtype == GH_CBF16 ? doppler_fft_kernel<GH_CBF16> : doppler_fft_kernel<GH_C64>;
    GH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    gh_launch_begin(ctx, GH_K_DOPPLER_FFT, &ev);
    kern<<<dim3(d.Nr / IB, d.Q), 256, smem2, ctx->stream>>>((const float2*)zr, maps, d.Ms, d.Mc, logNr, logNd, IB,
                                                            twd, oscale, rowlim, d.Q);
    return gh_launch_end(ctx, GH_K_DOPPLER_FFT, ev, "doppler_fft_kernel");
}

int gh_launch_maps_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* range_items, int n_range,
                         int rows_alloc, size_t smem_range, const BatchItem* dop_items, int n_dop, size_t smem_dop,
                         int k) {
    if (n_range > 0) {
        GH_CUDA(cudaFuncSetAttribute(range_fft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_range));
        cudaEvent_t ev;
        gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
        range_fft_batch_kernel<<<n_range, 256, smem_range, ctx->stream>>>(frames, range_items, k, rows_alloc);
        GH_TRY(gh_launch_end(ctx, GH_K_RANGE_FFT, ev, "range_fft_batch_kernel"));
    }
    if (n_dop > 0) {
        GH_CUDA(cudaFuncSetAttribute(doppler_fft_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_dop));
        cudaEvent_t ev;
        gh_launch_begin(ctx, GH_K_DOPPLER_FFT, &ev);
        doppler_fft_batch_kernel<<<n_dop, 256, smem_dop, ctx->stream>>>(frames, dop_items);
        GH_TRY(gh_launch_end(ctx, GH_K_DOPPLER_FFT, ev, "doppler_fft_batch_kernel"));
    }
    return GH_OK;
}
