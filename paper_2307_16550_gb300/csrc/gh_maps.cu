// Range-Doppler maps (Sec. III: the 2D FFT of each Y_q; Sec. IV: the FFT bins
// are correlations with the atoms on the FFT's frequency grid).
//
// Two kernels, both radix-2 Stockham FFTs in shared memory with float32 data
// and twiddles rounded from float64:
//   range_fft   : per (q, mc) row, the Ms samples zero-padded to Nr = pad*Ms,
//                 written [Q][Mc][Nr];
//   doppler_fft : per (q, block of IB range bins), the Mc chirps zero-padded to
//                 Nd = pad*Mc, times the range-centring factor
//                 exp(j pi (i/Nr)(Ms-1)), written [Q][Nr][Nd] so that one
//                 range bin's Doppler row is contiguous for the scorer.
#include <math.h>

#include <vector>

#include "gh_internal.cuh"

namespace {

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// In-place (ping-pong) radix-2 Stockham FFT of `ncol` columns of length
// N = 2^logN stored at x + c*ld. tw[t] = exp(-j 2 pi t / N), t < N/2.
// Returns the buffer holding the transform (x or y).
__device__ float2* fft_columns(float2* x, float2* y, int logN, int ncol, int ld, const float2* __restrict__ tw) {
    const int half = 1 << (logN - 1);
    const int total = ncol << (logN - 1);
    for (int s = 0; s < logN; ++s) {
        const int Ns = 1 << s;
        const int twshift = logN - 1 - s;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int c = idx >> (logN - 1);
            const int j = idx & (half - 1);
            const int k = j & (Ns - 1);
            const float2* xc = x + c * ld;
            float2* yc = y + c * ld;
            float2 a = xc[j];
            float2 b = cmul(xc[j + half], __ldg(&tw[k << twshift]));
            const int o = ((j - k) << 1) + k;
            yc[o] = f2add(a, b);
            yc[o + Ns] = f2sub(a, b);
        }
        __syncthreads();
        float2* t = x;
        x = y;
        y = t;
    }
    return x;
}

__global__ void __launch_bounds__(256) range_fft_kernel(const float2* __restrict__ Y, float2* __restrict__ out,
                                                        int Ms, int logNr, int rows, int rows_per_cta,
                                                        const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int Nr = 1 << logNr;
    const int r0 = blockIdx.x * rows_per_cta;
    const int nrow = min(rows_per_cta, rows - r0);
    float2* x = smem;
    float2* y = smem + rows_per_cta * Nr;
    for (int idx = threadIdx.x; idx < nrow * Nr; idx += blockDim.x) {
        const int c = idx >> logNr;
        const int n = idx & (Nr - 1);
        x[idx] = n < Ms ? Y[(size_t)(r0 + c) * Ms + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_columns(x, y, logNr, nrow, Nr, tw);
    for (int idx = threadIdx.x; idx < nrow * Nr; idx += blockDim.x) out[(size_t)r0 * Nr + idx] = res[idx];
}

__global__ void __launch_bounds__(256) doppler_fft_kernel(const float2* __restrict__ Zr, float2* __restrict__ maps,
                                                          int Ms, int Mc, int logNr, int logNd, int IB,
                                                          const float2* __restrict__ tw) {
    extern __shared__ float2 smem[];
    const int Nr = 1 << logNr;
    const int Nd = 1 << logNd;
    const int ld = Nd + 1;
    const int q = blockIdx.y;
    const int i0 = blockIdx.x * IB;
    float2* x = smem;
    float2* y = smem + IB * ld;
    float2* ramp = y + IB * ld;
    const float2* src = Zr + (size_t)q * Mc * Nr + i0;
    for (int idx = threadIdx.x; idx < Mc * IB; idx += blockDim.x) {
        const int mc = idx / IB;
        const int c = idx - mc * IB;
        x[c * ld + mc] = src[(size_t)mc * Nr + c];
    }
    for (int idx = threadIdx.x; idx < (Nd - Mc) * IB; idx += blockDim.x) {
        const int c = idx / (Nd - Mc);
        const int n = Mc + (idx - c * (Nd - Mc));
        x[c * ld + n] = make_float2(0.f, 0.f);
    }
    if (threadIdx.x < IB) {
        // exp(j pi (i/Nr)(Ms-1)) with the angle reduced exactly modulo 2 pi
        const long long t = ((long long)(i0 + threadIdx.x) * (Ms - 1)) % (2LL * Nr);
        float s, c;
        sincospif((float)t / (float)Nr, &s, &c);
        ramp[threadIdx.x] = make_float2(c, s);
    }
    __syncthreads();
    float2* res = fft_columns(x, y, logNd, IB, ld, tw);
    float2* dst = maps + ((size_t)q * Nr + i0) * Nd;
    for (int idx = threadIdx.x; idx < IB * Nd; idx += blockDim.x) {
        const int c = idx >> logNd;
        const int j = idx & (Nd - 1);
        dst[idx] = cmul(res[c * ld + j], ramp[c]);
    }
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// Uploads exp(-j 2 pi t / N), t < N/2, for N = Nr then N = Nd (float64 -> float32).
int ensure_twiddles(gh_ctx* ctx, int Nr, int Nd, const float2** twr, const float2** twd) {
    size_t bytes = (size_t)(Nr / 2 + Nd / 2) * sizeof(float2);
    void* p;
    GH_TRY(gh_ws(ctx, WS_TWIDDLE, bytes, &p));
    if (ctx->tw_n[0] != Nr || ctx->tw_n[1] != Nd) {
        std::vector<float2> h(Nr / 2 + Nd / 2);
        const double two_pi = 6.283185307179586476925286766559;
        for (int t = 0; t < Nr / 2; ++t) {
            double a = -two_pi * (double)t / (double)Nr;
            h[t] = make_float2((float)cos(a), (float)sin(a));
        }
        for (int t = 0; t < Nd / 2; ++t) {
            double a = -two_pi * (double)t / (double)Nd;
            h[Nr / 2 + t] = make_float2((float)cos(a), (float)sin(a));
        }
        GH_CUDA(cudaMemcpyAsync(p, h.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
        ctx->tw_n[0] = Nr;
        ctx->tw_n[1] = Nd;
    }
    *twr = (const float2*)p;
    *twd = (const float2*)p + Nr / 2;
    return GH_OK;
}

}  // namespace

int gh_launch_maps(gh_ctx* ctx, const Dims& d, const float2* Y, float2* maps) {
    const float2 *twr, *twd;
    GH_TRY(ensure_twiddles(ctx, d.Nr, d.Nd, &twr, &twd));
    void* zr;
    GH_TRY(gh_ws(ctx, WS_RANGE, (size_t)d.Q * d.Mc * d.Nr * sizeof(float2), &zr));

    // range FFT: rows of Nr points, as many rows per CTA as fit in ~32 KB
    const int logNr = ilog2(d.Nr), logNd = ilog2(d.Nd);
    int rpc = 2048 / d.Nr;
    if (rpc < 1) rpc = 1;
    const int rows = d.Q * d.Mc;
    size_t smem1 = (size_t)2 * rpc * d.Nr * sizeof(float2);
    GH_CUDA(cudaFuncSetAttribute(range_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_RANGE_FFT, &ev);
    range_fft_kernel<<<(rows + rpc - 1) / rpc, 256, smem1, ctx->stream>>>(Y, (float2*)zr, d.Ms, logNr, rows, rpc,
                                                                          twr);
    GH_TRY(gh_launch_end(ctx, GH_K_RANGE_FFT, ev, "range_fft_kernel"));

    // Doppler FFT: IB range bins per CTA
    int IB = 4096 / d.Nd;
    if (IB < 1) IB = 1;
    if (IB > 16) IB = 16;
    if (IB > d.Nr) IB = d.Nr;
    size_t smem2 = ((size_t)2 * IB * (d.Nd + 1) + IB) * sizeof(float2);
    GH_CUDA(cudaFuncSetAttribute(doppler_fft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    gh_launch_begin(ctx, GH_K_DOPPLER_FFT, &ev);
    doppler_fft_kernel<<<dim3(d.Nr / IB, d.Q), 256, smem2, ctx->stream>>>((const float2*)zr, maps, d.Ms, d.Mc,
                                                                          logNr, logNd, IB, twd);
    return gh_launch_end(ctx, GH_K_DOPPLER_FFT, ev, "doppler_fft_kernel");
}
