// Block orthogonal matching pursuit (BOMP, the paper's acronym list; several
// targets by iterative direct detection, Sec. VI) and the measurement
// synthesiser of the signal model (Sec. II).
//
// One BOMP iteration k, after the scorer has written the selected cell to
// sel[k] on the device (no host round trip):
//   bomp_atoms    : (r, u) of the selected cell at every receiver (float64) and
//                   its atoms a(r) (Ms) and b(u) (Mc), phases reduced exactly;
//   bomp_corr     : c_{k,q} = <Y_q, b(u) (x) a(r)>, float32 row sums added in float64;
//   bomp_solve    : per receiver, the normal equations of all k+1 selected
//                   atoms, in float64. With centred atoms (phase
//                   exp(-j pi (r (Ms-1) + u (Mc-1)))) the Gram matrix is real,
//                   G[s][t] = D_Ms(r_t - r_s) D_Mc(u_t - u_s),
//                   D_M(f) = sin(pi M f) / sin(pi f); Cholesky solve, then the
//                   amplitudes are rotated back to the atoms of Sec. II;
//   bomp_residual : R_q = Y_q - sum_t alpha_{t,q} b(u_t) (x) a(r_t).
#include <math.h>

#include "gh_internal.cuh"

namespace {

constexpr int kCorrRows = 8;  // chirps per correlation CTA (one per warp)

struct BompLayout {
    size_t alpha, corr, ru, phase, gram, corrp, atoms_a, atoms_b, total;
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
    L.total = o;
    return L;
}

__device__ double dirichlet(double f, int M) {
    const double s = sinpi(f);
    if (fabs(s) < 1e-13) {
        // f is (numerically) an integer n: D_M(n) = M (-1)^(n (M - 1))
        const double n = rint(f);
        return M * cospi(n * (double)(M - 1));
    }
    return sinpi((double)M * f) / s;
}

// One CTA per receiver: (r, u) of the cell selected in iteration k, its
// centring phase, row k of the real Gram matrix, and the atoms a(r), b(u).
__global__ void bomp_atoms_kernel(GeoParams g, const ArgResult* __restrict__ sel, int k, int K,
                                  double2* __restrict__ ru, double2* __restrict__ phase, double* __restrict__ gram,
                                  float2* __restrict__ atoms_a, float2* __restrict__ atoms_b) {
    const int q = blockIdx.x;
    __shared__ unsigned long long s_rf, s_uf;
    __shared__ double s_r, s_u;
    if (threadIdx.x == 0) {
        long long cell = sel[k].cell;
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
        ru[(size_t)k * g.Q + q] = make_double2(r, u);
        double sn, cs;
        sincospi(r * (g.Ms - 1) + u * (g.Mc - 1), &sn, &cs);
        phase[(size_t)k * g.Q + q] = make_double2(cs, sn);
        s_r = r;
        s_u = u;
        s_rf = gh_phase_fix(r);
        s_uf = gh_phase_fix(u);
    }
    __syncthreads();
    if (threadIdx.x <= k) {
        const int t = threadIdx.x;
        const double2 rut = t == k ? make_double2(s_r, s_u) : ru[(size_t)t * g.Q + q];
        const double v = dirichlet(s_r - rut.x, g.Ms) * dirichlet(s_u - rut.y, g.Mc);
        double* G = gram + (size_t)q * K * K;
        G[k * K + t] = v;
        G[t * K + k] = v;
    }
    float2* a = atoms_a + ((size_t)k * g.Q + q) * g.Ms;
    float2* b = atoms_b + ((size_t)k * g.Q + q) * g.Mc;
    for (int m = threadIdx.x; m < g.Ms; m += blockDim.x) a[m] = gh_cis_fix(s_rf * (unsigned long long)m);
    for (int m = threadIdx.x; m < g.Mc; m += blockDim.x) b[m] = gh_cis_fix(s_uf * (unsigned long long)m);
}

// CTA (chunk, q): partial <Y_q, b(u) (x) a(r)> over kCorrRows chirps; each warp
// sums one chirp in float32 and the chirps are added in float64.
__global__ void __launch_bounds__(256) bomp_corr_kernel(const float2* __restrict__ Y, GeoParams g, int k, int chunks,
                                                        const float2* __restrict__ atoms_a,
                                                        const float2* __restrict__ atoms_b,
                                                        double2* __restrict__ corrp) {
    const int ch = blockIdx.x, q = blockIdx.y;
    const float2* a = atoms_a + ((size_t)k * g.Q + q) * g.Ms;
    const float2* b = atoms_b + ((size_t)k * g.Q + q) * g.Mc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mc = ch * kCorrRows + warp;
    __shared__ double rx[kCorrRows], ry[kCorrRows];
    double sx = 0.0, sy = 0.0;
    if (warp < kCorrRows && mc < g.Mc) {
        const float2* row = Y + ((size_t)q * g.Mc + mc) * g.Ms;
        float2 s = make_float2(0.f, 0.f);
        for (int m = lane; m < g.Ms; m += 32) {
            const float2 y = row[m];
            const float2 w = a[m];
            s.x += y.x * w.x + y.y * w.y;  // y * conj(a)
            s.y += y.y * w.x - y.x * w.y;
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
    if (threadIdx.x == 0) {
        double tx = 0, ty = 0;
        for (int w = 0; w < kCorrRows; ++w) {
            tx += rx[w];
            ty += ry[w];
        }
        corrp[((size_t)k * g.Q + q) * chunks + ch] = make_double2(tx, ty);
    }
}

// One thread per receiver: sums the correlation partials of atom k, then
// solves the normal equations of atoms 0..k with the stored Gram matrix
// (Cholesky, dependent atoms dropped) and rotates the amplitudes back to the
// atoms of the signal model. Float64 arithmetic only.
__global__ void bomp_solve_kernel(int Q, int Ms, int Mc, int k, int K, int chunks,
                                  const double2* __restrict__ corrp, double2* __restrict__ corr,
                                  const double2* __restrict__ phase, const double* __restrict__ gram,
                                  double2* __restrict__ alpha) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const int n = k + 1;
    {
        double cx = 0.0, cy = 0.0;
        const double2* pp = corrp + ((size_t)k * Q + q) * chunks;
        for (int c = 0; c < chunks; ++c) {
            cx += pp[c].x;
            cy += pp[c].y;
        }
        corr[(size_t)k * Q + q] = make_double2(cx, cy);
    }
    double L[GH_MAX_K][GH_MAX_K];
    double zr[GH_MAX_K], zi[GH_MAX_K];
    bool dep[GH_MAX_K];
    for (int t = 0; t < n; ++t) {
        const double2 ph = phase[(size_t)t * Q + q];
        const double2 ct = corr[(size_t)t * Q + q];
        zr[t] = ph.x * ct.x - ph.y * ct.y;  // exp(+j pi ph) <Y, atom>
        zi[t] = ph.x * ct.y + ph.y * ct.x;
    }
    const double* G = gram + (size_t)q * K * K;
    const double floor_v = 1e-9 * (double)Ms * (double)Mc;
    for (int j = 0; j < n; ++j) {
        for (int i = j; i < n; ++i) {
            double v = G[i * K + j];
            for (int t = 0; t < j; ++t) v -= L[i][t] * L[j][t];
            if (i == j) {
                dep[j] = !(v > floor_v);
                L[j][j] = dep[j] ? 0.0 : sqrt(v);
            } else {
                L[i][j] = dep[j] ? 0.0 : v / L[j][j];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        if (dep[i]) {
            zr[i] = zi[i] = 0.0;
            continue;
        }
        for (int t = 0; t < i; ++t) {
            zr[i] -= L[i][t] * zr[t];
            zi[i] -= L[i][t] * zi[t];
        }
        zr[i] /= L[i][i];
        zi[i] /= L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        if (dep[i]) {
            zr[i] = zi[i] = 0.0;
            continue;
        }
        for (int t = i + 1; t < n; ++t) {
            zr[i] -= L[t][i] * zr[t];
            zi[i] -= L[t][i] * zi[t];
        }
        zr[i] /= L[i][i];
        zi[i] /= L[i][i];
    }
    for (int t = 0; t < n; ++t) {
        const double2 ph = phase[(size_t)t * Q + q];  // alpha = alpha~ exp(-j pi ph)
        alpha[(size_t)t * Q + q] = make_double2(ph.x * zr[t] + ph.y * zi[t], ph.x * zi[t] - ph.y * zr[t]);
    }
}

__global__ void __launch_bounds__(256) bomp_residual_kernel(const float2* __restrict__ Y, GeoParams g, int n,
                                                            const double2* __restrict__ alpha,
                                                            const float2* __restrict__ atoms_a,
                                                            const float2* __restrict__ atoms_b,
                                                            float2* __restrict__ R) {
    const size_t per_q = (size_t)g.Mc * g.Ms;
    const size_t total = per_q * g.Q;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(idx / per_q);
        const size_t e = idx - (size_t)q * per_q;
        const int mc = (int)(e / g.Ms), m = (int)(e - (size_t)mc * g.Ms);
        float2 v = Y[idx];
        for (int t = 0; t < n; ++t) {
            const double2 al = alpha[(size_t)t * g.Q + q];
            const float2 ab = cmul(atoms_b[((size_t)t * g.Q + q) * g.Mc + mc], atoms_a[((size_t)t * g.Q + q) * g.Ms + m]);
            const float2 c = cmul(make_float2((float)al.x, (float)al.y), ab);
            v.x -= c.x;
            v.y -= c.y;
        }
        R[idx] = v;
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

int gh_launch_bomp_iter(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, float2* R, int k, int K,
                        const ArgResult* sel, void* ws) {
    const BompLayout L = bomp_layout(d, K);
    char* base = (char*)ws;
    double2* alpha = (double2*)(base + L.alpha);
    double2* corr = (double2*)(base + L.corr);
    double2* ru = (double2*)(base + L.ru);
    double2* phase = (double2*)(base + L.phase);
    double* gram = (double*)(base + L.gram);
    double2* corrp = (double2*)(base + L.corrp);
    float2* aa = (float2*)(base + L.atoms_a);
    float2* ab = (float2*)(base + L.atoms_b);
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_atoms_kernel<<<d.Q, 256, 0, ctx->stream>>>(g, sel, k, K, ru, phase, gram, aa, ab);
    GH_TRY(gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_atoms_kernel"));
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_corr_kernel<<<dim3(L.chunks, d.Q), 32 * kCorrRows, 0, ctx->stream>>>(Y, g, k, L.chunks, aa, ab, corrp);
    GH_TRY(gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_corr_kernel"));
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_solve_kernel<<<(d.Q + 31) / 32, 32, 0, ctx->stream>>>(d.Q, d.Ms, d.Mc, k, K, L.chunks, corrp, corr, phase,
                                                              gram, alpha);
    GH_TRY(gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_solve_kernel"));
    const size_t total = (size_t)d.Q * d.Mc * d.Ms;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (blocks > (unsigned)ctx->num_sms * 8) blocks = (unsigned)ctx->num_sms * 8;
    gh_launch_begin(ctx, GH_K_BOMP, &ev);
    bomp_residual_kernel<<<blocks, 256, 0, ctx->stream>>>(Y, g, k + 1, alpha, aa, ab, R);
    return gh_launch_end(ctx, GH_K_BOMP, ev, "bomp_residual_kernel");
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
