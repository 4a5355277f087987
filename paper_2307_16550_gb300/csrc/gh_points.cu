// Differentiable hopping score at continuous points, its adjoint, and an
// on-device gradient-ascent refinement (off-grid estimates; Sec. VI names
// refined estimation as future work).
//
// The score of a point (x, y, vx, vy) interpolates both map axes with the
// three-bin polar model of Sec. IV: the range coefficients c_k(tau) as in the
// grid scorer, and, because the nearest Doppler bin of the grid scorer makes
// the score piecewise constant in v, the same construction on the Doppler axis
// with centred Doppler atoms (coefficients d_l(sigma), half-angle from Mc, Nd):
//   s_q = sum_{k,l} c_k(tau_q) d_l(sigma_q) V_q(i_q + k, j_q + l),  S = sum_q |s_q|^2,
//   V_q(n, m) = maps[q][n mod Nr][m mod Nd] (-1)^((Ms-1) floor(n/Nr)) exp(j pi m (Mc-1)/Nd)
// with rho = Nr r_q, i = floor(rho + 1/2), tau = rho - i, eta = Nd u_q,
// j = floor(eta + 1/2), sigma = eta - j, all in float64 (Eq. 1; each
// distance and its reciprocal from one reciprocal square root, so bin choices
// may differ from a square-root-and-division evaluation within a few ulps of a
// bin edge, where the score is continuous to the interpolation error);
// derivatives in float32.
//
// Adjoint (i, j fixed between bin switches): dS/drho_q = 2 Re(conj(s) sum c_k' d_l V),
// dS/deta_q = 2 Re(conj(s) sum c_k d_l' V), chained through
//   drho/dx = Nr B/(c Ms) w_q,   drho/drx_q = -Nr B/(c Ms) u_rx,
//   deta/dv = Nd kappa w_q,      deta/dx = Nd kappa (J_tx + J_rx) v,   deta/drx_q = -Nd kappa J_rx v,
// J_p = (I - u_p u_p^T)/|x - p|; and into the maps as d|s|^2/d(bin) = 2 s conj(weight).
//
// One warp per point, lanes over receivers, warp-shuffle sums over q.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "gh_internal.cuh"

namespace {

struct PtParams {
    double tx0, tx1;
    double B, cMs, kappa;
    double gr, ge;     // Nr B / (c Ms) and Nd kappa
    float grf, gef;    // the same in float32 (derivative factors)
    int Q, Ms, Mc, Nr, Nd;
    int lgNr;          // log2 of Nr (a power of two, as Nd)
    float thr, thd;    // polar half-angles (range, Doppler)
    float mscale;      // 2^s of reduced-precision maps
};

struct Coef {
    float c[3], dc[3];
};

// Polar coefficients (c_{-1}, c_0, c_{+1}) at offset t and their derivatives.
__device__ __forceinline__ Coef polar(float theta, float t) {
    float sh, ch, sf, cf;
    sincosf(0.5f * theta * t, &sh, &ch);
    sincosf(theta * t, &sf, &cf);
    float s2, c2, st, ct;
    sincosf(0.5f * theta, &s2, &c2);
    sincosf(theta, &st, &ct);
    const float inv_h = 1.0f / (s2 * s2);  // 1 / sin^2(theta/2) = 2 / (1 - cos theta)
    const float kap = sh * sh * inv_h;
    const float sig = sf / st;
    const float dkap = 0.5f * theta * sf * inv_h;
    const float dsig = theta * cf / st;
    Coef r;
    r.c[0] = 0.5f * (kap - sig);
    r.c[1] = 1.0f - kap;
    r.c[2] = 0.5f * (kap + sig);
    r.dc[0] = 0.5f * (dkap - dsig);
    r.dc[1] = -dkap;
    r.dc[2] = 0.5f * (dkap + dsig);
    return r;
}

template <int MT>
__device__ __forceinline__ float2 load_bin(const void* maps, size_t idx) {
    if constexpr (MT == GH_C64) {
        return __ldg((const float2*)maps + idx);
    } else if constexpr (MT == GH_C16) {
        const unsigned w = __ldg((const unsigned*)maps + idx);
        return __half22float2(*reinterpret_cast<const __half2*>(&w));
    } else {
        const unsigned w = __ldg((const unsigned*)maps + idx);
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    }
}

// Geometry of one (point, receiver) in float64 and its stencil.
struct PtGeo {
    float ux1, uy1, r1, ux2, uy2, r2, wx, wy;  // unit vectors, 1/|x - p| (0 on p), gradient w (for derivatives)
    long long i, j;
    float tau, sig;
};

// Unit vector from p to x, |x - p| and 1/|x - p| in float64 from one
// reciprocal square root (zero below 1e-9 m, as Eq. 1's gradient of a point
// on p).
__device__ __forceinline__ void unit_recip(double dx, double dy, double* n, double* ux, double* uy, double* r) {
    const double d2 = dx * dx + dy * dy;
    if (d2 < 1e-18) {
        *n = sqrt(d2);
        *r = 0.0;
    } else {
        *r = rsqrt(d2);
        *n = d2 * *r;
    }
    *ux = dx * *r;
    *uy = dy * *r;
}

// Range and Doppler positions of a point at one receiver in float64 (bins
// and offsets: rho = Nr B d / (c Ms), eta = Nd kappa <w, v>); derivative
// factors in float32.
__device__ __forceinline__ PtGeo pt_geo(const PtParams& p, double x, double y, double vx, double vy, double rxx,
                                        double rxy) {
    double n1, ux1, uy1, r1, n2, ux2, uy2, r2;
    unit_recip(x - p.tx0, y - p.tx1, &n1, &ux1, &uy1, &r1);
    unit_recip(x - rxx, y - rxy, &n2, &ux2, &uy2, &r2);
    const double wx = ux1 + ux2, wy = uy1 + uy2;
    const double rho = p.gr * (n1 + n2);
    const double eta = p.ge * (wx * vx + wy * vy);
    const double fi = floor(rho + 0.5), fj = floor(eta + 0.5);
    PtGeo g;
    g.ux1 = (float)ux1;
    g.uy1 = (float)uy1;
    g.r1 = (float)r1;
    g.ux2 = (float)ux2;
    g.uy2 = (float)uy2;
    g.r2 = (float)r2;
    g.wx = (float)wx;
    g.wy = (float)wy;
    g.i = (long long)fi;
    g.j = (long long)fj;
    g.tau = (float)(rho - fi);
    g.sig = (float)(eta - fj);
    return g;
}


// Stencil values V(i+k, j+l) of receiver q (range sign and Doppler centring applied).
template <int MT>
__device__ __forceinline__ void stencil(const void* maps, const PtParams& p, int q, long long i, long long j,
                                        float2 V[3][3], size_t idx[3][3], float2 wph[3][3]) {
    float2 ph[3];
    long long mm[3];
    for (int l = 0; l < 3; ++l) {
        const long long m = j + (l - 1);
        mm[l] = m & (long long)(p.Nd - 1);  // m mod Nd (Nd a power of two)
        // exp(j pi m (Mc-1)/Nd), angle reduced exactly modulo 2 pi
        const long long t2 = 2LL * p.Nd - 1;
        const long long t = ((m & t2) * (long long)(p.Mc - 1)) & t2;
        float s, c;
        sincospif((float)t / (float)p.Nd, &s, &c);
        ph[l] = make_float2(c, s);
    }
    for (int k = 0; k < 3; ++k) {
        const long long n = i + (k - 1);
        const long long w = n >> p.lgNr;  // floor(n / Nr)
        const long long nr = n & (long long)(p.Nr - 1);
        const float sg = (((p.Ms - 1) & 1) && (w & 1)) ? -p.mscale : p.mscale;
        for (int l = 0; l < 3; ++l) {
            idx[k][l] = ((size_t)q * p.Nr + (size_t)nr) * p.Nd + (size_t)mm[l];
            wph[k][l] = make_float2(sg * ph[l].x, sg * ph[l].y);
            V[k][l] = cmul(load_bin<MT>(maps, idx[k][l]), wph[k][l]);
        }
    }
}

__device__ __forceinline__ float2 contract(const float* a, const float* b, float2 V[3][3]) {
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
            const float w = a[k] * b[l];
            s.x += w * V[k][l].x;
            s.y += w * V[k][l].y;
        }
    return s;
}

// Sum over a group of G lanes (G a power of two <= 32; butterfly, so every
// lane of the group gets the same bits). All 32 lanes must call it.
__device__ __forceinline__ double group_sum(double v, int G) {
    for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// S of one point, evaluated by a group of G lanes (receivers strided over the
// group); every lane of the group returns the sum over receivers.
template <int MT>
__device__ double point_score(const void* maps, const PtParams& p, const double* __restrict__ rx, double x, double y,
                              double vx, double vy, int G) {
    const int sub = threadIdx.x & (G - 1);
    double acc = 0.0;
    for (int q = sub; q < p.Q; q += G) {
        const PtGeo g = pt_geo(p, x, y, vx, vy, rx[2 * q], rx[2 * q + 1]);
        const Coef cr = polar(p.thr, g.tau), cd = polar(p.thd, g.sig);
        float2 V[3][3], wph[3][3];
        size_t idx[3][3];
        stencil<MT>(maps, p, q, g.i, g.j, V, idx, wph);
        const float2 s = contract(cr.c, cd.c, V);
        acc += (double)(s.x * s.x + s.y * s.y);
    }
    return group_sum(acc, G);
}

// Gradient of S of one point (group of G lanes as point_score): dS/d(x, y, vx, vy)
// summed over receivers (every lane of the group returns it); per-receiver RX
// gradients and map gradients, scaled by gs, are accumulated when drx / dmaps
// are non-NULL and `live` is set.
template <int MT>
__device__ double point_grad(const void* maps, const PtParams& p, const double* __restrict__ rx, double x, double y,
                             double vx, double vy, float gs, double* __restrict__ drx, float2* __restrict__ dmaps,
                             double grad[4], int G, bool live = true) {
    const int sub = threadIdx.x & (G - 1);
    double acc = 0.0;
    float gx = 0.f, gy = 0.f, gvx = 0.f, gvy = 0.f;
    // receiver gradient of this lane's receiver (Q <= G: at most one per
    // lane), summed over the warp's point groups before the atomics
    const bool one_rx = p.Q <= G;
    float rgx = 0.f, rgy = 0.f;
    for (int q = sub; q < p.Q; q += G) {
        const PtGeo g = pt_geo(p, x, y, vx, vy, rx[2 * q], rx[2 * q + 1]);
        const Coef cr = polar(p.thr, g.tau), cd = polar(p.thd, g.sig);
        float2 V[3][3], wph[3][3];
        size_t idx[3][3];
        stencil<MT>(maps, p, q, g.i, g.j, V, idx, wph);
        const float2 s = contract(cr.c, cd.c, V);
        const float2 ar = contract(cr.dc, cd.c, V);
        const float2 ae = contract(cr.c, cd.dc, V);
        acc += (double)(s.x * s.x + s.y * s.y);
        const float dSr = 2.0f * (s.x * ar.x + s.y * ar.y);  // 2 Re(conj(s) ar)
        const float dSe = 2.0f * (s.x * ae.x + s.y * ae.y);
        // J_p v = (v - u (u.v)) / |x - p| (zero for a point on p: r = 0)
        const float fvx = (float)vx, fvy = (float)vy;
        const float uv1 = g.ux1 * fvx + g.uy1 * fvy, uv2 = g.ux2 * fvx + g.uy2 * fvy;
        const float j1x = (fvx - g.ux1 * uv1) * g.r1, j1y = (fvy - g.uy1 * uv1) * g.r1;
        const float j2x = (fvx - g.ux2 * uv2) * g.r2, j2y = (fvy - g.uy2 * uv2) * g.r2;
        const float fr = dSr * p.grf, fe = dSe * p.gef;
        gx += fr * g.wx + fe * (j1x + j2x);
        gy += fr * g.wy + fe * (j1y + j2y);
        gvx += fe * g.wx;
        gvy += fe * g.wy;
        if (drx && live) {
            if (one_rx) {
                rgx = gs * (-fr * g.ux2 - fe * j2x);
                rgy = gs * (-fr * g.uy2 - fe * j2y);
            } else {
                atomicAdd(&drx[2 * q], (double)(gs * (-fr * g.ux2 - fe * j2x)));
                atomicAdd(&drx[2 * q + 1], (double)(gs * (-fr * g.uy2 - fe * j2y)));
            }
        }
        if (dmaps && live) {
            // d|s|^2 / d(stored bin) = 2 s conj(c_k d_l wph) (stored bins are 2^-s times the values)
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    const float w = 2.0f * gs * cr.c[k] * cd.c[l];
                    const float2 t = cmulc(s, wph[k][l]);  // s conj(wph)
                    atomicAdd(&dmaps[idx[k][l]].x, w * t.x);
                    atomicAdd(&dmaps[idx[k][l]].y, w * t.y);
                }
        }
    }
    if (drx && one_rx) {  // every lane takes part (drx is the same for the whole warp)
        double sx = rgx, sy = rgy;
        for (int o = G; o < 32; o <<= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if ((threadIdx.x & 31) < G && sub < p.Q) {
            atomicAdd(&drx[2 * sub], sx);
            atomicAdd(&drx[2 * sub + 1], sy);
        }
    }
    grad[0] = group_sum((double)gx, G);
    grad[1] = group_sum((double)gy, G);
    grad[2] = group_sum((double)gvx, G);
    grad[3] = group_sum((double)gvy, G);
    return group_sum(acc, G);
}

// One group of G lanes per point (G = the power of two >= Q, at most 32).
// Groups past the last point evaluate the last point and write nothing, so
// that every lane takes part in the shuffles.
template <int MT>
__global__ void __launch_bounds__(128) points_fwd_kernel(const void* __restrict__ maps, PtParams p,
                                                        const double* __restrict__ rx,
                                                        const double* __restrict__ pts, long long P, int G,
                                                        float* __restrict__ S) {
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if ((gid - (threadIdx.x & 31) / G) >= P) return;  // the warp's first point is past the end: whole warp leaves
    const long long pt = gid < P ? gid : P - 1;
    const double* a = pts + 4 * pt;
    const double v = point_score<MT>(maps, p, rx, a[0], a[1], a[2], a[3], G);
    if ((threadIdx.x & (G - 1)) == 0 && gid < P) S[pt] = (float)v;
}

// Receiver gradients are summed per CTA in shared memory first (one global
// atomic per receiver coordinate and CTA instead of one per point).
template <int MT>
__global__ void __launch_bounds__(128) points_adj_kernel(const void* __restrict__ maps, PtParams p,
                                                        const double* __restrict__ rx,
                                                        const double* __restrict__ pts, long long P, int G,
                                                        const float* __restrict__ gS, double* __restrict__ dpts,
                                                        double* __restrict__ drx, float2* __restrict__ dmaps) {
    __shared__ double sdrx[2 * GH_MAX_Q];
    for (int i = threadIdx.x; i < 2 * p.Q; i += blockDim.x) sdrx[i] = 0.0;
    __syncthreads();
    const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if ((gid - (threadIdx.x & 31) / G) < P) {  // warp-uniform
        const bool live = gid < P;
        const long long pt = live ? gid : P - 1;
        const double* a = pts + 4 * pt;
        const float gs = gS[pt];
        double grad[4];
        point_grad<MT>(maps, p, rx, a[0], a[1], a[2], a[3], gs, drx ? sdrx : nullptr, dmaps, grad, G, live);
        if (dpts && live && (threadIdx.x & (G - 1)) == 0)
            for (int c = 0; c < 4; ++c) dpts[4 * pt + c] = (double)gs * grad[c];
    }
    __syncthreads();
    if (drx)
        for (int i = threadIdx.x; i < 2 * p.Q; i += blockDim.x) atomicAdd(&drx[i], sdrx[i]);
}

// Solves A x = b for a symmetric 4 x 4 A by Cholesky; false if A is not
// positive definite.
__device__ __forceinline__ bool chol4_solve(double A[4][4], const double b[4], double x[4]) {
    double L[4][4] = {{0}};
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    double y[4];
    for (int i = 0; i < 4; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = 3; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 4; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return true;
}

// Damped Newton (Levenberg-Marquardt) ascent of every point for at most
// `iters` iterations. The Hessian comes from central differences of the
// analytic gradient (steps 1e-3 of the per-axis scales sc); a step solves
// (-H + lambda diag(1/sc^2)) d = g (Cholesky); if it increases S the step is
// taken and lambda shrinks by 3, otherwise lambda grows by 4 (at most 40
// trials). The first lambda makes the step about `step` scale units long.
// One warp per point, split into 32/G groups of G lanes (G = the power of two
// >= Q, at most 32; a group evaluates one point, receivers over its lanes).
// The groups evaluate the 8 displaced gradients of the Hessian side by side,
// and consecutive damping trials lambda, 4 lambda, 16 lambda, ... side by side
// (the first improving one in that order is taken, as a sequential search
// would). Every lane ends each stage with the same values, so control flow
// stays warp-uniform.
template <int MT>
__global__ void __launch_bounds__(128) refine_kernel(const void* __restrict__ maps, PtParams p,
                                                    const double* __restrict__ rx, double* __restrict__ pts,
                                                    long long P, int iters, double sx, double sv, double step,
                                                    float* __restrict__ S, int G) {
    const long long pt = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (pt >= P) return;
    const int lane = threadIdx.x & 31, gi = lane / G, NG = 32 / G;
    double* a = pts + 4 * pt;
    double x[4] = {a[0], a[1], a[2], a[3]};
    const double sc[4] = {sx, sx, sv, sv};
    double g[4];
    double cur = point_grad<MT>(maps, p, rx, x[0], x[1], x[2], x[3], 0.f, nullptr, nullptr, g, G);
    double lam = -1.0;
    for (int it = 0; it < iters; ++it) {
        // gradients at x +- del e_c, evaluation e = 2 c + (0: +, 1: -)
        double gpm[8][4];
        for (int e0 = 0; e0 < 8; e0 += NG) {
            const int e = e0 + gi;
            double xe[4] = {x[0], x[1], x[2], x[3]};
            if (e < 8) {
                const int c = e >> 1;
                const double del = 1e-3 * sc[c];
                if (e & 1)
                    xe[c] -= del;
                else
                    xe[c] += del;
            }
            double ge[4];
            point_grad<MT>(maps, p, rx, xe[0], xe[1], xe[2], xe[3], 0.f, nullptr, nullptr, ge, G);
            for (int k = 0; k < NG && e0 + k < 8; ++k)
                for (int r = 0; r < 4; ++r) gpm[e0 + k][r] = __shfl_sync(0xffffffffu, ge[r], k * G);
        }
        double H[4][4];
        for (int c = 0; c < 4; ++c) {
            const double del = 1e-3 * sc[c];
            for (int r = 0; r < 4; ++r) H[r][c] = (gpm[2 * c][r] - gpm[2 * c + 1][r]) / (2.0 * del);
        }
        for (int r = 0; r < 4; ++r)
            for (int c = r + 1; c < 4; ++c) H[r][c] = H[c][r] = 0.5 * (H[r][c] + H[c][r]);
        if (lam < 0.0) {
            double n = 0.0;
            for (int c = 0; c < 4; ++c) n += (sc[c] * g[c]) * (sc[c] * g[c]);
            lam = sqrt(n) / step;
            if (!(lam > 0.0)) break;  // zero gradient: nothing to do
        }
        bool moved = false;
        for (int t0 = 0; t0 < 40 && !moved; t0 += NG) {
            double lt = lam;  // lambda of trial t0 + gi: lam 4^gi (exact: powers of two)
            for (int i = 0; i < gi; ++i) lt *= 4.0;
            double A[4][4], d[4] = {0.0, 0.0, 0.0, 0.0};
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) A[r][c] = -H[r][c] + (r == c ? lt / (sc[r] * sc[r]) : 0.0);
            const bool ok = t0 + gi < 40 && chol4_solve(A, g, d);
            const double y0 = x[0] + d[0], y1 = x[1] + d[1], y2 = x[2] + d[2], y3 = x[3] + d[3];
            double gy[4];
            const double val = point_grad<MT>(maps, p, rx, y0, y1, y2, y3, 0.f, nullptr, nullptr, gy, G);
            const unsigned win = __ballot_sync(0xffffffffu, ok && val > cur && (lane % G) == 0);
            if (win) {
                const int src = __ffs(win) - 1;  // the smallest improving lambda
                x[0] = __shfl_sync(0xffffffffu, y0, src);
                x[1] = __shfl_sync(0xffffffffu, y1, src);
                x[2] = __shfl_sync(0xffffffffu, y2, src);
                x[3] = __shfl_sync(0xffffffffu, y3, src);
                for (int c = 0; c < 4; ++c) g[c] = __shfl_sync(0xffffffffu, gy[c], src);
                cur = __shfl_sync(0xffffffffu, val, src);
                lam = __shfl_sync(0xffffffffu, lt, src) / 3.0;
                moved = true;
            } else {
                for (int i = 0; i < NG; ++i) lam *= 4.0;
            }
        }
        if (!moved) break;  // no improving step at any damping: converged
    }
    if ((threadIdx.x & 31) == 0) {
        for (int c = 0; c < 4; ++c) a[c] = x[c];
        if (S) S[pt] = (float)cur;
    }
}

double dirichlet_d(double f, int M) {
    const double pi = 3.14159265358979323846264338327950288;
    return sin(pi * M * f) / sin(pi * f);
}

double half_angle(int M, int N) {
    const double D1 = dirichlet_d(1.0 / N, M), D2 = dirichlet_d(2.0 / N, M);
    return 2.0 * acos(0.5 * sqrt((M - D2) / (M - D1)));
}

PtParams pt_params(const Dims& d, const GeoParams& g, int map_dtype) {
    PtParams p;
    p.tx0 = g.tx[0];
    p.tx1 = g.tx[1];
    p.B = g.B;
    p.cMs = g.cMs;
    p.kappa = g.kappa;
    p.gr = (double)d.Nr * g.B / g.cMs;
    p.ge = (double)d.Nd * g.kappa;
    p.grf = (float)p.gr;
    p.gef = (float)p.ge;
    p.Q = d.Q;
    p.Ms = d.Ms;
    p.Mc = d.Mc;
    p.Nr = d.Nr;
    p.Nd = d.Nd;
    p.lgNr = 0;
    while ((1 << p.lgNr) < d.Nr) ++p.lgNr;
    p.thr = (float)half_angle(d.Ms, d.Nr);
    p.thd = (float)half_angle(d.Mc, d.Nd);
    p.mscale = ldexpf(1.0f, gh_map_scale_log2(d, map_dtype));
    return p;
}

// Lanes per point: the power of two >= Q, at most 32.
int group_width(int Q) {
    int G = 1;
    while (G < Q && G < 32) G <<= 1;
    return G;
}

}  // namespace

int gh_launch_points(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                     const double* rx_dev, const double* pts, long long P, float* S) {
    if (P == 0) return GH_OK;
    const PtParams p = pt_params(d, g, map_dtype);
    const int G = group_width(d.Q);
    const unsigned blocks = (unsigned)((P * G + 127) / 128);
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_POINTS, &ev);
    if (map_dtype == GH_C16)
        points_fwd_kernel<GH_C16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, S);
    else if (map_dtype == GH_CBF16)
        points_fwd_kernel<GH_CBF16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, S);
    else
        points_fwd_kernel<GH_C64><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, S);
    return gh_launch_end(ctx, GH_K_POINTS, ev, "points_fwd_kernel");
}

int gh_launch_points_adjoint(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                             const double* rx_dev, const double* pts, long long P, const float* gS, double* dpts,
                             double* drx, float2* dmaps) {
    if (P == 0) return GH_OK;
    const PtParams p = pt_params(d, g, map_dtype);
    const int G = group_width(d.Q);
    const unsigned blocks = (unsigned)((P * G + 127) / 128);
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_POINTS, &ev);
    if (map_dtype == GH_C16)
        points_adj_kernel<GH_C16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, gS, dpts, drx, dmaps);
    else if (map_dtype == GH_CBF16)
        points_adj_kernel<GH_CBF16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, gS, dpts, drx,
                                                                      dmaps);
    else
        points_adj_kernel<GH_C64><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, G, gS, dpts, drx, dmaps);
    return gh_launch_end(ctx, GH_K_POINTS, ev, "points_adj_kernel");
}

int gh_launch_refine(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                     const double* rx_dev, double* pts, long long P, int iters, double sx, double sv, double step,
                     float* S) {
    if (P == 0) return GH_OK;
    const PtParams p = pt_params(d, g, map_dtype);
    const unsigned blocks = (unsigned)((P * 32 + 127) / 128);
    const int G = group_width(d.Q);
    cudaEvent_t ev;
    gh_launch_begin(ctx, GH_K_POINTS, &ev);
    if (map_dtype == GH_C16)
        refine_kernel<GH_C16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, iters, sx, sv, step, S, G);
    else if (map_dtype == GH_CBF16)
        refine_kernel<GH_CBF16><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, iters, sx, sv, step, S,
                                                                 G);
    else
        refine_kernel<GH_C64><<<blocks, 128, 0, ctx->stream>>>(maps, p, rx_dev, pts, P, iters, sx, sv, step, S, G);
    return gh_launch_end(ctx, GH_K_POINTS, ev, "refine_kernel");
}
