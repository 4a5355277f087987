// Internal declarations of libgh: context, workspace, launch bookkeeping and
// the float64 geometry (Eq. 1) shared by the coordinate, exact-direct, BOMP
// and synthesis kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <functional>
#include <vector>

#include "../../include/gh.h"

#define GH_C_LIGHT 299792458.0

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
enum WsSlot {
    WS_RANGE = 0,   // range-FFT intermediate [Q][Mc][Nr] complex64
    WS_TABLE,       // hopping coordinate table
    WS_PART,        // per-CTA argmax partials
    WS_RESULT,      // small device results (argmax, BOMP selections)
    WS_Y,           // staged measurement (host input) [Q][Mc][Ms]
    WS_R,           // BOMP residual [Q][Mc][Ms]
    WS_MAPS,        // maps of the residual [Q][Nr][Nd]
    WS_BOMP,        // BOMP atoms, correlations, amplitudes
    WS_EXACT_P,     // exact stage 1 output [Q][nxy][Mc] complex64
    WS_DIAG,        // coordinate-table diagnostics
    WS_TWIDDLE,     // FFT twiddle tables
    WS_EXACT_TAB,   // exact-path phase table [nxy][Q]
    WS_EXACT_B,     // stage-1 split-BF16 tiles of Y
    WS_BATCH,       // per-frame buffers of gh_detect_batch
    WS_BATCH_META,  // batch descriptors, work items, twiddles, packed results
    WS_COUNT
};

struct TimedLaunch {
    int kind;
    cudaEvent_t start, stop;
};

struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;             // kernels per replay
    std::vector<TimedLaunch> events;  // timing event pairs recorded by each replay
    uint64_t used = 0;                // last use, for eviction
};
constexpr int kMaxGraphs = 8;

struct gh_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    size_t smem_optin = 0;
    char err[512] = {0};

    void* ws[WS_COUNT] = {nullptr};
    size_t ws_bytes[WS_COUNT] = {0};
    void* pinned = nullptr;
    size_t pinned_bytes = 0;

    // twiddle table currently in WS_TWIDDLE: sizes it holds
    int tw_n[2] = {0, 0};

    uint32_t timing = 0;  // bit mask over GH_K_* classes

    // CUDA graphs of the gh_detect launch sequence, one per configuration
    // (recorded on the second call with that configuration, replayed
    // afterwards; all dropped whenever a workspace buffer moves or the
    // twiddle tables change).
    int detect_maps = GH_C64;  // map storage type of gh_detect (GH_HOP)
    bool graphs = true;
    bool capturing = false;
    cudaStream_t capture_stream = nullptr;  // records graphs (the legacy stream cannot be captured)
    std::vector<GraphEntry> graph_cache;
    std::vector<std::vector<unsigned char>> seen_keys;  // configurations met once
    uint64_t graph_tick = 0;
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    double ms[GH_K_COUNT] = {0};
    int64_t nlaunch[GH_K_COUNT] = {0};
    int64_t launches = 0;

    // host-side fault injection (gh_inject_fault): the status to report and
    // how many of its sites still pass before it fires
    int fault_status = 0;
    int fault_after = 0;
};

// True (and disarmed) when an injected fault of this status fires at this site.
bool gh_fault_hit(gh_ctx* ctx, int status);

// Records a failed CUDA call in the context and returns GH_ECUDA.
int gh_fail_cuda(gh_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);
int gh_fail(gh_ctx* ctx, int status, const char* fmt, ...);

#define GH_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return gh_fail_cuda(ctx, e_, #call, __FILE__, __LINE__); \
    } while (0)

#define GH_TRY(expr)                 \
    do {                             \
        int s_ = (expr);             \
        if (s_ != GH_OK) return s_;  \
    } while (0)

// Makes a device current for the scope of an entry point.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Frees the batch planner state of a context (gh_batch.cu).
void gh_batch_release(gh_ctx* ctx);

// Drops the cached gh_detect graph (its kernels hold workspace pointers).
void gh_graph_invalidate(gh_ctx* ctx);

// A launch sequence on ctx->stream that ends with an asynchronous copy of its
// results into the context's pinned buffer and sets *h to that buffer.
using GhSequence = std::function<int(void**)>;
// Runs seq eagerly, records it into a CUDA graph (second call with the same
// key) or replays the recorded graph (later calls); key NULL: always eager.
// Synchronises the stream and adds the replay's kernel timers.
int gh_run_sequence(gh_ctx* ctx, const std::vector<unsigned char>* key, const GhSequence& seq, void** h);

// Grow-only workspace slot; returns GH_OK and sets *p.
int gh_ws(gh_ctx* ctx, WsSlot slot, size_t bytes, void** p);
int gh_pinned(gh_ctx* ctx, size_t bytes, void** p);

// Device status word (0 = ok, else a GH_E* code written by a kernel), kept in
// the result workspace; gh_status_reset zeroes it on the context's stream.
int* gh_status_dev(gh_ctx* ctx);
int gh_status_reset(gh_ctx* ctx);

// Launch bookkeeping: call gh_launch_begin before a kernel launch and
// gh_launch_end right after it (checks the launch error, records events).
void gh_launch_begin(gh_ctx* ctx, int kind, cudaEvent_t* start);
int gh_launch_end(gh_ctx* ctx, int kind, cudaEvent_t start, const char* name);

// ---------------------------------------------------------------------------
// Argument validation shared by the entry points
// ---------------------------------------------------------------------------
struct Dims {
    int Q, Ms, Mc, pad, Nr, Nd;
    int nx, ny, nvx, nvy;
    int64_t nxy, nv, ncells;
};

// ---------------------------------------------------------------------------
// Kernel parameter blocks shared by the single-frame and batched launches
// ---------------------------------------------------------------------------
// Coordinate-table entry of one (x, y, q) (gh_hop.cu).
struct __align__(16) HopEntry {
    long long base;  // (eta(0,0) - j_ref + 1/2) * 2^32 + tol
    long long ax;    // d eta / d ivx * 2^32
    long long by;    // d eta / d ivy * 2^32
    double wx, wy;   // bistatic gradient (float64 bin decisions)
    int row[3];      // map rows (i + k) mod Nr, k = -1, 0, 1
    float cs[3];     // polar coefficients times the wrap sign
    int j_ref;       // Doppler bin of power-row entry 0, a multiple of 4 (entry u is bin (j_ref + u) mod Nd)
    int npair;       // power-row entries to build, in pairs
    int wrap;        // 1 if the velocity grid reaches more than Nd - 1 bins (entries wrap mod Nd)
};
static_assert(sizeof(HopEntry) == 80, "HopEntry layout");

// Hopping scorer (gh_hop.cu).
struct HopParams {
    int Q, Nr, Nd, nvx, nvy;
    float cscale;         // 2^s of reduced-precision maps (folded into the polar coefficients)
    int NB, SA;           // lane mapping: b = lane % NB (stride NB), a = lane / NB (stride SA)
    uint32_t tol2;        // 2 * tol
    long long nxy, nv;
    long long xy_per_cta;
    double lo2, step2, lo3, step3, kappa;
};

// Coordinate table (gh_hop.cu).
struct CoordParams {
    float theta_f;               // polar half-arc angle theta
    float inv_sin2_half;         // 1 / sin^2(theta / 2)
    float inv_sin_t;             // 1 / sin(theta)
    int Ms_odd_sign;             // 1 if (Ms - 1) is odd (wrap flips the sign)
    uint32_t tol;                // hop_tol(nvx, nvy)
};

// BOMP workspace pointers (gh_bomp.cu).
struct BompPtrs {
    double2 *alpha, *corr, *ru, *phase, *corrp;
    double2* alpha_prev;     // the amplitudes the residual maps hold (see Deflate)
    double* gram;
    float2 *atoms_a, *atoms_b;
    float2 *tab_a, *tab_b;   // maps of the atoms: range [K][Q][Nr], Doppler [K][Q][Nd]
    unsigned int* counter;   // CTAs done with the current iteration
    unsigned int* tab_counter;  // [K][Q] table entries handed out (zeroed with counter)
    int chunks;
};

// Map storage: bytes per bin and the power-of-two scale exponent s of the
// reduced-precision types (stored value = 2^-s * map value).
inline size_t gh_map_bin_bytes(int map_dtype) { return map_dtype == GH_C64 ? 8 : 4; }
inline int gh_map_scale_log2(const Dims& d, int map_dtype) {
    if (map_dtype == GH_C64) return 0;
    int s = 0;
    while ((1LL << s) < (long long)d.Ms * d.Mc) ++s;
    return s;
}
inline bool gh_map_dtype_ok(int map_dtype) {
    return map_dtype == GH_C64 || map_dtype == GH_C16 || map_dtype == GH_CBF16;
}

int gh_check_radar(gh_ctx* ctx, const gh_radar* radar, int32_t Q, Dims* d);
int gh_check_grid(gh_ctx* ctx, const gh_grid* grid, Dims* d);
int gh_check_positions(gh_ctx* ctx, const double* tx, const double* rx, int32_t Q);

// Classifies a pointer: 1 = device-accessible, 0 = host, <0 = error status.
int gh_is_device_ptr(gh_ctx* ctx, const void* p);

// ---------------------------------------------------------------------------
// Geometry parameters passed by value to kernels
// ---------------------------------------------------------------------------
struct GeoParams {
    double tx[2];
    double rx[2 * GH_MAX_Q];
    double B, cMs;        // bandwidth and c*Ms (range: r = (B*d)/(c*Ms))
    double kappa;         // (f0*Tc)/c (speed: u = kappa*(wx*vx + wy*vy))
    double lo[4], step[4];
    int32_t n[4];
    int32_t Q, Ms, Mc, Nr, Nd;
};

void gh_fill_geo(GeoParams* g, const gh_radar* radar, const double* tx, const double* rx,
                 int32_t Q, const gh_grid* grid);

// float64 helpers with no contraction, so that every rounding matches the
// documented expression order (bin decisions must agree with a plain float64
// evaluation of the same expressions).
__device__ __forceinline__ double gh_axis(double lo, double step, int i) {
    return __dadd_rn(lo, __dmul_rn((double)i + 0.5, step));
}

__device__ __forceinline__ void gh_unit(double dx, double dy, double* n, double* ux, double* uy) {
    double nn = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    *n = nn;
    if (nn < 1e-9) {
        *ux = 0.0;
        *uy = 0.0;
    } else {
        *ux = __ddiv_rn(dx, nn);
        *uy = __ddiv_rn(dy, nn);
    }
}

// Bistatic path d = |x - tx| + |x - rx| and gradient w (Eq. 1).
// The receiver half of gh_bistatic, given the transmitter's distance n1 and
// unit vector (ux1, uy1) at the same point (shared by all receivers).
__device__ __forceinline__ void gh_bistatic_rx(const GeoParams& g, int q, double x, double y, double n1, double ux1,
                                               double uy1, double* d, double* wx, double* wy) {
    double n2, ux2, uy2;
    gh_unit(__dsub_rn(x, g.rx[2 * q]), __dsub_rn(y, g.rx[2 * q + 1]), &n2, &ux2, &uy2);
    *d = __dadd_rn(n1, n2);
    *wx = __dadd_rn(ux1, ux2);
    *wy = __dadd_rn(uy1, uy2);
}

__device__ __forceinline__ void gh_bistatic(const GeoParams& g, int q, double x, double y,
                                            double* d, double* wx, double* wy) {
    double n1, ux1, uy1;
    gh_unit(__dsub_rn(x, g.tx[0]), __dsub_rn(y, g.tx[1]), &n1, &ux1, &uy1);
    gh_bistatic_rx(g, q, x, y, n1, ux1, uy1, d, wx, wy);
}

// r = (B*d)/(c*Ms), cycles per sample.
__device__ __forceinline__ double gh_range(const GeoParams& g, double d) {
    return __ddiv_rn(__dmul_rn(g.B, d), g.cMs);
}

// u = kappa*(wx*vx + wy*vy), cycles per chirp.
__device__ __forceinline__ double gh_speed(const GeoParams& g, double wx, double wy, double vx, double vy) {
    return __dmul_rn(g.kappa, __dadd_rn(__dmul_rn(wx, vx), __dmul_rn(wy, vy)));
}

// Fraction of x (cycles) as an unsigned 64-bit fixed-point phase (2^64 = one
// cycle). Integer products of such phases with sample indices wrap modulo one
// cycle exactly, so large phase arguments are reduced without rounding.
__device__ __forceinline__ uint64_t gh_phase_fix(double x) {
    double f = x - floor(x);                       // [0, 1)
    double s = f * 18446744073709551616.0;         // * 2^64
    if (s >= 18446744073709551615.0) return 0ull;  // f rounded up to one cycle
    return __double2ull_rz(s);
}

// sin/cos of 2*pi*phase for a fixed-point phase (top 32 bits used).
__device__ __forceinline__ float2 gh_cis_fix(uint64_t ph) {
    float t = (float)(uint32_t)(ph >> 32) * 4.656612873077392578125e-10f;  // 2^-31: turns * 2
    float s, c;
    sincospif(t, &s, &c);
    return make_float2(c, s);
}

// cos and sin of 2*pi*phase for a fixed-point phase (top 32 bits used), by
// reduction to the nearest quarter turn (exact, in integer arithmetic) and the
// Taylor series of sin and cos on |x| <= pi/4 to the x^9 and x^10 terms (the
// remainders, below x^11/11! and x^12/12!, are under 2e-9), then the exact
// rotation by that many quarter turns. Float32; about 1e-7 absolute error.
__device__ __forceinline__ float2 gh_cis_fix_poly(uint64_t ph) {
    const uint32_t u = (uint32_t)(ph >> 32);
    const uint32_t qi = (u + (1u << 29)) >> 30;        // nearest quarter turn, mod 4
    const int32_t r = (int32_t)(u - (qi << 30));       // in [-2^29, 2^29)
    const float x = (float)r * 1.46291807926715968e-9f;  // 2 pi / 2^32
    const float x2 = x * x;
    float sp = fmaf(x2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);  // 1/9!, -1/7!
    sp = fmaf(x2, sp, 8.33333333333333333e-3f);                               // 1/5!
    sp = fmaf(x2, sp, -1.66666666666666667e-1f);                              // -1/3!
    const float sn = fmaf(x * x2, sp, x);
    float cp = fmaf(x2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);   // -1/10!, 1/8!
    cp = fmaf(x2, cp, -1.38888888888888889e-3f);                              // -1/6!
    cp = fmaf(x2, cp, 4.16666666666666667e-2f);                               // 1/4!
    cp = fmaf(x2, cp, -0.5f);                                                 // -1/2!
    const float cs = fmaf(x2, cp, 1.0f);
    const float c = (qi & 1) ? -sn : cs, sv = (qi & 1) ? cs : sn;  // times i^qi
    return (qi & 2) ? make_float2(-c, -sv) : make_float2(c, sv);
}

// sin(2 pi x 2^-64) with full relative precision: x is reduced to its distance
// v <= 2^62 from the nearest multiple of half a cycle before the float
// conversion.
__device__ __forceinline__ float gh_sin2pi_fix(uint64_t x) {
    const uint64_t w = x & 0x7fffffffffffffffull;
    const uint64_t v = w < (1ull << 62) ? w : (1ull << 63) - w;
    const float s = sinpif((float)v * 1.08420217248550443e-19f);  // 2^-63
    return (x >> 63) ? -s : s;
}

// F_M(f) = sum_{m < M} exp(j 2 pi f m) = exp(j pi f (M-1)) sin(pi M f) / sin(pi f)
// for f = ph 2^-64 (a fixed-point phase; F is 1-periodic), M an even power of
// two. The arguments are reduced exactly in integer arithmetic: M f mod 2 from
// ph M/2 mod 2^64, the phase f (M-1)/2 mod 1 from the 128-bit product
// ph (M-1), sin(pi f) from the distance of f to the nearest integer.
__device__ __forceinline__ float2 gh_dtft_fix(uint64_t ph, int M) {
    const uint64_t h = ph < (1ull << 63) ? ph : (0ull - ph);
    if (h == 0) return make_float2((float)M, 0.f);
    const float sf = sinpif((float)h * 5.42101086242752217e-20f);  // sin(pi f) > 0, 2^-64
    const float sm = gh_sin2pi_fix(ph * (uint64_t)(M >> 1));           // sin(pi M f)
    const uint64_t lo = ph * (uint64_t)(M - 1), hi = __umul64hi(ph, (uint64_t)(M - 1));
    const float2 e = gh_cis_fix((lo >> 1) | (hi << 63));
    const float d = sm / sf;
    return make_float2(e.x * d, e.y * d);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// ---------------------------------------------------------------------------
// On-the-fly deflation of a measurement (BOMP residual):
//   R_q[mc][m] = Y_q[mc][m] - sum_{t < n} alpha[t][q] b_t,q[mc] a_t,q[m]
// ---------------------------------------------------------------------------
struct Deflate {
    const double2* alpha;    // [K][Q] amplitudes
    const float2* atoms_a;   // [K][Q][Ms] a(r_t,q)
    const float2* atoms_b;   // [K][Q][Mc] b(u_t,q)
    int n;                   // atoms to subtract (0: Y unchanged)
    // Maps of the residual by linearity (gh_launch_maps_deflate): the map of
    // atom t at receiver q is tab_a[t][q][i] tab_b[t][q][j]; the maps hold the
    // amplitudes alpha_prev, so alpha - alpha_prev is what is left to subtract.
    const double2* alpha_prev;  // [K][Q]
    const float2* tab_a;        // [K][Q][Nr]
    const float2* tab_b;        // [K][Q][Nd]
    const double2* ru;          // [K][Q] (r, u) of the atoms (the exact path's stage-1 update)
};


__device__ __forceinline__ float2 gh_deflate(const Deflate& f, int Q, int Ms, int Mc, int q, int mc, int m,
                                             float2 y) {
    for (int t = 0; t < f.n; ++t) {
        const double2 al = f.alpha[(size_t)t * Q + q];
        const float2 b = f.atoms_b[((size_t)t * Q + q) * Mc + mc];
        const float2 a = f.atoms_a[((size_t)t * Q + q) * Ms + m];
        const float2 ab = make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
        const float ax = (float)al.x, ay = (float)al.y;
        y.x -= ax * ab.x - ay * ab.y;
        y.y -= ax * ab.y + ay * ab.x;
    }
    return y;
}


// ---------------------------------------------------------------------------
// Per-kernel launchers (one per .cu file)
// ---------------------------------------------------------------------------
struct ArgPartial {
    float score;
    int32_t pad;
    int64_t cell;
};

// Result slot of an argmax: best cell and score.
struct ArgResult {
    int64_t cell;
    float score;
    int32_t valid;
};

// ---------------------------------------------------------------------------
// Batches of frames (gh_detect_batch): one device-resident descriptor per frame
// and work items that name a frame and a range of its rows, columns or cells.
// ---------------------------------------------------------------------------
struct BatchFrame {
    GeoParams g;
    Dims d;
    HopParams hp;
    CoordParams cp;
    BompPtrs bw;
    Deflate df;                 // atoms of the frame's BOMP workspace (n set per iteration)
    int K;
    const float2* Y;            // [Q][Mc][Ms]
    float2* zr;                 // range-FFT intermediate [Q][Mc][Nr]
    float2* maps;               // [Q][Nr][Nd]
    void* table;                // hopping coordinate table [nxy][Q]
    int* rowlim;                // [2Q]: per receiver the smallest, then the largest map row the table reads
    int64_t* mask;              // [K] selected cells
    unsigned long long* key;    // [K] packed argmax: score bits << 32 | (2^32 - 1 - cell)
    ArgResult* sel;             // [K]
    const float2* twr;          // exp(-j 2 pi t / Nr), t < Nr / 2
    const float2* twd;          // exp(-j 2 pi t / Nd), t < Nd / 2
};

struct BatchItem {
    int frame;
    int aux;          // FFT items: receiver q (Doppler) / unused
    long long start;  // first row, range bin or (x, y) cell
    long long count;
};

// rowlim (optional): per receiver the row bounds from gh_launch_coord; rows
// outside them are not computed (gh_detect's own maps only).
int gh_launch_maps(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate* df, void* maps, int map_dtype,
                   const int* rowlim = nullptr);
// Zero-padded range FFT of every chirp alone: *zr = [Q][Mc][Nr] complex64 (context workspace).
int gh_launch_range_rows(gh_ctx* ctx, const Dims& d, const float2* Y, void** zr);
// Shared-memory column length of an N-point FFT (one float2 of padding per 16).
__host__ __device__ inline int gh_fft_ld(int N) { return N + (N >> 4); }
// Range FFT: rows of Nr points per CTA; Doppler FFT: range bins per CTA.
inline int gh_fft_rows_per_cta(int Nr) { return Nr >= 2048 ? 1 : 2048 / Nr; }
inline int gh_fft_bins_per_cta(int Nr, int Nd) {
    const int IB = Nd >= 4096 ? 1 : 4096 / Nd;
    return IB > 16 ? (Nr < 16 ? Nr : 16) : (IB > Nr ? Nr : IB);
}
// Shared memory of the two FFT kernels: the columns (+ the Doppler centring
// factors) + the twiddle table of N/2 entries.
inline size_t gh_fft_smem_range(int rows, int Nr) {
    return ((size_t)rows * gh_fft_ld(Nr) + Nr / 2) * sizeof(float2);
}
inline size_t gh_fft_smem_dop(int IB, int Nd) {
    return ((size_t)IB * (gh_fft_ld(Nd) + 2) + IB + Nd / 2) * sizeof(float2);
}
// Threads of an FFT CTA over `points` points: one per radix-16 butterfly
// (the in-place passes need at least that many), in [32, 512].
inline int gh_fft_threads(int points) {
    const int t = points / 16;
    return t < 32 ? 32 : t > 512 ? 512 : t;
}
// exp(-j 2 pi t / N), t < N/2, rounded from float64 (the FFT twiddle table).
void gh_twiddles(int N, float2* out);
// Maps of the residual by linearity, in place (complex float32 maps): the
// maps of the previous iteration's residual minus
// sum_{t < df.n} (alpha_t - alpha_prev_t) tab_a_t[i] tab_b_t[j] per receiver;
// rows outside rowlim (if given) are left as they are.
int gh_launch_maps_deflate(gh_ctx* ctx, const Dims& d, const Deflate& df, void* maps, const int* rowlim);
// The same for the frames listed in items (frame, receiver, first range bin,
// count), iteration k.
int gh_launch_maps_deflate_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, int k);
// Batched maps (iteration k's residual applied on load); items as built by gh_batch.cu.
int gh_launch_maps_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* range_items, int n_range,
                         int thr_range, size_t smem_range, const BatchItem* dop_items, int n_dop, int thr_dop,
                         size_t smem_dop, int k);
// Scorer and coordinate-table parameters of one frame.
void gh_hop_frame_params(const Dims& d, const GeoParams& g, HopParams* hp, CoordParams* cp);
// Scoring slots per lane (cells, partial runs included) of frame d with AC
// cells per run: lanes b = lane % NB, a = lane / NB; NB = min(nvy, 32) for
// AC = 8, 16, 32 and NB = 8 (SA = 4) for AC = 6, 10 (the scorer's layouts).
inline int lane_slots(const Dims& d, int ac) {
    const int NB = (ac == 6 || ac == 10) ? 8 : (d.nvy < 32 ? d.nvy : 32), SA = 32 / NB;
    const int rows = (d.nvy + NB - 1) / NB, cells = (d.nvx + SA - 1) / SA;
    return rows * ((cells + ac - 1) / ac) * ac;
}

// 6 or 10 when the 8 x 4 layout with that many cells per run needs fewer
// slots than every standard configuration, else 0.
inline int lane_layout_ac(const Dims& d) {
    int best = 0, best_slots = 1 << 30;
    for (int ac : {8, 16, 32, 6, 10}) {
        const int sl = lane_slots(d, ac);
        if (sl < best_slots) {
            best_slots = sl;
            best = ac;
        }
    }
    return (best == 6 || best == 10) ? best : 0;
}

// Shared memory of one batched-scorer warp whose power rows hold at most
// row_floats floats (Q * Nd, or Nd with one receiver's row at a time).
size_t gh_hop_batch_warp_bytes(int ac, int row_floats, int max_q);
// Shared memory of one paired-scorer CTA (two warps per (x, y) cell, all
// receivers' rows: row_floats >= Q * Nd).
size_t gh_hop_pair_bytes(int ac, int row_floats, int max_q);
// Batched coordinate tables (items: frame, first (x, y) cell, count <= 16).
int gh_launch_coord_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n);
// Persistent batched scorer: warps take items (frame, first (x, y) cell, count)
// from *counter (zeroed here) and fold each frame's best cell into key[k];
// ac cells per lane (8, 16, 32; 6, 10 in the 8 x 4 lane layout), warps per
// CTA; per_rx: one receiver's power row at a time (every frame's cells of a
// lane form one run: nvy <= 32 and nvx <= SA ac); pair: the paired scorer
// (two warps per (x, y) cell sharing one set of power rows; warps = 2,
// !per_rx; ac 3 or 5 in the 8 x 4 layout, 8 or 16 in the standard one).
// max_nd, max_q_nd, max_q: largest Nd, Q * Nd and Q of the frames the items
// name.
int gh_launch_hop_batch(gh_ctx* ctx, const BatchFrame* frames, const BatchItem* items, int n, unsigned* counter,
                        int k, int ac, int warps, bool per_rx, bool pair, int max_nd, int max_q_nd, int max_q);
// Batched BOMP selection and correlation of iteration k for the listed frames.
int gh_launch_bomp_select_batch(gh_ctx* ctx, const BatchFrame* frames, const int* active, int n, int k);
int gh_launch_bomp_corr_batch(gh_ctx* ctx, const BatchFrame* frames, const int* active, int n, int k, int max_chunks,
                              int max_q);
// BOMP workspace pointers of one frame and its correlation chunk count.
BompPtrs gh_bomp_ptrs(void* ws, const Dims& d, int K);
int gh_bomp_chunks(const Dims& d);
// Zeroes every frame's BOMP counter (one CTA per frame).
int gh_launch_batch_reset(gh_ctx* ctx, const BatchFrame* frames, int nframes);
// Packs every frame's selections and amplitudes into out (see gh_batch.cu).
int gh_launch_batch_gather(gh_ctx* ctx, const BatchFrame* frames, int nframes, const long long* offsets, void* out);
// rowlim, rw: optional outputs, see coord_kernel.
int gh_launch_coord(gh_ctx* ctx, const Dims& d, const GeoParams& g, void* table, int32_t* diag_i,
                    double* diag_tau, float* diag_c, double* diag_w, int* rowlim = nullptr,
                    double* rw = nullptr);
size_t gh_hop_table_bytes(const Dims& d);
// Scorer: per-CTA argmax partials into the context workspace (*parts, *nparts);
// gh_launch_hop also reduces them into *result.
int gh_launch_hop_parts(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                        const void* table, float* scores, const int64_t* mask, int nmask,
                        ArgPartial** parts, int* nparts);
int gh_launch_hop(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                  const void* table, float* scores, const int64_t* mask, int nmask,
                  ArgResult* result);
int gh_launch_argmax_finalize(gh_ctx* ctx, const ArgPartial* parts, int nparts, ArgResult* out);
// Continuous-point scores, their adjoint and the refinement (gh_points.cu).
int gh_launch_points(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                     const double* rx_dev, const double* pts, long long P, float* S);
int gh_launch_points_adjoint(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                             const double* rx_dev, const double* pts, long long P, const float* gS, double* dpts,
                             double* drx, float2* dmaps);
int gh_launch_refine(gh_ctx* ctx, const Dims& d, const GeoParams& g, const void* maps, int map_dtype,
                     const double* rx_dev, double* pts, long long P, int iters, double sx, double sv, double step,
                     float* S);
// Stage 1 of the exact path alone (Eq. 4's g_q for every (x, y)): *P planar
// [Q][nxy][Re row | Im row][Mc] float32 in the context workspace.
int gh_launch_exact_stage1(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y, const float** P);
// Exact direct scores of the (deflated) measurement; partials as gh_launch_hop_parts.
int gh_launch_exact_parts(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y,
                          const Deflate* df, float* scores, const int64_t* mask, int nmask,
                          ArgPartial** parts, int* nparts);
int gh_launch_exact(gh_ctx* ctx, const Dims& d, const GeoParams& g, const float2* Y,
                    float* scores, const int64_t* mask, int nmask, ArgResult* result);
int gh_launch_synth(gh_ctx* ctx, const Dims& d, const GeoParams& g, int T,
                    const double* targets_alpha_dev, const float2* noise, float2* Y);
int gh_launch_residual(gh_ctx* ctx, const Dims& d, const float2* Y, const Deflate& df, float2* R);

// BOMP (workspace of gh_bomp_ws_bytes(d, K) bytes; the amplitudes, double2
// [K][Q], sit at its start). Iteration k, one launch (gh_launch_bomp_step):
// the scorer's partials -> sel[k] and mask[k], the new atom, its correlation
// with Y and the least squares of atoms 0..k. rw (optional): the coordinate
// kernel's float64 (r, wx, wy) per (x, y, q) entry, which saves recomputing
// the new atom's geometry. gh_bomp_reset zeroes the workspace's completion
// counter.
size_t gh_bomp_ws_bytes(const Dims& d, int K);
Deflate gh_bomp_deflate(void* bomp_ws, const Dims& d, int K, int n);
int gh_bomp_reset(gh_ctx* ctx, const Dims& d, int K, void* bomp_ws);
int gh_launch_bomp_step(gh_ctx* ctx, const Dims& d, const GeoParams& g, const ArgPartial* parts, int nparts,
                        const float2* Y, ArgResult* sel, int64_t* mask, int k, int K, void* bomp_ws,
                        const double* rw = nullptr);
