/*
 * gh.h - C-ABI of the GB300 grid-hopping library (libgh.so).
 *
 * Implements the hot path of "Grid Hopping: Accelerating Direct Estimation
 * Algorithms for Multistatic FMCW Radar" (Monnoyer, Feuillen, Drouguet,
 * Jacques, Vandendorpe): range-Doppler maps, the grid-hopping score over a 4D
 * location-velocity grid, its argmax, a BOMP detect-and-deflate loop, and the
 * exact direct decision function.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Problem statement (Sec. II): one TX at tx[0..1] (metres, 2D ground plane),
 * Q receivers at rx[2q], rx[2q+1]; chirps of carrier f0 [Hz], bandwidth B [Hz]
 * and duration Tc [s]; a frame of Mc chirps x Ms samples per receiver.
 *
 * Measurement Y: complex float32, interleaved (re, im), layout [Q][Mc][Ms]
 * (row mc is chirp mc; Sec. II). Range-Doppler maps: layout [Q][Nr][Nd]
 * (range bin major, Doppler bin contiguous), Nr = pad*Ms, Nd = pad*Mc.
 *
 * Sensing functions (Eq. 1, read as cycles per sample / per chirp):
 *   r_q(x)    = B * d_q(x) / (c * Ms),  d_q = |x - tx| + |x - rx_q|
 *   u_q(x, v) = (f0 * Tc / c) * <w_q(x), v>,
 *   w_q = (x - tx)/|x - tx| + (x - rx_q)/|x - rx_q|   (a length < 1e-9 m gives 0)
 * with c = 299792458 m/s. Atoms a_m(r) = exp(j 2 pi r m), b_mc(u) = exp(j 2 pi u mc).
 *
 * Grid (gh_grid): axes x, y, vx, vy; point i of axis a is
 * lo[a] + (i + 1/2) * step[a], i < n[a]. Linear cell index
 * ((ix * ny + iy) * nvx + ivx) * nvy + ivy (int64).
 *
 * Pointers: "_dev" arguments are device memory of the context's device;
 * "_host" arguments are host memory. Arguments documented as "host or device"
 * are classified with cudaPointerGetAttributes. The caller owns every buffer it
 * passes; the context owns its workspace and frees it in gh_destroy.
 *
 * Errors: every int-returning call returns GH_OK (0) or a negative GH_E* code
 * and never throws. GH_EINVAL is returned before any GPU work for bad
 * arguments; GH_ECUDA keeps the CUDA error text, readable with gh_last_error.
 * Calls are ordered on the context's stream; calls that return host results
 * synchronise that stream before returning. A context is not thread safe.
 */
#ifndef GH_H
#define GH_H

#include <stdint.h>

#if defined(__GNUC__)
#define GH_API __attribute__((visibility("default")))
#else
#define GH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define GH_OK        0
#define GH_EINVAL   (-1)  /* bad argument (NULL, size out of range, ...)       */
#define GH_ENOMEM   (-2)  /* device or pinned-host allocation failed           */
#define GH_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed       */
#define GH_ETIMEOUT (-4)  /* a bounded device-side wait gave up                */
#define GH_ENOTSUP  (-5)  /* valid but unsupported combination                 */

/* Map storage types (gh_make_maps, gh_score_grid, gh_set_detect_maps).
 * The reduced-precision types store 2^-s times each map value, with
 * s = log2(Ms) + log2(Mc) (a unit-amplitude on-bin tone becomes 1), so that
 * the float16 range holds every map; gh_score_grid undoes the scale exactly. */
#define GH_C64      0     /* complex float32 (8 bytes per bin)                 */
#define GH_C16      1     /* complex float16, (re, im) pair (4 bytes per bin)  */
#define GH_CBF16    2     /* complex bfloat16, (re, im) pair (4 bytes per bin) */

/* Scoring methods (gh_detect). */
#define GH_HOP      0     /* grid hopping (Sec. IV)                            */
#define GH_EXACT    1     /* exact direct decision function (Sec. III)        */
#define GH_INDIRECT 2     /* indirect method: map peaks + multilateration (Eq. 2), gh_factorized only */

/* Kernel classes for gh_kernel_stats. */
#define GH_K_RANGE_FFT   0
#define GH_K_DOPPLER_FFT 1
#define GH_K_COORD       2
#define GH_K_HOP_SCORE   3
#define GH_K_ARGMAX      4
#define GH_K_BOMP        5
#define GH_K_EXACT_S1    6
#define GH_K_EXACT_S2    7
#define GH_K_SYNTH       8
#define GH_K_POINTS      9   /* continuous-point scores, adjoint, refinement */
#define GH_K_DEFLATE     10  /* maps of a BOMP residual by linearity (atom maps subtracted) */
#define GH_K_COUNT       11

/* Size limits checked by every entry point (GH_EINVAL beyond them). */
#define GH_MAX_Q        64
#define GH_MIN_M        4       /* Ms, Mc: powers of two in [GH_MIN_M, GH_MAX_M] */
#define GH_MAX_M        4096
#define GH_MAX_NFFT     8192    /* pad*Ms and pad*Mc at most this               */
#define GH_MAX_K        16      /* BOMP iterations                              */

/* FMCW frame parameters (Sec. II). pad: zero-padding factor of both FFT axes,
 * a power of two in [1, 16]. */
typedef struct gh_radar {
    double  f0;        /* carrier frequency [Hz]          */
    double  B;         /* chirp bandwidth [Hz]            */
    double  Tc;        /* chirp duration [s]              */
    int32_t Ms;        /* samples per chirp               */
    int32_t Mc;        /* chirps per frame                */
    int32_t pad;       /* zero-padding factor             */
    int32_t reserved;  /* must be 0                       */
} gh_radar;

/* Cell-centred 4D grid (x [m], y [m], vx [m/s], vy [m/s]); step > 0, n >= 1,
 * total cells < 2^62. */
typedef struct gh_grid {
    double  lo[4];
    double  step[4];
    int32_t n[4];
} gh_grid;

typedef struct gh_ctx gh_ctx;

/* Create a context on CUDA device `device`. `stream` is a cudaStream_t to run
 * on (NULL: the context creates and owns a non-blocking stream). */
GH_API int gh_create(gh_ctx** ctx, int32_t device, void* stream);
/* Free the context, its workspace and (if owned) its stream. NULL is a no-op. */
GH_API void gh_destroy(gh_ctx* ctx);
/* Build id of the library: the first 16 hex digits of the SHA-256 of its
 * CUDA sources and this header, fixed at compile time (no counterpart in the
 * paper; it tells which sources a loaded library was built from). */
GH_API const char* gh_build_id(void);
/* Static text for a status code. */
GH_API const char* gh_status_str(int32_t status);
/* Text of the last error recorded in the context ("" if none). */
GH_API const char* gh_last_error(const gh_ctx* ctx);

/*
 * gh_make_maps - zero-padded 2D DFT range-Doppler maps of every receiver
 * (Sec. III: the 2D FFT of Y_q; Sec. IV: bin i is the correlation with the
 * atom at the FFT's i-th grid frequency).
 *   maps[q][i][j] = exp(j pi (i/Nr)(Ms-1)) *
 *                   sum_mc sum_m Y[q][mc][m] exp(-j 2 pi (j mc/Nd + i m/Nr))
 * The range-centring factor makes bin (i, j) the correlation with the centred
 * atom exp(j 2 pi r (m - (Ms-1)/2)), whose Gram is real (used by the polar
 * interpolation of gh_score_grid).
 *   Y_dev    : device, complex float32 [Q][Mc][Ms]
 *   maps_dev : device, [Q][Nr][Nd] bins of type map_dtype (written): complex
 *              float32 (GH_C64), or 2^-s times the values rounded to
 *              nearest-even complex float16 (GH_C16) / bfloat16 (GH_CBF16)
 *              from the float32 transform
 * No host synchronisation.
 */
GH_API int gh_make_maps(gh_ctx* ctx, const gh_radar* radar, int32_t Q,
                 const void* Y_dev, void* maps_dev, int32_t map_dtype);

/*
 * gh_score_grid - grid-hopping score of every cell and its argmax (Sec. IV,
 * Eq. 5, with the sum over receivers of Eq. 3):
 *   S(x, v) = sum_q | sum_{k=-1,0,1} c_k(tau_q) maps[q][(i_q+k) mod Nr][j_q] |^2
 * where rho_q = Nr * r_q(x), i_q = floor(rho_q + 1/2), tau_q = rho_q - i_q,
 * c_k are the three-bin polar interpolation coefficients (range axis) and
 * j_q = floor(Nd * u_q(x, v) + 1/2) mod Nd is the nearest Doppler bin (single
 * index, Sec. IV). Bin decisions i_q and j_q are taken in float64; scores
 * accumulate in float32. Range reads that wrap around the map carry the
 * centring phase of the unwrapped index.
 *   tx_host      : host, double[2]
 *   rx_host      : host, double[2*Q]
 *   maps_dev     : device, from gh_make_maps with the same map_dtype
 *                  (reduced-precision maps are read as float32 values and
 *                  accumulated in float32)
 *   scores_dev   : device float[ncells] or NULL (argmax only)
 *   best_cell    : host int64, argmax (ties: smallest index); may be NULL
 *   best_score   : host float, its score; may be NULL
 * Synchronises the stream when best_cell or best_score is non-NULL.
 */
GH_API int gh_score_grid(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                  const double* rx_host, int32_t Q, const void* maps_dev,
                  int32_t map_dtype, const gh_grid* grid, float* scores_dev,
                  int64_t* best_cell, float* best_score);

/*
 * gh_direct_exact - exact direct decision function of every cell (Sec. III,
 * the joint location-velocity form behind Eqs. 3-4):
 *   S(x, v) = sum_q | <Y_q, b(u_q(x, v)) (x) a(r_q(x))> |^2,  <y, a> = sum y conj(a)
 * computed as two contractions: P_q[x][mc] = sum_m Y[q][mc][m] conj(a_m(r_q(x)))
 * (the g_q of Eq. 4), then per (x, q) the Doppler correlation of P_q with the
 * separable atom b_mc(u) = exp(j2pi k wx vx mc) exp(j2pi k wy vy mc), k = f0 Tc/c.
 *   Y_host_or_dev: complex float32 [Q][Mc][Ms], host or device
 *   scores_dev   : device float[ncells] or NULL
 *   best_cell, best_score: as gh_score_grid
 */
GH_API int gh_direct_exact(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                    const double* rx_host, int32_t Q, const void* Y_host_or_dev,
                    const gh_grid* grid, float* scores_dev, int64_t* best_cell,
                    float* best_score);

/*
 * gh_score_points - differentiable hopping score at P continuous points
 * (x, y, vx, vy), for off-grid refinement of detections and calibration of
 * receiver positions (Sec. VI names refined estimation as future work). Both
 * map axes are interpolated with the three-bin polar model of Sec. IV (range:
 * c_k(tau) as in gh_score_grid; Doppler: the same construction on centred
 * Doppler atoms, coefficients d_l(sigma), in place of the nearest bin, so that
 * the score varies smoothly with v):
 *   S(p) = sum_q | sum_{k,l} c_k(tau_q) d_l(sigma_q) V_q(i_q+k, j_q+l) |^2
 *   V_q(n, m) = maps[q][n mod Nr][m mod Nd] (-1)^((Ms-1) floor(n/Nr)) exp(j pi m (Mc-1)/Nd)
 * with i_q, tau_q from Nr r_q and j_q, sigma_q from Nd u_q (float64, Eq. 1).
 *   tx_host    : host double[2]
 *   rx_dev     : device double[Q][2] receiver positions (device memory so that
 *                their gradient can be taken)
 *   maps_dev   : device, from gh_make_maps with map_dtype
 *   points_dev : device double[P][4] (x, y, vx, vy); P >= 0
 *   scores_dev : device float[P] (written)
 * Non-finite positions give non-finite scores. No host synchronisation.
 */
GH_API int gh_score_points(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                    const double* rx_dev, int32_t Q, const void* maps_dev, int32_t map_dtype,
                    const double* points_dev, int64_t P, float* scores_dev);

/*
 * gh_score_points_adjoint - gradients of L = sum_p g_p S(p) (gh_score_points)
 * for upstream weights g = dscores_dev (device float[P]):
 *   dpoints_dev : device double[P][4], written with dL/d(x, y, vx, vy), or NULL
 *   drx_dev     : device double[Q][2], dL/drx ADDED to its contents, or NULL
 *   dmaps_dev   : device complex float32 [Q][Nr][Nd], dL/dRe + j dL/dIm of each
 *                 map bin ADDED to its contents (scatter-add), or NULL; needs
 *                 map_dtype GH_C64
 * The score is differentiated between bin switches (tau, sigma = +-1/2, where
 * the three-bin stencil moves by one bin). Uses atomics (the summation order
 * of drx and dmaps is not deterministic).
 */
GH_API int gh_score_points_adjoint(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                    const double* rx_dev, int32_t Q, const void* maps_dev, int32_t map_dtype,
                    const double* points_dev, int64_t P, const float* dscores_dev,
                    double* dpoints_dev, double* drx_dev, void* dmaps_dev);

/*
 * gh_refine_points - off-grid refinement of P points by damped Newton
 * (Levenberg-Marquardt) ascent of gh_score_points, all iterations in one
 * launch (one warp per point). Per iteration: the Hessian from central
 * differences of the analytic gradient (steps of 1e-3 scale units), then
 * steps d solving (-H + lambda D) d = grad, D = diag(1/scale^2) with scales
 * (scale_xy, scale_xy, scale_v, scale_v); an improving step is taken and
 * lambda shrinks by 3, otherwise lambda grows by 4 (at most 40 trials; no
 * improving step ends the iterations). The first lambda makes the first step
 * about `step` scale units long.
 *   points_dev : device double[P][4], read and overwritten with the refined points
 *   scores_dev : device float[P], their scores (may be NULL)
 *   iters in [0, 100000]; scale_xy, scale_v, step > 0.
 */
GH_API int gh_refine_points(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                    const double* rx_dev, int32_t Q, const void* maps_dev, int32_t map_dtype,
                    double* points_dev, int64_t P, int32_t iters, double scale_xy,
                    double scale_v, double step, float* scores_dev);

/*
 * One frame of a batch (gh_detect_batch): the arguments of gh_detect for one
 * measurement, with the measurement in device memory.
 */
typedef struct {
    gh_radar radar;
    double tx[2];          /* TX position (m)                                  */
    const double* rx;      /* host double[2*Q], RX positions (m)               */
    int32_t Q;             /* receivers, 1..GH_MAX_Q                           */
    int32_t K;             /* BOMP iterations, 1..min(GH_MAX_K, cells)         */
    gh_grid grid;          /* at most 2^32 - 1 cells                           */
    const void* Y;         /* device complex float32 [Q][Mc][Ms]               */
} gh_frame;

/*
 * gh_detect_batch - gh_detect with grid hopping (GH_HOP, complex float32
 * maps) for nframes independent frames of any sizes, each step launched once
 * for the whole batch (coordinate tables, maps of the rows the tables read,
 * persistent scorers whose warps take (frame, cells) work items from a
 * counter, one per group of frames with the same shared-memory need, lane
 * layout and run shape, the groups of an iteration side by side, BOMP
 * selection and correlation); frames whose K is reached drop out of later
 * iterations.
 * Each frame's results equal those of gh_detect on that frame. Outputs are
 * concatenated in frame order:
 *   cells_host  : host int64[sum K]
 *   scores_host : host float[sum K] (may be NULL)
 *   alpha_host  : host double[sum K*Q][2] (may be NULL), per frame [K][Q][2]
 * Each scorer group's cells per lane (8, 16, 32, or 6 and 10 in the 8 x 4
 * lane layout for velocity axes of about 24 and 40 cells; with two warps
 * sharing each (x, y) cell's power rows, 3 and 5 in that layout and 8 and 16
 * in the standard one), warps per CTA,
 * power-row mode and (x, y) cells per work item are chosen by timing the
 * candidates on the first iteration of a batch shape (cached in the context),
 * unless fixed with gh_set_batch_tuning, gh_set_batch_row_mode and
 * gh_set_batch_tile. From the second call with an unchanged batch on, the
 * whole sequence is a replayed CUDA graph.
 */
GH_API int gh_detect_batch(gh_ctx* ctx, int32_t nframes, const gh_frame* frames, int64_t* cells_host,
                    float* scores_host, double* alpha_host);
/* Fixes the batched scorer's configuration: cells per lane in {8, 16, 32},
 * warps per CTA in {2, 4, 8}; (0, 0) returns to autotuning (the default). */
GH_API int gh_set_batch_tuning(gh_ctx* ctx, int32_t cells_per_lane, int32_t warps);
/* The configuration the last gh_detect_batch call used for its scorer group
 * with the most work (cells per lane 6 and 10: the 8 x 4 lane layout; with
 * row mode 2 the paired scorer, 2 warps per CTA). */
GH_API int gh_batch_tuning(gh_ctx* ctx, int32_t* cells_per_lane, int32_t* warps);
/* Fixes the number of consecutive (x, y) cells in one work item of the
 * batched scorer: 4, 8, 16 or 32; 0 returns to tuning (the default: after the
 * cells per lane and warps, the autotuner times the four item sizes; a
 * configuration fixed with gh_set_batch_tuning uses 8 unless an item size is
 * fixed here). Larger items keep a warp on neighbouring cells (map rows
 * shared in L1), smaller ones balance the last items of a launch. */
GH_API int gh_set_batch_tile(gh_ctx* ctx, int32_t cells_per_item);
/* The item size the last gh_detect_batch call used for its scorer group with
 * the most work (0 before the first call). */
GH_API int gh_batch_tile(gh_ctx* ctx, int32_t* cells_per_item);
/* The power-row mode of the last gh_detect_batch call's scorer group with
 * the most work: 1 one receiver's Doppler power row at a time, 0 the rows of
 * all its receivers at once, 2 the rows of all receivers shared by the two
 * warps of a CTA that score each (x, y) cell together. One row at a time
 * needs a lane's velocity cells to fit one run per vy row it takes (nvy <=
 * 32, or the 8 x 4 layout); it and the paired mode leave room for more
 * warps per SM when Q * Nd is large; the
 * autotuner times every mode that applies (a configuration fixed with
 * gh_set_batch_tuning builds all rows at once, one warp per cell). */
GH_API int gh_batch_row_mode(gh_ctx* ctx, int32_t* per_receiver);
/* Keeps the autotuner to one power-row mode: 0 all receivers' rows, 1 one
 * receiver's row at a time, 2 paired (1 and 2 for the scorer groups where
 * they apply, 2 wherever a group's rows fit one CTA; all rows elsewhere); -1
 * (the default) lets it time every mode.
 * Results do not depend on the mode. Other values: GH_EINVAL. */
GH_API int gh_set_batch_row_mode(gh_ctx* ctx, int32_t row_mode);

/*
 * gh_factorized - the paper's factorised single-target estimators: location
 * first over the (x, y) part of the grid, then velocity over its (vx, vy) part
 * at that location (Sec. III, Eqs. 3-4), and the indirect method (Eq. 2).
 *   GH_HOP      grid hopping (Sec. IV): Eq. 3 with the three-bin polar
 *               interpolation of the zero-padded range FFT of every chirp;
 *               Eq. 4 with g_q[mc] = <Y_q[mc], a(r_q(x^))> and the nearest bin
 *               of its Doppler DFT zero-padded to Nd
 *   GH_EXACT    the direct method: Eq. 3 exactly (the exact path's stage 1),
 *               Eq. 4 exactly
 *   GH_INDIRECT per receiver the peak (i, j) of |RD map|: r^ = i / Nr,
 *               u^ = j / Nd in [-1/2, 1/2); x^ = argmin sum_q (r_q(x) - r^_q)^2,
 *               then v^ = argmin sum_q (u_q(x^, v) - u^_q)^2, in float64
 * Ties go to the smallest index.
 *   Y_host_or_dev  : complex float32 [Q][Mc][Ms]
 *   cell_host      : host int64, the 4D cell (ix, iy, ivx, ivy) of the estimate
 *   values_host    : host double[2] (may be NULL): GH_HOP / GH_EXACT: S_loc at
 *                    x^ and S_vel at v^; GH_INDIRECT: the two costs at x^, v^
 *   loc_scores_dev : device float[nx*ny] location scores (may be NULL;
 *                    GH_HOP and GH_EXACT)
 * Synchronises the stream.
 */
GH_API int gh_factorized(gh_ctx* ctx, int32_t method, const gh_radar* radar, const double* tx_host,
                  const double* rx_host, int32_t Q, const void* Y_host_or_dev, const gh_grid* grid,
                  int64_t* cell_host, double* values_host, float* loc_scores_dev);

/*
 * gh_set_detect_maps - storage type (GH_C64 default, GH_C16, GH_CBF16) of the
 * range-Doppler maps gh_detect makes on the context for method GH_HOP.
 */
GH_API int gh_set_detect_maps(gh_ctx* ctx, int32_t map_dtype);

/*
 * gh_detect - K iterations of block orthogonal matching pursuit (BOMP, named
 * in the paper's acronym list; multi-target iterative direct detection is its
 * stated future work, Sec. VI). A block is the Q per-receiver atoms of one grid
 * cell with independent amplitudes. Iteration k:
 *   1. score the residual on the grid (method GH_HOP: maps + gh_score_grid;
 *      GH_EXACT: gh_direct_exact), cells already selected excluded;
 *   2. append the argmax cell;
 *   3. per receiver, solve the float64 least-squares problem for the
 *      amplitudes of all selected atoms (at their exact r, u) against Y;
 *   4. residual R_q = Y_q - sum_t alpha_{t,q} b(u_{t,q}) (x) a(r_{t,q}).
 *   Y_host_or_dev : complex float32 [Q][Mc][Ms], host or device
 *   cells_host    : host int64[K], selected cells in order
 *   scores_host   : host float[K], residual score at each selected cell (may be NULL)
 *   alpha_host    : host double[K][Q][2] (re, im) amplitudes multiplying the
 *                   atoms b(u) (x) a(r) of Sec. II, from the last solve (may be NULL)
 * All K iterations run on the device without host round trips; the stream is
 * synchronised once at the end. 1 <= K <= min(GH_MAX_K, ncells).
 * The residual's maps (GH_HOP with complex float32 maps) and stage-1
 * correlations (GH_EXACT) are reached by linearity after the first iteration:
 * the previous ones minus the newly solved part of the atoms' own maps or
 * correlations, which are known in closed form (equal to recomputing them
 * from R_q up to float32 rounding). Reduced-precision maps are remade from
 * R_q by FFT every iteration.
 */
GH_API int gh_detect(gh_ctx* ctx, int32_t method, const gh_radar* radar,
              const double* tx_host, const double* rx_host, int32_t Q,
              const void* Y_host_or_dev, const gh_grid* grid, int32_t K,
              int64_t* cells_host, float* scores_host, double* alpha_host);

/*
 * gh_synth - synthetic measurement from the signal model (Sec. II, Eq.
 * general-model): Y_q = sum_t alpha_{t,q} b(u_q(x_t, v_t)) (x) a(r_q(x_t)) + W_q.
 *   targets_host : host double[T][4] (x, y, vx, vy)
 *   alpha_host   : host double[T][Q][2] (re, im)
 *   noise_dev    : device complex float32 [Q][Mc][Ms] added to Y, or NULL
 *   Y_dev        : device complex float32 [Q][Mc][Ms] (written)
 * Phases are reduced in float64 before a float32 sincos. 0 <= T <= 64.
 */
GH_API int gh_synth(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
             const double* rx_host, int32_t Q, int32_t T,
             const double* targets_host, const double* alpha_host,
             const void* noise_dev, void* Y_dev);

/*
 * gh_coord_table - the coordinate mapping of the hopping scorer for every
 * (ix, iy, q), copied to the host (diagnostic; Eq. 1 and the polar
 * coefficients of Sec. IV):
 *   ibin_host  : host int32[nx][ny][Q]   nearest range bin i_q (unwrapped)
 *   tau_host   : host double[nx][ny][Q]  fractional offset tau_q
 *   coef_host  : host float[nx][ny][Q][3] polar coefficients c_{-1}, c_0, c_{+1}
 *   w_host     : host double[nx][ny][Q][2] bistatic gradient w_q (may be NULL)
 */
GH_API int gh_coord_table(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                   const double* rx_host, int32_t Q, const gh_grid* grid,
                   int32_t* ibin_host, double* tau_host, float* coef_host,
                   double* w_host);

/*
 * gh_score_grid_noalloc - the same scores and argmax as gh_score_grid, for
 * callers that must not allocate device memory. The paper has no counterpart:
 * this entry point exists for the software around it. Typical such callers are
 * a real-time radar pipeline with a deadline per frame, where cudaMalloc and
 * cudaFree may block on or synchronise with work already queued on the GPU,
 * and a plug-in inside a host framework that owns the device memory budget
 * and forbids allocations outside its own pool.
 *
 * It needs no context and calls no cudaMalloc, cudaFree, cudaMallocHost or
 * other allocating routine. Its scratch (coordinate table, argmax partials,
 * result slot) is one fixed 8 MiB array in device memory, reserved on every
 * GPU that loads the library until the process exits; problems with
 * nx * ny * Q > GH_NOALLOC_MAX_XYQ return GH_EINVAL. The array's device
 * address is looked up on the first call made on each device (with that device
 * current); make that first call before any stream capture. All calls share
 * the array and leave their contents in it: calls whose GPU work overlaps (on
 * two streams or from two host threads) race and must be serialised by the
 * caller.
 *   stream       : cudaStream_t to run on (NULL: the legacy default stream); the
 *                  current device must own maps_dev and scores_dev
 *   maps_dev     : device, complex float32 [Q][Nr][Nd] from gh_make_maps
 *   scores_dev   : device float[ncells] or NULL
 *   best_cell, best_score: host, may be NULL; when either is given the call
 *                  copies the result with cudaMemcpyAsync and synchronises the stream
 * The address is cached per device ordinal for the life of the process:
 * resetting a device (cudaDeviceReset) after its first call here is not
 * supported, since later calls would pass the old address.
 * Errors: GH_EINVAL for bad arguments or a problem beyond the scratch size,
 * GH_ENOTSUP when shared memory is too small or the current device's ordinal
 * is 64 or more, GH_ECUDA for CUDA failures (no error text is kept: there is
 * no context). Launch failures are read from each launch's own status: a CUDA
 * error that other code left pending in the calling thread is neither
 * reported nor cleared.
 */
#define GH_NOALLOC_MAX_XYQ 98304   /* max nx * ny * Q of gh_score_grid_noalloc */
GH_API int gh_score_grid_noalloc(void* stream, const gh_radar* radar,
                                 const double* tx_host, const double* rx_host,
                                 int32_t Q, const void* maps_dev, const gh_grid* grid,
                                 float* scores_dev, int64_t* best_cell, float* best_score);

/*
 * gh_selftest_tcgen05 - diagnostic of the tensor-core plumbing the exact
 * direct path uses (no counterpart in the paper): D = A * B^T with M = 128,
 * A and B rounded to BF16, FP32 accumulation in tensor memory.
 *   A_host : host float[128][K]; B_host : host float[N][K]; D_host : host float[128][N]
 *   N a multiple of 32 in [32, 256]; K a multiple of 16 in [16, 256].
 * GH_ETIMEOUT if the completion barrier does not arrive within its wait limit.
 */
GH_API int gh_selftest_tcgen05(gh_ctx* ctx, const float* A_host, const float* B_host,
                               float* D_host, int32_t N, int32_t K);

/*
 * gh_selftest_tcgen05_ex - gh_selftest_tcgen05 with a choice of operand
 * layout and of the wait limit (diagnostic; no counterpart in the paper):
 *   layout     : GH_TC_NOSWIZZLE (the canonical K-major layout of 8 x 16-byte
 *                core matrices) or GH_TC_SW128 (K-major, 128-byte swizzle;
 *                K a multiple of 64)
 *   flags      : 0, or GH_TC_SKIP_MMA: no MMA and no commit are issued, so
 *                nothing arrives on the completion barrier; the kernel's
 *                bounded wait gives up after wait_polls polls, the kernel frees
 *                its tensor memory, and the call returns GH_ETIMEOUT with the
 *                context still usable (the test of that failure path)
 *   wait_polls : polls of the completion barrier before giving up (0: the
 *                library's default, 2^22)
 * D_host is written only when the wait succeeds.
 */
#define GH_TC_NOSWIZZLE 0
#define GH_TC_SW128     1
#define GH_TC_SKIP_MMA  1
GH_API int gh_selftest_tcgen05_ex(gh_ctx* ctx, const float* A_host, const float* B_host,
                                  float* D_host, int32_t N, int32_t K, int32_t layout,
                                  int32_t flags, int32_t wait_polls);

/*
 * gh_probe_read_bandwidth - diagnostic read-bandwidth probe (no counterpart in
 * the paper): streams 16-byte loads over a device buffer of `bytes` bytes
 * (1 MiB .. 64 GiB), `reps` times (1 .. 1000), and returns GB/s in *gbs. A
 * buffer well below the L2 size measures L2-to-SM bandwidth; one well above it
 * measures DRAM read bandwidth. Allocates its buffer in the context workspace
 * (a growth drops the context's recorded gh_detect graphs).
 */
GH_API int gh_probe_read_bandwidth(gh_ctx* ctx, int64_t bytes, int32_t reps, double* gbs);

/*
 * gh_probe_smem_bandwidth - diagnostic (no counterpart in the paper): shared-
 * memory load bandwidth of the GPU in GB/s (conflict-free 16-byte loads, 64
 * warps per SM, every SM).
 * gh_probe_issue_rate - diagnostic: warp instructions issued per second by
 * the whole GPU for a stream of independent FP32 FMAs (the issue limit that
 * bounds an instruction-bound kernel).
 */
GH_API int gh_probe_smem_bandwidth(gh_ctx* ctx, double* gbs);
GH_API int gh_probe_issue_rate(gh_ctx* ctx, double* warp_inst_per_s);

/*
 * gh_inject_fault - host-side fault injection for testing the failure paths
 * (no counterpart in the paper; nothing faults on the GPU). Arms one fault
 * of `status` on the context: the (after + 1)-th site of that kind reached
 * by later calls reports it, then the fault is disarmed.
 *   GH_ENOMEM   : a workspace or pinned-buffer acquisition fails
 *   GH_ECUDA    : a kernel-launch check reports a failure (the kernel itself
 *                 was launched and runs)
 *   GH_ETIMEOUT : the device status word read after a synchronising call
 *                 reports a bounded wait that gave up (gh_make_maps has no
 *                 such read)
 *   GH_OK       : disarms an armed fault
 * The call that meets the fault returns its status with the message in
 * gh_last_error; the context stays usable (no partial state survives into
 * the next call). after >= 0.
 */
GH_API int gh_inject_fault(gh_ctx* ctx, int32_t status, int32_t after);

/*
 * Instrumentation. gh_set_timing(ctx, mask) brackets every launch of the
 * kernel classes whose bit (1 << GH_K_*) is set in `mask` with CUDA events on
 * the context's stream (mask 0: off; -1: all classes). gh_kernel_stats
 * returns, for kernel class `kind`, the summed device time of the timed
 * launches [ms] and their count (it synchronises the stream).
 * gh_reset_stats clears both. gh_launch_count returns the number of kernels
 * the context has launched.
 */
GH_API int     gh_set_timing(gh_ctx* ctx, int32_t mask);
/* gh_set_graphs(ctx, 1) (the default) lets gh_detect record its launch
 * sequence into a CUDA graph on the second call with an unchanged
 * configuration (method, radar, grid, positions, Q, K, measurement address,
 * timing mask; device or pinned-host measurement) and replay it afterwards.
 * The graph is dropped when any workspace buffer is reallocated. 0 disables. */
GH_API int     gh_set_graphs(gh_ctx* ctx, int32_t enable);
GH_API int     gh_kernel_stats(gh_ctx* ctx, int32_t kind, double* ms_total, int64_t* launches);
GH_API int     gh_reset_stats(gh_ctx* ctx);
GH_API int64_t gh_launch_count(const gh_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GH_H */
