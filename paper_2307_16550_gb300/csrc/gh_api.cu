// C-ABI entry points of libgh: argument validation, context and workspace
// management, launch bookkeeping and the orchestration of the kernels.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <cmath>

#include "gh_internal.cuh"

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
int gh_fail(gh_ctx* ctx, int status, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return status;
}

int gh_fail_cuda(gh_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    gh_fail(ctx, GH_ECUDA, "%s: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
    return e == cudaErrorMemoryAllocation ? GH_ENOMEM : GH_ECUDA;
}

#ifndef GH_BUILD_ID
#define GH_BUILD_ID "unknown"
#endif
extern "C" const char* gh_build_id(void) { return GH_BUILD_ID; }

extern "C" const char* gh_status_str(int32_t status) {
    switch (status) {
        case GH_OK: return "ok";
        case GH_EINVAL: return "invalid argument";
        case GH_ENOMEM: return "out of memory";
        case GH_ECUDA: return "CUDA error";
        case GH_ETIMEOUT: return "device wait timed out";
        case GH_ENOTSUP: return "unsupported";
        default: return "unknown status";
    }
}

extern "C" const char* gh_last_error(const gh_ctx* ctx) { return ctx ? ctx->err : "null context"; }

// ---------------------------------------------------------------------------
// Host-side fault injection: the failure paths of the entry points are
// exercised without a GPU fault. Sites: workspace and pinned-buffer
// acquisitions (GH_ENOMEM), kernel-launch checks (GH_ECUDA) and the read of
// the device status word (GH_ETIMEOUT).
// ---------------------------------------------------------------------------
bool gh_fault_hit(gh_ctx* ctx, int status) {
    if (!ctx || ctx->fault_status == 0 || ctx->fault_status != status) return false;
    if (ctx->fault_after > 0) {
        --ctx->fault_after;
        return false;
    }
    ctx->fault_status = 0;
    return true;
}

extern "C" int gh_inject_fault(gh_ctx* ctx, int32_t status, int32_t after) {
    if (!ctx) return GH_EINVAL;
    if (status != GH_OK && status != GH_ENOMEM && status != GH_ECUDA && status != GH_ETIMEOUT)
        return gh_fail(ctx, GH_EINVAL, "cannot inject status %d", status);
    if (after < 0) return gh_fail(ctx, GH_EINVAL, "after must be >= 0");
    ctx->fault_status = status;
    ctx->fault_after = after;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// Device guard: makes the context's device current for the duration of a call.
// ---------------------------------------------------------------------------


// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
extern "C" int gh_create(gh_ctx** out, int32_t device, void* stream) {
    if (!out) return GH_EINVAL;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return GH_ECUDA;
    if (device < 0 || device >= ndev) return GH_EINVAL;
    gh_ctx* ctx = new (std::nothrow) gh_ctx();
    if (!ctx) return GH_ENOMEM;
    ctx->device = device;
    DeviceGuard g(device);
    if (!g.ok) {
        delete ctx;
        return GH_ECUDA;
    }
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete ctx;
        return GH_ECUDA;
    }
    ctx->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) {
        delete ctx;
        return GH_ECUDA;
    }
    ctx->smem_optin = (size_t)v;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return GH_ECUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return GH_OK;
}

extern "C" void gh_destroy(gh_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    gh_graph_invalidate(ctx);
    gh_batch_release(ctx);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    for (auto& t : ctx->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
    for (int i = 0; i < WS_COUNT; ++i)
        if (ctx->ws[i]) cudaFree(ctx->ws[i]);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

static void graph_entry_free(GraphEntry& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (auto& t : g.events) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    g.events.clear();
}

void gh_graph_invalidate(gh_ctx* ctx) {
    for (auto& g : ctx->graph_cache) graph_entry_free(g);
    ctx->graph_cache.clear();
    ctx->seen_keys.clear();
}

int gh_ws(gh_ctx* ctx, WsSlot slot, size_t bytes, void** p) {
    if (gh_fault_hit(ctx, GH_ENOMEM)) return gh_fail(ctx, GH_ENOMEM, "injected fault: workspace acquisition refused");
    if (bytes == 0) bytes = 256;
    if (ctx->ws_bytes[slot] < bytes) {
        if (ctx->capturing) return gh_fail(ctx, GH_ECUDA, "workspace growth during graph capture");
        gh_graph_invalidate(ctx);
        if (ctx->ws[slot]) {
            GH_CUDA(cudaStreamSynchronize(ctx->stream));
            GH_CUDA(cudaFree(ctx->ws[slot]));
            ctx->ws[slot] = nullptr;
            ctx->ws_bytes[slot] = 0;
        }
        size_t want = (bytes + 4095) & ~(size_t)4095;
        GH_CUDA(cudaMalloc(&ctx->ws[slot], want));
        ctx->ws_bytes[slot] = want;
        if (slot == WS_TWIDDLE) ctx->tw_n[0] = ctx->tw_n[1] = 0;
    }
    *p = ctx->ws[slot];
    return GH_OK;
}

int gh_pinned(gh_ctx* ctx, size_t bytes, void** p) {
    if (gh_fault_hit(ctx, GH_ENOMEM)) return gh_fail(ctx, GH_ENOMEM, "injected fault: pinned buffer refused");
    if (ctx->pinned_bytes < bytes) {
        if (ctx->capturing) return gh_fail(ctx, GH_ECUDA, "pinned buffer growth during graph capture");
        gh_graph_invalidate(ctx);
        if (ctx->pinned) {
            GH_CUDA(cudaStreamSynchronize(ctx->stream));
            cudaFreeHost(ctx->pinned);
            ctx->pinned = nullptr;
            ctx->pinned_bytes = 0;
        }
        size_t want = (bytes + 4095) & ~(size_t)4095;
        GH_CUDA(cudaMallocHost(&ctx->pinned, want));
        ctx->pinned_bytes = want;
    }
    *p = ctx->pinned;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// Launch bookkeeping
// ---------------------------------------------------------------------------
static cudaEvent_t take_event(gh_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t ev = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
    return ev;
}

// While a graph is being captured the timing events become event-record
// nodes of the graph (external records), so every replay times its kernels.
static void record_event(gh_ctx* ctx, cudaEvent_t ev) {
    cudaEventRecordWithFlags(ev, ctx->stream, ctx->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

void gh_launch_begin(gh_ctx* ctx, int kind, cudaEvent_t* start) {
    *start = nullptr;
    if (!((ctx->timing >> kind) & 1u)) return;
    *start = take_event(ctx);
    if (*start) record_event(ctx, *start);
}

int gh_launch_end(gh_ctx* ctx, int kind, cudaEvent_t start, const char* name) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && gh_fault_hit(ctx, GH_ECUDA)) {
        if (start) ctx->event_pool.push_back(start);
        ctx->launches++;  // the kernel did launch
        return gh_fail(ctx, GH_ECUDA, "injected fault: launch of %s reported as failed", name);
    }
    if (e != cudaSuccess) {
        if (start) ctx->event_pool.push_back(start);
        return gh_fail_cuda(ctx, e, name, __FILE__, __LINE__);
    }
    ctx->launches++;
    if (start) {
        cudaEvent_t stop = take_event(ctx);
        if (stop) {
            record_event(ctx, stop);
            ctx->pending.push_back({kind, start, stop});
        } else {
            ctx->event_pool.push_back(start);
        }
    }
    return GH_OK;
}

static int drain_timing(gh_ctx* ctx) {
    if (ctx->pending.empty()) return GH_OK;
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    for (auto& t : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            ctx->ms[t.kind] += ms;
            ctx->nlaunch[t.kind] += 1;
        }
        ctx->event_pool.push_back(t.start);
        ctx->event_pool.push_back(t.stop);
    }
    ctx->pending.clear();
    return GH_OK;
}

extern "C" int gh_set_timing(gh_ctx* ctx, int32_t mask) {
    if (!ctx) return GH_EINVAL;
    ctx->timing = (uint32_t)mask;
    return GH_OK;
}

// Common checks of the continuous-point entry points.
static int points_prologue(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_dev,
                           int32_t Q, const void* maps_dev, int32_t map_dtype, const double* points_dev, int64_t P,
                           Dims* d, GeoParams* geo) {
    GH_TRY(gh_check_radar(ctx, radar, Q, d));
    if (!tx_host || !std::isfinite(tx_host[0]) || !std::isfinite(tx_host[1]))
        return gh_fail(ctx, GH_EINVAL, "tx_host must hold two finite values");
    if (!gh_map_dtype_ok(map_dtype)) return gh_fail(ctx, GH_EINVAL, "map_dtype %d unknown", map_dtype);
    if (P < 0) return gh_fail(ctx, GH_EINVAL, "P must be >= 0");
    if (!rx_dev || !maps_dev || (P > 0 && !points_dev))
        return gh_fail(ctx, GH_EINVAL, "rx_dev, maps_dev and points_dev must be non-NULL");
    for (const void* ptr : {(const void*)rx_dev, maps_dev, (const void*)points_dev}) {
        if (!ptr) continue;
        const int dv = gh_is_device_ptr(ctx, ptr);
        if (dv < 0) return dv;
        if (!dv) return gh_fail(ctx, GH_EINVAL, "rx_dev, maps_dev and points_dev must be device memory");
    }
    double rx0[2 * GH_MAX_Q] = {0};
    gh_fill_geo(geo, radar, tx_host, rx0, Q, nullptr);
    return GH_OK;
}

extern "C" int gh_score_points(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_dev,
                               int32_t Q, const void* maps_dev, int32_t map_dtype, const double* points_dev,
                               int64_t P, float* scores_dev) {
    if (!ctx) return GH_EINVAL;
    DeviceGuard dg(ctx->device);
    Dims d = {};
    GeoParams geo;
    GH_TRY(points_prologue(ctx, radar, tx_host, rx_dev, Q, maps_dev, map_dtype, points_dev, P, &d, &geo));
    if (P > 0 && !scores_dev) return gh_fail(ctx, GH_EINVAL, "scores_dev is NULL");
    return gh_launch_points(ctx, d, geo, maps_dev, map_dtype, rx_dev, points_dev, P, scores_dev);
}

extern "C" int gh_score_points_adjoint(gh_ctx* ctx, const gh_radar* radar, const double* tx_host,
                                       const double* rx_dev, int32_t Q, const void* maps_dev, int32_t map_dtype,
                                       const double* points_dev, int64_t P, const float* dscores_dev,
                                       double* dpoints_dev, double* drx_dev, void* dmaps_dev) {
    if (!ctx) return GH_EINVAL;
    DeviceGuard dg(ctx->device);
    Dims d = {};
    GeoParams geo;
    GH_TRY(points_prologue(ctx, radar, tx_host, rx_dev, Q, maps_dev, map_dtype, points_dev, P, &d, &geo));
    if (P > 0 && !dscores_dev) return gh_fail(ctx, GH_EINVAL, "dscores_dev is NULL");
    if (dmaps_dev && map_dtype != GH_C64)
        return gh_fail(ctx, GH_ENOTSUP, "map gradients need complex float32 maps (GH_C64)");
    return gh_launch_points_adjoint(ctx, d, geo, maps_dev, map_dtype, rx_dev, points_dev, P, dscores_dev,
                                    dpoints_dev, drx_dev, (float2*)dmaps_dev);
}

extern "C" int gh_refine_points(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_dev,
                                int32_t Q, const void* maps_dev, int32_t map_dtype, double* points_dev, int64_t P,
                                int32_t iters, double scale_xy, double scale_v, double step, float* scores_dev) {
    if (!ctx) return GH_EINVAL;
    DeviceGuard dg(ctx->device);
    Dims d = {};
    GeoParams geo;
    GH_TRY(points_prologue(ctx, radar, tx_host, rx_dev, Q, maps_dev, map_dtype, points_dev, P, &d, &geo));
    if (iters < 0 || iters > 100000) return gh_fail(ctx, GH_EINVAL, "iters must be in [0, 100000]");
    if (!(scale_xy > 0.0) || !(scale_v > 0.0) || !(step > 0.0) || !std::isfinite(scale_xy) ||
        !std::isfinite(scale_v) || !std::isfinite(step))
        return gh_fail(ctx, GH_EINVAL, "scale_xy, scale_v and step must be finite and > 0");
    return gh_launch_refine(ctx, d, geo, maps_dev, map_dtype, rx_dev, points_dev, P, iters, scale_xy, scale_v, step,
                            scores_dev);
}

extern "C" int gh_set_detect_maps(gh_ctx* ctx, int32_t map_dtype) {
    if (!ctx) return GH_EINVAL;
    if (!gh_map_dtype_ok(map_dtype)) return gh_fail(ctx, GH_EINVAL, "map_dtype %d unknown", map_dtype);
    ctx->detect_maps = map_dtype;
    return GH_OK;
}

extern "C" int gh_set_graphs(gh_ctx* ctx, int32_t enable) {
    if (!ctx) return GH_EINVAL;
    ctx->graphs = enable != 0;
    if (!ctx->graphs) {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        gh_graph_invalidate(ctx);
    }
    return GH_OK;
}

extern "C" int gh_kernel_stats(gh_ctx* ctx, int32_t kind, double* ms_total, int64_t* launches) {
    if (!ctx || kind < 0 || kind >= GH_K_COUNT) return GH_EINVAL;
    DeviceGuard g(ctx->device);
    GH_TRY(drain_timing(ctx));
    if (ms_total) *ms_total = ctx->ms[kind];
    if (launches) *launches = ctx->nlaunch[kind];
    return GH_OK;
}

extern "C" int gh_reset_stats(gh_ctx* ctx) {
    if (!ctx) return GH_EINVAL;
    DeviceGuard g(ctx->device);
    GH_TRY(drain_timing(ctx));
    for (int i = 0; i < GH_K_COUNT; ++i) {
        ctx->ms[i] = 0;
        ctx->nlaunch[i] = 0;
    }
    return GH_OK;
}

extern "C" int64_t gh_launch_count(const gh_ctx* ctx) { return ctx ? ctx->launches : -1; }

// ---------------------------------------------------------------------------
// Validation
// ---------------------------------------------------------------------------
static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int gh_check_radar(gh_ctx* ctx, const gh_radar* r, int32_t Q, Dims* d) {
    if (!r) return gh_fail(ctx, GH_EINVAL, "radar is NULL");
    if (Q < 1 || Q > GH_MAX_Q) return gh_fail(ctx, GH_EINVAL, "Q=%d outside [1, %d]", Q, GH_MAX_Q);
    if (!is_pow2(r->Ms) || r->Ms < GH_MIN_M || r->Ms > GH_MAX_M)
        return gh_fail(ctx, GH_EINVAL, "Ms=%d must be a power of two in [%d, %d]", r->Ms, GH_MIN_M, GH_MAX_M);
    if (!is_pow2(r->Mc) || r->Mc < GH_MIN_M || r->Mc > GH_MAX_M)
        return gh_fail(ctx, GH_EINVAL, "Mc=%d must be a power of two in [%d, %d]", r->Mc, GH_MIN_M, GH_MAX_M);
    if (!is_pow2(r->pad) || r->pad > 16)
        return gh_fail(ctx, GH_EINVAL, "pad=%d must be a power of two in [1, 16]", r->pad);
    if ((int64_t)r->pad * r->Ms > GH_MAX_NFFT || (int64_t)r->pad * r->Mc > GH_MAX_NFFT)
        return gh_fail(ctx, GH_EINVAL, "pad*Ms and pad*Mc must be at most %d", GH_MAX_NFFT);
    if (r->reserved != 0) return gh_fail(ctx, GH_EINVAL, "radar.reserved must be 0");
    if (!(r->f0 > 0) || !(r->B > 0) || !(r->Tc > 0) || !isfinite(r->f0) || !isfinite(r->B) || !isfinite(r->Tc))
        return gh_fail(ctx, GH_EINVAL, "f0, B, Tc must be finite and positive");
    d->Q = Q;
    d->Ms = r->Ms;
    d->Mc = r->Mc;
    d->pad = r->pad;
    d->Nr = r->pad * r->Ms;
    d->Nd = r->pad * r->Mc;
    return GH_OK;
}

int gh_check_grid(gh_ctx* ctx, const gh_grid* g, Dims* d) {
    if (!g) return gh_fail(ctx, GH_EINVAL, "grid is NULL");
    int64_t cells = 1;
    for (int a = 0; a < 4; ++a) {
        if (g->n[a] < 1) return gh_fail(ctx, GH_EINVAL, "grid.n[%d]=%d must be >= 1", a, g->n[a]);
        if (!(g->step[a] > 0) || !isfinite(g->step[a]) || !isfinite(g->lo[a]))
            return gh_fail(ctx, GH_EINVAL, "grid.step[%d] must be finite and > 0, lo finite", a);
        if (cells > ((int64_t)1 << 62) / g->n[a]) return gh_fail(ctx, GH_EINVAL, "grid has >= 2^62 cells");
        cells *= g->n[a];
    }
    d->nx = g->n[0];
    d->ny = g->n[1];
    d->nvx = g->n[2];
    d->nvy = g->n[3];
    d->nxy = (int64_t)g->n[0] * g->n[1];
    d->nv = (int64_t)g->n[2] * g->n[3];
    d->ncells = cells;
    return GH_OK;
}

int gh_check_positions(gh_ctx* ctx, const double* tx, const double* rx, int32_t Q) {
    if (!tx || !rx) return gh_fail(ctx, GH_EINVAL, "tx or rx is NULL");
    for (int i = 0; i < 2; ++i)
        if (!isfinite(tx[i])) return gh_fail(ctx, GH_EINVAL, "tx not finite");
    for (int i = 0; i < 2 * Q; ++i)
        if (!isfinite(rx[i])) return gh_fail(ctx, GH_EINVAL, "rx not finite");
    return GH_OK;
}

int gh_is_device_ptr(gh_ctx* ctx, const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gh_fail(ctx, GH_EINVAL, "cannot classify pointer %p: %s", p, cudaGetErrorString(e));
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        if (at.device != ctx->device && at.type == cudaMemoryTypeDevice)
            return gh_fail(ctx, GH_EINVAL, "device pointer belongs to device %d, context is on %d", at.device,
                           ctx->device);
        return 1;
    }
    return 0;
}

void gh_fill_geo(GeoParams* g, const gh_radar* radar, const double* tx, const double* rx, int32_t Q,
                 const gh_grid* grid) {
    memset(g, 0, sizeof(*g));
    g->tx[0] = tx[0];
    g->tx[1] = tx[1];
    for (int i = 0; i < 2 * Q; ++i) g->rx[i] = rx[i];
    volatile double c = GH_C_LIGHT;  // keep the two roundings of (B*d)/(c*Ms) and (f0*Tc)/c
    g->B = radar->B;
    g->cMs = c * (double)radar->Ms;
    double f0Tc = radar->f0 * radar->Tc;
    g->kappa = f0Tc / c;
    if (grid) {
        for (int a = 0; a < 4; ++a) {
            g->lo[a] = grid->lo[a];
            g->step[a] = grid->step[a];
            g->n[a] = grid->n[a];
        }
    }
    g->Q = Q;
    g->Ms = radar->Ms;
    g->Mc = radar->Mc;
    g->Nr = radar->pad * radar->Ms;
    g->Nd = radar->pad * radar->Mc;
}

// Stages a host-or-device measurement in device memory.
static int stage_Y(gh_ctx* ctx, const Dims& d, const void* Y, const float2** Ydev) {
    if (!Y) return gh_fail(ctx, GH_EINVAL, "Y is NULL");
    int dev = gh_is_device_ptr(ctx, Y);
    if (dev < 0) return dev;
    if (dev) {
        *Ydev = (const float2*)Y;
        return GH_OK;
    }
    size_t bytes = (size_t)d.Q * d.Mc * d.Ms * sizeof(float2);
    void* p;
    GH_TRY(gh_ws(ctx, WS_Y, bytes, &p));
    GH_CUDA(cudaMemcpyAsync(p, Y, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *Ydev = (const float2*)p;
    return GH_OK;
}

// The result workspace holds kResultSlots ArgResults; the last slot's first
// int is the device status word written by kernels with bounded waits.
constexpr int kResultSlots = 64;

int* gh_status_dev(gh_ctx* ctx) { return (int*)((ArgResult*)ctx->ws[WS_RESULT] + (kResultSlots - 1)); }

int gh_status_reset(gh_ctx* ctx) {
    GH_CUDA(cudaMemsetAsync(gh_status_dev(ctx), 0, sizeof(int), ctx->stream));
    return GH_OK;
}

static int check_status(gh_ctx* ctx, const ArgResult* host_slots) {
    int st = *(const int*)(host_slots + (kResultSlots - 1));
    if (st == 0 && gh_fault_hit(ctx, GH_ETIMEOUT)) st = GH_ETIMEOUT;
    if (st != 0) return gh_fail(ctx, st, "a device-side wait gave up (status %d)", st);
    return GH_OK;
}

// Copies the whole result block (results and status word) to pinned memory.
static int read_result(gh_ctx* ctx, const ArgResult* res, int64_t* best_cell, float* best_score) {
    void* h;
    GH_TRY(gh_pinned(ctx, kResultSlots * sizeof(ArgResult), &h));
    GH_CUDA(cudaMemcpyAsync(h, ctx->ws[WS_RESULT], kResultSlots * sizeof(ArgResult), cudaMemcpyDeviceToHost,
                            ctx->stream));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    GH_TRY(check_status(ctx, (const ArgResult*)h));
    const ArgResult* r = (const ArgResult*)h + (res - (const ArgResult*)ctx->ws[WS_RESULT]);
    if (best_cell) *best_cell = r->cell;
    if (best_score) *best_score = r->score;
    return GH_OK;
}

// ---------------------------------------------------------------------------
// Entry points
// ---------------------------------------------------------------------------
extern "C" int gh_make_maps(gh_ctx* ctx, const gh_radar* radar, int32_t Q, const void* Y_dev, void* maps_dev,
                            int32_t map_dtype) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    if (!Y_dev || !maps_dev) return gh_fail(ctx, GH_EINVAL, "Y_dev or maps_dev is NULL");
    if (!gh_map_dtype_ok(map_dtype)) return gh_fail(ctx, GH_EINVAL, "map_dtype %d unknown", map_dtype);
    DeviceGuard g(ctx->device);
    int dv = gh_is_device_ptr(ctx, Y_dev);
    if (dv < 0) return dv;
    int dm = gh_is_device_ptr(ctx, maps_dev);
    if (dm < 0) return dm;
    if (!dv || !dm) return gh_fail(ctx, GH_EINVAL, "Y_dev and maps_dev must be device memory");
    return gh_launch_maps(ctx, d, (const float2*)Y_dev, nullptr, maps_dev, map_dtype);
}

// Coordinate table; with rowlim, also the per-receiver bounds of the map rows
// it reads (stored after the table).
// Coordinate table; optionally also the map row bounds (rowlim) and the
// float64 (r, wx, wy) of every entry (rw), after the table in WS_TABLE.
static int build_table(gh_ctx* ctx, const Dims& d, const GeoParams& geo, void** table, int** rowlim = nullptr,
                       double** rw = nullptr) {
    const size_t tb = (gh_hop_table_bytes(d) + 255) & ~(size_t)255;
    const size_t lb = 2 * GH_MAX_Q * sizeof(int);
    const size_t rb = rw ? (size_t)d.nxy * d.Q * 3 * sizeof(double) : 0;
    GH_TRY(gh_ws(ctx, WS_TABLE, tb + lb + rb, table));
    int* lim = rowlim ? (int*)((char*)*table + tb) : nullptr;
    if (rowlim) *rowlim = lim;
    double* r = rw ? (double*)((char*)*table + tb + lb) : nullptr;
    if (rw) *rw = r;
    return gh_launch_coord(ctx, d, geo, *table, nullptr, nullptr, nullptr, nullptr, lim, r);
}

extern "C" int gh_score_grid(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_host,
                             int32_t Q, const void* maps_dev, int32_t map_dtype, const gh_grid* grid,
                             float* scores_dev, int64_t* best_cell, float* best_score) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_grid(ctx, grid, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    if (!maps_dev) return gh_fail(ctx, GH_EINVAL, "maps_dev is NULL");
    if (!gh_map_dtype_ok(map_dtype)) return gh_fail(ctx, GH_EINVAL, "map_dtype %d unknown", map_dtype);
    DeviceGuard dg(ctx->device);
    int dm = gh_is_device_ptr(ctx, maps_dev);
    if (dm < 0) return dm;
    if (!dm) return gh_fail(ctx, GH_EINVAL, "maps_dev must be device memory");
    if (scores_dev) {
        int ds = gh_is_device_ptr(ctx, scores_dev);
        if (ds < 0) return ds;
        if (!ds) return gh_fail(ctx, GH_EINVAL, "scores_dev must be device memory");
    }
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, grid);
    void* table;
    GH_TRY(build_table(ctx, d, geo, &table));
    void* res;
    GH_TRY(gh_ws(ctx, WS_RESULT, kResultSlots * sizeof(ArgResult), &res));
    GH_TRY(gh_status_reset(ctx));
    GH_TRY(gh_launch_hop(ctx, d, geo, maps_dev, map_dtype, table, scores_dev, nullptr, 0, (ArgResult*)res));
    if (!best_cell && !best_score) return GH_OK;
    return read_result(ctx, (const ArgResult*)res, best_cell, best_score);
}

extern "C" int gh_direct_exact(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_host,
                               int32_t Q, const void* Y, const gh_grid* grid, float* scores_dev,
                               int64_t* best_cell, float* best_score) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_grid(ctx, grid, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    DeviceGuard dg(ctx->device);
    if (scores_dev) {
        int ds = gh_is_device_ptr(ctx, scores_dev);
        if (ds < 0) return ds;
        if (!ds) return gh_fail(ctx, GH_EINVAL, "scores_dev must be device memory");
    }
    const float2* Yd;
    GH_TRY(stage_Y(ctx, d, Y, &Yd));
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, grid);
    void* res;
    GH_TRY(gh_ws(ctx, WS_RESULT, kResultSlots * sizeof(ArgResult), &res));
    GH_TRY(gh_status_reset(ctx));
    GH_TRY(gh_launch_exact(ctx, d, geo, Yd, scores_dev, nullptr, 0, (ArgResult*)res));
    return read_result(ctx, (const ArgResult*)res, best_cell, best_score);
}

// The gh_detect launch sequence (from the staged measurement to the results
// copied into pinned host memory); recorded into a CUDA graph when capturing.
static int detect_sequence(gh_ctx* ctx, int32_t method, const Dims& d, const GeoParams& geo, const void* Y,
                           int Ydev, int K, void** host_out) {
    const float2* Yd;
    if (Ydev) {
        Yd = (const float2*)Y;
    } else {
        size_t bytes = (size_t)d.Q * d.Mc * d.Ms * sizeof(float2);
        void* p;
        GH_TRY(gh_ws(ctx, WS_Y, bytes, &p));
        GH_CUDA(cudaMemcpyAsync(p, Y, bytes, cudaMemcpyHostToDevice, ctx->stream));
        Yd = (const float2*)p;
    }
    size_t mbytes = (size_t)d.Q * d.Nr * d.Nd * gh_map_bin_bytes(ctx->detect_maps);
    void *maps = nullptr, *table = nullptr, *res, *bws;
    GH_TRY(gh_ws(ctx, WS_RESULT, kResultSlots * sizeof(ArgResult), &res));
    GH_TRY(gh_ws(ctx, WS_BOMP, gh_bomp_ws_bytes(d, K), &bws));
    int64_t* mask;  // selected cells, excluded from later argmaxes
    GH_TRY(gh_ws(ctx, WS_DIAG, (size_t)GH_MAX_K * sizeof(int64_t) + 256, (void**)&mask));
    if (method == GH_HOP) GH_TRY(gh_ws(ctx, WS_MAPS, mbytes, &maps));
    size_t sel_bytes = (size_t)kResultSlots * sizeof(ArgResult);
    size_t alpha_bytes = (size_t)K * d.Q * 2 * sizeof(double);
    void* h;
    GH_TRY(gh_pinned(ctx, sel_bytes + alpha_bytes, &h));
    GH_TRY(gh_status_reset(ctx));
    GH_TRY(gh_bomp_reset(ctx, d, K, bws));
    int* rowlim = nullptr;  // map rows the scorer can read: the Doppler FFT skips the others
    double* rw = nullptr;   // (r, wx, wy) per coordinate entry, for the new atoms
    if (method == GH_HOP) GH_TRY(build_table(ctx, d, geo, &table, &rowlim, &rw));
    ArgResult* sel = (ArgResult*)res;  // sel[k] = selection of iteration k
    for (int k = 0; k < K; ++k) {
        // the residual of iteration k subtracts atoms 0..k-1 (amplitudes of the last solve)
        const Deflate df = gh_bomp_deflate(bws, d, K, k);
        ArgPartial* parts;
        int nparts;
        if (method == GH_HOP) {
            if (k > 0 && ctx->detect_maps == GH_C64)  // residual maps by linearity, in place
                GH_TRY(gh_launch_maps_deflate(ctx, d, df, maps, rowlim));
            else
                GH_TRY(gh_launch_maps(ctx, d, Yd, &df, maps, ctx->detect_maps, rowlim));
            GH_TRY(gh_launch_hop_parts(ctx, d, geo, maps, ctx->detect_maps, table, nullptr, mask, k, &parts,
                                       &nparts));
        } else {
            GH_TRY(gh_launch_exact_parts(ctx, d, geo, Yd, &df, nullptr, mask, k, &parts, &nparts));
        }
        GH_TRY(gh_launch_bomp_step(ctx, d, geo, parts, nparts, Yd, sel, mask, k, K, bws, rw));
    }
    // results: selections, status word and the final amplitudes (double2 [K][Q]
    // at the start of the BOMP workspace)
    GH_CUDA(cudaMemcpyAsync(h, sel, sel_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaMemcpyAsync((char*)h + sel_bytes, bws, alpha_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    *host_out = h;
    return GH_OK;
}

static void key_append(std::vector<unsigned char>& k, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    k.insert(k.end(), b, b + n);
}

static GraphEntry* find_graph(gh_ctx* ctx, const std::vector<unsigned char>& key) {
    for (auto& g : ctx->graph_cache)
        if (g.key == key) {
            g.used = ++ctx->graph_tick;
            return &g;
        }
    return nullptr;
}

static bool seen_before(gh_ctx* ctx, const std::vector<unsigned char>& key) {
    for (auto& k : ctx->seen_keys)
        if (k == key) return true;
    return false;
}

// Runs the launch sequence of one configuration (this call's results), then
// records it into a new cache entry without running it again (evicting the
// least recently used entry when the cache is full).
static int record_graph(gh_ctx* ctx, const std::vector<unsigned char>& key, const GhSequence& seq, void** h) {
    // the plain run makes sure every buffer of this configuration exists, so
    // that the capture allocates nothing (a growth would drop all graphs)
    GH_TRY(seq(h));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    if ((int)ctx->graph_cache.size() >= kMaxGraphs) {
        size_t lru = 0;
        for (size_t i = 1; i < ctx->graph_cache.size(); ++i)
            if (ctx->graph_cache[i].used < ctx->graph_cache[lru].used) lru = i;
        graph_entry_free(ctx->graph_cache[lru]);
        ctx->graph_cache.erase(ctx->graph_cache.begin() + lru);
    }
    if (!ctx->capture_stream) GH_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    const int64_t n0 = ctx->launches;
    const size_t p0 = ctx->pending.size();
    // recorded on a private stream, launched on the context's stream
    cudaStream_t user_stream = ctx->stream;
    GH_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeRelaxed));
    ctx->stream = ctx->capture_stream;
    ctx->capturing = true;
    void* h2 = nullptr;
    const int st = seq(&h2);
    ctx->capturing = false;
    ctx->stream = user_stream;
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->capture_stream, &graph);
    GraphEntry e;
    e.key = key;
    // events recorded while capturing are nodes of the graph now
    e.events.assign(ctx->pending.begin() + p0, ctx->pending.end());
    ctx->pending.resize(p0);
    e.launches = ctx->launches - n0;
    ctx->launches = n0;  // the capture ran nothing; replays count their kernels
    int rc = st;
    if (rc == GH_OK && ec != cudaSuccess) rc = gh_fail_cuda(ctx, ec, "cudaStreamEndCapture", __FILE__, __LINE__);
    if (rc == GH_OK && h2 != *h) rc = gh_fail(ctx, GH_ECUDA, "graph capture moved the result buffer");
    if (rc == GH_OK) {
        const cudaError_t ei = cudaGraphInstantiate(&e.exec, graph, 0);
        if (ei != cudaSuccess) {
            e.exec = nullptr;
            rc = gh_fail_cuda(ctx, ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
    }
    if (graph) cudaGraphDestroy(graph);
    if (rc != GH_OK) {
        graph_entry_free(e);
        return rc;
    }
    e.used = ++ctx->graph_tick;
    ctx->graph_cache.push_back(std::move(e));
    return GH_OK;
}

int gh_run_sequence(gh_ctx* ctx, const std::vector<unsigned char>* key, const GhSequence& seq, void** h) {
    GraphEntry* g = key ? find_graph(ctx, *key) : nullptr;
    if (g) {
        GH_CUDA(cudaGraphLaunch(g->exec, ctx->stream));
        ctx->launches += g->launches;
        *h = ctx->pinned;
    } else if (key && seen_before(ctx, *key)) {
        GH_TRY(record_graph(ctx, *key, seq, h));
    } else {
        GH_TRY(seq(h));
        if (key) {
            if (ctx->seen_keys.size() >= 4 * kMaxGraphs) ctx->seen_keys.erase(ctx->seen_keys.begin());
            ctx->seen_keys.push_back(*key);
        }
    }
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    if (g) {
        for (auto& t : g->events) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
                ctx->ms[t.kind] += ms;
                ctx->nlaunch[t.kind] += 1;
            }
        }
    }
    return GH_OK;
}

extern "C" int gh_detect(gh_ctx* ctx, int32_t method, const gh_radar* radar, const double* tx_host,
                         const double* rx_host, int32_t Q, const void* Y, const gh_grid* grid, int32_t K,
                         int64_t* cells_host, float* scores_host, double* alpha_host) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_grid(ctx, grid, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    if (method != GH_HOP && method != GH_EXACT) return gh_fail(ctx, GH_EINVAL, "method %d unknown", method);
    if (K < 1 || K > GH_MAX_K || K > d.ncells)
        return gh_fail(ctx, GH_EINVAL, "K=%d outside [1, min(%d, ncells)]", K, GH_MAX_K);
    if (!cells_host) return gh_fail(ctx, GH_EINVAL, "cells_host is NULL");
    if (!Y) return gh_fail(ctx, GH_EINVAL, "Y is NULL");
    DeviceGuard dg(ctx->device);
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, grid);
    const int ydev = gh_is_device_ptr(ctx, Y);
    if (ydev < 0) return ydev;
    bool pinned_host = false;
    if (!ydev) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, Y) == cudaSuccess) pinned_host = at.type == cudaMemoryTypeHost;
        cudaGetLastError();
    }
    // graphs replay fixed addresses: device or pinned-host measurements only
    const bool graphable = ctx->graphs && (ydev || pinned_host);
    std::vector<unsigned char> key;
    if (graphable) {
        key_append(key, &method, sizeof(method));
        key_append(key, radar, sizeof(*radar));
        key_append(key, grid, sizeof(*grid));
        key_append(key, tx_host, 2 * sizeof(double));
        key_append(key, rx_host, 2 * (size_t)Q * sizeof(double));
        key_append(key, &Q, sizeof(Q));
        key_append(key, &K, sizeof(K));
        key_append(key, &Y, sizeof(Y));
        key_append(key, &ctx->timing, sizeof(ctx->timing));
        key_append(key, &ctx->detect_maps, sizeof(ctx->detect_maps));
    }
    void* h = nullptr;
    const GhSequence seq = [&](void** out) { return detect_sequence(ctx, method, d, geo, Y, ydev, K, out); };
    GH_TRY(gh_run_sequence(ctx, graphable ? &key : nullptr, seq, &h));
    const size_t sel_bytes = (size_t)kResultSlots * sizeof(ArgResult);
    const ArgResult* hs = (const ArgResult*)h;
    GH_TRY(check_status(ctx, hs));
    for (int k = 0; k < K; ++k) {
        cells_host[k] = hs[k].cell;
        if (scores_host) scores_host[k] = hs[k].score;
    }
    if (alpha_host) memcpy(alpha_host, (char*)h + sel_bytes, (size_t)K * d.Q * 2 * sizeof(double));
    return GH_OK;
}

extern "C" int gh_synth(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_host,
                        int32_t Q, int32_t T, const double* targets_host, const double* alpha_host,
                        const void* noise_dev, void* Y_dev) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    if (T < 0 || T > 64) return gh_fail(ctx, GH_EINVAL, "T=%d outside [0, 64]", T);
    if (T > 0 && (!targets_host || !alpha_host)) return gh_fail(ctx, GH_EINVAL, "targets or alpha is NULL");
    if (!Y_dev) return gh_fail(ctx, GH_EINVAL, "Y_dev is NULL");
    for (int i = 0; i < 4 * T; ++i)
        if (!isfinite(targets_host[i])) return gh_fail(ctx, GH_EINVAL, "targets not finite");
    DeviceGuard dg(ctx->device);
    int dy = gh_is_device_ptr(ctx, Y_dev);
    if (dy < 0) return dy;
    if (!dy) return gh_fail(ctx, GH_EINVAL, "Y_dev must be device memory");
    if (noise_dev) {
        int dn = gh_is_device_ptr(ctx, noise_dev);
        if (dn < 0) return dn;
        if (!dn) return gh_fail(ctx, GH_EINVAL, "noise_dev must be device memory");
    }
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, nullptr);
    size_t tb = (size_t)T * 4 * sizeof(double), ab = (size_t)T * Q * 2 * sizeof(double);
    void* buf;
    GH_TRY(gh_ws(ctx, WS_DIAG, tb + ab + 256, &buf));
    if (T > 0) {
        void* h;
        GH_TRY(gh_pinned(ctx, tb + ab, &h));
        GH_CUDA(cudaStreamSynchronize(ctx->stream));  // pinned buffer may be in use by an earlier copy
        memcpy(h, targets_host, tb);
        memcpy((char*)h + tb, alpha_host, ab);
        GH_CUDA(cudaMemcpyAsync(buf, h, tb + ab, cudaMemcpyHostToDevice, ctx->stream));
    }
    return gh_launch_synth(ctx, d, geo, T, (const double*)buf, (const float2*)noise_dev, (float2*)Y_dev);
}

extern "C" int gh_coord_table(gh_ctx* ctx, const gh_radar* radar, const double* tx_host, const double* rx_host,
                              int32_t Q, const gh_grid* grid, int32_t* ibin_host, double* tau_host,
                              float* coef_host, double* w_host) {
    if (!ctx) return GH_EINVAL;
    Dims d = {};
    GH_TRY(gh_check_radar(ctx, radar, Q, &d));
    GH_TRY(gh_check_grid(ctx, grid, &d));
    GH_TRY(gh_check_positions(ctx, tx_host, rx_host, Q));
    if (!ibin_host || !tau_host || !coef_host) return gh_fail(ctx, GH_EINVAL, "output is NULL");
    if (d.nxy * d.Q > ((int64_t)1 << 28)) return gh_fail(ctx, GH_EINVAL, "table too large for diagnostics");
    DeviceGuard dg(ctx->device);
    GeoParams geo;
    gh_fill_geo(&geo, radar, tx_host, rx_host, Q, grid);
    size_t n = (size_t)d.nxy * d.Q;
    size_t bytes = n * (sizeof(int32_t) + sizeof(double) + 3 * sizeof(float) + 2 * sizeof(double)) + 1024;
    void *table, *diag;
    GH_TRY(gh_ws(ctx, WS_TABLE, gh_hop_table_bytes(d), &table));
    GH_TRY(gh_ws(ctx, WS_DIAG, bytes, &diag));
    char* p = (char*)diag;
    double* dtau = (double*)p;
    double* dw = dtau + n;
    int32_t* di = (int32_t*)(dw + 2 * n);
    float* dc = (float*)(di + n);
    GH_TRY(gh_launch_coord(ctx, d, geo, table, di, dtau, dc, dw));
    GH_CUDA(cudaMemcpyAsync(ibin_host, di, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaMemcpyAsync(tau_host, dtau, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaMemcpyAsync(coef_host, dc, 3 * n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    if (w_host) GH_CUDA(cudaMemcpyAsync(w_host, dw, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));
    return GH_OK;
}
