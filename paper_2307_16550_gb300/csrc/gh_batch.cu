// gh_detect_batch: the grid-hopping detect-and-deflate loop of gh_detect
// (Sec. IV scores, BOMP iterations) over many independent frames of uneven
// size at once. Every step is one launch for the whole batch:
//   coordinate tables         coord_batch_kernel       (once; also each frame's
//                             map row limits)
//   per iteration k:
//     maps                    k = 0: range_fft_batch_kernel, doppler_fft_batch_kernel;
//                             k > 0: maps_deflate_batch_kernel (the residual's
//                             maps by linearity, as gh_detect does); rows
//                             outside the row limits are skipped
//     scores + argmax         hop_batch_kernel or hop_pair_kernel, one launch per class
//                             (persistent; warps take work items from the
//                             class's counter; per-frame packed argmax)
//     selection, new atom     bomp_select_batch_kernel (one CTA per frame)
//     correlation + solve     bomp_corr_batch_kernel
//   results                   batch_gather_kernel + one copy to the host
// Frames whose K is reached drop out of later iterations. Every frame runs
// the kernels of the single-frame path on the same data in the same order, so
// its results are those of gh_detect bit for bit.
//
// Frames are classed by the shared memory a scorer warp needs (Q * Nd rounded
// up to a power of two), by whether a lane's velocity cells form one run (the
// one-receiver-row mode's condition) and by the lane layout that fits their
// velocity axes best; each class has its own scorer launch per iteration
// (the classes of an iteration on side streams), whose cells per lane, warps
// per CTA, row mode (all receivers' rows, one receiver's row at a time, or
// all rows shared by two warps per (x, y) cell: hop_pair_kernel) and cells
// per work item are picked by timing the
// candidates on the class's first iteration (once per batch shape, cached in
// the context) unless fixed with gh_set_batch_tuning, gh_set_batch_row_mode
// and gh_set_batch_tile. The whole sequence is a CUDA graph from the second
// call with an unchanged batch on (gh_run_sequence).
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <mutex>
#include <vector>

#include "gh_internal.cuh"

namespace {

// (x, y) cells per scorer work item: the tile sizes the autotuner tries
constexpr int kTiles[] = {4, 8, 16, 32};
constexpr int kNumTiles = 4;
constexpr int kDefaultTile = 1;  // 8 cells
constexpr int kBatchMaxFrames = 65536;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Plan {
    std::vector<unsigned char> key;    // whole batch (graph key)
    std::vector<unsigned char> shape;  // sizes only (tuning key)
    int nframes = 0, Kmax = 0, max_q = 0, max_chunks = 0;
    std::vector<int> K;                      // per frame
    std::vector<long long> out_off;          // byte offset of each frame in the packed results
    size_t out_bytes = 0;
    // device pointers (inside WS_BATCH / WS_BATCH_META)
    BatchFrame* frames = nullptr;
    BatchItem *coord_items = nullptr, *range_items = nullptr, *dop_items = nullptr;
    // frames grouped by the shared memory their scorer warps need (Q * Nd
    // rounded up to a power of two, at least 1024 floats): one scorer launch
    // per class and iteration, each sized and tuned for its class
    struct ScoreClass {
        int bound = 0, max_q = 0, max_nd = 0;
        // cells per lane of the frame with the most (one run per lane), or a
        // large value when a frame has nvy > 32: the per-receiver scorer
        // needs ac >= pr_need
        int pr_need = 0;
        int layout_ac = 0;  // 6 or 10: the 8 x 4 lane layout fits the class's frames best
        int layout_run = 0;  // largest ceil(nvx / 4): cells per vy row and lane in the 8 x 4 layout
        double work = 0.0;                    // cell * receiver * iteration evals
        // per tile size: the class's items, frames in decreasing K (so the
        // items of the frames still iterating at k are a prefix), and per k
        // that prefix's length
        BatchItem* items[kNumTiles] = {};
        std::vector<int> n[kNumTiles];
    };
    std::vector<ScoreClass> classes;
    std::vector<int*> active;                // per k
    std::vector<int> n_active;               // per k
    std::vector<BatchItem*> defl_items;      // per k: residual maps by linearity (k >= 1, active frames)
    std::vector<int> n_defl;                 // per k
    int n_coord = 0, n_range = 0, n_dop = 0;
    size_t smem_range = 0, smem_dop = 0;
    int thr_range = 32, thr_dop = 32;  // threads of the FFT kernels (enough for every item)
    unsigned long long* keys = nullptr;      // all frames' keys, contiguous
    size_t keys_bytes = 0;
    unsigned* counter = nullptr;
    long long* out_off_dev = nullptr;
    void* out_dev = nullptr;
};

struct Tuning {
    int ac = 0, warps = 0, tile = kDefaultTile;  // tile: index into kTiles
    bool per_rx = false;                         // one receiver's power row at a time
    bool pair = false;                           // two warps per (x, y) cell (warps = 2, all rows)
};

int class_bound(int q_nd) {
    int b = 1024;
    while (b < q_nd) b <<= 1;
    return b;
}

constexpr int kMaxClasses = 256;  // scorer classes of a batch (shared-memory bound x run x lane layout: far fewer)
constexpr int kSideStreams = 4;  // streams the scorer classes of one iteration run on side by side

// Context-side state of the batch path (one per context).
struct BatchState {
    // side streams and events of the scorer classes' fork and join (created on
    // first use, released with the state)
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork = nullptr, join[kSideStreams] = {};
    ~BatchState() {
        for (int i = 0; i < kSideStreams; ++i) {
            if (side[i]) cudaStreamDestroy(side[i]);
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
    }
    Plan plan;
    bool plan_valid = false;
    int force_ac = 0, force_warps = 0;
    int force_tile = -1;  // index into kTiles, -1: tuned
    int force_rm = -1;    // row mode the autotuner keeps to (0 all rows, 1 one row at a time, 2 paired), -1: any
    Tuning last;                                         // of the class with the most work
    std::map<std::vector<unsigned char>, Tuning> tuned;  // per batch shape and class
};

std::mutex g_state_mu;
std::map<const gh_ctx*, BatchState*> g_state;

BatchState* state_of(gh_ctx* ctx) {
    std::lock_guard<std::mutex> lk(g_state_mu);
    auto it = g_state.find(ctx);
    if (it != g_state.end()) return it->second;
    BatchState* s = new BatchState();
    g_state[ctx] = s;
    return s;
}

template <class T>
void append(std::vector<unsigned char>& k, const T& v) {
    const unsigned char* b = (const unsigned char*)&v;
    k.insert(k.end(), b, b + sizeof(T));
}

int validate(gh_ctx* ctx, int nframes, const gh_frame* frames) {
    if (nframes < 1 || nframes > kBatchMaxFrames)
        return gh_fail(ctx, GH_EINVAL, "nframes=%d outside [1, %d]", nframes, kBatchMaxFrames);
    if (!frames) return gh_fail(ctx, GH_EINVAL, "frames is NULL");
    for (int f = 0; f < nframes; ++f) {
        const gh_frame& fr = frames[f];
        Dims d = {};
        int st = gh_check_radar(ctx, &fr.radar, fr.Q, &d);
        if (st == GH_OK) st = gh_check_grid(ctx, &fr.grid, &d);
        if (st == GH_OK) st = gh_check_positions(ctx, fr.tx, fr.rx, fr.Q);
        if (st != GH_OK) return gh_fail(ctx, st, "frame %d: %s", f, gh_last_error(ctx));
        if (fr.K < 1 || fr.K > GH_MAX_K || fr.K > d.ncells)
            return gh_fail(ctx, GH_EINVAL, "frame %d: K=%d outside [1, min(%d, ncells)]", f, fr.K, GH_MAX_K);
        if (d.ncells >= ((int64_t)1 << 32))
            return gh_fail(ctx, GH_EINVAL, "frame %d: %lld cells (at most 2^32 - 1 per frame)", f,
                           (long long)d.ncells);
        if (!fr.Y) return gh_fail(ctx, GH_EINVAL, "frame %d: Y is NULL", f);
        const int dv = gh_is_device_ptr(ctx, fr.Y);
        if (dv < 0) return dv;
        if (!dv) return gh_fail(ctx, GH_EINVAL, "frame %d: Y must be device memory", f);
    }
    return GH_OK;
}

// Builds the descriptors and work items of a batch and uploads them.
int build_plan(gh_ctx* ctx, int nframes, const gh_frame* frames, Plan& P) {
    P = Plan();
    P.nframes = nframes;
    std::vector<Dims> dims(nframes);
    std::vector<GeoParams> geos(nframes);
    for (int f = 0; f < nframes; ++f) {
        const gh_frame& fr = frames[f];
        GH_TRY(gh_check_radar(ctx, &fr.radar, fr.Q, &dims[f]));
        GH_TRY(gh_check_grid(ctx, &fr.grid, &dims[f]));
        gh_fill_geo(&geos[f], &fr.radar, fr.tx, fr.rx, fr.Q, &fr.grid);
        P.K.push_back(fr.K);
        P.Kmax = std::max(P.Kmax, fr.K);
        P.max_q = std::max(P.max_q, fr.Q);
        P.max_chunks = std::max(P.max_chunks, gh_bomp_chunks(dims[f]));
        // graph key: everything the sequence reads from the host
        append(P.key, fr.radar);
        append(P.key, fr.grid);
        append(P.key, fr.Q);
        append(P.key, fr.K);
        append(P.key, fr.Y);
        P.key.insert(P.key.end(), (const unsigned char*)fr.tx, (const unsigned char*)(fr.tx + 2));
        P.key.insert(P.key.end(), (const unsigned char*)fr.rx, (const unsigned char*)(fr.rx + 2 * fr.Q));
        append(P.shape, fr.radar.Ms);
        append(P.shape, fr.radar.Mc);
        append(P.shape, fr.radar.pad);
        append(P.shape, fr.Q);
        append(P.shape, fr.K);
        P.shape.insert(P.shape.end(), (const unsigned char*)fr.grid.n, (const unsigned char*)(fr.grid.n + 4));
    }
    // per-frame device buffers
    std::vector<size_t> off_zr(nframes), off_maps(nframes), off_tab(nframes), off_bomp(nframes), off_mask(nframes),
        off_sel(nframes), off_key(nframes), off_lim(nframes);
    size_t o = 0, okeys = 0;
    for (int f = 0; f < nframes; ++f) {
        const Dims& d = dims[f];
        const int K = P.K[f];
        off_zr[f] = o;
        o += align256((size_t)d.Q * d.Mc * d.Nr * sizeof(float2));
        off_maps[f] = o;
        o += align256((size_t)d.Q * d.Nr * d.Nd * sizeof(float2));
        off_tab[f] = o;
        o += align256(gh_hop_table_bytes(d));
        off_bomp[f] = o;
        o += align256(gh_bomp_ws_bytes(d, K));
        off_mask[f] = o;
        o += align256((size_t)K * sizeof(int64_t));
        off_sel[f] = o;
        o += align256((size_t)K * sizeof(ArgResult));
        off_lim[f] = o;
        o += align256((size_t)2 * d.Q * sizeof(int));
        off_key[f] = okeys;
        okeys += (size_t)K * sizeof(unsigned long long);
    }
    const size_t keys_off = o;
    o += align256(okeys);
    const size_t counter_off = o;
    o += kMaxClasses * sizeof(unsigned);  // work counters, one per scorer class
    void* big;
    GH_TRY(gh_ws(ctx, WS_BATCH, o, &big));
    char* B = (char*)big;
    P.keys = (unsigned long long*)(B + keys_off);
    P.keys_bytes = okeys;
    P.counter = (unsigned*)(B + counter_off);

    // twiddle tables of every transform size of the batch
    std::map<int, size_t> tw_off;
    size_t ntw = 0;
    for (int f = 0; f < nframes; ++f)
        for (int N : {dims[f].Nr, dims[f].Nd})
            if (!tw_off.count(N)) {
                tw_off[N] = ntw;
                ntw += (size_t)(N / 2);
            }
    std::vector<float2> tw(ntw);
    for (auto& kv : tw_off) gh_twiddles(kv.first, tw.data() + kv.second);

    // work items
    std::vector<BatchItem> coord, range, dop;
    // classes: (shared-memory bound, whether every lane's cells form one run,
    // which the per-receiver scorer needs, and the 8 x 4 lane layout's cells
    // per run when that layout fills the runs best: 6 or 10, else 0)
    auto class_key = [&](const Dims& d) {
        const int NB = d.nvy < 32 ? d.nvy : 32, SA = 32 / NB;
        const bool one_run = d.nvy <= 32 && (d.nvx + SA - 1) / SA <= 32;
        return std::make_tuple(class_bound(d.Q * d.Nd), one_run ? 1 : 0, lane_layout_ac(d));
    };
    std::map<std::tuple<int, int, int>, int> class_of_key;
    for (int f = 0; f < nframes; ++f) class_of_key[class_key(dims[f])] = 0;
    for (auto& kv : class_of_key) {
        kv.second = (int)P.classes.size();
        Plan::ScoreClass c;
        c.bound = std::get<0>(kv.first);
        c.layout_ac = std::get<2>(kv.first);
        P.classes.push_back(c);
    }
    if ((int)P.classes.size() > kMaxClasses)
        return gh_fail(ctx, GH_ENOTSUP, "batch: %zu scorer classes, at most %d", P.classes.size(), kMaxClasses);
    std::vector<std::vector<int>> class_frames(P.classes.size());
    std::vector<std::vector<int>> active(P.Kmax);
    std::vector<std::vector<BatchItem>> defl(P.Kmax);
    for (int f = 0; f < nframes; ++f) {
        const Dims& d = dims[f];
        for (long long s = 0; s < d.nxy; s += 16) coord.push_back({f, 0, s, std::min(16LL, d.nxy - s)});
        const int rpc = gh_fft_rows_per_cta(d.Nr);
        const int rows = d.Q * d.Mc;
        for (int r = 0; r < rows; r += rpc) {
            const int c = std::min(rpc, rows - r);
            range.push_back({f, 0, r, c});
            P.smem_range = std::max(P.smem_range, gh_fft_smem_range(c, d.Nr));
            P.thr_range = std::max(P.thr_range, gh_fft_threads(c * d.Nr));
        }
        const int IB = gh_fft_bins_per_cta(d.Nr, d.Nd);
        for (int q = 0; q < d.Q; ++q)
            for (int i0 = 0; i0 < d.Nr; i0 += IB) dop.push_back({f, q, i0, IB});
        P.smem_dop = std::max(P.smem_dop, gh_fft_smem_dop(IB, d.Nd));
        P.thr_dop = std::max(P.thr_dop, gh_fft_threads(IB * d.Nd));
        const int cls = class_of_key[class_key(d)];
        P.classes[cls].max_q = std::max(P.classes[cls].max_q, d.Q);
        P.classes[cls].max_nd = std::max(P.classes[cls].max_nd, d.Nd);
        P.classes[cls].layout_run = std::max(P.classes[cls].layout_run, (d.nvx + 3) / 4);
        {
            const int NB = d.nvy < 32 ? d.nvy : 32, SA = 32 / NB;
            const int cells = d.nvy <= 32 ? (d.nvx + SA - 1) / SA : (1 << 20);
            P.classes[cls].pr_need = std::max(P.classes[cls].pr_need, cells);
        }
        P.classes[cls].work += (double)d.ncells * d.Q * P.K[f];
        for (int k = 1; k < P.K[f]; ++k)
            for (int q = 0; q < d.Q; ++q)
                for (int i0 = 0; i0 < d.Nr; i0 += IB) defl[k].push_back({f, q, i0, IB});
        for (int k = 0; k < P.K[f]; ++k) active[k].push_back(f);
        class_frames[cls].push_back(f);
    }
    // scorer items per class and tile size: frames in decreasing K (ties in
    // frame order), runs of `tile` consecutive (x, y) cells; n[t][k] = items
    // of the frames with K > k (a prefix)
    std::vector<std::vector<std::vector<BatchItem>>> score(P.classes.size(),
                                                          std::vector<std::vector<BatchItem>>(kNumTiles));
    for (size_t c = 0; c < P.classes.size(); ++c) {
        std::vector<int>& cf = class_frames[c];
        std::stable_sort(cf.begin(), cf.end(), [&](int a, int b) { return P.K[a] > P.K[b]; });
        for (int t = 0; t < kNumTiles; ++t) {
            const long long T = kTiles[t];
            P.classes[c].n[t].assign(P.Kmax, 0);
            for (int f : cf) {
                for (long long s = 0; s < dims[f].nxy; s += T)
                    score[c][t].push_back({f, 0, s, std::min(T, dims[f].nxy - s)});
                for (int k = 0; k < P.K[f]; ++k) P.classes[c].n[t][k] = (int)score[c][t].size();
            }
        }
    }
    // packed results: per frame ArgResult[K] then double2[K][Q]
    for (int f = 0; f < nframes; ++f) {
        P.out_off.push_back((long long)P.out_bytes);
        P.out_bytes += (size_t)P.K[f] * sizeof(ArgResult) + (size_t)P.K[f] * dims[f].Q * 2 * sizeof(double);
    }

    // metadata buffer: frames, items, active lists, twiddles, result offsets, packed results
    size_t m = 0;
    auto take = [&](size_t bytes) {
        const size_t at = m;
        m += align256(bytes);
        return at;
    };
    const size_t m_frames = take(nframes * sizeof(BatchFrame));
    const size_t m_coord = take(coord.size() * sizeof(BatchItem));
    const size_t m_range = take(range.size() * sizeof(BatchItem));
    const size_t m_dop = take(dop.size() * sizeof(BatchItem));
    std::vector<std::vector<size_t>> m_score(P.classes.size(), std::vector<size_t>(kNumTiles));
    for (size_t c = 0; c < P.classes.size(); ++c)
        for (int t = 0; t < kNumTiles; ++t) m_score[c][t] = take(score[c][t].size() * sizeof(BatchItem));
    std::vector<size_t> m_active(P.Kmax), m_defl(P.Kmax);
    for (int k = 0; k < P.Kmax; ++k) {
        m_active[k] = take(active[k].size() * sizeof(int));
        m_defl[k] = take(defl[k].size() * sizeof(BatchItem));
    }
    const size_t m_tw = take(ntw * sizeof(float2));
    const size_t m_outoff = take(nframes * sizeof(long long));
    const size_t m_out = take(P.out_bytes);
    void* meta;
    GH_TRY(gh_ws(ctx, WS_BATCH_META, m, &meta));
    char* M = (char*)meta;
    // workspace pointers are final now (both slots allocated)
    B = (char*)ctx->ws[WS_BATCH];
    P.keys = (unsigned long long*)(B + keys_off);
    P.counter = (unsigned*)(B + counter_off);

    std::vector<unsigned char> host(m, 0);
    auto put = [&](size_t at, const void* src, size_t bytes) {
        if (bytes) memcpy(host.data() + at, src, bytes);
    };
    std::vector<BatchFrame> bf(nframes);
    const float2* twdev = (const float2*)(M + m_tw);
    for (int f = 0; f < nframes; ++f) {
        BatchFrame& F = bf[f];
        memset(&F, 0, sizeof(F));
        F.g = geos[f];
        F.d = dims[f];
        gh_hop_frame_params(dims[f], geos[f], &F.hp, &F.cp);
        void* bomp = B + off_bomp[f];
        F.bw = gh_bomp_ptrs(bomp, dims[f], P.K[f]);
        F.df = gh_bomp_deflate(bomp, dims[f], P.K[f], 0);
        F.K = P.K[f];
        F.Y = (const float2*)frames[f].Y;
        F.zr = (float2*)(B + off_zr[f]);
        F.maps = (float2*)(B + off_maps[f]);
        F.table = B + off_tab[f];
        F.rowlim = (int*)(B + off_lim[f]);
        F.mask = (int64_t*)(B + off_mask[f]);
        F.key = (unsigned long long*)((char*)P.keys + off_key[f]);
        F.sel = (ArgResult*)(B + off_sel[f]);
        F.twr = twdev + tw_off[dims[f].Nr];
        F.twd = twdev + tw_off[dims[f].Nd];
    }
    put(m_frames, bf.data(), nframes * sizeof(BatchFrame));
    put(m_coord, coord.data(), coord.size() * sizeof(BatchItem));
    put(m_range, range.data(), range.size() * sizeof(BatchItem));
    put(m_dop, dop.data(), dop.size() * sizeof(BatchItem));
    for (int k = 0; k < P.Kmax; ++k) {
        put(m_active[k], active[k].data(), active[k].size() * sizeof(int));
        put(m_defl[k], defl[k].data(), defl[k].size() * sizeof(BatchItem));
    }
    for (size_t c = 0; c < P.classes.size(); ++c)
        for (int t = 0; t < kNumTiles; ++t)
            put(m_score[c][t], score[c][t].data(), score[c][t].size() * sizeof(BatchItem));
    put(m_tw, tw.data(), ntw * sizeof(float2));
    put(m_outoff, P.out_off.data(), nframes * sizeof(long long));
    GH_CUDA(cudaMemcpyAsync(meta, host.data(), m, cudaMemcpyHostToDevice, ctx->stream));
    GH_CUDA(cudaStreamSynchronize(ctx->stream));  // host staging goes out of scope

    P.frames = (BatchFrame*)(M + m_frames);
    P.coord_items = (BatchItem*)(M + m_coord);
    P.range_items = (BatchItem*)(M + m_range);
    P.dop_items = (BatchItem*)(M + m_dop);
    P.n_coord = (int)coord.size();
    P.n_range = (int)range.size();
    P.n_dop = (int)dop.size();
    for (int k = 0; k < P.Kmax; ++k) {
        P.active.push_back((int*)(M + m_active[k]));
        P.n_active.push_back((int)active[k].size());
        P.defl_items.push_back((BatchItem*)(M + m_defl[k]));
        P.n_defl.push_back((int)defl[k].size());
    }
    for (size_t c = 0; c < P.classes.size(); ++c)
        for (int t = 0; t < kNumTiles; ++t) P.classes[c].items[t] = (BatchItem*)(M + m_score[c][t]);
    P.out_off_dev = (long long*)(M + m_outoff);
    P.out_dev = M + m_out;
    return GH_OK;
}

// Zeroes the argmax keys and the BOMP counters of every frame.
int reset_frames(gh_ctx* ctx, const Plan& P) {
    GH_CUDA(cudaMemsetAsync(P.keys, 0, P.keys_bytes, ctx->stream));
    return gh_launch_batch_reset(ctx, P.frames, P.nframes);
}

int side_streams(gh_ctx* ctx, BatchState* S) {
    for (int i = 0; i < kSideStreams; ++i) {
        if (!S->side[i]) GH_CUDA(cudaStreamCreateWithFlags(&S->side[i], cudaStreamNonBlocking));
        if (!S->join[i]) GH_CUDA(cudaEventCreateWithFlags(&S->join[i], cudaEventDisableTiming));
    }
    if (!S->fork) GH_CUDA(cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming));
    return GH_OK;
}

// The scorer launches of iteration k, one per class, each with its own work
// counter. Without kernel timers they run on side streams after a fork from
// the context's stream and are joined back (graph branches when captured):
// the classes score disjoint frames, and a class's first CTAs fill the SMs
// the previous class's last items leave idle.
int score_classes(gh_ctx* ctx, BatchState* S, const Plan& P, const std::vector<Tuning>& t, int k) {
    const int nc = (int)P.classes.size();
    auto launch = [&](int c) {
        const Plan::ScoreClass& C = P.classes[c];
        return gh_launch_hop_batch(ctx, P.frames, C.items[t[c].tile], C.n[t[c].tile][k], P.counter + c, k, t[c].ac,
                                   t[c].warps, t[c].per_rx, t[c].pair, C.max_nd, C.bound, C.max_q);
    };
    if (ctx->timing != 0 || nc < 2) {
        for (int c = 0; c < nc; ++c) GH_TRY(launch(c));
        return GH_OK;
    }
    GH_TRY(side_streams(ctx, S));
    cudaStream_t main = ctx->stream;
    GH_CUDA(cudaEventRecord(S->fork, main));
    int st = GH_OK;
    for (int c = 0; c < nc && st == GH_OK; ++c) {
        cudaStream_t s = S->side[c % kSideStreams];
        if (c < kSideStreams && cudaStreamWaitEvent(s, S->fork, 0) != cudaSuccess) {
            st = gh_fail(ctx, GH_ECUDA, "fork of the scorer classes failed");
            break;
        }
        ctx->stream = s;
        st = launch(c);
        ctx->stream = main;
    }
    for (int i = 0; i < kSideStreams && i < nc; ++i) {  // join (also after a failed launch)
        GH_CUDA(cudaEventRecord(S->join[i], S->side[i]));
        GH_CUDA(cudaStreamWaitEvent(main, S->join[i], 0));
    }
    return st;
}

int batch_sequence(gh_ctx* ctx, BatchState* S, const Plan& P, const std::vector<Tuning>& t, void** h) {
    GH_TRY(reset_frames(ctx, P));
    GH_TRY(gh_launch_coord_batch(ctx, P.frames, P.coord_items, P.n_coord));
    for (int k = 0; k < P.Kmax; ++k) {
        if (k == 0)  // maps of the measurements
            GH_TRY(gh_launch_maps_batch(ctx, P.frames, P.range_items, P.n_range, P.thr_range, P.smem_range,
                                        P.dop_items, P.n_dop, P.thr_dop, P.smem_dop, 0));
        else  // maps of the residuals by linearity, frames still iterating
            GH_TRY(gh_launch_maps_deflate_batch(ctx, P.frames, P.defl_items[k], P.n_defl[k], k));
        GH_TRY(score_classes(ctx, S, P, t, k));
        GH_TRY(gh_launch_bomp_select_batch(ctx, P.frames, P.active[k], P.n_active[k], k));
        GH_TRY(gh_launch_bomp_corr_batch(ctx, P.frames, P.active[k], P.n_active[k], k, P.max_chunks, P.max_q));
    }
    GH_TRY(gh_launch_batch_gather(ctx, P.frames, P.nframes, P.out_off_dev, P.out_dev));
    void* hp;
    GH_TRY(gh_pinned(ctx, P.out_bytes, &hp));
    GH_CUDA(cudaMemcpyAsync(hp, P.out_dev, P.out_bytes, cudaMemcpyDeviceToHost, ctx->stream));
    *h = hp;
    return GH_OK;
}

// Maps of the batch's first iteration (what the autotuner scores).
int autotune_prepare(gh_ctx* ctx, const Plan& P) {
    GH_TRY(reset_frames(ctx, P));
    GH_TRY(gh_launch_coord_batch(ctx, P.frames, P.coord_items, P.n_coord));
    return gh_launch_maps_batch(ctx, P.frames, P.range_items, P.n_range, P.thr_range, P.smem_range, P.dop_items,
                                P.n_dop, P.thr_dop, P.smem_dop, 0);
}

// Times the scorer on the first iteration of one class and returns the
// fastest configuration: cells per lane (8, 16, 32, and 6 or 10 in the 8 x 4
// lane layout for classes it fits) x warps per CTA (8, 4, 2, as shared memory
// allows) x power rows of all receivers or of one receiver at a time (where
// every frame's cells of a lane form one run), and the paired scorer (two
// warps per (x, y) cell: 3 or 5 cells per run in the 8 x 4 layout, 8 or 16 in
// the standard one), with 8-cell items, then, for that configuration, items
// of 4, 8, 16 and 32 (x, y) cells (`tile` >= 0 fixes the item size). rm: the
// row mode kept to (-1 any, 0 all rows, 1 one row at a time, 2 paired).
int autotune(gh_ctx* ctx, const Plan& P, const Plan::ScoreClass& C, int tile, int rm, Tuning* best) {
    cudaEvent_t a, b;
    GH_CUDA(cudaEventCreate(&a));
    GH_CUDA(cudaEventCreate(&b));
    float best_ms = 1e30f;
    *best = Tuning();
    int st = GH_OK;
    auto time_one = [&](const Tuning& c) {
        for (int rep = 0; rep < 2 && st == GH_OK; ++rep) {  // first launch warms up
            cudaEventRecord(a, ctx->stream);
            st = gh_launch_hop_batch(ctx, P.frames, C.items[c.tile], C.n[c.tile][0], P.counter, 0, c.ac, c.warps,
                                     c.per_rx, c.pair, C.max_nd, C.bound, C.max_q);
            cudaEventRecord(b, ctx->stream);
        }
        if (st != GH_OK) return;
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            st = gh_fail(ctx, GH_ECUDA, "autotune timing failed");
            return;
        }
        if (ms < best_ms) {
            best_ms = ms;
            *best = c;
        }
    };
    const int t0 = tile >= 0 ? tile : kDefaultTile;
    // two warps per (x, y) cell, where the class's rows fit one CTA: runs of
    // 3 or 5 in the 8 x 4 layout, of 8 or 16 in the standard one; where it is
    // asked for but does not apply, all rows
    const bool pair_ok =
        gh_hop_pair_bytes(C.layout_ac ? C.layout_ac / 2 : 16, C.bound, C.max_q) <= ctx->smem_optin;
    if (rm == 2 && !pair_ok) rm = 0;
    if (pair_ok && (rm == -1 || rm == 2)) {
        if (C.layout_ac) {
            if (st == GH_OK) time_one({C.layout_ac / 2, 2, t0, false, true});
        } else {
            for (int ac : {8, 16})
                if (st == GH_OK) time_one({ac, 2, t0, false, true});
        }
    }
    // one row at a time where it applies and is wanted; all rows otherwise
    // (also when one row at a time is asked for but applies to no configuration)
    const bool pr_any = rm != 0 && (C.pr_need <= 32 || (C.layout_ac && C.layout_run <= C.layout_ac));
    for (int ac : {8, 16, 32, 6, 10}) {
        if (rm == 2) break;
        if ((ac == 6 || ac == 10) && ac != C.layout_ac) continue;
        for (int warps : {8, 4, 2}) {
            if (st == GH_OK && (rm != 1 || !pr_any) &&
                gh_hop_batch_warp_bytes(ac, C.bound, C.max_q) * warps <= ctx->smem_optin)
                time_one({ac, warps, t0, false});
            // one row at a time: one run per lane (standard layout) or per vy row (8 x 4 layout)
            const bool pr_ok = (ac == 6 || ac == 10) ? C.layout_run <= ac : ac >= C.pr_need;
            if (st == GH_OK && rm != 0 && pr_ok &&
                gh_hop_batch_warp_bytes(ac, C.max_nd, C.max_q) * warps <= ctx->smem_optin)
                time_one({ac, warps, t0, true});
        }
    }
    if (st == GH_OK && best->ac == 0)
        st = gh_fail(ctx, GH_ENOTSUP, "batched scorer: frames too large for shared memory");
    if (tile < 0) {
        const Tuning cfg = *best;
        for (int t = 0; t < kNumTiles && st == GH_OK; ++t)
            if (t != t0) time_one({cfg.ac, cfg.warps, t, cfg.per_rx, cfg.pair});
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

}  // namespace

extern "C" int gh_detect_batch(gh_ctx* ctx, int32_t nframes, const gh_frame* frames, int64_t* cells_host,
                               float* scores_host, double* alpha_host) {
    if (!ctx) return GH_EINVAL;
    if (!cells_host) return gh_fail(ctx, GH_EINVAL, "cells_host is NULL");
    DeviceGuard dg(ctx->device);
    GH_TRY(validate(ctx, nframes, frames));
    BatchState* S = state_of(ctx);
    // the plan (descriptors, items) is rebuilt when the batch changes
    std::vector<unsigned char> key;
    for (int f = 0; f < nframes; ++f) {
        const gh_frame& fr = frames[f];
        append(key, fr.radar);
        append(key, fr.grid);
        append(key, fr.Q);
        append(key, fr.K);
        append(key, fr.Y);
        key.insert(key.end(), (const unsigned char*)fr.tx, (const unsigned char*)(fr.tx + 2));
        key.insert(key.end(), (const unsigned char*)fr.rx, (const unsigned char*)(fr.rx + 2 * fr.Q));
    }
    const bool same = S->plan_valid && S->plan.key == key && ctx->ws[WS_BATCH] && ctx->ws[WS_BATCH_META];
    if (!same) {
        S->plan_valid = false;
        GH_TRY(build_plan(ctx, nframes, frames, S->plan));
        S->plan_valid = true;
    }
    Plan& P = S->plan;
    std::vector<Tuning> t(P.classes.size());
    bool prepared = false;
    size_t heaviest = 0;
    for (size_t c = 0; c < P.classes.size(); ++c) {
        if (P.classes[c].work > P.classes[heaviest].work) heaviest = c;
        if (S->force_ac) {
            t[c].ac = S->force_ac;
            t[c].warps = S->force_warps;
            t[c].tile = S->force_tile >= 0 ? S->force_tile : kDefaultTile;
            continue;
        }
        std::vector<unsigned char> tkey = P.shape;
        append(tkey, P.classes[c].bound);
        append(tkey, P.classes[c].pr_need);
        append(tkey, P.classes[c].layout_ac);
        append(tkey, S->force_tile);
        append(tkey, S->force_rm);
        auto it = S->tuned.find(tkey);
        if (it != S->tuned.end()) {
            t[c] = it->second;
            continue;
        }
        if (!prepared) {
            GH_TRY(autotune_prepare(ctx, P));
            prepared = true;
        }
        GH_TRY(autotune(ctx, P, P.classes[c], S->force_tile, S->force_rm, &t[c]));
        S->tuned[tkey] = t[c];
    }
    S->last = t[heaviest];
    // graph key: the batch, the scorer configurations and the timing mask
    std::vector<unsigned char> gkey = P.key;
    for (const Tuning& tc : t) {
        append(gkey, tc.ac);
        append(gkey, tc.warps);
        append(gkey, tc.tile);
        append(gkey, tc.per_rx);
        append(gkey, tc.pair);
    }
    append(gkey, ctx->timing);
    const char tag[] = "batch";
    gkey.insert(gkey.begin(), tag, tag + sizeof(tag));
    void* h = nullptr;
    const GhSequence seq = [&](void** out) { return batch_sequence(ctx, S, P, t, out); };
    GH_TRY(gh_run_sequence(ctx, ctx->graphs ? &gkey : nullptr, seq, &h));
    // unpack: per frame ArgResult[K] then double2[K][Q]
    size_t oc = 0, oa = 0;
    for (int f = 0; f < nframes; ++f) {
        const unsigned char* base = (const unsigned char*)h + P.out_off[f];
        const ArgResult* sel = (const ArgResult*)base;
        const double* al = (const double*)(sel + P.K[f]);
        for (int k = 0; k < P.K[f]; ++k) {
            if (!sel[k].valid) return gh_fail(ctx, GH_ECUDA, "frame %d: iteration %d selected no cell", f, k);
            cells_host[oc + k] = sel[k].cell;
            if (scores_host) scores_host[oc + k] = sel[k].score;
        }
        if (alpha_host) memcpy(alpha_host + oa, al, (size_t)P.K[f] * frames[f].Q * 2 * sizeof(double));
        oc += P.K[f];
        oa += (size_t)P.K[f] * frames[f].Q * 2;
    }
    return GH_OK;
}

extern "C" int gh_set_batch_tuning(gh_ctx* ctx, int32_t cells_per_lane, int32_t warps) {
    if (!ctx) return GH_EINVAL;
    if (cells_per_lane == 0 && warps == 0) {
        state_of(ctx)->force_ac = 0;
        return GH_OK;
    }
    if ((cells_per_lane != 8 && cells_per_lane != 16 && cells_per_lane != 32) ||
        (warps != 2 && warps != 4 && warps != 8))
        return gh_fail(ctx, GH_EINVAL, "tuning (%d, %d): cells per lane in {8, 16, 32}, warps in {2, 4, 8}",
                       cells_per_lane, warps);
    BatchState* S = state_of(ctx);
    S->force_ac = cells_per_lane;
    S->force_warps = warps;
    return GH_OK;
}

extern "C" int gh_batch_tuning(gh_ctx* ctx, int32_t* cells_per_lane, int32_t* warps) {
    if (!ctx || !cells_per_lane || !warps) return GH_EINVAL;
    const BatchState* S = state_of(ctx);
    *cells_per_lane = S->last.ac;
    *warps = S->last.warps;
    return GH_OK;
}

extern "C" int gh_set_batch_tile(gh_ctx* ctx, int32_t cells_per_item) {
    if (!ctx) return GH_EINVAL;
    int idx = -1;
    for (int t = 0; t < kNumTiles; ++t)
        if (kTiles[t] == cells_per_item) idx = t;
    if (cells_per_item != 0 && idx < 0)
        return gh_fail(ctx, GH_EINVAL, "cells per item %d: 0 (tuned) or one of 4, 8, 16, 32", cells_per_item);
    state_of(ctx)->force_tile = idx;
    return GH_OK;
}

extern "C" int gh_set_batch_row_mode(gh_ctx* ctx, int32_t row_mode) {
    if (!ctx) return GH_EINVAL;
    if (row_mode < -1 || row_mode > 2)
        return gh_fail(ctx, GH_EINVAL, "row mode %d: -1 (tuned), 0, 1 or 2", row_mode);
    state_of(ctx)->force_rm = row_mode;
    return GH_OK;
}

extern "C" int gh_batch_row_mode(gh_ctx* ctx, int32_t* per_receiver) {
    if (!ctx || !per_receiver) return GH_EINVAL;
    const Tuning& t = state_of(ctx)->last;
    *per_receiver = t.per_rx ? 1 : t.pair ? 2 : 0;
    return GH_OK;
}

extern "C" int gh_batch_tile(gh_ctx* ctx, int32_t* cells_per_item) {
    if (!ctx || !cells_per_item) return GH_EINVAL;
    *cells_per_item = state_of(ctx)->last.ac ? kTiles[state_of(ctx)->last.tile] : 0;
    return GH_OK;
}

void gh_batch_release(gh_ctx* ctx) {
    std::lock_guard<std::mutex> lk(g_state_mu);
    auto it = g_state.find(ctx);
    if (it != g_state.end()) {
        delete it->second;
        g_state.erase(it);
    }
}
