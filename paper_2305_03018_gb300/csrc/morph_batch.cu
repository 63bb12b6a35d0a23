// Heterogeneous batches: many images of uneven sizes, tonal ranges, SEs and
// operations.  Every problem is planned on the host (route, tiles, SE
// blocks, cached per SE and shape); then all FP8-direct problems share
//   one encoder launch (a job list; each thread finds its job by binary search)
//   one persistent k_direct_fp8 launch over the concatenated tile list, with
//     the problems' tensor maps in device memory (tiles of the most expensive
//     problems first, so the cheap ones fill the tail),
// and the transform-route problems (FFT, NTT) follow with their own launch
// sequences, spread over up to four branch streams (heaviest first onto the
// least-loaded branch, each with its own workspace slice) that fork from and
// join back into the caller's stream, so small problems run side by side.
// The same
// enqueue serves morph_run_batch (direct launches into the context's batch
// workspace) and morph_batch_capture (launches recorded once into a CUDA
// graph that owns its workspace).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "morph_internal.h"
#include "ptx.cuh"

using namespace morph;

struct morph_batch {
    morph_ctx* ctx = nullptr;
    struct Item {
        morph_image f;
        int erode;
        int32_t* out;
        int32_t* cnt;
        std::shared_ptr<Plan> plan;
        size_t planes_off = 0;
        size_t band_off = 0;
    };
    std::vector<Item> items;
    std::vector<int> direct_order;       // items on the direct route, heaviest tiles first
    std::vector<int> fft_items;
    std::vector<int> empty_items;
    int nbranch = 1;                          // branch streams for the transform-route problems
    std::vector<std::vector<int>> branch_items;
    size_t fft_stride = 0;                    // workspace slice per branch
    size_t jobs_off = 0, probs_off = 0, fft_off = 0, total_bytes = 0;
    long long enc_items = 0, total_tiles = 0;
    std::vector<EncodeJob> jobs;
    std::vector<DirectProblemDev> probs;
    void* ws = nullptr;                  // owned when captured
    bool owns_ws = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float* count_err = nullptr;
    int validate = 0;
    uint64_t graph_launches = 0;         // kernel nodes per replay
    ~morph_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (owns_ws && ws) cudaFree(ws);
    }
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

constexpr int kBatchBranches = 4;

// The context's branch streams and events (created once, kept until the context is destroyed).
int ensure_branches(morph_ctx* ctx, int n) {
    if (!ctx->fork_ev) MORPH_CUDA_TRY(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
    while (static_cast<int>(ctx->branch.size()) < n) {
        cudaStream_t s = nullptr;
        MORPH_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        ctx->branch.push_back(s);
        cudaEvent_t e = nullptr;
        MORPH_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->branch_ev.push_back(e);
    }
    return MORPH_OK;
}

int launch_transform_item(morph_batch* b, int i, uint8_t* ws, cudaStream_t st) {
    const auto& it = b->items[i];
    return it.plan->route == ROUTE_NTT
               ? launch_ntt_in(b->ctx, it.plan->ntt, &it.f, it.erode, it.out, it.cnt, ws, st)
               : launch_fft_in(b->ctx, it.plan->fft, &it.f, it.erode, it.out, it.cnt, b->count_err, b->validate, ws,
                               st);
}

// Host planning of every problem and the layout of the batch workspace.
int batch_setup(morph_ctx* ctx, const morph_problem* p, int n, const morph_opts* opts, morph_batch* b,
                cudaStream_t tune_stream) {
    if (!ctx || (n > 0 && !p) || n < 0) return MORPH_E_INVAL;
    b->ctx = ctx;
    b->items.resize(n);
    for (int i = 0; i < n; ++i) {
        if (p[i].op != 0 && p[i].op != 1) return MORPH_E_INVAL;
        if (!p[i].out) return MORPH_E_INVAL;
        auto& it = b->items[i];
        it.f = p[i].f;
        it.erode = p[i].op;
        it.out = p[i].out;
        it.cnt = p[i].out_count;
        if (opts && (opts->flags & MORPH_F_AUTOTUNE) && opts->method == MORPH_AUTO) {
            // measured route choice on this problem's own buffers (before any capture)
            int rc = tune_problem(ctx, &p[i].f, &p[i].se, p[i].op, opts, p[i].out, p[i].out_count, tune_stream);
            if (rc) return rc;
        }
        int rc = prepare_problem(ctx, &p[i].f, &p[i].se, p[i].op, opts, &it.plan, true);
        if (rc) return rc;
        if (it.plan->route == ROUTE_DIRECT) b->direct_order.push_back(i);
        else if (it.plan->route == ROUTE_EMPTY) b->empty_items.push_back(i);
        else b->fft_items.push_back(i);
    }
    // heaviest units first: MMA work per unit = active SE rows x K-steps x tiles
    std::stable_sort(b->direct_order.begin(), b->direct_order.end(), [&](int a, int c) {
        const DirectPlan& x = b->items[a].plan->direct;
        const DirectPlan& y = b->items[c].plan->direct;
        return x.active_rows_total * x.ksteps * x.T > y.active_rows_total * y.ksteps * y.T;
    });
    size_t off = 0;
    b->jobs_off = off;
    off = align_up(off + sizeof(EncodeJob) * std::max<size_t>(1, b->direct_order.size()), 256);
    b->probs_off = off;
    off = align_up(off + sizeof(DirectProblemDev) * std::max<size_t>(1, b->direct_order.size()), 256);
    for (int i : b->direct_order) {
        b->items[i].planes_off = off;
        off = align_up(off + planes_bytes(&b->items[i].f), 256);
        b->items[i].band_off = off;
        off = align_up(off + direct_band_bytes(&b->items[i].f), 256);
    }
    size_t fft_need = 0;
    for (int i : b->fft_items) {
        const Plan& pl = *b->items[i].plan;
        fft_need = std::max(fft_need, pl.route == ROUTE_NTT ? pl.ntt.ws_bytes : pl.fft.ws_bytes);
    }
    // branches: up to 4, within 8 GB of transform workspace in total
    int S = std::min<int>(kBatchBranches, static_cast<int>(b->fft_items.size()));
    while (S > 1 && fft_need * static_cast<size_t>(S) > (size_t(8) << 30)) --S;
    b->nbranch = std::max(S, 1);
    b->branch_items.assign(b->nbranch, {});
    std::vector<std::pair<double, int>> cost;
    for (int i : b->fft_items) {
        const Plan& pl = *b->items[i].plan;
        const double c = pl.route == ROUTE_NTT ? ntt_time_estimate(pl.ntt)
                                               : pl.fft.flop / (pl.fft.prec == 4 ? 5.55e12 : 7.25e11);
        cost.push_back({c, i});
    }
    std::stable_sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<double> load(b->nbranch, 0.0);
    for (const auto& c : cost) {
        const int s = static_cast<int>(std::min_element(load.begin(), load.end()) - load.begin());
        b->branch_items[s].push_back(c.second);
        load[s] += c.first;
    }
    b->fft_stride = align_up(fft_need, 256);
    b->fft_off = off;
    off = align_up(off + b->fft_stride * b->nbranch, 256);
    b->total_bytes = std::max<size_t>(off, 256);
    b->count_err = opts ? opts->count_err : nullptr;
    b->validate = (opts && (opts->flags & MORPH_F_VALIDATE)) ? 1 : 0;
    return MORPH_OK;
}

// Descriptors of the encoder jobs and of the direct problems for a workspace
// at `ws`; uploaded with one copy each.
int batch_descriptors(morph_batch* b, uint8_t* ws) {
    b->jobs.clear();
    b->probs.clear();
    b->enc_items = 0;
    b->total_tiles = 0;
    for (int i : b->direct_order) {
        const auto& it = b->items[i];
        const DirectPlan& dp = it.plan->direct;
        EncodeJob job;
        job.src = it.f.data;
        job.dtype = it.f.dtype;
        job.n = it.f.n;
        job.h = it.f.h;
        job.w = it.f.w;
        job.row_stride = it.f.row_stride;
        job.batch_stride = it.f.batch_stride;
        job.L = it.f.L;
        job.flip = it.erode;
        job.planes = ws + it.planes_off;
        job.w_pad = dp.w_pad;
        job.shift = dp.shift;
        job.item_base = b->enc_items;
        b->enc_items += static_cast<long long>(it.f.n) * it.f.h * (dp.w_pad / 16);
        DirectProblemDev d;
        int rc = MORPH_OK;
        direct_fill_problem(dp, &d, ws + it.planes_off, it.out, it.cnt, b->total_tiles, &rc);
        if (rc) return rc;
        direct_fill_band(&d, &it.f, reinterpret_cast<DirectBand*>(ws + it.band_off));
        job.lev_range = d.lev_range;      // written by the band range kernel before the encoder runs
        b->jobs.push_back(job);
        b->total_tiles += dp.tiles;
        b->probs.push_back(d);
    }
    return MORPH_OK;
}

int batch_enqueue(morph_batch* b, uint8_t* ws, cudaStream_t st) {
    morph_ctx* ctx = b->ctx;
    for (int i : b->empty_items) {
        const auto& it = b->items[i];
        int rc = launch_fill_empty(ctx, it.out, it.cnt, static_cast<long long>(it.f.n) * it.f.h * it.f.w,
                                   it.erode ? it.f.L - 1 : 0, st);
        if (rc) return rc;
    }
    if (!b->direct_order.empty()) {
        EncodeJob* d_jobs = reinterpret_cast<EncodeJob*>(ws + b->jobs_off);
        int rc = MORPH_OK;
        DirectLaunch dl;
        std::memset(static_cast<void*>(&dl), 0, sizeof(dl));
        dl.many = reinterpret_cast<const DirectProblemDev*>(ws + b->probs_off);
        dl.nprob = static_cast<int>(b->probs.size());
        dl.total_tiles = b->total_tiles;
        dl.err = ctx->d_err;
        dl.mma_count = ctx->d_mma;
        dl.band_work = ctx->d_mma + 1;
        dl.wait_ns = ctx->wait_ns;
        if (b->probs.size() == 1) {       // one problem: descriptor as a kernel parameter
            dl.single = b->probs[0];
            dl.many = nullptr;
        }
        int kind = b->probs.empty() ? 0 : direct_kind(b->probs[0]);
        for (const auto& d : b->probs)
            if (direct_kind(d) != kind) kind = 0;
        int win = 0;
        int slabs = 1;
        for (const auto& d : b->probs) {
            win = std::max(win, direct_band_window(d));
            slabs = std::max(slabs, direct_band_slabs(d));
        }
        // the launch's unit counter: in the band buffer of its first problem with bands (the band
        // kernel, which zeroes it, runs only when some problem has bands)
        dl.next_unit = nullptr;
        for (size_t k = 0; k < b->probs.size() && dl.next_unit == nullptr; ++k)
            if (b->probs[k].band != nullptr) {
                const auto& it = b->items[b->direct_order[k]];
                dl.next_unit = direct_unit_counter(reinterpret_cast<DirectBand*>(ws + it.band_off), &it.f);
            }
        rc = launch_band(ctx, dl, win, slabs, st);
        if (rc) return rc;
        // the planes after the bands: only the levels some unit's chunks read are written
        rc = launch_band_range(ctx, dl, st);
        if (rc) return rc;
        rc = launch_encode(ctx, b->jobs.data(), static_cast<int>(b->jobs.size()), b->enc_items, d_jobs, st);
        if (rc) return rc;
        rc = launch_direct(ctx, dl, st, kind);
        if (rc) return rc;
    }
    if (b->count_err && !b->fft_items.empty())
        MORPH_CUDA_TRY(cudaMemsetAsync(b->count_err, 0, sizeof(float), st));
    if (b->fft_items.empty()) return MORPH_OK;
    if (b->nbranch == 1) {
        for (int i : b->fft_items) {
            int rc = launch_transform_item(b, i, ws + b->fft_off, st);
            if (rc) return rc;
        }
        return MORPH_OK;
    }
    int rc = ensure_branches(ctx, b->nbranch);
    if (rc) return rc;
    MORPH_CUDA_TRY(cudaEventRecord(ctx->fork_ev, st));
    int first_err = MORPH_OK;
    for (int s = 0; s < b->nbranch; ++s) {
        cudaStream_t bs = ctx->branch[s];
        MORPH_CUDA_TRY(cudaStreamWaitEvent(bs, ctx->fork_ev, 0));
        for (int i : b->branch_items[s]) {
            if (first_err) break;
            first_err = launch_transform_item(b, i, ws + b->fft_off + s * b->fft_stride, bs);
        }
        // join even after an error, so a capture in progress stays well-formed
        MORPH_CUDA_TRY(cudaEventRecord(ctx->branch_ev[s], bs));
        MORPH_CUDA_TRY(cudaStreamWaitEvent(st, ctx->branch_ev[s], 0));
    }
    return first_err;
}

int upload_descriptors(morph_batch* b, uint8_t* ws, cudaStream_t st, bool sync_copy) {
    if (b->direct_order.empty()) return MORPH_OK;
    const size_t jb = sizeof(EncodeJob) * b->jobs.size();
    const size_t pb = sizeof(DirectProblemDev) * b->probs.size();
    if (sync_copy) {
        MORPH_CUDA_TRY(cudaMemcpy(ws + b->jobs_off, b->jobs.data(), jb, cudaMemcpyHostToDevice));
        MORPH_CUDA_TRY(cudaMemcpy(ws + b->probs_off, b->probs.data(), pb, cudaMemcpyHostToDevice));
    } else {
        // pageable source: each call returns once its bytes are staged, so the
        // host vectors may be released right after
        MORPH_CUDA_TRY(cudaMemcpyAsync(ws + b->jobs_off, b->jobs.data(), jb, cudaMemcpyHostToDevice, st));
        MORPH_CUDA_TRY(cudaMemcpyAsync(ws + b->probs_off, b->probs.data(), pb, cudaMemcpyHostToDevice, st));
    }
    return MORPH_OK;
}

}  // namespace

extern "C" {

int morph_run_batch(morph_ctx* ctx, const morph_problem* p, int n, const morph_opts* opts, morph_stream_t stream) {
    if (!ctx) return MORPH_E_INVAL;
    if (n == 0) return MORPH_OK;
    morph_batch b;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = batch_setup(ctx, p, n, opts, &b, st);
    if (rc) return rc;
    void* ws = nullptr;
    rc = ctx_workspace(ctx, b.total_bytes, &ws);
    if (rc) return rc;
    rc = batch_descriptors(&b, static_cast<uint8_t*>(ws));
    if (rc) return rc;
    rc = upload_descriptors(&b, static_cast<uint8_t*>(ws), st, false);
    if (rc) return rc;
    return batch_enqueue(&b, static_cast<uint8_t*>(ws), st);
}

int morph_batch_capture(morph_ctx* ctx, const morph_problem* p, int n, const morph_opts* opts, morph_batch** out) {
    if (!out) return MORPH_E_INVAL;
    *out = nullptr;
    morph_batch* b = new (std::nothrow) morph_batch();
    if (!b) return MORPH_E_NOMEM;
    int rc = batch_setup(ctx, p, n, opts, b, nullptr);
    if (rc) {
        delete b;
        return rc;
    }
    if (cudaMalloc(&b->ws, b->total_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return MORPH_E_NOMEM;
    }
    b->owns_ws = true;
    uint8_t* ws = static_cast<uint8_t*>(b->ws);
    rc = batch_descriptors(b, ws);
    if (!rc) rc = upload_descriptors(b, ws, nullptr, true);
    if (rc) {
        delete b;
        return rc;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return MORPH_E_CUDA;
    }
    const uint64_t launches0 = ctx->launches;
    const bool prof = ctx->prof_on;
    ctx->prof_on = false;   // no event records inside the graph
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = batch_enqueue(b, ws, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        b->graph = g;
    }
    ctx->prof_on = prof;
    ctx->launches = launches0;   // counted when the graph is launched
    cudaStreamDestroy(cs);
    if (e != cudaSuccess || rc != MORPH_OK) {
        cudaGetLastError();
        delete b;
        return rc ? rc : MORPH_E_CUDA;
    }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return MORPH_E_CUDA;
    }
    // kernel launches per replay, for the context's counter
    size_t nn = 0;
    cudaGraphGetNodes(b->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(b->graph, nodes.data(), &nn);
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++b->graph_launches;
    }
    *out = b;
    return MORPH_OK;
}

int morph_batch_launch(morph_batch* b, morph_stream_t stream) {
    if (!b || !b->exec) return MORPH_E_INVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    prof_begin(b->ctx, st, "batch_graph");
    const cudaError_t e = cudaGraphLaunch(b->exec, st);
    prof_end(b->ctx, st);
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaGraphLaunch", __FILE__, __LINE__);
        return MORPH_E_CUDA;
    }
    b->ctx->launches += b->graph_launches;
    return MORPH_OK;
}

int morph_batch_destroy(morph_batch* b) {
    if (!b) return MORPH_E_INVAL;
    cudaDeviceSynchronize();   // replays in flight still read the batch's workspace
    delete b;
    return MORPH_OK;
}

}  // extern "C"
