// C ABI of the library: context, argument validation (the S0 step: check
// 0 <= b, 2 <= L, shapes), planning and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

static thread_local char g_last_error[512] = {0};

void set_last_cuda_error(cudaError_t e, const char* expr, const char* file, int line) {
    std::snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", expr, cudaGetErrorString(e), file, line);
}

// ------------------------------------------------------------ tensor maps
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode_fn() {
    static PFN_encodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    });
    return fn;
}

int encode_tmap(CUtensorMap* m, CUtensorMapDataType dt, int rank, void* base, const uint64_t* dims,
                const uint64_t* strides_bytes, const uint32_t* box, CUtensorMapSwizzle swz) {
    PFN_encodeTiled fn = get_encode_fn();
    if (!fn) {
        std::snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled entry point not found");
        return MORPH_E_CUDA;
    }
    cuuint64_t gd[5];
    cuuint64_t gs[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gd[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) gs[i] = strides_bytes[i];
    }
    CUresult r = fn(m, dt, static_cast<cuuint32_t>(rank), base, gd, gs, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        std::snprintf(g_last_error, sizeof(g_last_error), "cuTensorMapEncodeTiled failed (%d), rank %d", (int)r, rank);
        return MORPH_E_CUDA;
    }
    return MORPH_OK;
}

static cudaEvent_t prof_event(morph_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void prof_begin(morph_ctx* ctx, cudaStream_t st, const char* name) {
    if (!ctx->prof_on) return;
    morph_prof_rec r;
    r.name = name;
    r.a = prof_event(ctx);
    r.b = prof_event(ctx);
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    ctx->prof.push_back(r);
}

void prof_end(morph_ctx* ctx, cudaStream_t st) {
    if (!ctx->prof_on || ctx->prof.empty()) return;
    cudaEventRecord(ctx->prof.back().b, st);
}

static std::mutex g_ready_mu;
static std::vector<uint32_t> g_ready;   // per device: bit g = kernel group g set up

bool kernels_ready(int device, KernelGroup group) {
    std::lock_guard<std::mutex> lk(g_ready_mu);
    return device >= 0 && device < static_cast<int>(g_ready.size()) && ((g_ready[device] >> group) & 1u);
}

void mark_kernels_ready(int device, KernelGroup group) {
    std::lock_guard<std::mutex> lk(g_ready_mu);
    if (device < 0) return;
    if (device >= static_cast<int>(g_ready.size())) g_ready.resize(device + 1, 0u);
    g_ready[device] |= 1u << group;
}

int ctx_workspace(morph_ctx* ctx, size_t bytes, void** out) {
    if (bytes <= ctx->ws_bytes) {
        *out = ctx->ws;
        return MORPH_OK;
    }
    // Growing: earlier calls on any stream may still read the old buffer.
    MORPH_CUDA_TRY(cudaDeviceSynchronize());
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = (bytes + (size_t(1) << 20) - 1) & ~((size_t(1) << 20) - 1);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return MORPH_E_NOMEM;
    }
    ctx->ws_bytes = want;
    *out = ctx->ws;
    return MORPH_OK;
}

int ctx_workspace2(morph_ctx* ctx, size_t bytes, void** out) {
    if (bytes > ctx->ws2_bytes) {
        MORPH_CUDA_TRY(cudaDeviceSynchronize());
        if (ctx->ws2) cudaFree(ctx->ws2);
        ctx->ws2 = nullptr;
        ctx->ws2_bytes = 0;
        if (cudaMalloc(&ctx->ws2, bytes) != cudaSuccess) {
            cudaGetLastError();
            return MORPH_E_NOMEM;
        }
        ctx->ws2_bytes = bytes;
    }
    *out = ctx->ws2;
    return MORPH_OK;
}

// ------------------------------------------------------------------ plans

// SE after the erosion-by-duality reflection (Sec. 2.1): b_reflected(y) = b(-y),
// i.e. the box is flipped in both axes and the origin moves to (kh-1-oy, kw-1-ox).
struct EffSE {
    std::vector<uint8_t> mask;
    std::vector<int32_t> off;
    morph_se se;
};

static void effective_se(const morph_se* b, int erode, EffSE* e) {
    const int kh = b->kh, kw = b->kw;
    e->mask.resize(kh * kw);
    e->off.resize(kh * kw);
    for (int r = 0; r < kh; ++r)
        for (int c = 0; c < kw; ++c) {
            const int src = erode ? (kh - 1 - r) * kw + (kw - 1 - c) : r * kw + c;
            e->mask[r * kw + c] = b->mask[src] ? 1 : 0;
            e->off[r * kw + c] = b->mask[src] ? b->offset[src] : 0;
        }
    e->se = *b;
    e->se.mask = e->mask.data();
    e->se.offset = e->off.data();
    if (erode) {
        e->se.oy = kh - 1 - b->oy;
        e->se.ox = kw - 1 - b->ox;
    }
}

static int inval(const char* why) {
    std::snprintf(g_last_error, sizeof(g_last_error), "invalid argument: %s", why);
    return MORPH_E_INVAL;
}

static int validate_image(const morph_image* f) {
    if (!f) return inval("null image");
    if (!f->data) return inval("null image data");
    if (f->dtype < MORPH_U8 || f->dtype > MORPH_I32) return inval("dtype");
    if (f->n < 1 || f->h < 1 || f->w < 1) return inval("image shape");
    if (f->L < 2 || f->L > 256) return inval("L outside [2, 256]");
    if (f->row_stride < f->w) return inval("row_stride < w");
    if (f->batch_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w) return inval("batch_stride");
    return MORPH_OK;
}

static int validate(const morph_image* f, const morph_se* b) {
    if (!f || !b) return inval("null image or SE");
    if (!f->data) return inval("null image data");
    if (f->dtype < MORPH_U8 || f->dtype > MORPH_I32) return inval("dtype");
    if (f->n < 1 || f->h < 1 || f->w < 1) return inval("image shape");
    if (f->L < 2 || f->L > 256) return inval("L outside [2, 256]");
    if (f->row_stride < f->w) return inval("row_stride < w");
    if (f->batch_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w) return inval("batch_stride");
    if (b->kh < 1 || b->kw < 1 || b->kh > 512 || b->kw > 512) return inval("SE box outside 1..512");
    if (!b->mask || !b->offset) return inval("null SE mask or offset");
    if (b->oy < -4096 || b->oy > 4096 || b->ox < -4096 || b->ox > 4096) return inval("SE origin");
    for (int t = 0; t < b->kh * b->kw; ++t)
        if (b->mask[t] && (b->offset[t] < 0 || b->offset[t] > 65535)) return inval("SE offset outside [0, 65535]");
    return MORPH_OK;
}

static std::string plan_key(const morph_image* f, const morph_se* se, int erode, int route, bool unproven = false) {
    std::string k;
    char head[160];
    std::snprintf(head, sizeof(head), "r%d%s|e%d|L%d|n%d|h%d|w%d|k%dx%d|o%d,%d|", route, unproven ? "u" : "", erode,
                  f->L, f->n, f->h, f->w, se->kh, se->kw, se->oy, se->ox);
    k = head;
    k.append(reinterpret_cast<const char*>(se->mask), static_cast<size_t>(se->kh) * se->kw);
    k.append(reinterpret_cast<const char*>(se->offset), static_cast<size_t>(se->kh) * se->kw * sizeof(int32_t));
    return k;
}

static size_t plan_device_bytes(const Plan& p) {
    if (p.route == ROUTE_DIRECT)
        return static_cast<size_t>(p.direct.toeplitz_blocks) * 128 * 128 + p.direct.meta.size() * sizeof(int);
    if (p.route == ROUTE_NTT) {
        const NttPlan& q = p.ntt;
        return static_cast<size_t>(q.Rf) * q.ay.N * q.ax.N * sizeof(uint32_t) +
               (static_cast<size_t>(q.ax.N) + q.ay.N + q.Rf) * sizeof(uint2) + q.Rf * sizeof(uint32_t);
    }
    if (p.route == ROUTE_FFT32 || p.route == ROUTE_FFT64) {
        const FftPlan& q = p.fft;
        return static_cast<size_t>(q.K) * q.ay.N * q.ax.N * 2 * q.prec +
               (static_cast<size_t>(q.ax.N) + q.ay.N + q.Rf) * 2 * q.prec;
    }
    return 0;
}

static int get_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, int erode, int route,
                    std::shared_ptr<Plan>* out, bool unproven = false) {
    const std::string key = plan_key(f, se, erode, route, unproven);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        it->second->last_use = ++ctx->plan_tick;
        *out = it->second;
        return MORPH_OK;
    }
    auto p = std::make_shared<Plan>();
    int taps = 0;
    for (int t = 0; t < se->kh * se->kw; ++t) taps += se->mask[t] ? 1 : 0;
    if (taps == 0) {
        p->route = ROUTE_EMPTY;
    } else if (route == ROUTE_DIRECT) {
        p->route = ROUTE_DIRECT;
        int rc = build_direct_plan(ctx, f, se, erode, &p->direct);
        if (rc) return rc;
    } else if (route == ROUTE_NTT) {
        p->route = ROUTE_NTT;
        int rc = build_ntt_plan(ctx, f, se, &p->ntt);
        if (rc) return rc;
    } else {
        p->route = route;
        int rc = build_fft_plan(ctx, f, se, route == ROUTE_FFT32 ? 4 : 8, unproven, &p->fft);
        if (rc) return rc;
    }
    p->dev_bytes = plan_device_bytes(*p);
    p->last_use = ++ctx->plan_tick;
    // keep the cache within its budget: drop least-recently-used plans
    while (ctx->plan_bytes + p->dev_bytes > ctx->plan_budget && !ctx->plans.empty()) {
        auto lru = ctx->plans.begin();
        for (auto jt = ctx->plans.begin(); jt != ctx->plans.end(); ++jt)
            if (jt->second->last_use < lru->second->last_use) lru = jt;
        ctx->plan_bytes -= lru->second->dev_bytes;
        ctx->plans.erase(lru);
    }
    ctx->plan_bytes += p->dev_bytes;
    ctx->plans.emplace(key, p);
    *out = p;
    return MORPH_OK;
}

size_t planes_bytes(const morph_image* f) {
    const size_t w_pad = (static_cast<size_t>(f->w) + 62) & ~size_t(31);   // the direct plan's pitch
    return (static_cast<size_t>(f->n) * f->h * f->L * w_pad + 255) & ~size_t(255);
}

size_t direct_ws_bytes(const morph_image* f) { return planes_bytes(f) + direct_band_bytes(f); }

// Route for a request.  AUTO estimates each exact route's time on the host
// (no device work) and takes the fastest among the FP8 direct route, the FP32
// FFT route where its a-priori bound proves it exact, and the NTT route (exact
// for any size it supports); the FP64 FFT route is the fallback where neither
// transform route applies.  Each estimate is a fixed cost plus the route's
// work at rates fitted to GB300 runs:
//   direct: 70 us + 94.7 ns per MMA and 2.69 us per accumulation (epilogue)
//           along the busiest SM (waves of units over the SMs) + 0.77 ps
//           per pixel level (encoder), fitted over 180 shapes (images 64^2
//           to 2048^2, L = 16 / 64 / 256, flat disks and full non-flat SEs
//           3^2..63^2; 83 % within 1.5x).  The MMAs and accumulations depend
//           on each unit's level band, which depends on the data; the
//           estimate takes ceil((0.12 L + max b) / Lc) chunks of Lc levels,
//           the band of uniformly distributed pixel values;
//   FFT32 : 70 us + FFT FLOP / 5.55e12;  FFT64: 92 us + FFT FLOP / 7.25e11;
//   NTT   : 80 us + 1.2 x its own estimate (operations, bytes, CTAs).
static double direct_time(const DirectPlan& dp, const morph_image* f, int num_sms) {
    if (dp.tiles <= 0) return 70e-6;
    const int full = (dp.L + dp.Lc - 1) / dp.Lc;
    const int est = static_cast<int>(std::ceil((0.12 * dp.L + dp.maxb) / dp.Lc));
    const double nch = std::min(full, std::max(1, est));
    const double waves = std::ceil(static_cast<double>(dp.tiles) / std::max(1, num_sms));
    const double unit_mmas = dp.issued_flop / (2.0 * kDirectM * kDirectN * 32.0) / dp.tiles * nch / full;
    return 70e-6 + 94.7e-9 * waves * unit_mmas + 2.69e-6 * waves * dp.n_pass * nch * dp.T +
           0.77e-12 * static_cast<double>(f->n) * f->h * f->w * f->L;
}

// in_batch: the problem is one of a batch, whose FP8-route problems share one
// encoder, band and tcgen05 launch, so the FP8 route's fixed cost is not this
// problem's; the transform routes still launch their own kernels per problem.
static int choose_route(morph_ctx* ctx, const morph_image* f, const morph_se* se, int erode, int method,
                        bool unproven, int* route, bool in_batch = false) {
    if (method == MORPH_DIRECT_FP8) { *route = ROUTE_DIRECT; return MORPH_OK; }
    if (method == MORPH_FFT_F64) { *route = ROUTE_FFT64; return MORPH_OK; }
    if (method == MORPH_FFT_F32) { *route = ROUTE_FFT32; return MORPH_OK; }
    if (method == MORPH_NTT) { *route = ROUTE_NTT; return MORPH_OK; }
    if (method != MORPH_AUTO) return MORPH_E_INVAL;
    const std::string key = (in_batch ? "autob|" : "auto|") + plan_key(f, se, erode, 0);
    if (ctx) {
        auto tt = ctx->route_cache.find("tuned|auto|" + plan_key(f, se, erode, 0));   // a measured choice wins
        if (tt != ctx->route_cache.end()) { *route = tt->second; return MORPH_OK; }
        auto it = ctx->route_cache.find(key);
        if (it != ctx->route_cache.end()) { *route = it->second; return MORPH_OK; }
    }
    DirectPlan dp;
    int rc = plan_direct_host(f, se, erode, &dp);
    if (rc) return rc;
    *route = ROUTE_DIRECT;
    if (dp.taps > 0) {
        double best = direct_time(dp, f, ctx ? ctx->num_sms : 152) - (in_batch ? 70e-6 : 0.0);
        FftPlan fp;
        const bool f32_ok = plan_fft_tiles(f, se, 4, false, &fp) == MORPH_OK;
        if (f32_ok) {
            const double t = 70e-6 + fp.flop / 5.55e12;
            if (t < best) { best = t; *route = ROUTE_FFT32; }
        }
        NttPlan np;
        if (plan_ntt_tiles(f, se, &np) == MORPH_OK) {
            const double t = 80e-6 + 1.2 * ntt_time_estimate(np);
            if (t < best) { best = t; *route = ROUTE_NTT; }
        } else if (!f32_ok) {
            FftPlan f64;
            if (plan_fft_tiles(f, se, 8, false, &f64) == MORPH_OK) {
                const double t = 92e-6 + f64.flop / 7.25e11;
                if (t < best) { best = t; *route = ROUTE_FFT64; }
            }
        }
    }
    (void)unproven;
    if (ctx) {
        if (ctx->route_cache.size() >= kRouteCacheEntries) ctx->route_cache.clear();   // keys hold whole SEs
        ctx->route_cache.emplace(key, *route);
    }
    return MORPH_OK;
}

int prepare_problem(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, const morph_opts* opts,
                    std::shared_ptr<Plan>* plan, bool in_batch) {
    if (!ctx) return inval("null context");
    int rc = validate(f, b);
    if (rc) return rc;
    const int method = opts ? opts->method : MORPH_AUTO;
    const bool unproven = opts && (opts->flags & MORPH_F_ALLOW_UNPROVEN_F32);
    EffSE e;
    effective_se(b, erode, &e);
    int route = ROUTE_DIRECT;
    rc = choose_route(ctx, f, &e.se, erode, method, unproven, &route, in_batch);
    if (rc) return rc;
    return get_plan(ctx, f, &e.se, erode, route, plan, route == ROUTE_FFT32 && unproven);
}

static int run_plan(morph_ctx* ctx, const Plan& pl, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                    const morph_opts* opts, cudaStream_t st, const OutAdjust* adj = nullptr);

// Autotuning (MORPH_F_AUTOTUNE with AUTO): time each exact route that the
// models do not rule out -- FP8 direct, the FP32 FFT where its bound is
// proven, the NTT (the FP64 FFT only where neither transform route applies)
// -- once after a warm-up run, on the caller's stream and output buffers
// (every route writes the same result), and cache the fastest for this
// problem key.  Routes whose model estimate is more than 8x the best
// estimate are not timed.  Synchronises the stream; a cached decision is
// reused by later AUTO calls with or without the flag.
int tune_problem(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, const morph_opts* opts,
                 int32_t* out, int32_t* cnt, cudaStream_t st) {
    int rc = validate(f, b);
    if (rc) return rc;
    EffSE e;
    effective_se(b, erode, &e);
    const std::string key = "tuned|auto|" + plan_key(f, &e.se, erode, 0);
    if (ctx->route_cache.count(key)) return MORPH_OK;
    DirectPlan dp;
    rc = plan_direct_host(f, &e.se, erode, &dp);
    if (rc) return rc;
    if (dp.taps == 0) return MORPH_OK;
    std::vector<std::pair<int, double>> cand;        // route, model estimate (s)
    cand.push_back({ROUTE_DIRECT, direct_time(dp, f, ctx ? ctx->num_sms : 152)});
    FftPlan fp;
    const bool f32_ok = plan_fft_tiles(f, &e.se, 4, false, &fp) == MORPH_OK;
    if (f32_ok) cand.push_back({ROUTE_FFT32, 70e-6 + fp.flop / 5.55e12});
    NttPlan np;
    const bool ntt_ok = plan_ntt_tiles(f, &e.se, &np) == MORPH_OK;
    if (ntt_ok) cand.push_back({ROUTE_NTT, 80e-6 + 1.2 * ntt_time_estimate(np)});
    if (!f32_ok && !ntt_ok) {
        FftPlan f64;
        if (plan_fft_tiles(f, &e.se, 8, false, &f64) == MORPH_OK) cand.push_back({ROUTE_FFT64, 92e-6 + f64.flop / 7.25e11});
    }
    double best_est = 1e30;
    for (const auto& c : cand) best_est = std::min(best_est, c.second);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MORPH_CUDA_TRY(cudaEventCreate(&e0));
    MORPH_CUDA_TRY(cudaEventCreate(&e1));
    int best = -1;
    float best_ms = 0.f;
    for (const auto& c : cand) {
        if (c.second > 8.0 * best_est) continue;
        std::shared_ptr<Plan> plan;
        rc = get_plan(ctx, f, &e.se, erode, c.first, &plan);
        if (rc) break;
        rc = run_plan(ctx, *plan, f, erode, out, cnt, opts, st);         // warm-up (workspace, caches)
        if (rc) break;
        cudaEventRecord(e0, st);
        rc = run_plan(ctx, *plan, f, erode, out, cnt, opts, st);
        if (rc) break;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = MORPH_E_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best < 0 || ms < best_ms) {
            best = c.first;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best >= 0) {
        if (ctx->route_cache.size() >= kRouteCacheEntries) ctx->route_cache.clear();
        ctx->route_cache[key] = best;
    }
    return MORPH_OK;
}

int run_one(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, int32_t* out, int32_t* cnt,
            const morph_opts* opts, cudaStream_t st, const OutAdjust* adj) {
    if (!out) return inval("null output");
    int rc = MORPH_OK;
    if (opts && (opts->flags & MORPH_F_AUTOTUNE) && opts->method == MORPH_AUTO) {
        rc = tune_problem(ctx, f, b, erode, opts, out, cnt, st);
        if (rc) return rc;
    }
    std::shared_ptr<Plan> plan;
    rc = prepare_problem(ctx, f, b, erode, opts, &plan);
    if (rc) return rc;
    return run_plan(ctx, *plan, f, erode, out, cnt, opts, st, adj);
}

// Steps 1-3 of one problem with a built plan.
static int run_plan(morph_ctx* ctx, const Plan& pl, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                    const morph_opts* opts, cudaStream_t st, const OutAdjust* adj) {
    const Plan* plan = &pl;
    int rc = MORPH_OK;
    const long long npx = static_cast<long long>(f->n) * f->h * f->w;
    if (plan->route == ROUTE_EMPTY) return launch_fill_empty(ctx, out, cnt, npx, erode ? f->L - 1 : 0, st, adj);
    if (plan->route == ROUTE_NTT) return launch_ntt(ctx, plan->ntt, f, erode, out, cnt, st, adj);
    if (plan->route == ROUTE_FFT32 || plan->route == ROUTE_FFT64)
        return launch_fft(ctx, plan->fft, f, erode, out, cnt, opts ? opts->count_err : nullptr,
                          (opts && (opts->flags & MORPH_F_VALIDATE)) ? 1 : 0, st, adj);

    const DirectPlan& dp = plan->direct;
    void* ws = nullptr;
    rc = ctx_workspace(ctx, direct_ws_bytes(f), &ws);
    if (rc) return rc;
    uint8_t* planes = static_cast<uint8_t*>(ws);
    DirectBand* band = reinterpret_cast<DirectBand*>(planes + planes_bytes(f));

    EncodeJob job;
    job.src = f->data;
    job.dtype = f->dtype;
    job.n = f->n;
    job.h = f->h;
    job.w = f->w;
    job.row_stride = f->row_stride;
    job.batch_stride = f->batch_stride;
    job.L = f->L;
    job.flip = erode;
    job.planes = planes;
    job.w_pad = dp.w_pad;
    job.shift = dp.shift;
    job.item_base = 0;
    job.lev_range = nullptr;
    const long long items = static_cast<long long>(f->n) * f->h * (dp.w_pad / 16);

    DirectLaunch dl;
    std::memset(static_cast<void*>(&dl), 0, sizeof(dl));
    direct_fill_problem(dp, &dl.single, planes, out, cnt, 0, &rc);
    if (rc) return rc;
    direct_fill_band(&dl.single, f, band);
    if (adj) {
        dl.single.out_add = adj->add;
        dl.single.out_sub = adj->sub;
    }
    dl.many = nullptr;
    dl.nprob = 1;
    dl.total_tiles = dp.tiles;
    dl.err = ctx->d_err;
    dl.mma_count = ctx->d_mma;
    dl.band_work = ctx->d_mma + 1;
    dl.next_unit = dl.single.band != nullptr ? direct_unit_counter(band, f) : nullptr;
    dl.wait_ns = ctx->wait_ns;
    rc = launch_band(ctx, dl, direct_band_window(dl.single), direct_band_slabs(dl.single), st);
    if (rc) return rc;
    // the planes after the bands: only the levels some unit's chunks read are written
    rc = launch_band_range(ctx, dl, st);
    if (rc) return rc;
    job.lev_range = dl.single.lev_range;
    rc = launch_encode(ctx, &job, 1, items, nullptr, st);
    if (rc) return rc;
    return launch_direct(ctx, dl, st);
}

// One dilation / erosion by an SE with device-resident offsets (FP8 route).
// The plan depends on the mask, the bound and the shape only; each call writes
// the SE's Toeplitz blocks from the device offsets into the workspace.
int run_one_dev(morph_ctx* ctx, const morph_image* f, const morph_se_dev* b, int erode, int32_t* out, int32_t* cnt,
                cudaStream_t st) {
    if (!ctx) return inval("null context");
    if (!out) return inval("null output");
    int rc = validate_image(f);
    if (rc) return rc;
    if (!b || !b->mask || !b->offset) return inval("null SE, mask or offsets");
    if (b->kh < 1 || b->kw < 1 || b->kh > 512 || b->kw > 512) return inval("SE box outside 1..512");
    if (b->oy < -4096 || b->oy > 4096 || b->ox < -4096 || b->ox > 4096) return inval("SE origin");
    if (b->max_offset < 0 || b->max_offset > 255) return inval("max_offset outside [0, 255]");
    const int kh = b->kh, kw = b->kw;
    std::vector<uint8_t> mask(static_cast<size_t>(kh) * kw);
    for (int r = 0; r < kh; ++r)
        for (int c = 0; c < kw; ++c)
            mask[r * kw + c] = b->mask[erode ? (kh - 1 - r) * kw + (kw - 1 - c) : r * kw + c] ? 1 : 0;
    morph_se e;
    e.kh = kh;
    e.kw = kw;
    e.oy = erode ? kh - 1 - b->oy : b->oy;
    e.ox = erode ? kw - 1 - b->ox : b->ox;
    e.mask = mask.data();
    e.offset = nullptr;
    char head[160];
    std::snprintf(head, sizeof(head), "dev|e%d|L%d|n%d|h%d|w%d|k%dx%d|o%d,%d|b%d|", erode, f->L, f->n, f->h, f->w, kh,
                  kw, e.oy, e.ox, b->max_offset);
    std::string key = head;
    key.append(reinterpret_cast<const char*>(mask.data()), mask.size());
    std::shared_ptr<Plan> plan;
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        it->second->last_use = ++ctx->plan_tick;
        plan = it->second;
    } else {
        plan = std::make_shared<Plan>();
        plan->route = ROUTE_DIRECT;
        rc = build_direct_plan_dev(f, &e, b->max_offset, erode, &plan->direct);
        if (rc) return rc;
        if (plan->direct.taps == 0) plan->route = ROUTE_EMPTY;
        plan->dev_bytes = plan->direct.meta.size() * sizeof(int) + mask.size();
        plan->last_use = ++ctx->plan_tick;
        ctx->plan_bytes += plan->dev_bytes;
        ctx->plans.emplace(key, plan);
    }
    const long long npx = static_cast<long long>(f->n) * f->h * f->w;
    if (plan->route == ROUTE_EMPTY) return launch_fill_empty(ctx, out, cnt, npx, erode ? f->L - 1 : 0, st);
    const DirectPlan& dp = plan->direct;
    const size_t toe_off = (direct_ws_bytes(f) + 1023) & ~size_t(1023);
    void* ws = nullptr;
    rc = ctx_workspace(ctx, toe_off + direct_toeplitz_bytes(dp), &ws);
    if (rc) return rc;
    uint8_t* planes = static_cast<uint8_t*>(ws);
    DirectBand* band = reinterpret_cast<DirectBand*>(planes + planes_bytes(f));
    CUtensorMap tmA;
    rc = launch_toeplitz_dev(ctx, dp, b->offset, erode, planes + toe_off, &tmA, st);
    if (rc) return rc;
    EncodeJob job;
    job.src = f->data;
    job.dtype = f->dtype;
    job.n = f->n;
    job.h = f->h;
    job.w = f->w;
    job.row_stride = f->row_stride;
    job.batch_stride = f->batch_stride;
    job.L = f->L;
    job.flip = erode;
    job.planes = planes;
    job.w_pad = dp.w_pad;
    job.shift = dp.shift;
    job.item_base = 0;
    job.lev_range = nullptr;
    const long long items = static_cast<long long>(f->n) * f->h * (dp.w_pad / 16);
    DirectLaunch dl;
    std::memset(static_cast<void*>(&dl), 0, sizeof(dl));
    direct_fill_problem(dp, &dl.single, planes, out, cnt, 0, &rc);
    if (rc) return rc;
    dl.single.tmA = tmA;
    direct_fill_band(&dl.single, f, band);
    dl.single.dev_off = b->offset;
    dl.single.dev_reflect = erode;
    dl.many = nullptr;
    dl.nprob = 1;
    dl.total_tiles = dp.tiles;
    dl.err = ctx->d_err;
    dl.mma_count = ctx->d_mma;
    dl.band_work = ctx->d_mma + 1;
    dl.next_unit = dl.single.band != nullptr ? direct_unit_counter(band, f) : nullptr;
    dl.wait_ns = ctx->wait_ns;
    rc = launch_band(ctx, dl, direct_band_window(dl.single), direct_band_slabs(dl.single), st);
    if (rc) return rc;
    // the planes after the bands: only the levels some unit's chunks read are written
    rc = launch_band_range(ctx, dl, st);
    if (rc) return rc;
    job.lev_range = dl.single.lev_range;
    rc = launch_encode(ctx, &job, 1, items, nullptr, st);
    if (rc) return rc;
    return launch_direct(ctx, dl, st);
}

}  // namespace morph

using namespace morph;

extern "C" {

int morph_dilate_dev_se(morph_ctx* ctx, const morph_image* f, const morph_se_dev* b, int32_t* out,
                        int32_t* out_count, morph_stream_t stream) {
    return run_one_dev(ctx, f, b, 0, out, out_count, reinterpret_cast<cudaStream_t>(stream));
}

int morph_erode_dev_se(morph_ctx* ctx, const morph_image* f, const morph_se_dev* b, int32_t* out,
                       int32_t* out_count, morph_stream_t stream) {
    return run_one_dev(ctx, f, b, 1, out, out_count, reinterpret_cast<cudaStream_t>(stream));
}

int morph_ctx_create(int device, morph_ctx** out) {
    if (!out) return MORPH_E_INVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return MORPH_E_CUDA;
    }
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    if (major != 10 || minor != 3) return MORPH_E_UNSUPPORTED;   // built for sm_103a only
    morph_ctx* c = new (std::nothrow) morph_ctx();
    if (!c) return MORPH_E_NOMEM;
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&c->d_err, sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(c->d_err, 0, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&c->d_mma, 2 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(c->d_mma, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (c->d_err) cudaFree(c->d_err);
        if (c->d_mma) cudaFree(c->d_mma);
        delete c;
        return MORPH_E_NOMEM;
    }
    *out = c;
    return MORPH_OK;
}

int morph_ctx_destroy(morph_ctx* ctx) {
    if (!ctx) return MORPH_E_INVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->plans.clear();
    ctx->aux_plans.clear();
    ctx->route_cache.clear();
    for (auto& r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    for (auto s : ctx->branch) cudaStreamDestroy(s);
    for (auto e : ctx->branch_ev) cudaEventDestroy(e);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->ws2) cudaFree(ctx->ws2);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_mma) cudaFree(ctx->d_mma);
    delete ctx;
    return MORPH_OK;
}

int morph_dilate(morph_ctx* ctx, const morph_image* f, const morph_se* b, int32_t* out, int32_t* out_count,
                 const morph_opts* opts, morph_stream_t stream) {
    return run_one(ctx, f, b, 0, out, out_count, opts, reinterpret_cast<cudaStream_t>(stream));
}

int morph_erode(morph_ctx* ctx, const morph_image* f, const morph_se* b, int32_t* out, int32_t* out_count,
                const morph_opts* opts, morph_stream_t stream) {
    return run_one(ctx, f, b, 1, out, out_count, opts, reinterpret_cast<cudaStream_t>(stream));
}

int morph_plan_query(morph_ctx* ctx, const morph_image* f, const morph_se* b, int op, const morph_opts* opts,
                     morph_plan_info* out) {
    if (!out) return MORPH_E_INVAL;
    int rc = validate(f, b);
    if (rc) return rc;
    const int method = opts ? opts->method : MORPH_AUTO;
    const bool unproven = opts && (opts->flags & MORPH_F_ALLOW_UNPROVEN_F32);
    const int erode = op ? 1 : 0;
    EffSE e;
    effective_se(b, erode, &e);
    int route = ROUTE_DIRECT;
    rc = choose_route(ctx, f, &e.se, erode, method, unproven, &route);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    int taps = 0, maxb = 0;
    for (int t = 0; t < b->kh * b->kw; ++t)
        if (b->mask[t]) {
            ++taps;
            maxb = std::max(maxb, static_cast<int>(b->offset[t]));
        }
    out->R = f->L + maxb;
    out->taps = taps;
    // bound of the tiling an FP32 (FP64) request would run: the cheapest tiling
    // whose bound is below 0.5 if one exists, else the cheapest tiling
    FftPlan f32, f64;
    if (taps > 0) {
        if (plan_fft_tiles(f, &e.se, 4, false, &f32) == MORPH_OK ||
            plan_fft_tiles(f, &e.se, 4, true, &f32) == MORPH_OK)
            out->f32_bound = f32.bound;
        if (plan_fft_tiles(f, &e.se, 8, false, &f64) == MORPH_OK ||
            plan_fft_tiles(f, &e.se, 8, true, &f64) == MORPH_OK)
            out->f64_bound = f64.bound;
    }
    if (route == ROUTE_DIRECT) {
        std::shared_ptr<Plan> plan;
        DirectPlan host_only;
        const DirectPlan* dpp = &host_only;
        if (ctx) {
            rc = get_plan(ctx, f, &e.se, erode, ROUTE_DIRECT, &plan);
            if (rc) return rc;
            dpp = &plan->direct;
        } else {
            rc = plan_direct_host(f, &e.se, erode, &host_only);
            if (rc) return rc;
        }
        const DirectPlan& d = *dpp;
        out->method = MORPH_DIRECT_FP8;
        out->k_steps = d.ksteps;
        out->level_chunks = (d.L + d.Lc - 1) / std::max(1, d.Lc);
        out->ring_stages = direct_stages(d.T);
        out->unit_queue = direct_unit_queue();
        out->groups = d.G;
        out->passes = d.n_pass;
        out->tile_w = d.J;
        out->tile_h = d.rows_n;
        out->unit_tiles = d.T;
        out->unit_blocks = d.nb;
        out->est_flop = d.issued_flop;
        out->workspace_bytes = direct_ws_bytes(f);
    } else if (route == ROUTE_NTT) {
        NttPlan q;
        rc = plan_ntt_tiles(f, &e.se, &q);
        if (rc) return rc;
        out->method = MORPH_NTT;
        out->fft_nx = q.ax.N;
        out->fft_ny = q.ay.N;
        out->tile_w = q.To_x;
        out->tile_h = q.To_y;
        out->est_flop = q.ops;
        out->workspace_bytes = q.ws_bytes;
    } else {
        FftPlan q;
        rc = plan_fft_tiles(f, &e.se, route == ROUTE_FFT32 ? 4 : 8, unproven, &q);
        if (rc) return rc;
        out->method = route == ROUTE_FFT32 ? MORPH_FFT_F32 : MORPH_FFT_F64;
        out->fft_nx = q.ax.N;
        out->fft_ny = q.ay.N;
        out->tile_w = q.To_x;
        out->tile_h = q.To_y;
        out->est_flop = q.flop;
        out->workspace_bytes = q.ws_bytes;
    }
    return MORPH_OK;
}

int morph_ctx_set_cache_limit(morph_ctx* ctx, size_t bytes) {
    if (!ctx) return MORPH_E_INVAL;
    ctx->plan_budget = bytes;
    while (ctx->plan_bytes > ctx->plan_budget && !ctx->plans.empty()) {
        auto lru = ctx->plans.begin();
        for (auto jt = ctx->plans.begin(); jt != ctx->plans.end(); ++jt)
            if (jt->second->last_use < lru->second->last_use) lru = jt;
        ctx->plan_bytes -= lru->second->dev_bytes;
        ctx->plans.erase(lru);
    }
    return MORPH_OK;
}

int morph_ctx_cache_info(const morph_ctx* ctx, size_t* bytes, int* nplans) {
    if (!ctx) return MORPH_E_INVAL;
    if (bytes) *bytes = ctx->plan_bytes;
    if (nplans) *nplans = static_cast<int>(ctx->plans.size());
    return MORPH_OK;
}

int morph_workspace_size(morph_ctx* ctx, const morph_image* f, const morph_se* b, int op, const morph_opts* opts,
                         size_t* bytes) {
    if (!bytes || op < 0 || op > 3) return MORPH_E_INVAL;
    int rc = validate(f, b);
    if (rc) return rc;
    *bytes = 0;
    if (op >= 2) {
        *bytes = backward_workspace_bytes(f, b);
        return MORPH_OK;
    }
    const int erode = op;
    const int method = opts ? opts->method : MORPH_AUTO;
    const bool unproven = opts && (opts->flags & MORPH_F_ALLOW_UNPROVEN_F32);
    EffSE e;
    effective_se(b, erode, &e);
    int taps = 0;
    for (int t = 0; t < b->kh * b->kw; ++t) taps += b->mask[t] ? 1 : 0;
    if (taps == 0) return MORPH_OK;
    int route = ROUTE_DIRECT;
    rc = choose_route(ctx, f, &e.se, erode, method, unproven, &route);
    if (rc) return rc;
    if (route == ROUTE_DIRECT) {
        *bytes = direct_ws_bytes(f);
    } else if (route == ROUTE_NTT) {
        NttPlan q;
        rc = plan_ntt_tiles(f, &e.se, &q);
        if (rc) return rc;
        *bytes = q.ws_bytes;
    } else {
        FftPlan q;
        rc = plan_fft_tiles(f, &e.se, route == ROUTE_FFT32 ? 4 : 8, unproven, &q);
        if (rc) return rc;
        *bytes = q.ws_bytes;
    }
    return MORPH_OK;
}

int morph_stream_check(morph_ctx* ctx, morph_stream_t stream) {
    if (!ctx) return MORPH_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_last_cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        return MORPH_E_CUDA;
    }
    unsigned int h = 0;
    MORPH_CUDA_TRY(cudaMemcpy(&h, ctx->d_err, sizeof(h), cudaMemcpyDeviceToHost));
    if (h) MORPH_CUDA_TRY(cudaMemset(ctx->d_err, 0, sizeof(h)));
    if (h & MORPH_DEVERR_TIMEOUT) return MORPH_E_TIMEOUT;
    if (h & MORPH_DEVERR_RANGE) return MORPH_E_RANGE;
    if (h & MORPH_DEVERR_CONFIG) return MORPH_E_UNSUPPORTED;
    return MORPH_OK;
}

const char* morph_strerror(int s) {
    switch (s) {
        case MORPH_OK: return "ok";
        case MORPH_E_INVAL: return g_last_error[0] ? g_last_error : "invalid argument";
        case MORPH_E_RANGE: return "pixel value outside [0, L)";
        case MORPH_E_NOMEM: return "out of memory";
        case MORPH_E_PRECISION: return "FP32 FFT round-off bound fails for this problem";
        case MORPH_E_CUDA: return g_last_error[0] ? g_last_error : "CUDA error";
        case MORPH_E_TIMEOUT: return "a bounded device wait timed out";
        case MORPH_E_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

uint64_t morph_launch_count(const morph_ctx* ctx) { return ctx ? ctx->launches : 0; }

int morph_ctx_set_wait_limit(morph_ctx* ctx, uint64_t ns) {
    if (!ctx) return MORPH_E_INVAL;
    ctx->wait_ns = static_cast<unsigned long long>(ns);
    return MORPH_OK;
}

int morph_band_work(morph_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) return MORPH_E_INVAL;
    MORPH_CUDA_TRY(cudaSetDevice(ctx->device));
    MORPH_CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long v = 0;
    MORPH_CUDA_TRY(cudaMemcpy(&v, ctx->d_mma + 1, sizeof(v), cudaMemcpyDeviceToHost));
    *out = static_cast<uint64_t>(v);
    return MORPH_OK;
}

int morph_mma_count(morph_ctx* ctx, uint64_t* out) {
    if (!ctx || !out) return MORPH_E_INVAL;
    MORPH_CUDA_TRY(cudaSetDevice(ctx->device));
    MORPH_CUDA_TRY(cudaDeviceSynchronize());
    unsigned long long v = 0;
    MORPH_CUDA_TRY(cudaMemcpy(&v, ctx->d_mma, sizeof(v), cudaMemcpyDeviceToHost));
    *out = static_cast<uint64_t>(v);
    return MORPH_OK;
}

int morph_profile_enable(morph_ctx* ctx, int on) {
    if (!ctx) return MORPH_E_INVAL;
    ctx->prof_on = on != 0;
    return MORPH_OK;
}

int morph_profile_read(morph_ctx* ctx, morph_kernel_time* out, int cap, int* n) {
    if (!ctx || (cap > 0 && !out)) return MORPH_E_INVAL;
    MORPH_CUDA_TRY(cudaDeviceSynchronize());
    std::vector<morph_kernel_time> acc;
    for (const morph_prof_rec& r : ctx->prof) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        morph_kernel_time* slot = nullptr;
        for (auto& k : acc)
            if (std::strncmp(k.name, r.name, sizeof(k.name)) == 0) slot = &k;
        if (!slot) {
            morph_kernel_time k;
            std::memset(&k, 0, sizeof(k));
            std::strncpy(k.name, r.name, sizeof(k.name) - 1);
            acc.push_back(k);
            slot = &acc.back();
        }
        slot->launches += 1;
        slot->total_ms += ms;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof.clear();
    if (n) *n = static_cast<int>(acc.size());
    for (int i = 0; i < cap && i < static_cast<int>(acc.size()); ++i) out[i] = acc[i];
    return MORPH_OK;
}

}  // extern "C"
