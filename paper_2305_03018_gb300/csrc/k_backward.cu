// Backward of the dilation (and of the erosion) for a learnable
// morphological layer.
//
// The forward value at x is the top degree D(x) of the count polynomial
// (Step 3, Eq. 9) and its top coefficient cD(x) counts the SE taps attaining
// it.  The upstream gradient g(x) is split equally among those taps:
//   grad_in(p)  = sum_{y in B, p + y in F, f(p) + b(y) = D(p + y)} g(p + y) / cD(p + y)
//   grad_se(y)  = sum_{x in F, x - y in F, f(x - y) + b(y) = D(x)} g(x) / cD(x)
// grad_se(y) is the coefficient of t^b(y) in the lag-y cross-correlation
// sum_x (g / cD)(x) t^D(x) t^-f(x - y); the kernel evaluates that single
// coefficient.  Both sums run in a fixed order (taps in box order; pixels in
// fixed chunks reduced by a fixed tree), so results are deterministic.
// Erosion (Eq. Erosion, E(x) = min f(x + y) - b(y), count cE) is the same
// with the tap direction and the sign of b reversed (sgn = -1):
//   grad_in(p)  = sum_{y, p - y in F, f(p) - b(y) = E(p - y)} g(p - y) / cE(p - y)
//   grad_se(y)  = - sum_{x, x + y in F, f(x + y) - b(y) = E(x)} g(x) / cE(x)
#include <algorithm>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

struct BwdTap {
    int dy, dx, b, box;   // y = (dy, dx), b(y), box index r * kw + c
};

template <int DT>
__device__ __forceinline__ int load_px(const void* src, long long idx) {
    if (DT == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (DT == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

struct BwdRow {
    int dy, t0, t1;       // SE row offset and its taps [t0, t1) in the tap list
};

// A device-resident SE's tap list for one call: the cached list (offsets 0)
// with each tap's offset read from the caller's device array, clamped into
// [0, bound] (an offset outside it is reported by the forward call).
__global__ void k_bwd_taps_dev(const BwdTap* __restrict__ src, int ntaps, const int32_t* __restrict__ off, int bound,
                               BwdTap* __restrict__ dst) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntaps; t += gridDim.x * blockDim.x) {
        BwdTap tp = src[t];
        tp.b = min(max(off[tp.box], 0), bound);
        dst[t] = tp;
    }
}

struct BwdImage {
    const void* f;
    int dtype, n, h, w;
    long long row_stride, batch_stride;
    int sgn;        // +1 dilation, -1 erosion
};

// q(x) = g(x) / cD(x), or 0 where no tap was valid: the share of the upstream
// gradient each attaining tap receives (one division per pixel, reused by
// every tap).
__global__ void k_bwd_share(const float* __restrict__ g, const int32_t* __restrict__ cD, float* __restrict__ q,
                            long long total) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int c = cD[x];
        q[x] = c > 0 ? g[x] / static_cast<float>(c) : 0.f;
    }
}

// grid (ceil(w / blockDim), rows): pixel (n, i, j) of image row blockIdx.y
// (grid-strided over the n h rows) gathers its taps in box order, SE row by
// SE row.  SGN = +1 dilation, -1 erosion; DT the pixel type.
template <int SGN, int DT>
__global__ void __launch_bounds__(256) k_bwd_input(BwdImage im, const int32_t* __restrict__ D,
                                                   const float* __restrict__ q, const BwdTap* __restrict__ taps,
                                                   const BwdRow* __restrict__ trows, int nrows,
                                                   float* __restrict__ grad_in) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= im.w) return;
    const long long rows = static_cast<long long>(im.n) * im.h;
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int n = static_cast<int>(row / im.h);
        const int i = static_cast<int>(row - static_cast<long long>(n) * im.h);
        const int fp = load_px<DT>(im.f, n * im.batch_stride + i * im.row_stride + j);
        const long long img0 = static_cast<long long>(n) * im.h;
        float acc = 0.f;
        for (int rr = 0; rr < nrows; ++rr) {
            const BwdRow R = trows[rr];
            const int xi = i + SGN * R.dy;
            if (xi < 0 || xi >= im.h) continue;
            const int32_t* Dr = D + (img0 + xi) * im.w;
            const float* qr = q + (img0 + xi) * im.w;
            for (int t = R.t0; t < R.t1; ++t) {
                const BwdTap tp = taps[t];
                const int xj = j + SGN * tp.dx;
                if (static_cast<unsigned>(xj) >= static_cast<unsigned>(im.w)) continue;
                if (fp + SGN * tp.b == Dr[xj]) acc += qr[xj];
            }
        }
        grad_in[row * im.w + j] = acc;
    }
}

constexpr int kSeChunk = 8192;      // pixels per partial sum
constexpr int kSeThreads = 256;
constexpr int kSeTaps = 8;          // taps per CTA of k_bwd_se_partial (D and q loaded once for all)

struct SeChunks {
    int CB, RB;              // chunk = RB rows x CB columns of one image (RB CB <= kSeChunk)
    int cx, cy;              // chunks across, down
    uint32_t cbm;            // ceil(2^32 / CB): k / CB for k < kSeChunk
};

// partial[t][chunk] = sum over the chunk's pixels x of the tap-t terms, each
// thread summing its pixels in order, then a fixed warp and block tree.
// grid (nchunks, ceil(ntaps / kSeTaps)).
template <int SGN, int DT>
__global__ void __launch_bounds__(kSeThreads) k_bwd_se_partial(BwdImage im, const int32_t* __restrict__ D,
                                                               const float* __restrict__ q,
                                                               const BwdTap* __restrict__ taps, int ntaps,
                                                               SeChunks ch, int nchunks,
                                                               float* __restrict__ partial) {
    const int chunk = blockIdx.x;
    const int t0 = blockIdx.y * kSeTaps;
    const int nt = min(kSeTaps, ntaps - t0);
    const int cxi = chunk % ch.cx;
    const int rest = chunk / ch.cx;
    const int cyi = rest % ch.cy;
    const int n = rest / ch.cy;
    const int i0 = cyi * ch.RB, j0 = cxi * ch.CB;
    BwdTap tp[kSeTaps];
#pragma unroll
    for (int u = 0; u < kSeTaps; ++u) tp[u] = taps[t0 + (u < nt ? u : 0)];
    float acc[kSeTaps];
#pragma unroll
    for (int u = 0; u < kSeTaps; ++u) acc[u] = 0.f;
    const long long img0 = static_cast<long long>(n) * im.h;
    for (int k = threadIdx.x; k < ch.RB * ch.CB; k += kSeThreads) {
        const int r = ch.CB == 1 ? k : static_cast<int>(__umulhi(static_cast<uint32_t>(k), ch.cbm));   // k / CB
        const int i = i0 + r, j = j0 + (k - r * ch.CB);
        if (i >= im.h) break;
        if (j >= im.w) continue;
        const long long x = (img0 + i) * im.w + j;
        const int dx = D[x];
        const float qx = q[x];
#pragma unroll
        for (int u = 0; u < kSeTaps; ++u) {
            if (u >= nt) break;
            const int si = i - SGN * tp[u].dy, sj = j - SGN * tp[u].dx;
            if (static_cast<unsigned>(si) >= static_cast<unsigned>(im.h) ||
                static_cast<unsigned>(sj) >= static_cast<unsigned>(im.w))
                continue;
            const int fs = load_px<DT>(im.f, n * im.batch_stride + si * im.row_stride + sj);
            if (fs + SGN * tp[u].b == dx) acc[u] += qx;
        }
    }
    __shared__ float red[kSeTaps][kSeThreads / 32];
#pragma unroll
    for (int u = 0; u < kSeTaps; ++u) {
        float a = acc[u];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) red[u][threadIdx.x >> 5] = a;
    }
    __syncthreads();
    if (threadIdx.x < nt) {
        float s = 0.f;
        for (int k = 0; k < kSeThreads / 32; ++k) s += red[threadIdx.x][k];
        partial[static_cast<long long>(t0 + threadIdx.x) * nchunks + chunk] = s;
    }
}

// Both gradients at once.  Every (source pixel p, tap y) term
//   [f(p) + sgn b(y) = D(p + sgn y)] q(p + sgn y)
// adds to grad_in(p) and to grad_se(y) (substituting x = p + sgn y in the
// grad_se sum), so one pass over the terms serves both.  A CTA owns a chunk of
// 256 M consecutive source pixels of one image in row-major order (thread k:
// pixels k + 256 m of the chunk, m < M), keeps their f values
// and grad_in sums in registers, and walks the taps in box order -- the order
// k_bwd_input sums in; per tap each warp reduces its M-pixel sums with a fixed
// shuffle tree into wsum[warp][tap], and the CTA adds its warps in order into
// partial[tap][chunk] (taps <= kFusedMaxTaps).
constexpr int kFusedMaxTaps = 1024;

template <int SGN, int DT, int M>
__global__ void __launch_bounds__(kSeThreads) k_bwd_fused(BwdImage im, const int32_t* __restrict__ D,
                                                          const float* __restrict__ q,
                                                          const BwdTap* __restrict__ taps, int ntaps,
                                                          int chunks_per_img, int nchunks,
                                                          float* __restrict__ partial, float* __restrict__ grad_in) {
    extern __shared__ float wsum[];   // [kSeThreads / 32][ntaps]
    const int chunk = blockIdx.x;
    const int n = chunk / chunks_per_img;
    const long long flat0 = static_cast<long long>(chunk - n * chunks_per_img) * (kSeThreads * M);
    const long long npx = static_cast<long long>(im.h) * im.w;
    const long long img0 = static_cast<long long>(n) * im.h;
    int pi[M], pj[M], fp[M];
    long long px[M];   // flat index of the pixel in D and q
    float acc[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const long long flat = flat0 + threadIdx.x + kSeThreads * m;
        const bool in = flat < npx;
        pi[m] = in ? static_cast<int>(flat / im.w) : -(1 << 20);   // outside: every tap's row is off the image
        pj[m] = in ? static_cast<int>(flat - static_cast<long long>(pi[m]) * im.w) : 0;
        px[m] = img0 * im.w + flat;
        fp[m] = in ? load_px<DT>(im.f, n * im.batch_stride + pi[m] * im.row_stride + pj[m]) : 0;
        acc[m] = 0.f;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = 0; t < ntaps; ++t) {
        const BwdTap tp = taps[t];
        // the tap as row / column steps, a flat-index step and a level shift
        const int sy = SGN * tp.dy, sx = SGN * tp.dx, sb = SGN * tp.b;
        const long long so = static_cast<long long>(sy) * im.w + sx;
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            if (static_cast<unsigned>(pi[m] + sy) < static_cast<unsigned>(im.h) &&
                static_cast<unsigned>(pj[m] + sx) < static_cast<unsigned>(im.w)) {
                const long long x = px[m] + so;
                if (fp[m] + sb == D[x]) {
                    const float v = q[x];
                    acc[m] += v;
                    s += v;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) wsum[warp * ntaps + t] = s;
    }
    if (grad_in) {
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (pi[m] >= 0) grad_in[(img0 + pi[m]) * im.w + pj[m]] = acc[m];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntaps; t += kSeThreads) {
        float s = 0.f;
        for (int w = 0; w < kSeThreads / 32; ++w) s += wsum[w * ntaps + t];
        partial[static_cast<long long>(t) * nchunks + chunk] = s;
    }
}

// grad_se[box of tap t] = the sum of tap t's partials in fp64, one CTA per tap:
// thread k adds chunks k, k + 256, ... in order, then a fixed tree over the
// threads (boxes off B are zeroed beforehand on the same stream).
constexpr int kFinalThreads = 256;

__global__ void __launch_bounds__(kFinalThreads) k_bwd_se_final(const float* __restrict__ partial, int nchunks,
                                                                const BwdTap* __restrict__ taps, int sgn,
                                                                float* __restrict__ grad_se) {
    __shared__ double red[kFinalThreads];
    const int t = blockIdx.x;
    const float* pt = partial + static_cast<long long>(t) * nchunks;
    double s = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += kFinalThreads) s += pt[c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = kFinalThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) grad_se[taps[t].box] = static_cast<float>(sgn * red[0]);
}

}  // namespace morph

using namespace morph;

namespace morph {

struct BwdPlan {
    BwdTap* d_taps = nullptr;
    BwdRow* d_rows = nullptr;
    int ntaps = 0, nrows = 0;
    ~BwdPlan() {
        if (d_taps) cudaFree(d_taps);
        if (d_rows) cudaFree(d_rows);
    }
};

typedef void (*BwdInputKernel)(BwdImage, const int32_t*, const float*, const BwdTap*, const BwdRow*, int, float*);
typedef void (*BwdSeKernel)(BwdImage, const int32_t*, const float*, const BwdTap*, int, SeChunks, int, float*);

template <int SGN>
static BwdInputKernel input_kernel(int dt) {
    return dt == MORPH_U8 ? k_bwd_input<SGN, MORPH_U8> : dt == MORPH_U16 ? k_bwd_input<SGN, MORPH_U16>
                                                                          : k_bwd_input<SGN, MORPH_I32>;
}
typedef void (*BwdFusedKernel)(BwdImage, const int32_t*, const float*, const BwdTap*, int, int, int, float*,
                               float*);

template <int SGN, int DT>
static BwdFusedKernel fused_kernel_m(int M) {
    return M >= 8 ? k_bwd_fused<SGN, DT, 8> : M == 4 ? k_bwd_fused<SGN, DT, 4>
                                            : M == 2 ? k_bwd_fused<SGN, DT, 2> : k_bwd_fused<SGN, DT, 1>;
}
template <int SGN>
static BwdFusedKernel fused_kernel(int dt, int M) {
    return dt == MORPH_U8 ? fused_kernel_m<SGN, MORPH_U8>(M) : dt == MORPH_U16 ? fused_kernel_m<SGN, MORPH_U16>(M)
                                                                               : fused_kernel_m<SGN, MORPH_I32>(M);
}

template <int SGN>
static BwdSeKernel se_kernel(int dt) {
    return dt == MORPH_U8 ? k_bwd_se_partial<SGN, MORPH_U8> : dt == MORPH_U16 ? k_bwd_se_partial<SGN, MORPH_U16>
                                                                               : k_bwd_se_partial<SGN, MORPH_I32>;
}

}  // namespace morph

static SeChunks se_chunks(const morph_image* f) {
    SeChunks ch;
    ch.CB = std::min(f->w, kSeChunk);
    ch.RB = std::max(1, kSeChunk / ch.CB);
    ch.cx = (f->w + ch.CB - 1) / ch.CB;
    ch.cy = (f->h + ch.RB - 1) / ch.RB;
    ch.cbm = ch.CB == 1 ? 0u : static_cast<uint32_t>(((uint64_t(1) << 32) + ch.CB - 1) / ch.CB);
    return ch;
}

static size_t share_bytes(const morph_image* f) {
    const size_t total = static_cast<size_t>(f->n) * f->h * f->w;
    return (total * sizeof(float) + 255) & ~size_t(255);
}

// How the SE-gradient partial sums are laid out: the fused kernel for SEs of up
// to kFusedMaxTaps taps (chunks of 256 M consecutive pixels, M the largest of
// 8, 4, 2, 1 that still gives four CTAs per SM of a 152-SM GB300, where the
// batch allows), else the pixel-chunked gather (chunks of <= 8192 pixels).
struct BwdLayout {
    bool fused = false;
    int M = 1;
    int chunks_per_img = 0;
    SeChunks ch{};
    long long nchunks = 0;
};

static BwdLayout bwd_layout(const morph_image* f, int ntaps) {
    BwdLayout L;
    const long long npx = static_cast<long long>(f->h) * f->w;
    L.fused = ntaps > 0 && ntaps <= kFusedMaxTaps;
    if (L.fused) {
        L.M = 8;
        while (L.M > 1 && npx * f->n / (kSeThreads * L.M) < 4LL * 152) L.M /= 2;
        const long long per = (npx + kSeThreads * L.M - 1) / (kSeThreads * L.M);
        if (per > (1LL << 30)) L.fused = false;
        else {
            L.chunks_per_img = static_cast<int>(per);
            L.nchunks = per * f->n;
            return L;
        }
    }
    L.ch = se_chunks(f);
    L.nchunks = static_cast<long long>(f->n) * L.ch.cy * L.ch.cx;
    return L;
}

size_t morph::backward_workspace_bytes(const morph_image* f, const morph_se* b) {
    int ntaps = 0;
    for (int t = 0; t < b->kh * b->kw; ++t) ntaps += b->mask[t] ? 1 : 0;
    const BwdLayout L = bwd_layout(f, ntaps);
    return share_bytes(f) + static_cast<size_t>(ntaps) * static_cast<size_t>(L.nchunks) * sizeof(float);
}

// dev_off != nullptr: the SE's offsets are in device memory (b->offset is not
// read) and lie in [0, dev_bound]; the cached tap list then depends on the mask
// only and each call writes its offsets into a workspace copy.
static int backward_impl(morph_ctx* ctx, const morph_image* f, const morph_se* b, const int32_t* D,
                         const int32_t* cD, const float* grad_out, float* grad_in, float* grad_se,
                         morph_stream_t stream, int sgn, const int32_t* dev_off = nullptr, int dev_bound = 0) {
    if (!ctx || !f || !b || !f->data || !D || !cD || !grad_out) return MORPH_E_INVAL;
    if (f->dtype < MORPH_U8 || f->dtype > MORPH_I32 || f->n < 1 || f->h < 1 || f->w < 1) return MORPH_E_INVAL;
    if (f->row_stride < f->w || f->batch_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w)
        return MORPH_E_INVAL;
    if (b->kh < 1 || b->kw < 1 || b->kh > 512 || b->kw > 512 || !b->mask || (!b->offset && !dev_off))
        return MORPH_E_INVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // tap list, cached per SE (per mask for device-resident offsets)
    std::string key = dev_off ? "bwddev|" : "bwd|";
    key.append(reinterpret_cast<const char*>(&b->kh), 4 * sizeof(int));
    key.append(reinterpret_cast<const char*>(b->mask), static_cast<size_t>(b->kh) * b->kw);
    if (!dev_off)
        key.append(reinterpret_cast<const char*>(b->offset), static_cast<size_t>(b->kh) * b->kw * sizeof(int32_t));
    std::shared_ptr<BwdPlan> plan;
    auto it = ctx->aux_plans.find(key);
    if (it != ctx->aux_plans.end()) {
        plan = std::static_pointer_cast<BwdPlan>(it->second);
    } else {
        std::vector<BwdTap> taps;
        for (int r = 0; r < b->kh; ++r)
            for (int c = 0; c < b->kw; ++c) {
                const int t = r * b->kw + c;
                if (!b->mask[t]) continue;
                if (!dev_off && b->offset[t] < 0) return MORPH_E_INVAL;
                taps.push_back(BwdTap{r - b->oy, c - b->ox, dev_off ? 0 : b->offset[t], t});
            }
        if (taps.size() > 65535) return MORPH_E_UNSUPPORTED;   // one grid row of partial sums per tap
        plan = std::make_shared<BwdPlan>();
        plan->ntaps = static_cast<int>(taps.size());
        std::vector<BwdRow> trows;            // taps are in box order, so each SE row's taps are contiguous
        for (int t = 0; t < plan->ntaps; ++t) {
            if (trows.empty() || trows.back().dy != taps[t].dy) trows.push_back(BwdRow{taps[t].dy, t, t});
            trows.back().t1 = t + 1;
        }
        plan->nrows = static_cast<int>(trows.size());
        if (plan->ntaps > 0) {
            MORPH_CUDA_TRY(cudaMalloc(&plan->d_taps, taps.size() * sizeof(BwdTap)));
            MORPH_CUDA_TRY(cudaMemcpy(plan->d_taps, taps.data(), taps.size() * sizeof(BwdTap),
                                      cudaMemcpyHostToDevice));
            MORPH_CUDA_TRY(cudaMalloc(&plan->d_rows, trows.size() * sizeof(BwdRow)));
            MORPH_CUDA_TRY(cudaMemcpy(plan->d_rows, trows.data(), trows.size() * sizeof(BwdRow),
                                      cudaMemcpyHostToDevice));
        }
        ctx->aux_plans.emplace(key, plan);
    }
    BwdImage im{f->data, f->dtype, f->n, f->h, f->w, f->row_stride, f->batch_stride, sgn};
    const long long total = static_cast<long long>(f->n) * f->h * f->w;
    // chunks of the SE-gradient sums
    const BwdLayout lay = bwd_layout(f, plan->ntaps);
    if (lay.nchunks > (1LL << 30)) return MORPH_E_UNSUPPORTED;
    const int nchunks = static_cast<int>(lay.nchunks);
    const SeChunks ch = lay.ch;
    const bool fused = grad_se && lay.fused;
    // workspace: q (one float per pixel), then the partial sums
    const size_t q_bytes = share_bytes(f);
    const size_t part_bytes = grad_se ? static_cast<size_t>(plan->ntaps) * nchunks * sizeof(float) : 0;
    const size_t taps_bytes = dev_off ? (static_cast<size_t>(plan->ntaps) * sizeof(BwdTap) + 255) & ~size_t(255) : 0;
    void* ws = nullptr;
    int rc = ctx_workspace(ctx, q_bytes + part_bytes + taps_bytes, &ws);
    if (rc) return rc;
    float* q = static_cast<float*>(ws);
    const BwdTap* taps_dev = plan->d_taps;
    if (dev_off && plan->ntaps > 0) {
        BwdTap* dst = reinterpret_cast<BwdTap*>(static_cast<unsigned char*>(ws) + q_bytes + part_bytes);
        const unsigned nb = static_cast<unsigned>(std::min(64, (plan->ntaps + 255) / 256));
        prof_begin(ctx, st, "k_bwd_taps_dev");
        k_bwd_taps_dev<<<nb, 256, 0, st>>>(plan->d_taps, plan->ntaps, dev_off, dev_bound, dst);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
        taps_dev = dst;
    }
    if (plan->ntaps > 0) {
        const unsigned blocks = static_cast<unsigned>(std::min<long long>((total + 255) / 256, ctx->num_sms * 16LL));
        prof_begin(ctx, st, "k_bwd_share");
        k_bwd_share<<<blocks, 256, 0, st>>>(grad_out, cD, q, total);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    if (fused) {
        // one pass over the (pixel, tap) terms for both gradients
        float* partial = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + q_bytes);
        const size_t smem = sizeof(float) * (kSeThreads / 32) * plan->ntaps;
        prof_begin(ctx, st, "k_bwd_fused");
        const BwdFusedKernel kf = sgn > 0 ? fused_kernel<1>(f->dtype, lay.M) : fused_kernel<-1>(f->dtype, lay.M);
        kf<<<nchunks, kSeThreads, smem, st>>>(im, D, q, taps_dev, plan->ntaps, lay.chunks_per_img, nchunks,
                                              partial, grad_in);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    if (grad_in && !fused) {
        const int bx = std::min(256, ((f->w + 31) / 32) * 32);
        const long long rows = static_cast<long long>(f->n) * f->h;
        dim3 grid(static_cast<unsigned>((f->w + bx - 1) / bx), static_cast<unsigned>(std::min<long long>(rows, 65535)));
        prof_begin(ctx, st, "k_bwd_input");
        const BwdInputKernel kin = sgn > 0 ? input_kernel<1>(f->dtype) : input_kernel<-1>(f->dtype);
        kin<<<grid, bx, 0, st>>>(im, D, q, taps_dev, plan->d_rows, plan->nrows, grad_in);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    if (grad_se) {
        const int nbox = b->kh * b->kw;
        float* partial = nullptr;
        if (plan->ntaps > 0) partial = reinterpret_cast<float*>(static_cast<unsigned char*>(ws) + q_bytes);
        if (plan->ntaps > 0 && !fused) {
            dim3 grid(nchunks, (plan->ntaps + kSeTaps - 1) / kSeTaps);
            prof_begin(ctx, st, "k_bwd_se_partial");
            const BwdSeKernel kse = sgn > 0 ? se_kernel<1>(f->dtype) : se_kernel<-1>(f->dtype);
            kse<<<grid, kSeThreads, 0, st>>>(im, D, q, taps_dev, plan->ntaps, ch, nchunks, partial);
            prof_end(ctx, st);
            ctx->launches += 1;
            MORPH_CUDA_TRY(cudaGetLastError());
        }
        MORPH_CUDA_TRY(cudaMemsetAsync(grad_se, 0, sizeof(float) * static_cast<size_t>(nbox), st));
        if (plan->ntaps > 0) {
            prof_begin(ctx, st, "k_bwd_se_final");
            k_bwd_se_final<<<plan->ntaps, kFinalThreads, 0, st>>>(partial, nchunks, taps_dev, sgn, grad_se);
            prof_end(ctx, st);
            ctx->launches += 1;
            MORPH_CUDA_TRY(cudaGetLastError());
        }
    }
    return MORPH_OK;
}

extern "C" int morph_dilate_backward(morph_ctx* ctx, const morph_image* f, const morph_se* b, const int32_t* D,
                                     const int32_t* cD, const float* grad_out, float* grad_in, float* grad_se,
                                     morph_stream_t stream) {
    return backward_impl(ctx, f, b, D, cD, grad_out, grad_in, grad_se, stream, +1);
}

extern "C" int morph_erode_backward(morph_ctx* ctx, const morph_image* f, const morph_se* b, const int32_t* E,
                                    const int32_t* cE, const float* grad_out, float* grad_in, float* grad_se,
                                    morph_stream_t stream) {
    return backward_impl(ctx, f, b, E, cE, grad_out, grad_in, grad_se, stream, -1);
}

static morph_se host_view(const morph_se_dev* b) {
    morph_se s;
    s.kh = b->kh;
    s.kw = b->kw;
    s.oy = b->oy;
    s.ox = b->ox;
    s.mask = b->mask;
    s.offset = nullptr;
    return s;
}

extern "C" int morph_dilate_backward_dev_se(morph_ctx* ctx, const morph_image* f, const morph_se_dev* b,
                                            const int32_t* D, const int32_t* cD, const float* grad_out,
                                            float* grad_in, float* grad_se, morph_stream_t stream) {
    if (!b || !b->offset || b->max_offset < 0 || b->max_offset > 255) return MORPH_E_INVAL;
    const morph_se s = host_view(b);
    return backward_impl(ctx, f, &s, D, cD, grad_out, grad_in, grad_se, stream, +1, b->offset, b->max_offset);
}

extern "C" int morph_erode_backward_dev_se(morph_ctx* ctx, const morph_image* f, const morph_se_dev* b,
                                           const int32_t* E, const int32_t* cE, const float* grad_out,
                                           float* grad_in, float* grad_se, morph_stream_t stream) {
    if (!b || !b->offset || b->max_offset < 0 || b->max_offset > 255) return MORPH_E_INVAL;
    const morph_se s = host_view(b);
    return backward_impl(ctx, f, &s, E, cE, grad_out, grad_in, grad_se, stream, -1, b->offset, b->max_offset);
}
