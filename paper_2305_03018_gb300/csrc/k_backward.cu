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
#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

struct BwdTap {
    int dy, dx, b, box;   // y = (dy, dx), b(y), box index r * kw + c
};

__device__ __forceinline__ int load_px(const void* src, int dtype, long long idx) {
    if (dtype == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (dtype == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

struct BwdImage {
    const void* f;
    int dtype, n, h, w;
    long long row_stride, batch_stride;
    int sgn;        // +1 dilation, -1 erosion
};

__global__ void __launch_bounds__(256) k_bwd_input(BwdImage im, const int32_t* __restrict__ D,
                                                   const int32_t* __restrict__ cD, const float* __restrict__ g,
                                                   const BwdTap* __restrict__ taps, int ntaps,
                                                   float* __restrict__ grad_in) {
    const long long total = static_cast<long long>(im.n) * im.h * im.w;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
         p += (long long)gridDim.x * blockDim.x) {
        const int j = static_cast<int>(p % im.w);
        const long long rr = p / im.w;
        const int i = static_cast<int>(rr % im.h);
        const int n = static_cast<int>(rr / im.h);
        const int fp = load_px(im.f, im.dtype, n * im.batch_stride + i * im.row_stride + j);
        float acc = 0.f;
        for (int t = 0; t < ntaps; ++t) {
            const BwdTap tp = taps[t];
            const int xi = i + im.sgn * tp.dy, xj = j + im.sgn * tp.dx;
            if (xi < 0 || xi >= im.h || xj < 0 || xj >= im.w) continue;
            const long long x = (static_cast<long long>(n) * im.h + xi) * im.w + xj;
            if (fp + im.sgn * tp.b == D[x]) {
                const int c = cD[x];
                if (c > 0) acc += g[x] / static_cast<float>(c);
            }
        }
        grad_in[p] = acc;
    }
}

constexpr int kSeChunk = 8192;      // pixels per partial sum
constexpr int kSeThreads = 256;

// partial[t][chunk] = sum over the chunk's pixels x of the tap-t terms, by a fixed tree.
__global__ void __launch_bounds__(kSeThreads) k_bwd_se_partial(BwdImage im, const int32_t* __restrict__ D,
                                                               const int32_t* __restrict__ cD,
                                                               const float* __restrict__ g,
                                                               const BwdTap* __restrict__ taps, int nchunks,
                                                               float* __restrict__ partial) {
    const int chunk = blockIdx.x;
    const int t = blockIdx.y;
    const BwdTap tp = taps[t];
    const long long total = static_cast<long long>(im.n) * im.h * im.w;
    const long long x0 = static_cast<long long>(chunk) * kSeChunk;
    float acc = 0.f;
    for (int k = threadIdx.x; k < kSeChunk; k += kSeThreads) {
        const long long x = x0 + k;
        if (x >= total) break;
        const int j = static_cast<int>(x % im.w);
        const long long rr = x / im.w;
        const int i = static_cast<int>(rr % im.h);
        const int n = static_cast<int>(rr / im.h);
        const int si = i - im.sgn * tp.dy, sj = j - im.sgn * tp.dx;
        if (si < 0 || si >= im.h || sj < 0 || sj >= im.w) continue;
        const int fs = load_px(im.f, im.dtype, n * im.batch_stride + si * im.row_stride + sj);
        if (fs + im.sgn * tp.b == D[x]) {
            const int c = cD[x];
            if (c > 0) acc += g[x] / static_cast<float>(c);
        }
    }
    __shared__ float red[kSeThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int k = 0; k < kSeThreads / 32; ++k) s += red[k];
        partial[static_cast<long long>(t) * nchunks + chunk] = s;
    }
}

// grad_se[box] = sum of the partials of its tap in chunk order (fp64 accumulator); 0 off B.
__global__ void k_bwd_se_final(const float* __restrict__ partial, int nchunks, const BwdTap* __restrict__ taps,
                               int ntaps, int nbox, int sgn, float* __restrict__ grad_se) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) grad_se[b] = 0.f;
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntaps; t += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += partial[static_cast<long long>(t) * nchunks + c];
        grad_se[taps[t].box] = static_cast<float>(sgn * s);
    }
}

}  // namespace morph

using namespace morph;

namespace morph {

struct BwdPlan {
    BwdTap* d_taps = nullptr;
    int ntaps = 0;
    ~BwdPlan() {
        if (d_taps) cudaFree(d_taps);
    }
};

}  // namespace morph

static int backward_impl(morph_ctx* ctx, const morph_image* f, const morph_se* b, const int32_t* D,
                         const int32_t* cD, const float* grad_out, float* grad_in, float* grad_se,
                         morph_stream_t stream, int sgn) {
    if (!ctx || !f || !b || !f->data || !D || !cD || !grad_out) return MORPH_E_INVAL;
    if (f->dtype < MORPH_U8 || f->dtype > MORPH_I32 || f->n < 1 || f->h < 1 || f->w < 1) return MORPH_E_INVAL;
    if (f->row_stride < f->w || f->batch_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w)
        return MORPH_E_INVAL;
    if (b->kh < 1 || b->kw < 1 || b->kh > 512 || b->kw > 512 || !b->mask || !b->offset) return MORPH_E_INVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // tap list, cached per SE
    std::string key = "bwd|";
    key.append(reinterpret_cast<const char*>(&b->kh), 4 * sizeof(int));
    key.append(reinterpret_cast<const char*>(b->mask), static_cast<size_t>(b->kh) * b->kw);
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
                if (b->offset[t] < 0) return MORPH_E_INVAL;
                taps.push_back(BwdTap{r - b->oy, c - b->ox, b->offset[t], t});
            }
        if (taps.size() > 65535) return MORPH_E_UNSUPPORTED;   // one grid row of partial sums per tap
        plan = std::make_shared<BwdPlan>();
        plan->ntaps = static_cast<int>(taps.size());
        if (plan->ntaps > 0) {
            MORPH_CUDA_TRY(cudaMalloc(&plan->d_taps, taps.size() * sizeof(BwdTap)));
            MORPH_CUDA_TRY(cudaMemcpy(plan->d_taps, taps.data(), taps.size() * sizeof(BwdTap),
                                      cudaMemcpyHostToDevice));
        }
        ctx->aux_plans.emplace(key, plan);
    }
    BwdImage im{f->data, f->dtype, f->n, f->h, f->w, f->row_stride, f->batch_stride, sgn};
    const long long total = static_cast<long long>(f->n) * f->h * f->w;
    if (grad_in) {
        long long blocks = (total + 255) / 256;
        if (blocks > ctx->num_sms * 16LL) blocks = ctx->num_sms * 16LL;
        prof_begin(ctx, st, "k_bwd_input");
        k_bwd_input<<<static_cast<unsigned>(blocks), 256, 0, st>>>(im, D, cD, grad_out, plan->d_taps, plan->ntaps,
                                                                  grad_in);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    if (grad_se) {
        const int nbox = b->kh * b->kw;
        const int nchunks = static_cast<int>((total + kSeChunk - 1) / kSeChunk);
        float* partial = nullptr;
        if (plan->ntaps > 0) {
            void* ws = nullptr;
            int rc = ctx_workspace(ctx, static_cast<size_t>(plan->ntaps) * nchunks * sizeof(float), &ws);
            if (rc) return rc;
            partial = static_cast<float*>(ws);
            dim3 grid(nchunks, plan->ntaps);
            prof_begin(ctx, st, "k_bwd_se_partial");
            k_bwd_se_partial<<<grid, kSeThreads, 0, st>>>(im, D, cD, grad_out, plan->d_taps, nchunks, partial);
            prof_end(ctx, st);
            ctx->launches += 1;
            MORPH_CUDA_TRY(cudaGetLastError());
        }
        prof_begin(ctx, st, "k_bwd_se_final");
        k_bwd_se_final<<<1, 1024, 0, st>>>(partial, nchunks, plan->d_taps, plan->ntaps, nbox, sgn, grad_se);
        prof_end(ctx, st);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
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
