// Composite operators built from the exact dilation and erosion: opening,
// closing and the Beucher gradient (the combinations the paper's conclusion
// names).  With the conventions of Sec. 2.1 (taps outside F skipped):
//   opening  (f o b) = (f (-) b) (+) b
//   closing  (f . b) = (f (+) b) (-) b
//   gradient         = (f (+) b) - (f (-) b)
// The intermediate result is an int32 image; its values lie in
// [-max b, L-1] (erosion) or [0, L-1+max b] (dilation), so it is shifted
// into the tonal range [0, L + max b) before the second operation and the
// shift is removed afterwards.  Every result is exact and unclamped.
#include "morph_internal.h"

namespace morph {

__global__ void k_add_const(const int32_t* __restrict__ in, int32_t* __restrict__ out, long long n, int add) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = in[k] + add;
}

__global__ void k_sub(const int32_t* __restrict__ a, const int32_t* __restrict__ b, int32_t* __restrict__ out,
                      long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = a[k] - b[k];
}

static unsigned blocks_for(morph_ctx* ctx, long long n) {
    long long b = (n + 255) / 256;
    if (b > ctx->num_sms * 8LL) b = ctx->num_sms * 8LL;
    return static_cast<unsigned>(b < 1 ? 1 : b);
}

static int add_const(morph_ctx* ctx, const int32_t* in, int32_t* out, long long n, int add, cudaStream_t st) {
    prof_begin(ctx, st, "k_add_const");
    k_add_const<<<blocks_for(ctx, n), 256, 0, st>>>(in, out, n, add);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

static int ws2(morph_ctx* ctx, size_t bytes, int32_t** out) {
    void* p = nullptr;
    const int rc = ctx_workspace2(ctx, bytes, &p);
    *out = static_cast<int32_t*>(p);
    return rc;
}

static int max_offset(const morph_se* b) {
    int m = 0;
    for (int t = 0; t < b->kh * b->kw; ++t)
        if (b->mask[t] && b->offset[t] > m) m = b->offset[t];
    return m;
}

static morph_image int_view(const morph_image* f, const int32_t* data, int L) {
    morph_image g = *f;
    g.data = data;
    g.dtype = MORPH_I32;
    g.row_stride = f->w;
    g.batch_stride = static_cast<int64_t>(f->h) * f->w;
    g.L = L;
    return g;
}

// op: 0 opening, 1 closing, 2 gradient
static int composite(morph_ctx* ctx, const morph_image* f, const morph_se* b, int op, int32_t* out,
                     const morph_opts* opts, cudaStream_t st) {
    if (!ctx || !f || !b || !out || !b->mask || !b->offset) return MORPH_E_INVAL;
    if (b->kh < 1 || b->kw < 1) return MORPH_E_INVAL;
    const int mb = max_offset(b);
    const long long n = static_cast<long long>(f->n) * f->h * f->w;
    if (n <= 0) return MORPH_E_INVAL;
    if (op != 2 && f->L + mb > 256) return MORPH_E_UNSUPPORTED;   // the second pass needs L + max b <= 256
    int32_t* t = nullptr;
    int rc = ws2(ctx, sizeof(int32_t) * static_cast<size_t>(n) * 2, &t);
    if (rc) return rc;
    int32_t* t2 = t + n;
    if (op == 0) {
        rc = run_one(ctx, f, b, 1, t, nullptr, opts, st);                 // E = f (-) b in [-mb, L-1]
        if (!rc) rc = add_const(ctx, t, t2, n, mb, st);                   // E + mb in [0, L-1+mb]
        if (rc) return rc;
        const morph_image g = int_view(f, t2, f->L + mb);
        rc = run_one(ctx, &g, b, 0, t, nullptr, opts, st);                // (E + mb) (+) b
        if (!rc) rc = add_const(ctx, t, out, n, -mb, st);
        return rc;
    }
    if (op == 1) {
        rc = run_one(ctx, f, b, 0, t, nullptr, opts, st);                 // D = f (+) b in [0, L-1+mb]
        if (rc) return rc;
        const morph_image g = int_view(f, t, f->L + mb);
        return run_one(ctx, &g, b, 1, out, nullptr, opts, st);            // D (-) b
    }
    rc = run_one(ctx, f, b, 0, t, nullptr, opts, st);
    if (!rc) rc = run_one(ctx, f, b, 1, t2, nullptr, opts, st);
    if (rc) return rc;
    prof_begin(ctx, st, "k_sub");
    k_sub<<<blocks_for(ctx, n), 256, 0, st>>>(t, t2, out, n);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

}  // namespace morph

using namespace morph;

extern "C" {

int morph_open(morph_ctx* ctx, const morph_image* f, const morph_se* b, int32_t* out, const morph_opts* opts,
               morph_stream_t stream) {
    return composite(ctx, f, b, 0, out, opts, reinterpret_cast<cudaStream_t>(stream));
}

int morph_close(morph_ctx* ctx, const morph_image* f, const morph_se* b, int32_t* out, const morph_opts* opts,
                morph_stream_t stream) {
    return composite(ctx, f, b, 1, out, opts, reinterpret_cast<cudaStream_t>(stream));
}

int morph_gradient(morph_ctx* ctx, const morph_image* f, const morph_se* b, int32_t* out, const morph_opts* opts,
                   morph_stream_t stream) {
    return composite(ctx, f, b, 2, out, opts, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
