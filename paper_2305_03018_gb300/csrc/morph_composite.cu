// Composite operators built from the exact dilation and erosion: opening,
// closing and the Beucher gradient (the combinations the paper's conclusion
// names).  With the conventions of Sec. 2.1 (taps outside F skipped):
//   opening  (f o b) = (f (-) b) (+) b
//   closing  (f . b) = (f (+) b) (-) b
//   gradient         = (f (+) b) - (f (-) b)
// The intermediate result is an int32 image; its values lie in
// [-max b, L-1] (erosion) or [0, L-1+max b] (dilation).  The opening's first
// pass writes the erosion shifted by max b into the tonal range
// [0, L + max b) of its second pass, whose epilogue removes the shift; the
// gradient's second pass subtracts the stored erosion as it writes.  Every
// result is exact and unclamped; where no tap is valid the second pass gives
// the lowest (dilation) or highest (erosion) value of its input's range.
#include "morph_internal.h"

namespace morph {

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

// op: 0 opening, 1 closing, 2 gradient.  Two passes each; the tonal shift and
// the gradient's difference are applied by the passes' own epilogues (OutAdjust).
static int composite(morph_ctx* ctx, const morph_image* f, const morph_se* b, int op, int32_t* out,
                     const morph_opts* opts, cudaStream_t st) {
    if (!ctx || !f || !b || !out || !b->mask || !b->offset) return MORPH_E_INVAL;
    if (b->kh < 1 || b->kw < 1) return MORPH_E_INVAL;
    const int mb = max_offset(b);
    const long long n = static_cast<long long>(f->n) * f->h * f->w;
    if (n <= 0) return MORPH_E_INVAL;
    if (op != 2 && f->L + mb > 256) return MORPH_E_UNSUPPORTED;   // the second pass needs L + max b <= 256
    int32_t* t = nullptr;
    int rc = ws2(ctx, sizeof(int32_t) * static_cast<size_t>(n), &t);
    if (rc) return rc;
    if (op == 0) {
        OutAdjust up;
        up.add = mb;
        rc = run_one(ctx, f, b, 1, t, nullptr, opts, st, &up);           // E + mb, in [0, L-1+mb]
        if (rc) return rc;
        const morph_image g = int_view(f, t, f->L + mb);
        OutAdjust down;
        down.add = -mb;
        return run_one(ctx, &g, b, 0, out, nullptr, opts, st, &down);     // ((E + mb) (+) b) - mb
    }
    if (op == 1) {
        rc = run_one(ctx, f, b, 0, t, nullptr, opts, st);                 // D = f (+) b in [0, L-1+mb]
        if (rc) return rc;
        const morph_image g = int_view(f, t, f->L + mb);
        return run_one(ctx, &g, b, 1, out, nullptr, opts, st);            // D (-) b
    }
    rc = run_one(ctx, f, b, 1, t, nullptr, opts, st);                     // E
    if (rc) return rc;
    OutAdjust diff;
    diff.sub = t;
    return run_one(ctx, f, b, 0, out, nullptr, opts, st, &diff);          // D - E
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
