// 3-D volumes.  The method is stated for N-D images (Sec. 2.1, Sec. 3):
// with a kd x kh x kw SE, the count polynomial at x = (z, p) is the sum over
// SE slices q of the 2-D count polynomials of input slice z - (q - oz)
// (dilation; z + (q - oz) for erosion) with SE slice q.  All coefficients
// are non-negative, so by the degree rules of Prop. 2.3 the 3-D result is the
// maximum (minimum) of the per-slice 2-D results and its count the sum of
// the per-slice counts attaining it.  Each SE slice runs through the exact
// 2-D routes over all slices of a volume as a batch of images; a small
// kernel folds the slice results into the output.
#include "morph_internal.h"

namespace morph {

// acc (value, count) <- combine(acc, slice result shifted by dz); count 0 = no tap yet
__global__ void k_fold_slice(const int32_t* __restrict__ sv, const int32_t* __restrict__ sc,
                             int32_t* __restrict__ av, int32_t* __restrict__ ac, int d, long long plane, int dz,
                             int erode) {
    const long long total = static_cast<long long>(d) * plane;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const int z = static_cast<int>(k / plane);
        const long long px = k - static_cast<long long>(z) * plane;
        const int zs = erode ? z + dz : z - dz;
        if (zs < 0 || zs >= d) continue;
        const long long src = static_cast<long long>(zs) * plane + px;
        const int c = sc[src];
        if (c == 0) continue;
        const int v = sv[src];
        const int cur = ac[k];
        if (cur == 0 || (erode ? v < av[k] : v > av[k])) {
            av[k] = v;
            ac[k] = c;
        } else if (v == av[k]) {
            ac[k] = cur + c;
        }
    }
}

__global__ void k_fill_pair(int32_t* __restrict__ v, int32_t* __restrict__ c, long long n, int value) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        v[k] = value;
        c[k] = 0;
    }
}

// pixels no tap reached: 0 (dilation, Eq. 6) or L - 1 (erosion)
__global__ void k_finish_empty(int32_t* __restrict__ v, const int32_t* __restrict__ c, long long n, int value) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        if (c[k] == 0) v[k] = value;
}

static unsigned grid_for(morph_ctx* ctx, long long n) {
    long long b = (n + 255) / 256;
    if (b > ctx->num_sms * 8LL) b = ctx->num_sms * 8LL;
    return static_cast<unsigned>(b < 1 ? 1 : b);
}

static int run3d(morph_ctx* ctx, const morph_volume* f, const morph_se3d* b, int erode, int32_t* out,
                 int32_t* out_count, const morph_opts* opts, cudaStream_t st) {
    if (!ctx || !f || !b || !out || !f->data || !b->mask || !b->offset) return MORPH_E_INVAL;
    if (f->n < 1 || f->d < 1 || f->h < 1 || f->w < 1) return MORPH_E_INVAL;
    if (b->kd < 1 || b->kd > 512) return MORPH_E_INVAL;
    if (f->slice_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w ||
        f->volume_stride < static_cast<int64_t>(f->d - 1) * f->slice_stride + (f->h - 1) * f->row_stride + f->w)
        return MORPH_E_INVAL;
    const long long plane = static_cast<long long>(f->h) * f->w;
    const long long vol = plane * f->d;
    void* w2 = nullptr;
    int rc = ctx_workspace2(ctx, sizeof(int32_t) * static_cast<size_t>(vol) * 3, &w2);
    if (rc) return rc;
    int32_t* sv = static_cast<int32_t*>(w2);
    int32_t* sc = sv + vol;
    int32_t* tmpc = sc + vol;
    const int slice = b->kh * b->kw;
    for (int n = 0; n < f->n; ++n) {
        int32_t* av = out + n * vol;
        int32_t* ac = out_count ? out_count + n * vol : tmpc;
        k_fill_pair<<<grid_for(ctx, vol), 256, 0, st>>>(av, ac, vol, 0);
        ctx->launches += 1;
        morph_image g;
        g.data = static_cast<const uint8_t*>(f->data) +
                 static_cast<size_t>(n) * f->volume_stride * (f->dtype == MORPH_U8 ? 1 : f->dtype == MORPH_U16 ? 2 : 4);
        g.dtype = f->dtype;
        g.n = f->d;
        g.h = f->h;
        g.w = f->w;
        g.row_stride = f->row_stride;
        g.batch_stride = f->slice_stride;
        g.L = f->L;
        for (int q = 0; q < b->kd; ++q) {
            int any = 0;
            for (int t = 0; t < slice && !any; ++t) any = b->mask[q * slice + t] != 0;
            if (!any) continue;
            morph_se s2;
            s2.kh = b->kh;
            s2.kw = b->kw;
            s2.oy = b->oy;
            s2.ox = b->ox;
            s2.mask = b->mask + static_cast<size_t>(q) * slice;
            s2.offset = b->offset + static_cast<size_t>(q) * slice;
            rc = run_one(ctx, &g, &s2, erode, sv, sc, opts, st);
            if (rc) return rc;
            prof_begin(ctx, st, "k_fold_slice");
            k_fold_slice<<<grid_for(ctx, vol), 256, 0, st>>>(sv, sc, av, ac, f->d, plane, q - b->oz, erode);
            prof_end(ctx, st);
            ctx->launches += 1;
        }
        k_finish_empty<<<grid_for(ctx, vol), 256, 0, st>>>(av, ac, vol, erode ? f->L - 1 : 0);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    return MORPH_OK;
}

}  // namespace morph

using namespace morph;

extern "C" {

int morph_dilate3d(morph_ctx* ctx, const morph_volume* f, const morph_se3d* b, int32_t* out, int32_t* out_count,
                   const morph_opts* opts, morph_stream_t stream) {
    return run3d(ctx, f, b, 0, out, out_count, opts, reinterpret_cast<cudaStream_t>(stream));
}

int morph_erode3d(morph_ctx* ctx, const morph_volume* f, const morph_se3d* b, int32_t* out, int32_t* out_count,
                  const morph_opts* opts, morph_stream_t stream) {
    return run3d(ctx, f, b, 1, out, out_count, opts, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
