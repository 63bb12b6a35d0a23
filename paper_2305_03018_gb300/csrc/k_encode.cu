// Step 1 of the method (Sec. 3, Eq. 7): the umbra f_Um of the image as FP8
// indicator planes.  f_Um(x, v) = 1 iff f(x) = v; the library stores it
// level-major per image row, planes[n][i][v][j], so that the tensor-core route
// can read a (row, level) x (column window) tile with one TMA box.
//
// HBM-bound: 1 pixel read, L bytes written per pixel -- or only the planes of
// the levels the tensor-core route will read, when its band range is known.
// Each thread owns 16 consecutive columns of one row and writes one 16-byte
// vector per level; a warp writes 512 contiguous bytes of one plane.
#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

__device__ __forceinline__ int load_pixel(const void* src, int dtype, long long idx) {
    if (dtype == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (dtype == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

// Byte k of the result is 0x38 (E4M3 1.0) iff byte k of `packed` equals v
// and byte k of `valid` is set.
__device__ __forceinline__ uint32_t onehot4(uint32_t packed, uint32_t valid, uint32_t v4) {
    return __vcmpeq4(packed, v4) & valid & 0x38383838u;
}

__global__ void __launch_bounds__(256) k_encode_planes(const EncodeJob* __restrict__ jobs, int njobs,
                                                        EncodeJob single, long long total_items,
                                                        unsigned int* __restrict__ err) {
    for (long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x; item < total_items;
         item += (long long)gridDim.x * blockDim.x) {
        const EncodeJob* J = &single;
        if (jobs != nullptr) {
            int lo = 0, hi = njobs - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (jobs[mid].item_base <= item) lo = mid; else hi = mid - 1;
            }
            J = &jobs[lo];
        }
        const long long local = item - J->item_base;
        const int cb_per_row = J->w_pad >> 4;
        const int cb = static_cast<int>(local % cb_per_row);
        const long long row = local / cb_per_row;           // n * h + i
        const int i = static_cast<int>(row % J->h);
        const int n = static_cast<int>(row / J->h);
        const int j0 = cb << 4;                              // plane column of the first byte
        // levels of the 16 pixels; `valid` has 0xFF in the bytes of present, in-range pixels
        uint32_t packed[4] = {0u, 0u, 0u, 0u};
        uint32_t valid[4] = {0u, 0u, 0u, 0u};
        const long long base = n * J->batch_stride + i * J->row_stride;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int j = j0 + k - J->shift;                  // image column
            if (j >= 0 && j < J->w) {
                int val = load_pixel(J->src, J->dtype, base + j);
                if (val < 0 || val >= J->L) {
                    bad = true;
                } else {
                    const uint32_t lev = J->flip ? static_cast<uint32_t>(J->L - 1 - val) : static_cast<uint32_t>(val);
                    packed[k >> 2] |= lev << (8 * (k & 3));
                    valid[k >> 2] |= 0xFFu << (8 * (k & 3));
                }
            }
        }
        if (bad) atomicOr(err, MORPH_DEVERR_RANGE);
        uint8_t* dst = J->planes + (row * J->L) * (long long)J->w_pad + j0;
        int v0 = 0, v1 = J->L - 1;
        if (J->lev_range != nullptr) {
            v0 = max(v0, J->lev_range[0]);
            v1 = min(v1, J->lev_range[1]);
        }
        for (int v = v0; v <= v1; ++v) {
            const uint32_t v4 = 0x01010101u * static_cast<uint32_t>(v);
            uint4 q;
            q.x = onehot4(packed[0], valid[0], v4);
            q.y = onehot4(packed[1], valid[1], v4);
            q.z = onehot4(packed[2], valid[2], v4);
            q.w = onehot4(packed[3], valid[3], v4);
            *reinterpret_cast<uint4*>(dst + (long long)v * J->w_pad) = q;
        }
    }
}

int launch_encode(morph_ctx* ctx, const EncodeJob* jobs, int njobs, long long total_items, EncodeJob* d_jobs,
                  cudaStream_t st) {
    if (total_items <= 0) return MORPH_OK;
    const int threads = 256;
    long long blocks = (total_items + threads - 1) / threads;
    const long long cap = static_cast<long long>(ctx->num_sms) * 16;
    if (blocks > cap) blocks = cap;
    EncodeJob single = jobs[0];
    prof_begin(ctx, st, "k_encode_planes");
    k_encode_planes<<<static_cast<unsigned>(blocks), threads, 0, st>>>(njobs > 1 ? d_jobs : nullptr, njobs, single,
                                                                      total_items, ctx->d_err);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

// Output fill for a problem whose SE has no tap: Eq. 6 gives 0 for dilation,
// the erosion convention gives L-1; the top count is 0.
__global__ void k_fill_empty(int32_t* out, int32_t* cnt, long long n, int value, const int32_t* sub) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        out[k] = value - (sub ? sub[k] : 0);
        if (cnt) cnt[k] = 0;
    }
}

int launch_fill_empty(morph_ctx* ctx, int32_t* out, int32_t* cnt, long long n, int value, cudaStream_t st,
                      const OutAdjust* adj) {
    if (n <= 0) return MORPH_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > ctx->num_sms * 8LL) blocks = ctx->num_sms * 8LL;
    prof_begin(ctx, st, "k_fill_empty");
    k_fill_empty<<<static_cast<unsigned>(blocks), 256, 0, st>>>(out, cnt, n, value + (adj ? adj->add : 0),
                                                                adj ? adj->sub : nullptr);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

}  // namespace morph
