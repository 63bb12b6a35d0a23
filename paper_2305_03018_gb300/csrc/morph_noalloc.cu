// Allocation-free entry point of the FP8 tensor-core route: morph_run_noalloc.
//
// Who needs it: code that must not call cudaMalloc / cudaFree -- for example a
// component that runs while another owner has reserved the device memory it
// may use, a host path that may not block on the device-wide synchronisation
// an allocation can imply, or an integration whose memory budget is fixed at
// start-up.  Such a caller passes its image and output buffers and this entry
// point uses only the fixed scratch array below for everything else: the
// device error word, the plan metadata, the Toeplitz blocks of the SE and the
// FP8 indicator planes.  No context is involved and nothing is cached.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds its 64 MiB until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a host-side shadow),
// so the first call on each device, with that device current, looks the
// address up with cudaGetSymbolAddress and keeps it.  That first call should
// come before any stream capture.  All calls share the one array and the last
// call's contents stay in it: the setup kernel clears the error word at the
// start of every call, and calls whose work overlaps on the GPU race with
// each other (serialise them, e.g. on one stream).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;     // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxMeta = (kDirectMaxPasses + 1) + 8 * kDirectMaxPasses + kDirectMaxPasses * 63;

// The SE and the plan metadata travel as a kernel parameter (about 21 KB),
// so no host-to-device copy and no staging buffer is needed.
struct InlineSE {
    int kh, kw, n_pass, nk, J, G, nmeta;
    unsigned char mask[63 * 63];
    unsigned short off[63 * 63];
    int meta[kMaxMeta];
};

// Clears the error word, writes the metadata the direct kernel reads, and
// builds the Toeplitz blocks of the SE rows (same layout as the cached plans).
__global__ void k_noalloc_setup(const __grid_constant__ InlineSE se, uint8_t* __restrict__ blocks, long long nbytes,
                                int* __restrict__ meta_dst, unsigned int* __restrict__ err) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (tid == 0) *err = 0u;
    for (long long i = tid; i < se.nmeta; i += stride) meta_dst[i] = se.meta[i];
    const int* rb = se.meta;
    const int* gw = rb + (se.n_pass + 1);
    const int* rows = gw + se.n_pass * 8;
    for (long long idx = tid; idx < nbytes; idx += stride) {
        const int k = static_cast<int>(idx & 127);
        const int m = static_cast<int>((idx >> 7) & 127);
        const long long blk = idx >> 14;
        const int q = static_cast<int>(blk / se.nk);
        const int kc = static_cast<int>(blk % se.nk);
        int p = 0;
        while (p + 1 < se.n_pass && rb[p + 1] <= q) ++p;
        const int r = rows[q];
        const int g = m / se.J, j = m % se.J;
        const int c = j + (se.kw - 1) - (128 * kc + k);
        uint8_t v = 0;
        if (g < se.G && c >= 0 && c < se.kw) {
            const int t = r * se.kw + c;
            if (se.mask[t] && static_cast<int>(se.off[t]) == gw[p * 8 + g]) v = 0x38;
        }
        blocks[idx] = v;
    }
}

__global__ void k_noalloc_status(const unsigned int* __restrict__ err, uint32_t* __restrict__ out) {
    *out = *err;
}

struct DevState {
    void* scratch = nullptr;
    int num_sms = 0;
    bool ready = false;
};

std::mutex g_noalloc_mu;
DevState g_noalloc_dev[64];

// Status for a failed check; `why` documents the cause at the call site.
int fail(int code, const char* why) {
    (void)why;
    return code;
}

// Once per device, with that device current: the device address of the
// scratch array and the SM count.
int noalloc_setup(int dev, DevState** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 64) return fail(MORPH_E_INVAL, "device ordinal outside 0..63");
    DevState& s = g_noalloc_dev[dev];
    if (!s.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return fail(MORPH_E_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
        }
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return fail(MORPH_E_CUDA, "device attribute query failed");
        }
        if (major != 10 || minor != 3) return fail(MORPH_E_UNSUPPORTED, "built for sm_103a only");
        s.scratch = p;
        s.num_sms = sms;
        s.ready = true;
    }
    *out = &s;
    return MORPH_OK;
}

int check_args(const morph_image* f, const morph_se* b, int op, const int32_t* out) {
    if (!f || !b || !f->data || !out) return fail(MORPH_E_INVAL, "null image, SE or output");
    if (op != 0 && op != 1) return fail(MORPH_E_INVAL, "op must be 0 (dilation) or 1 (erosion)");
    if (f->dtype < MORPH_U8 || f->dtype > MORPH_I32) return fail(MORPH_E_INVAL, "dtype");
    if (f->n < 1 || f->h < 1 || f->w < 1) return fail(MORPH_E_INVAL, "image shape");
    if (f->L < 2 || f->L > 256) return fail(MORPH_E_INVAL, "L outside [2, 256]");
    if (f->row_stride < f->w || f->batch_stride < static_cast<int64_t>(f->h - 1) * f->row_stride + f->w)
        return fail(MORPH_E_INVAL, "strides");
    if (b->kh < 1 || b->kw < 1 || b->kh > 63 || b->kw > 63 || !b->mask || !b->offset)
        return fail(MORPH_E_INVAL, "SE box outside 1..63 or null SE arrays");
    if (b->oy < -4096 || b->oy > 4096 || b->ox < -4096 || b->ox > 4096) return fail(MORPH_E_INVAL, "SE origin");
    for (int t = 0; t < b->kh * b->kw; ++t)
        if (b->mask[t] && (b->offset[t] < 0 || b->offset[t] > 65535))
            return fail(MORPH_E_INVAL, "SE offset outside [0, 65535]");
    return MORPH_OK;
}

// Host-side plan of the direct route for the (already reflected, for erosion)
// SE: the same choices as the cached plans, without any device work.
int plan_inline(const morph_image* f, const std::vector<uint8_t>& mask, const std::vector<int>& off, int kh, int kw,
                int oy, int ox, int erode, DirectPlan* p, InlineSE* ise) {
    p->L = f->L;
    p->Lc = kDirectLc;                  // every level, in chunks of Lc (no band buffer)
    p->rows_n = kDirectN / kDirectLc;
    p->kh = kh;
    p->kw = kw;
    p->oy = oy;
    p->ox = ox;
    p->erode = erode;
    p->h = f->h;
    p->w = f->w;
    p->nimg = f->n;
    p->w_pad = (f->w + 15) & ~15;
    std::vector<int> levels;
    int taps = 0;
    for (int t = 0; t < kh * kw; ++t)
        if (mask[t]) {
            ++taps;
            levels.push_back(off[t]);
        }
    std::sort(levels.begin(), levels.end());
    levels.erase(std::unique(levels.begin(), levels.end()), levels.end());
    p->taps = taps;
    p->n_levels = static_cast<int>(levels.size());
    if (taps == 0) return MORPH_OK;
    long long best = -1;
    for (int G = 1; G <= 8; G <<= 1) {
        const int J = 128 / G;
        const int ks = (J + kw - 1 + 31) / 32;
        const int passes = (p->n_levels + G - 1) / G;
        if (passes > kDirectMaxPasses) continue;
        const long long cost = static_cast<long long>(passes) * G * ks;
        if (best < 0 || cost <= best) {
            best = cost;
            p->G = G;
        }
    }
    if (best < 0) return fail(MORPH_E_UNSUPPORTED, "too many distinct SE offsets");
    p->J = 128 / p->G;
    p->ksteps = (p->J + kw - 1 + 31) / 32;
    p->nk = (p->J + kw - 1 + 127) / 128;
    p->nb = p->nk;   // one tile per unit: every staged block carries its A block
    p->n_pass = (p->n_levels + p->G - 1) / p->G;
    const int a = (((kw - 1 - ox) % 16) + 16) % 16;
    p->e = (16 - a) % 16;
    p->tiles_x = (f->w + p->e + p->J - 1) / p->J;
    p->tiles_y = (f->h + p->rows_n - 1) / p->rows_n;
    p->tiles = static_cast<long long>(f->n) * p->tiles_x * p->tiles_y;
    std::vector<int> rb(p->n_pass + 1, 0), gw(p->n_pass * 8, 0), rows;
    for (int ps = 0; ps < p->n_pass; ++ps) {
        rb[ps] = static_cast<int>(rows.size());
        for (int g = 0; g < p->G; ++g) {
            const int li = ps * p->G + g;
            gw[ps * 8 + g] = li < p->n_levels ? levels[li] : -1;
        }
        for (int r = 0; r < kh; ++r) {
            bool any = false;
            for (int c = 0; c < kw && !any; ++c) {
                const int t = r * kw + c;
                if (!mask[t]) continue;
                for (int g = 0; g < p->G; ++g)
                    if (gw[ps * 8 + g] == off[t]) {
                        any = true;
                        break;
                    }
            }
            if (any) rows.push_back(r);
        }
    }
    rb[p->n_pass] = static_cast<int>(rows.size());
    p->active_rows_total = static_cast<long long>(rows.size());
    p->toeplitz_blocks = p->active_rows_total * p->nk;
    std::vector<int> meta;
    meta.insert(meta.end(), rb.begin(), rb.end());
    meta.insert(meta.end(), gw.begin(), gw.end());
    meta.insert(meta.end(), rows.begin(), rows.end());
    if (static_cast<int>(meta.size()) > kMaxMeta) return fail(MORPH_E_UNSUPPORTED, "plan metadata too large");
    ise->kh = kh;
    ise->kw = kw;
    ise->n_pass = p->n_pass;
    ise->nk = p->nk;
    ise->J = p->J;
    ise->G = p->G;
    ise->nmeta = static_cast<int>(meta.size());
    for (int t = 0; t < kh * kw; ++t) {
        ise->mask[t] = mask[t];
        ise->off[t] = static_cast<unsigned short>(off[t]);
    }
    std::copy(meta.begin(), meta.end(), ise->meta);
    return MORPH_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace
}  // namespace morph

using namespace morph;

extern "C" int morph_run_noalloc(const morph_image* f, const morph_se* b, int op, int32_t* out, int32_t* out_count,
                                 uint32_t* dev_status, morph_stream_t stream) {
    int rc = check_args(f, b, op, out);
    if (rc) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MORPH_E_CUDA, "cudaGetDevice failed");
    }
    DevState* st = nullptr;
    rc = noalloc_setup(dev, &st);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    // SE reflected for erosion by duality (Sec. 2.1)
    const int kh = b->kh, kw = b->kw, erode = op;
    std::vector<uint8_t> mask(kh * kw);
    std::vector<int> off(kh * kw);
    for (int r = 0; r < kh; ++r)
        for (int c = 0; c < kw; ++c) {
            const int src = erode ? (kh - 1 - r) * kw + (kw - 1 - c) : r * kw + c;
            mask[r * kw + c] = b->mask[src] ? 1 : 0;
            off[r * kw + c] = b->mask[src] ? b->offset[src] : 0;
        }
    const int oy = erode ? kh - 1 - b->oy : b->oy;
    const int ox = erode ? kw - 1 - b->ox : b->ox;

    static thread_local InlineSE ise;   // 21 KB: kept off the stack
    DirectPlan p;
    rc = plan_inline(f, mask, off, kh, kw, oy, ox, erode, &p, &ise);
    if (rc) return rc;

    morph_ctx c;                        // launch bookkeeping only; owns no device memory
    c.device = dev;
    c.num_sms = st->num_sms;
    uint8_t* base = static_cast<uint8_t*>(st->scratch);
    unsigned int* err = reinterpret_cast<unsigned int*>(base);
    c.d_err = err;
    const long long npx = static_cast<long long>(f->n) * f->h * f->w;

    if (p.taps == 0) {   // no tap: Eq. 6 gives 0, the erosion convention L - 1; no pixel is read
        if (dev_status && cudaMemsetAsync(dev_status, 0, sizeof(uint32_t), s) != cudaSuccess)
            return fail(MORPH_E_CUDA, "status clear failed");
        return launch_fill_empty(&c, out, out_count, npx, erode ? f->L - 1 : 0, s);
    }

    // scratch layout: error word | metadata | Toeplitz blocks | indicator planes
    const size_t meta_off = 256;
    const size_t toe_off = align_up(meta_off + sizeof(int) * static_cast<size_t>(ise.nmeta), 1024);
    const size_t toe_bytes = static_cast<size_t>(p.toeplitz_blocks) * 128 * 128;
    const size_t planes_off = align_up(toe_off + toe_bytes, 256);
    const size_t planes_bytes = static_cast<size_t>(f->n) * f->h * f->L * static_cast<size_t>(p.w_pad);
    if (planes_off + planes_bytes > kNoAllocScratchBytes)
        return fail(MORPH_E_NOMEM, "n*h*L*round16(w) bytes of planes plus the SE blocks exceed the fixed scratch");
    uint8_t* toe = base + toe_off;
    int* meta = reinterpret_cast<int*>(base + meta_off);
    uint8_t* planes = base + planes_off;

    {
        long long blocks = (static_cast<long long>(toe_bytes) + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        if (blocks < 1) blocks = 1;
        k_noalloc_setup<<<static_cast<unsigned>(blocks), 256, 0, s>>>(ise, toe, static_cast<long long>(toe_bytes),
                                                                      meta, err);
        if (cudaGetLastError() != cudaSuccess) return fail(MORPH_E_CUDA, "setup kernel launch failed");
    }
    p.d_toeplitz = nullptr;   // scratch-resident: the plan must not free it
    p.d_meta = nullptr;
    const uint64_t dims[2] = {128, static_cast<uint64_t>(p.toeplitz_blocks) * 128};
    const uint64_t strides[1] = {128};
    const uint32_t box[2] = {128, 128};
    rc = encode_tmap(&p.tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, toe, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return fail(rc, "tensor map of the SE blocks");

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
    job.w_pad = p.w_pad;
    job.shift = 0;   // this planner shifts the tile grid by e instead
    job.item_base = 0;
    job.lev_range = nullptr;           // no band: every level
    rc = launch_encode(&c, &job, 1, static_cast<long long>(f->n) * f->h * (p.w_pad / 16), nullptr, s);
    if (rc) return rc;

    DirectLaunch dl;
    std::memset(static_cast<void*>(&dl), 0, sizeof(dl));
    direct_fill_problem(p, &dl.single, planes, out, out_count, 0, &rc);
    if (rc) return fail(rc, "tensor map of the indicator planes");
    dl.single.meta = meta;
    dl.many = nullptr;
    dl.nprob = 1;
    dl.total_tiles = p.tiles;
    dl.err = err;
    rc = launch_direct(&c, dl, s);
    if (rc) return rc;
    if (dev_status) {
        k_noalloc_status<<<1, 1, 0, s>>>(err, dev_status);
        if (cudaGetLastError() != cudaSuccess) return fail(MORPH_E_CUDA, "status kernel launch failed");
    }
    return MORPH_OK;
}
