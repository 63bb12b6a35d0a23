/*
 * morph.h -- C ABI of the GB300 (sm_103a) library for exact grey-value
 * dilation and erosion by umbra / polynomial convolution.
 *
 * Method (arxiv 2305.03018, Sec. 3): every pixel value f(x) becomes the
 * monomial t^f(x) (Step 1, Eq. 7), every structuring-element value b(y)
 * becomes t^b(y) (Eq. 8); their full-mode convolution over space x grey level
 * (Step 2) gives at each pixel a polynomial with non-negative integer
 * coefficients -- the number of SE taps y with f(x - y) + b(y) = d (Eq. Obs7)
 * -- and the dilation is the degree of its highest nonzero coefficient
 * (Step 3, Eq. 9).  Erosion is computed through duality (Sec. 2.1):
 * f (-) b = (L - 1) - ((L - 1 - f) (+) b_reflected).
 *
 * Conventions shared by every call:
 *   - Image f: N images of H x W pixels, integer values in [0, L-1]
 *     (Sec. 2.1, tonal range {0..l}, L = l + 1).  Device memory.
 *   - SE b on a kh x kw box; box entry (r, c) is the spatial offset
 *     y = (r - oy, c - ox).  mask[r*kw + c] != 0 puts y in B; offset[] gives
 *     b(y) >= 0 (Sec. 2.1 requires b >= 0).  Host memory, read during the
 *     call only.
 *   - Dilation output (Eq. 6): D(x) = max{f(x-y) + b(y) : x-y in F, y in B},
 *     0 where no tap is valid; int32, never clamped, in [0, L-1+max b].
 *   - Erosion output (Eq. Erosion): min{f(x+y) - b(y) : x+y in F, y in B},
 *     L-1 where no tap is valid; int32, never clamped, in [-max b, L-1].
 *   - Optional top count: the coefficient of the top degree, i.e. how many
 *     valid taps attain the result (0 where no tap is valid).
 *   - Outputs are int32 [N][H][W], contiguous, device memory, owned by the
 *     caller.  The library owns its context: plans, device workspace, the
 *     device error word.
 *   - Every call is stream-ordered and asynchronous unless stated otherwise.
 *     Calls return a status synchronously for argument errors; data errors
 *     found on the device (a pixel outside [0, L)) are reported by
 *     morph_stream_check().
 *   - A context is bound to one device and is not thread-safe: use one
 *     context per host thread.  Calls through one context share its device
 *     workspace: issue them on one stream (or order the streams).
 */
#ifndef MORPH_H
#define MORPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream; NULL is the legacy default stream. */
typedef struct CUstream_st *morph_stream_t;

typedef struct morph_ctx morph_ctx;

/* ------------------------------------------------------------- status */
enum morph_status {
    MORPH_OK = 0,
    MORPH_E_INVAL = 1,       /* bad argument: shape, stride, L, SE, pointer */
    MORPH_E_RANGE = 2,       /* data error found on the device (pixel not in [0, L)) */
    MORPH_E_NOMEM = 3,       /* device or host allocation failed */
    MORPH_E_PRECISION = 4,   /* FP32 FFT requested but its round-off bound fails */
    MORPH_E_CUDA = 5,        /* a CUDA runtime/driver call failed */
    MORPH_E_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    MORPH_E_UNSUPPORTED = 7  /* valid request outside what the library implements */
};

/* ------------------------------------------------------------- inputs */
enum morph_dtype { MORPH_U8 = 0, MORPH_U16 = 1, MORPH_I32 = 2 };

typedef struct {
    const void *data;        /* device pointer to pixel (0,0) of image 0 */
    int dtype;               /* enum morph_dtype */
    int n, h, w;             /* images, rows, columns (each >= 1) */
    int64_t row_stride;      /* elements between rows (>= w) */
    int64_t batch_stride;    /* elements between images (>= h * row_stride) */
    int L;                   /* number of grey levels, 2 <= L <= 256 */
} morph_image;

typedef struct {
    int kh, kw;              /* box size, 1..512 each (1..63 for morph_run_noalloc) */
    int oy, ox;              /* box entry of the spatial origin (any integers) */
    const uint8_t *mask;     /* host, kh*kw, row-major */
    const int32_t *offset;   /* host, kh*kw, >= 0 where mask != 0 */
} morph_se;

/* A structuring element whose offsets live in device memory -- a learnable
 * layer's parameter -- so that no call has to copy them to the host (which
 * would wait for the device).  The mask and the bound are host values; the
 * plan depends on them only.  Offsets outside [0, max_offset] at taps are a
 * data error reported by morph_stream_check (MORPH_E_RANGE). */
typedef struct {
    int kh, kw;              /* box size, 1..512 each */
    int oy, ox;              /* box entry of the spatial origin */
    const uint8_t *mask;     /* host, kh*kw, row-major */
    const int32_t *offset;   /* DEVICE, kh*kw int32, in [0, max_offset] where mask != 0 */
    int max_offset;          /* host bound on the offsets, 0..255 */
} morph_se_dev;

/* ------------------------------------------------------------ options */
enum morph_method {
    MORPH_AUTO = 0,          /* planner picks the fastest exact back-end */
    MORPH_DIRECT_FP8 = 1,    /* tcgen05 FP8 implicit GEMM, exact by construction */
    MORPH_FFT_F32 = 2,       /* FP32 FFT; refused (E_PRECISION) if the bound fails */
    MORPH_FFT_F64 = 3,       /* FP64 FFT, the plain form of the paper's Step 2 */
    MORPH_NTT = 4            /* number-theoretic transform mod a prime > |B|: exact integer
                                convolution (Sec. 2.2), no round-off bound needed */
};

enum morph_flags {
    MORPH_F_ALLOW_UNPROVEN_F32 = 1,  /* run FFT_F32 even where the a-priori bound fails */
    MORPH_F_VALIDATE = 2,            /* FFT routes: measure max |C - rint C| over every degree */
    MORPH_F_AUTOTUNE = 4             /* AUTO: on the first call for a problem key, time each exact
                                        route the models do not rule out (on the caller's stream and
                                        output buffers, synchronising it) and keep the fastest */
};

typedef struct {
    int method;              /* enum morph_method */
    int flags;               /* enum morph_flags, or-ed */
    float *count_err;        /* device, nullable: FFT routes write max |C - rint C| seen */
} morph_opts;

/* What the planner chose for one problem (morph_plan_query). */
typedef struct {
    int method;              /* enum morph_method actually used */
    int R;                   /* number of degrees: L + max b */
    int taps;                /* |B| */
    double f32_bound;        /* a-priori bound on the FP32 FFT count error of the tiling an
                                FP32 request runs (< 0.5: proven exact; else no tiling is) */
    double f64_bound;        /* the same bound for FP64 */
    int fft_nx, fft_ny;      /* FFT sizes of the FFT routes */
    int groups, passes;      /* direct route: offset levels stacked per pass, passes */
    int tile_w, tile_h;      /* direct route: output tile (columns x rows) */
    double est_flop;         /* issued dense FLOP (direct) or FFT FLOP (FFT routes) */
    size_t workspace_bytes;  /* device workspace the call needs */
    int unit_tiles;          /* direct route: horizontally adjacent tiles per work unit (1 or 2) */
    int unit_blocks;         /* direct route: 128-byte K blocks of image planes staged per SE row
                                and unit (two tiles share them) */
    int k_steps;             /* direct route: 32-column K steps per SE row and tile */
    int level_chunks;        /* direct route: chunks of grey levels (4, 8 or 16 levels each) a
                                unit contracts when its band holds every level (est_flop counts
                                that many); a unit's band usually needs fewer */
    int ring_stages;         /* direct route: stages of the kernel's shared-memory operand ring (4 for
                                one-tile units, 3 when units hold two tiles) */
    int unit_queue;          /* direct route: units the kernel's producer may publish ahead of
                                its MMA issuer and epilogue */
} morph_plan_info;

/* --------------------------------------------------------------- calls */

/* Create a context on `device` (the CUDA ordinal).  The call makes `device`
 * current on the calling thread.  Returns MORPH_OK and *out, or an error. */
int morph_ctx_create(int device, morph_ctx **out);

/* Wait for the context's work, release its device memory and free it. */
int morph_ctx_destroy(morph_ctx *ctx);

/* Plans (SE blocks, FFT / NTT tables and SE spectra) are cached per context,
 * keyed by shape, L, SE and route.  The cache holds at most `bytes` of device
 * memory (default 16 GiB); beyond it the least recently used plans are
 * dropped (launched work and captured batches keep their own references;
 * freeing waits for the device as cudaFree does).  Host-only otherwise. */
int morph_ctx_set_cache_limit(morph_ctx *ctx, size_t bytes);
/* Device bytes held by the plan cache and the number of cached plans (either nullable). */
int morph_ctx_cache_info(const morph_ctx *ctx, size_t *bytes, int *nplans);

/* Plan (without running) the dilation (op = 0) or erosion (op = 1) of `f` by
 * `b` under `opts` (nullable = AUTO).  With a context the plan is built and
 * cached (the direct route's SE blocks are written on the device); with
 * ctx = NULL nothing touches the device and only the host-side figures are
 * filled in. */
int morph_plan_query(morph_ctx *ctx, const morph_image *f, const morph_se *b, int op,
                     const morph_opts *opts, morph_plan_info *out);

/* Device workspace (bytes) that a call will grow the context's workspace to:
 * op 0 = morph_dilate, 1 = morph_erode, 2 = morph_dilate_backward, 3 =
 * morph_erode_backward, for `f` and `b` under `opts` (nullable = AUTO).
 * Host-only: no device work, no allocation; `ctx` may be NULL (then the AUTO
 * decision is not cached).  The workspace is owned by the context and reused
 * by later calls; composite and 3-D calls additionally use a second
 * workspace of 2 resp. 3 int32 images. */
int morph_workspace_size(morph_ctx *ctx, const morph_image *f, const morph_se *b, int op,
                         const morph_opts *opts, size_t *bytes);

/* Dilation, Eq. 6 (Steps 1-3 of Sec. 3).  out: int32 [n][h][w] device;
 * out_count: nullable int32 [n][h][w] device, the top coefficient.
 * The first call for a new (SE, L, shape, method) builds and caches a plan,
 * which may allocate device memory and synchronize the device. */
int morph_dilate(morph_ctx *ctx, const morph_image *f, const morph_se *b, int32_t *out,
                 int32_t *out_count, const morph_opts *opts, morph_stream_t stream);

/* Erosion, Eq. Erosion, by the duality of Sec. 2.1.  Arguments as morph_dilate;
 * out_count counts the taps attaining the minimum. */
int morph_erode(morph_ctx *ctx, const morph_image *f, const morph_se *b, int32_t *out,
                int32_t *out_count, const morph_opts *opts, morph_stream_t stream);

/* Dilation (Eq. 6new / Eq. 6) and erosion (Eq. Erosion) by an SE with
 * device-resident offsets, on the FP8 tensor-core route; arguments and results
 * as morph_dilate / morph_erode.  Every offset level 0..max_offset is planned
 * for, so a tight bound costs less.  The plan (cached per mask, bound and
 * shape) is built on the first call; later calls only read the offsets on the
 * device (each call writes the SE's Toeplitz blocks into the context's
 * workspace), so the call neither synchronizes nor copies to the host. */
int morph_dilate_dev_se(morph_ctx *ctx, const morph_image *f, const morph_se_dev *b, int32_t *out,
                        int32_t *out_count, morph_stream_t stream);
int morph_erode_dev_se(morph_ctx *ctx, const morph_image *f, const morph_se_dev *b, int32_t *out,
                       int32_t *out_count, morph_stream_t stream);

/* 3-D volumes (the method is stated for N-D images, Sec. 2.1 and Sec. 3). */
typedef struct {
    const void *data;        /* device pointer to voxel (0,0,0) of volume 0 */
    int dtype;               /* enum morph_dtype */
    int n, d, h, w;          /* volumes, slices, rows, columns (each >= 1) */
    int64_t row_stride;      /* elements between rows */
    int64_t slice_stride;    /* elements between slices */
    int64_t volume_stride;   /* elements between volumes */
    int L;                   /* grey levels, 2 <= L <= 256 */
} morph_volume;

typedef struct {
    int kd, kh, kw;          /* box size; kd 1..512, kh and kw as morph_se */
    int oz, oy, ox;          /* box entry of the origin */
    const uint8_t *mask;     /* host, kd*kh*kw, slice-major then row-major */
    const int32_t *offset;   /* host, kd*kh*kw, >= 0 where mask != 0 */
} morph_se3d;

/* 3-D dilation / erosion with the conventions of the 2-D calls (taps outside
 * the volume skipped; 0 resp. L-1 where no tap is valid; int32, unclamped).
 * out and nullable out_count: int32 [n][d][h][w] device, contiguous.  Each SE
 * slice runs through the 2-D routes over all slices of a volume; the
 * per-slice results are folded by max (min) with counts summed at ties.
 * Uses the context's second workspace (three int32 volumes). */
int morph_dilate3d(morph_ctx *ctx, const morph_volume *f, const morph_se3d *b, int32_t *out,
                   int32_t *out_count, const morph_opts *opts, morph_stream_t stream);
int morph_erode3d(morph_ctx *ctx, const morph_volume *f, const morph_se3d *b, int32_t *out,
                  int32_t *out_count, const morph_opts *opts, morph_stream_t stream);

/* Composite operators (the combinations named in the paper's conclusion),
 * computed exactly from the dilation and erosion above, with the same
 * conventions (taps outside F skipped; int32, unclamped):
 *   morph_open:     (f (-) b) (+) b   -- values in [-max b, L-1]
 *   morph_close:    (f (+) b) (-) b   -- values in [0, L-1+max b]
 *   morph_gradient: (f (+) b) - (f (-) b), the Beucher gradient
 * The intermediate result is shifted into [0, L + max b) before the second
 * operation, so opening and closing need L + max b <= 256
 * (MORPH_E_UNSUPPORTED otherwise).  out: int32 [n][h][w] device.  The
 * context keeps a device buffer of two int32 images for the intermediates
 * (grown with a device synchronize). */
int morph_open(morph_ctx *ctx, const morph_image *f, const morph_se *b, int32_t *out, const morph_opts *opts,
               morph_stream_t stream);
int morph_close(morph_ctx *ctx, const morph_image *f, const morph_se *b, int32_t *out, const morph_opts *opts,
                morph_stream_t stream);
int morph_gradient(morph_ctx *ctx, const morph_image *f, const morph_se *b, int32_t *out, const morph_opts *opts,
                   morph_stream_t stream);

/* Backward of the dilation for a learnable layer.  The upstream gradient
 * g = grad_out (fp32 [n][h][w], device) at x is routed to every tap attaining
 * the maximum, split equally among the cD(x) of them:
 *   grad_in(p)  = sum_{y in B, p+y in F, f(p)+b(y) = D(p+y)} g(p+y) / cD(p+y)
 *   grad_se(y)  = sum_{x in F, x-y in F, f(x-y)+b(y) = D(x)} g(x) / cD(x),
 * the latter being the coefficient of t^b(y) in the lag-y cross-correlation
 * of g/cD * t^D with t^-f.  D and cD are the forward outputs (device int32).
 * At most 65535 taps (MORPH_E_UNSUPPORTED beyond).
 * grad_in: nullable fp32 [n][h][w] device (overwritten).  grad_se: nullable
 * fp32 [kh][kw] device (overwritten; 0 outside B).  Deterministic: fixed
 * summation order, no atomics on floating point. */
int morph_dilate_backward(morph_ctx *ctx, const morph_image *f, const morph_se *b,
                          const int32_t *D, const int32_t *cD, const float *grad_out,
                          float *grad_in, float *grad_se, morph_stream_t stream);

/* Backward of the erosion: g(x) goes to every tap attaining the minimum,
 * split equally among the cE(x) of them, and b enters with a minus sign:
 *   grad_in(p)  =   sum_{y in B, p-y in F, f(p)-b(y) = E(p-y)} g(p-y) / cE(p-y)
 *   grad_se(y)  = - sum_{x in F, x+y in F, f(x+y)-b(y) = E(x)} g(x) / cE(x).
 * E and cE are morph_erode's outputs; other arguments as morph_dilate_backward. */
int morph_erode_backward(morph_ctx *ctx, const morph_image *f, const morph_se *b,
                         const int32_t *E, const int32_t *cE, const float *grad_out,
                         float *grad_in, float *grad_se, morph_stream_t stream);

/* The two backward passes for an SE with device-resident offsets (the outputs
 * of morph_dilate_dev_se / morph_erode_dev_se); arguments otherwise as
 * morph_dilate_backward / morph_erode_backward.  No host copy, no sync. */
int morph_dilate_backward_dev_se(morph_ctx *ctx, const morph_image *f, const morph_se_dev *b,
                                 const int32_t *D, const int32_t *cD, const float *grad_out,
                                 float *grad_in, float *grad_se, morph_stream_t stream);
int morph_erode_backward_dev_se(morph_ctx *ctx, const morph_image *f, const morph_se_dev *b,
                                const int32_t *E, const int32_t *cE, const float *grad_out,
                                float *grad_in, float *grad_se, morph_stream_t stream);

/* One problem of a heterogeneous batch. */
typedef struct {
    morph_image f;
    morph_se se;
    int op;                  /* 0 = dilation, 1 = erosion */
    int32_t *out;            /* device int32 [n][h][w] */
    int32_t *out_count;      /* nullable */
} morph_problem;

/* Run `n` problems on `stream`: one encoder launch and one persistent
 * tcgen05 launch cover every problem on the FP8 direct route (tiles of the
 * most expensive problems first); problems on an FFT route follow with their
 * own launches.  opts applies to every problem (AUTO: the planner chooses per
 * problem); opts->count_err, if given, receives the max over the FFT problems.
 * Plans are built on first use.  The problem descriptors are copied to the
 * context's workspace in stream order before the kernels are queued. */
int morph_run_batch(morph_ctx *ctx, const morph_problem *p, int n, const morph_opts *opts,
                    morph_stream_t stream);

typedef struct morph_batch morph_batch;

/* Plan the batch once and capture its launches into a CUDA graph with a
 * workspace of its own.  The problems' device pointers are baked into the
 * graph: each morph_batch_launch replays it on `stream`, reading the current
 * contents of the same buffers.  morph_batch_destroy waits for the device
 * and frees the graph and its workspace. */
int morph_batch_capture(morph_ctx *ctx, const morph_problem *p, int n, const morph_opts *opts,
                        morph_batch **out);
/* Replay a captured batch on `stream` (asynchronous). */
int morph_batch_launch(morph_batch *b, morph_stream_t stream);
/* Wait for the device, then free a captured batch. */
int morph_batch_destroy(morph_batch *b);

/* Synchronize `stream`, then return (and clear) the device error word:
 * MORPH_E_RANGE for a pixel outside [0, L), MORPH_E_TIMEOUT if a bounded wait
 * gave up, MORPH_OK otherwise. */
int morph_stream_check(morph_ctx *ctx, morph_stream_t stream);

/* Static text for a status code. */
const char *morph_strerror(int status);

/* Number of kernel launches the library issued through this context since
 * creation (every launch, every route). */
uint64_t morph_launch_count(const morph_ctx *ctx);

/* Limit, in nanoseconds, of every bounded device wait of the library's
 * pipelined kernels launched through this context from now on (ns = 0: the
 * default, 4 s).  A wait that reaches its limit makes its thread block stop:
 * it raises the device error word, lets the copies and tensor-core work it
 * already issued complete, frees its tensor memory and returns, so that
 * morph_stream_check reports MORPH_E_TIMEOUT and the context stays usable.
 * A failure-handling hook: a limit shorter than the kernel's ordinary waits
 * (a few microseconds) makes that path run on purpose.  Host-only. */
int morph_ctx_set_wait_limit(morph_ctx *ctx, uint64_t ns);

/* Number of tcgen05 MMA instructions (M = 128, N = 256, K = 32, FP8; each
 * 2 x 128 x 256 x 32 FLOP) that the FP8 direct route's kernel issued through
 * this context since creation, counted on the device by the issuing thread
 * (a measurement hook: the issued tensor work, zero-padding included).
 * Synchronises the device; *out receives the count. */
int morph_mma_count(morph_ctx *ctx, uint64_t *out);

/* Multiply-adds of the contraction the FP8 route's units needed -- for each
 * unit and offset-group pass, the pass's taps x the grey levels of its band x
 * the unit's pixels (Step 2 restricted to the degrees Step 3 can read) --
 * summed on the device by the direct kernel's epilogue over the calls through
 * this context (host-resident SEs with L > 16; a measurement hook, the
 * method's own work for the roofline).  Synchronises the device; *out
 * receives the sum. */
int morph_band_work(morph_ctx *ctx, uint64_t *out);

/* Measurement hook: the rate, in TFLOP/s, of the tensor-core instruction the
 * FP8 route issues (tcgen05.mma kind::f8f6f4, M = 128, N = 256, K = 32, FP32
 * accumulation) when every SM issues it back to back from shared memory, with
 * no copies and no waits: the tensor pipe's FP8 peak on this GPU at its
 * present clock (about 1 ms of device time, on a stream of its own; blocks
 * until done).  Its wait for the MMAs is bounded: a tensor pipe that does not
 * finish raises MORPH_E_TIMEOUT through morph_stream_check.  *tflops
 * receives the rate. */
int morph_tc_fp8_peak(morph_ctx *ctx, double *tflops);

/* Per-kernel device time, summed over the launches recorded while profiling
 * was on. */
typedef struct {
    char name[48];           /* kernel name */
    uint64_t launches;
    double total_ms;         /* sum of CUDA-event durations on the launching stream */
} morph_kernel_time;

/* on != 0: record a CUDA event pair on the launching stream around every
 * kernel the context launches from now on (a timing hook; adds a few
 * microseconds of host work per launch).  on == 0: stop recording. */
int morph_profile_enable(morph_ctx *ctx, int on);

/* Synchronize the device, turn the recorded event pairs into per-kernel
 * totals, write up to `cap` of them to `out`, set *n to the number of
 * kernels, and clear the record. */
int morph_profile_read(morph_ctx *ctx, morph_kernel_time *out, int cap, int *n);

/* Dilation (op = 0) or erosion (op = 1) by the FP8 tensor-core route,
 * without allocating any device memory and without a context.  The paper has
 * no counterpart: this serves callers that cannot call cudaMalloc / cudaFree,
 * such as code running where another component owns the device memory
 * budget, or host paths that must not block on the device-wide
 * synchronisation an allocation may imply.
 *
 * Inputs and outputs are as for morph_dilate / morph_erode (out and the
 * nullable out_count are int32 [n][h][w] device buffers of the caller).
 * dev_status: nullable device uint32; when given, it receives the device
 * error bits of this call (0 = ok, 1 = a pixel outside [0, L), 2 = a bounded
 * wait gave up), written in stream order after the result.
 *
 * Everything else (error word, plan metadata, SE Toeplitz blocks, FP8
 * indicator planes) lives in one fixed 64 MiB __device__ array that every GPU
 * loading the library holds until the process exits.  A problem fits when
 * n*h*L*round_up(w, 16) bytes of planes plus the SE blocks (up to 2 MB) fit in
 * 64 MiB; a larger one is rejected with MORPH_E_NOMEM before any work is
 * queued.  The first call on a device (with that device current) looks up the
 * array's device address once; make that first call before any stream
 * capture.  All calls share the array: each call clears the error word it
 * uses, and calls whose GPU work overlaps race with each other (issue them in
 * one stream).  Plans are rebuilt on every call. */
int morph_run_noalloc(const morph_image *f, const morph_se *b, int op, int32_t *out, int32_t *out_count,
                      uint32_t *dev_status, morph_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MORPH_H */
