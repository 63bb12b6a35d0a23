// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "morph.h"

namespace morph {

// ----------------------------------------------------------------- errors
#define MORPH_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t e__ = (expr);                              \
        if (e__ != cudaSuccess) {                              \
            morph::set_last_cuda_error(e__, #expr, __FILE__, __LINE__); \
            return MORPH_E_CUDA;                               \
        }                                                      \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* expr, const char* file, int line);

// --------------------------------------------------- encoder (Step 1, Eq. 7)
// One image batch is written as FP8 E4M3 indicator planes
//   planes[n][i][v][c] = 1.0 if level(f(n,i,c - shift)) == v else 0,
// with level(f) = f (dilation) or L-1-f (erosion by duality); row pitch
// w_pad (a multiple of 16 bytes), columns outside [shift, shift + w) zero.
// The shift (0..31) puts the K windows of the direct route's tiles on
// 32-byte boundaries without shifting the tile grid.
struct EncodeJob {
    const void* src;
    int dtype;              // morph_dtype
    int n, h, w;
    long long row_stride, batch_stride;
    int L;
    int flip;               // 1: level = L-1-f
    uint8_t* planes;
    int w_pad;
    int shift;              // plane column of image column 0
    long long item_base;    // first work item of this job (batched launch)
    const int* lev_range;   // nullable: planes are written for the levels r[0]..r[1] only (the rest
                            // are never read: the direct problem's band range)
};

// Output adjustment of one pass of a composite operator, applied by the route's
// epilogue: the stored value is v + add - (sub ? sub[pixel] : 0), v the
// dilation value (or the erosion's L - 1 - D).  The top counts are unchanged.
struct OutAdjust {
    int add = 0;
    const int32_t* sub = nullptr;   // int32 [n][h][w], same layout as the output
};

// ------------------------------------------- FP8 tcgen05 direct route (Step 2)
constexpr int kDirectMaxPasses = 32;
constexpr long long kDirectSplitMinUnits = 2 * 152;   // split two-tile units only with two waves on 152 SMs
constexpr int kDirectN = 256;        // MMA N: image rows x grey levels of one chunk
constexpr int kDirectM = 128;        // MMA M: offset groups x output columns
constexpr int kDirectLc = 16;        // grey levels per chunk of the N axis when L <= 16 or L > 64 (16 image rows)
constexpr int kDirectLcBand = 8;     // ... when 16 < L <= 64 and L + max b > kDirectNarrowMaxR (32 image rows)
constexpr int kDirectLcNarrow = 4;   // ... when 16 < L <= 64 and L + max b <= kDirectNarrowMaxR (64 image rows)
constexpr int kDirectNarrowMaxR = 4095;   // degrees + 1 of 4-level plans fit the 12 bits of a packed run entry
constexpr int kBandTapsMax = 264;    // taps of the per-unit lower bound on the top degree (16 x 16 cells + origin)

// Per unit of a direct launch: hi = the largest level in the unit's input
// window, lb = a lower bound on the smallest dilation value of the unit's
// pixels (-1: none).  A product f(x - y) + b(y) that reaches a top degree has
// level >= lb - b(y), so the pass of offset groups whose largest offset is
// wmax contracts only the levels [max(0, lb - wmax), hi] (none when
// lb - wmax > hi), in chunks of Lc levels from the top: chunk c covers
// hi - Lc (c + 1) + 1 .. hi - Lc c.
struct DirectBand {
    int hi;
    int lb;
};

struct DirectProblemDev {
    CUtensorMap tmA;        // Toeplitz blocks: [blocks * 128 rows][128 B]
    CUtensorMap tmB;        // planes: dims (w, L, h, n), box (128, Lc, rows_n, 1)
    int32_t* out;           // [n][h][w]
    int32_t* out_cnt;       // nullable
    int out_add;            // output adjustment (OutAdjust)
    const int32_t* out_sub;
    const int* meta;        // pass_row_begin[n_pass+1], group_w[n_pass*8], rows[...], band taps (3 ints each)
    const DirectBand* band; // per unit; nullptr: every level, ceil(L / Lc) chunks
    int* lev_range;         // with band: [lowest, highest] level any unit's chunks read (band range kernel)
    const int32_t* dev_off; // device-resident SE offsets (box order of the caller's SE), or nullptr
    int dev_reflect;        // 1: read dev_off at kh kw - 1 - t (the erosion's reflected SE)
    const void* src;        // the image (read by the band kernel)
    int dtype;
    long long row_stride, batch_stride;
    int kh, maxb, band_tap_off, n_band_taps;
    int band_seg_off, n_band_segs;   // runs of band taps with one offset (0: offsets on the device)
    int pass_taps_off;      // meta offset of the taps per pass (-1 entries: offsets on the device)
    int h, w, nimg, L;
    int Lc, rows_n, J, G;
    int n_pass, nk, ksteps, kw;
    int oy, ox, e, erode;
    int shift;              // plane column of image column 0 (TMA x = image column + shift)
    int T;                  // horizontally adjacent tiles per unit (1 or 2)
    int split;              // T = 2 with tile 1 one J-shift along a multi-block K window
    int nb;                 // 128-byte K blocks staged per SE row and unit (nk, or nk + 1 when split)
    int tiles_x, tiles_y;   // units (of T tiles) across, tile rows down
    long long tile_base;    // first global tile of this problem
    long long tiles;        // tiles of this problem
};

struct DirectLaunch {
    DirectProblemDev single;         // used when many == nullptr
    const DirectProblemDev* many;    // device array (batched launch)
    int nprob;
    long long total_tiles;
    unsigned int* err;
    unsigned long long* mma_count;   // nullable: MMAs issued, added once per CTA
    unsigned long long* band_work;   // nullable: multiply-adds of the band-limited contraction (direct kernel)
    unsigned long long* next_unit;   // nullable: units claimed after each CTA's first (zeroed by the band kernel);
                                     // nullptr: CTA b takes units b, b + grid, ...
    unsigned long long wait_ns;      // limit of each bounded wait; 0 = kWaitLimitNs
};

struct DirectPlan {
    int L = 0, Lc = 0, rows_n = 0, J = 0, G = 0, n_pass = 0, nk = 0, ksteps = 0, T = 1, split = 0, nb = 0;
    int band_tap_off = 0, n_band_taps = 0;   // lower-bound taps (oy - r, ox - c, b) in meta
    int band_seg_off = 0, n_band_segs = 0;   // ends of their runs of equal b (host offsets only)
    int pass_taps_off = 0;                    // taps of each pass in meta
    int kh = 0, kw = 0, oy = 0, ox = 0, e = 0, erode = 0, shift = 0;
    int h = 0, w = 0, nimg = 0, w_pad = 0;
    int tiles_x = 0, tiles_y = 0;
    long long tiles = 0;
    int n_levels = 0, taps = 0, maxb = 0;
    long long active_rows_total = 0;  // sum over passes of active SE rows
    std::vector<int> meta;
    uint8_t* d_toeplitz = nullptr;
    int* d_meta = nullptr;
    uint8_t* d_mask = nullptr;        // device-resident-SE plans: the (reflected) mask for the per-call Toeplitz build
    long long toeplitz_blocks = 0;
    CUtensorMap tmA;
    double issued_flop = 0;           // dense MMA FLOP per launch with every level (ceil(L / Lc) chunks)
    ~DirectPlan();
};

// -------------------------------------------------------- FFT route (Step 2)
struct FftAxis {
    int N;         // transform length (2^a 3^b 5^c, <= 2048)
    int nst;       // Stockham stages
    int rad[16];   // radix of each stage (4, 2, 3, 5)
    int tstep[16];       // N / (Ns R): twiddle stride of each stage
    uint32_t nsm[16];    // ceil(2^32 / Ns), Ns the product of the earlier radices (0 for Ns = 1)
};

struct FftPlan {
    int prec = 8;                 // 4 = FP32, 8 = FP64
    int taps = 0, R = 0, K = 0;   // |B|, degrees, grey frequencies (Rf/2 + 1)
    int Rf = 0;                   // grey-axis DFT length: smallest 2^a 3^b 5^c >= R
    int kh = 0, kw = 0, ry = 0, rx = 0;
    int To_y = 0, To_x = 0, Rin_y = 0, Win_x = 0;
    int tiles_y = 0, tiles_x = 0;
    long long ntiles = 0;
    int wave_tiles = 0, colgroup = 4, pixgroup = 16;
    int kgroup = 1;               // grey frequencies per pass of the row kernels (power of two)
    int col_threads = 256, pix_threads = 256, row_threads = 256;
    size_t buf_bytes = 0;         // spectra of one wave of tiles
    size_t ws_bytes = 0;          // buf_bytes + per-tile scan bounds
    bool range_fft = false;       // grey-axis inverse by FFT (long axes) or by direct evaluation
    double bound = 0;             // a-priori bound on |C - C_exact| for this precision
    double flop = 0;
    FftAxis ax, ay, ar;
    void* tw_x = nullptr;
    void* tw_y = nullptr;
    void* wr = nullptr;
    void* S = nullptr;
    ~FftPlan();
};

// ------------------------------------------------ exact NTT route (Step 2)
struct NttAxis {
    int N;                 // transform length (2^a 3^b 5^c, c <= 3, <= 2048)
    int nst;               // Stockham stages
    int rad[16];           // radix of each stage (16, 4, 2, 3, 5)
    int tstep[16];         // N / (Ns R): twiddle stride of each stage
    uint32_t nsm[16];      // ceil(2^32 / Ns) with Ns the product of the earlier radices (0 for Ns = 1)
};

struct NttPlan {
    int taps = 0, R = 0, Rf = 0;  // |B|, degrees, grey-axis length (= grey frequencies)
    int kh = 0, kw = 0, ry = 0, rx = 0;
    int To_y = 0, To_x = 0, Rin_y = 0, Win_x = 0;
    int tiles_y = 0, tiles_x = 0;
    long long ntiles = 0;
    int wave_tiles = 0, kgroup = 1, colgroup = 8, pixgroup = 16;
    int col_threads = 256, pix_threads = 256;
    size_t buf_bytes = 0, ws_bytes = 0;
    double ops = 0, bytes = 0;    // estimated integer operations and HBM bytes per call
    NttAxis ax, ay, ar;
    uint2* tw_x = nullptr;        // (omega_N^m, Shoup quotient) pairs
    uint2* tw_y = nullptr;
    uint2* tw_r = nullptr;
    uint32_t* wr = nullptr;       // omega_Rf^m
    uint32_t* S = nullptr;
    ~NttPlan();
};

// ------------------------------------------------------------------- plans
enum Route { ROUTE_EMPTY = 0, ROUTE_DIRECT = 1, ROUTE_FFT32 = 2, ROUTE_FFT64 = 3, ROUTE_NTT = 4 };

struct Plan {
    int route = ROUTE_EMPTY;
    DirectPlan direct;
    FftPlan fft;
    NttPlan ntt;
    size_t dev_bytes = 0;         // device memory the plan holds (tables, SE blocks or spectrum)
    uint64_t last_use = 0;        // context tick of the last lookup (LRU eviction)
};

// Device memory the context's plan cache may hold before least-recently-used
// plans are dropped (work already launched, and captured graphs, keep their
// own references to the plans they use).
constexpr size_t kPlanCacheBytes = size_t(16) << 30;
// AUTO decisions kept per context (host memory: each key holds the SE); the
// table is cleared when full, and decisions are recomputed on demand.
constexpr size_t kRouteCacheEntries = 4096;

}  // namespace morph

struct morph_prof_rec {
    const char* name;
    cudaEvent_t a, b;
};

struct morph_ctx {
    bool prof_on = false;
    std::vector<morph_prof_rec> prof;     // recorded event pairs
    std::vector<cudaEvent_t> prof_pool;   // free events
    int device = 0;
    int num_sms = 0;
    unsigned int* d_err = nullptr;        // device error word
    unsigned long long* d_mma = nullptr;  // [0] MMAs issued by the direct route, [1] its band-limited
                                          // method work in multiply-adds (measurement hooks)
    unsigned long long wait_ns = 0;       // limit of the kernels' bounded waits; 0 = the default
    void* ws = nullptr;                   // device workspace
    size_t ws_bytes = 0;
    void* ws2 = nullptr;                  // intermediate images of composite operators
    size_t ws2_bytes = 0;
    uint64_t launches = 0;
    std::vector<cudaStream_t> branch;     // batch branches for transform-route problems (created on demand)
    std::vector<cudaEvent_t> branch_ev;   // their join events
    cudaEvent_t fork_ev = nullptr;
    std::unordered_map<std::string, std::shared_ptr<morph::Plan>> plans;
    size_t plan_bytes = 0;                // sum of the cached plans' dev_bytes
    size_t plan_budget = morph::kPlanCacheBytes;
    uint64_t plan_tick = 0;
    std::unordered_map<std::string, std::shared_ptr<void>> aux_plans;   // backward tap lists, ...
    std::unordered_map<std::string, int> route_cache;                   // AUTO decisions
};

namespace morph {

// Kernel attributes (the dynamic shared-memory opt-in) belong to a device's
// context: each group of kernels is set up once per device.  kernels_ready
// tells whether `group` is set up on `device`; mark_kernels_ready records it
// after the setup succeeded (a race only repeats the idempotent setup).
enum KernelGroup { kGroupDirect = 0, kGroupFft32, kGroupFft64, kGroupFftPlane, kGroupNtt, kGroupBand, kGroupCount };
bool kernels_ready(int device, KernelGroup group);
void mark_kernels_ready(int device, KernelGroup group);

// Timing hook: event pair around one launch while profiling is on.
void prof_begin(morph_ctx* ctx, cudaStream_t st, const char* name);
void prof_end(morph_ctx* ctx, cudaStream_t st);

// Workspace of at least `bytes` (grows with a device synchronize).
int ctx_workspace(morph_ctx* ctx, size_t bytes, void** out);
// Second workspace for intermediate int32 images of composite and 3-D operators.
int ctx_workspace2(morph_ctx* ctx, size_t bytes, void** out);

// Encoding of tensor maps through the driver entry point.
int encode_tmap(CUtensorMap* m, CUtensorMapDataType dt, int rank, void* base, const uint64_t* dims,
                const uint64_t* strides_bytes, const uint32_t* box, CUtensorMapSwizzle swz);

// Kernel launchers (defined next to their kernels).
int launch_encode(morph_ctx* ctx, const EncodeJob* jobs, int njobs, long long total_items,
                  EncodeJob* d_jobs, cudaStream_t st);
int build_direct_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, int erode, DirectPlan* p);
int plan_direct_host(const morph_image* f, const morph_se* se, int erode, DirectPlan* p, int dev_bound = -1);
// uniform_T: tiles per unit shared by every problem of a batched launch (1 or 2), 0 if mixed
// unit kind: 1 = one tile, 2 = two tiles in one K block, 3 = two split tiles; 0 = per problem
int direct_kind(const DirectProblemDev& d);
int launch_direct(morph_ctx* ctx, const DirectLaunch& dl, cudaStream_t st, int uniform_kind = -1);
int direct_smem_bytes(int stages);
int direct_stages(int unit_tiles);   // ring depth of the direct kernel for units of that many tiles
int direct_unit_queue();   // slots of the direct kernel's unit queue
void direct_fill_problem(const DirectPlan& p, DirectProblemDev* d, const uint8_t* planes, int32_t* out,
                         int32_t* out_cnt, long long tile_base, int* status);
// device-resident SE offsets: plan (metadata and mask on the device), the per-call Toeplitz
// blocks and their size
int build_direct_plan_dev(const morph_image* f, const morph_se* se, int bound, int erode, DirectPlan* p);
size_t direct_toeplitz_bytes(const DirectPlan& p);
int launch_toeplitz_dev(morph_ctx* ctx, const DirectPlan& p, const int32_t* dev_off, int reflect, uint8_t* blocks,
                        CUtensorMap* tmA, cudaStream_t st);
// the image and the per-unit band buffer of a problem (band may be nullptr: every level)
void direct_fill_band(DirectProblemDev* d, const morph_image* f, DirectBand* band);
// bytes of the per-unit band buffer for an image of this shape (any plan), the launch's
// unit counter included
size_t direct_band_bytes(const morph_image* f);
// the unit counter in a band buffer of this image
unsigned long long* direct_unit_counter(DirectBand* band, const morph_image* f);
// per-unit grey-level bands of every problem of a direct launch (before launch_direct, same
// stream); win_bytes: shared memory per CTA for the unit windows (the largest
// direct_band_window of the launch's problems; larger windows take a slower path);
// slabs: the largest direct_band_slabs of the launch's problems
int launch_band(morph_ctx* ctx, const DirectLaunch& dl, int win_bytes, int slabs, cudaStream_t st);
// after launch_band: each problem's lev_range from its units' bands (the levels the encoder must
// write), one CTA per problem
int launch_band_range(morph_ctx* ctx, const DirectLaunch& dl, cudaStream_t st);
int direct_band_window(const DirectProblemDev& d);
int direct_band_slabs(const DirectProblemDev& d);   // band entries per unit (slabs of 32 image rows)
int launch_fill_empty(morph_ctx* ctx, int32_t* out, int32_t* cnt, long long n, int value, cudaStream_t st,
                      const OutAdjust* adj = nullptr);
// validation, erosion reflection, route choice and (cached) plan of one problem
int prepare_problem(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, const morph_opts* opts,
                    std::shared_ptr<Plan>* plan, bool in_batch = false);
size_t planes_bytes(const morph_image* f);
// workspace of one direct-route call: the planes, then the per-unit band buffer
size_t direct_ws_bytes(const morph_image* f);
// time the exact routes of one AUTO problem on its own buffers and cache the fastest (MORPH_F_AUTOTUNE)
int tune_problem(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, const morph_opts* opts,
                 int32_t* out, int32_t* cnt, cudaStream_t st);
// one dilation (erode = 0) or erosion (erode = 1), the body of morph_dilate / morph_erode
int run_one(morph_ctx* ctx, const morph_image* f, const morph_se* b, int erode, int32_t* out, int32_t* cnt,
            const morph_opts* opts, cudaStream_t st, const OutAdjust* adj = nullptr);
int plan_fft_tiles(const morph_image* f, const morph_se* se, int prec, bool unproven, FftPlan* p);
int build_fft_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, int prec, bool unproven, FftPlan* p);
int launch_fft(morph_ctx* ctx, const FftPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
               float* count_err, int validate, cudaStream_t st, const OutAdjust* adj = nullptr);
int launch_fft_in(morph_ctx* ctx, const FftPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                  float* count_err, int validate, void* buf, cudaStream_t st, const OutAdjust* adj = nullptr);
int plan_ntt_tiles(const morph_image* f, const morph_se* se, NttPlan* p);
double ntt_time_estimate(const NttPlan& p);
int build_ntt_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, NttPlan* p);
int launch_ntt(morph_ctx* ctx, const NttPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
               cudaStream_t st, const OutAdjust* adj = nullptr);
int launch_ntt_in(morph_ctx* ctx, const NttPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                  void* buf, cudaStream_t st, const OutAdjust* adj = nullptr);
// device workspace of morph_dilate_backward / morph_erode_backward (shares + partial sums)
size_t backward_workspace_bytes(const morph_image* f, const morph_se* b);
double fft_error_bound(const FftAxis& ax, const FftAxis& ay, const FftAxis& ar, double sqrtP, int taps, double u);

}  // namespace morph
