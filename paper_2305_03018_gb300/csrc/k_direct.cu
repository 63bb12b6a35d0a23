// Step 2 + Step 3 of the method (Sec. 3) on the 5th-generation tensor cores.
//
// Step 2 convolves the umbras: the count polynomial at pixel x has, at
// degree d, the number of SE taps y with f(x - y) + b(y) = d (Eq. Obs7).
// Split the taps by their offset level w = b(y): with
//     H_w(x, v) = #{ y in B : b(y) = w, x - y in F, f(x - y) = v }
// the polynomial is p_x(t) = sum_w t^w H_w(x, t).  All coefficients are
// non-negative, so by the degree rules of Prop. 2.3 (deg(p q) = deg p +
// deg q, deg(p + q) = max) Step 3 (Eq. 9) is
//     D(x) = max_w ( w + top{v : H_w(x, v) >= 1} ),
// and the top coefficient is the sum of H_w(x, D(x) - w) over the w that
// attain that maximum.
//
// H_w is a sum of one-hot level vectors over shifted pixels, computed as a
// dense FP8 GEMM per SE row r (exact: 0/1 operands, FP32 accumulation of
// counts <= |B| < 2^24):
//     acc[(g, j), (t, v)] += sum_k  T_r[(g, j), k] * U[i0 + t - (r - oy)][v][s + k]
//   A = T_r : 128 x K Toeplitz of SE row r; row (g, j) holds a 1 at
//             k = j + (kw - 1) - c for every tap (r, c) of offset group g;
//   B = U   : the FP8 indicator planes (Step 1, Eq. 7), rows (t, v) = image
//             row x grey level, K = a window of image columns;
//   D       : 128 x 256 FP32 accumulator in TMEM.
// M = 128 stacks G offset groups x J = 128 / G output columns, N = 256
// stacks rows_n image rows x Lc grey levels (16 x 16 when L <= 16 or L > 64,
// 64 x 4 -- or 32 x 8 with offsets beyond 4095 - L -- when 16 < L <= 64).
// A unit's levels are covered in chunks of Lc from the top of its
// level band (see "level bands" below): Step 3 needs only the degrees at or
// above each pixel's dilation value.  The epilogue reads a lane per (group,
// column), finds each group's top level by a descending scan and combines
// groups and chunks with (max, sum-at-max).
//
// Warp roles (192 threads, one persistent CTA per SM):
//   warp 0   : TMA producer (one lane) -- claims units (a per-launch counter, units with
//              two or more accumulations first), hands them to the other roles through a
//              shared-memory queue, and stages A and B tiles into a 4-stage ring (3 when
//              units hold two tiles);
//   warp 1   : TMEM allocator + MMA issuer (one lane), tcgen05.mma kind::f8f6f4;
//   warps 2-5: epilogue (TMEM -> registers -> SMEM reduction -> int32 output).
// Two TMEM accumulators (2 x 256 columns) let the epilogue of one unit
// overlap the MMAs of the next.  When two horizontally adjacent tiles fit in
// one 128-byte K window (2 J + kw - 1 <= 128), a unit holds both (T = 2):
// each A / B stage feeds the MMAs of both tiles, the second reading B from a
// start address J bytes further, which halves the operand bytes per MMA; the
// two accumulators then belong to the one unit.  When they do not fit but
// J >= 32 (flat or few-level SEs with wide rows), a unit may still hold two
// tiles ("split"): tile 1's K window is tile 0's shifted by J bytes, so K
// step ks of tile tt reads B byte 32 ks + tt J of the unit's window, i.e.
// block (32 ks + tt J) / 128, with A block ks / 4 -- the block staged with
// that B block or the one before it.  A row then stages ceil((J + 32 ksteps)
// / 128) blocks for both tiles instead of nk per tile, the blocks past the
// last A block carrying B only; each stage is released after the next
// stage's MMAs.
#include <cuda_fp16.h>

#include <algorithm>
#include <array>
#include <cstring>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

constexpr int kStageA = 128 * 128;             // 16 KB: 128 Toeplitz rows x 128 B of K
constexpr int kStageB = kDirectN * 128;        // 32 KB: 256 (row, level) rows x 128 B of K
constexpr int kStageBytes = kStageA + kStageB;
constexpr int kStagesMax = 4;

// Shared memory per unit kind TT (see k_direct_fp8): one-tile units (TT = 1) read one accumulator
// at a time, so `red` holds one tile's lane results (rows_n <= 64 x 128 lanes) and the ring takes
// a fourth stage; launches with two-tile units keep both tiles' results (both accumulators are
// read out before either is reduced) and three stages.  A stage of the disk's 190-byte K window
// carries 4 or 2 MMAs, and the commit-to-refill round trip of a stage (about 1700 cycles) needs
// that much MMA work queued behind it.
template <int TT>
struct DirectCfg {
    static constexpr int stages = TT == 1 ? 4 : 3;
    static constexpr int red = TT == 1 ? 64 * 128 : 2 * 64 * 128;   // 32-bit entries
};
constexpr int kRunEntries = 4096;              // pixels per unit, rows_n x J x T, with int2 running results
constexpr int kRunPacked = 2 * kRunEntries;    // ... with packed ones (4-level plans: 64 x 128)
constexpr int kRunWords = kRunPacked / 128;    // 32-bit words of running results per epilogue thread
constexpr int kDirectNarrowMinMmas = 96;       // MMAs per accumulation below which 4-level plans do not pay
constexpr int kDirectThreads = 192;
constexpr uint32_t kTmemCols = 2 * kDirectN;   // two accumulators

constexpr int kUnitQ = 4;                      // units the producer may publish ahead of the consumers

struct DirectSmemTail {
    uint64_t full[kStagesMax];
    uint64_t empty[kStagesMax];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t ufull[kUnitQ];                    // unit queue: published by the producer
    uint64_t uempty[kUnitQ];                   // ... read by the MMA issuer and the epilogue
    long long unit[kUnitQ];                    // unit index, -1: no more units
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

int direct_stages(int unit_tiles) { return unit_tiles == 1 ? DirectCfg<1>::stages : DirectCfg<2>::stages; }
int direct_unit_queue() { return kUnitQ; }
template <int TT>
int direct_smem_bytes() {
    return 1024 + DirectCfg<TT>::stages * kStageBytes + DirectCfg<TT>::red * 4 + static_cast<int>(sizeof(DirectSmemTail));
}

__device__ __forceinline__ const DirectProblemDev* direct_find(const DirectLaunch& dl, long long t) {
    if (dl.many == nullptr) return &dl.single;
    int lo = 0, hi = dl.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (dl.many[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return &dl.many[lo];
}

struct TileCoord {
    int n, i0, j0;
};

__device__ __forceinline__ TileCoord direct_tile(const DirectProblemDev* P, long long t) {
    const long long lt = t - P->tile_base;
    const long long per_img = static_cast<long long>(P->tiles_x) * P->tiles_y;
    TileCoord c;
    c.n = static_cast<int>(lt / per_img);
    const int rem = static_cast<int>(lt % per_img);
    c.i0 = (rem / P->tiles_x) * P->rows_n;
    c.j0 = (rem % P->tiles_x) * P->J * P->T - P->e;
    return c;
}

// Image rows of a unit that the band kernel takes at a time: as many as give 2048 pixel pairs
// (its largest per-CTA load: 8 pairs per thread), at most the unit's rows -- 32 for units 128
// columns wide, 64 for 64 columns, 16 for 256; a unit with more rows has several band entries,
// which the direct kernel combines.
__host__ __device__ __forceinline__ int band_slab_rows(int rows_n, int uw) { return min(rows_n, 4096 / uw); }

__host__ __device__ __forceinline__ int band_slabs(int rows_n, int uw) {
    const int r = band_slab_rows(rows_n, uw);
    return (rows_n + r - 1) / r;
}

// The unit's level band (see DirectBand), from its slabs' entries: hi = the
// largest level in their windows (-1: none read), lb = the smallest of their
// lower bounds (INT_MAX: no pixel).  Without a band buffer every level is
// covered.
__device__ __forceinline__ DirectBand direct_band(const DirectProblemDev* P, long long t) {
    DirectBand b;
    if (P->band == nullptr) {
        b.hi = P->L - 1;
        b.lb = -1;
        return b;
    }
    const int ns = band_slabs(P->rows_n, P->T * P->J);
    const DirectBand* e = P->band + (t - P->tile_base) * ns;
    b = e[0];
    for (int k = 1; k < ns; ++k) {
        b.hi = max(b.hi, e[k].hi);
        b.lb = min(b.lb, e[k].lb);
    }
    b.hi = b.hi < 0 ? P->L - 1 : b.hi;          // no pixel read: the unit's pixels have no valid tap
    // lb <= D(x) <= hi + max b for every pixel with a valid tap, so the pass holding the largest
    // offset always has a chunk; the clamp keeps that true for any input
    b.lb = min(b.lb, b.hi + P->maxb);
    return b;
}

// Chunks of Lc levels that pass p of the unit contracts (0: the pass cannot
// reach the unit's lower bound and is skipped).
__device__ __forceinline__ int direct_pass_chunks(const DirectProblemDev* P, const DirectBand& b, int p) {
    const int* gw = P->meta + (P->n_pass + 1) + p * 8;
    int wmax = 0;
    for (int g = 0; g < P->G; ++g) wmax = max(wmax, gw[g]);
    const int lo = b.lb - wmax;
    if (lo > b.hi) return 0;
    return (b.hi - max(lo, 0)) / P->Lc + 1;
}

// The unit the producer takes next.  With the launch's counter, claims run over 2 T indices (T
// units): index c < T offers unit c to a first round that takes the units of two or more
// accumulations, index c >= T offers unit c - T to a second round that takes the rest, so the
// long units go first and the launch ends on short ones.  Each CTA's first index is its own;
// later ones come from the counter.  Returns -1 when the indices are used up.
__device__ long long direct_claim(const DirectLaunch& dl, long long c) {
    const long long T = dl.total_tiles;
    while (c < 2 * T) {
        const long long t = c < T ? c : c - T;
        const DirectProblemDev* P = direct_find(dl, t);
        const DirectBand bd = direct_band(P, t);
        int n = 0;
        for (int p = 0; p < P->n_pass && n < 2; ++p) n += direct_pass_chunks(P, bd, p);
        if ((c < T) == (n >= 2)) return t;
        c = static_cast<long long>(gridDim.x) + static_cast<long long>(atomicAdd(dl.next_unit, 1ull));
    }
    return -1;
}

__device__ __forceinline__ bool epi_any_failed(bool failed) {
    uint32_t any;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(any) : "r"(static_cast<uint32_t>(failed)) : "memory");
    return any != 0;
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// One lane's read-out of an accumulator: N = 256 / LC image rows x LC levels, 32 columns
// (32 / LC rows) per TMEM load.  Each row's result is (top level in the chunk + 1) << 20 | its
// count (0: no level set; counts <= |B| <= 512^2 < 2^20), stored at red_m[row * 128].
template <int LC>
__device__ __forceinline__ void epi_read_rows(uint32_t trow, uint32_t* red_m) {
    constexpr int kRowsPerLoad = 32 / LC;
    for (int tr0 = 0; tr0 < kDirectN / LC; tr0 += kRowsPerLoad) {
        float v[32];
        tmem_ld_32x32b_x32(trow + static_cast<uint32_t>(tr0 * LC), v);
        tc_wait_ld();
#pragma unroll
        for (int a = 0; a < kRowsPerLoad; ++a) {
            int top = -1;
            float cnt = 0.f;
#pragma unroll
            for (int k = 0; k < LC; ++k)
                if (v[a * LC + k] > 0.5f) {
                    top = k;
                    cnt = v[a * LC + k];
                }
            red_m[(tr0 + a) * 128] =
                top >= 0 ? (static_cast<uint32_t>(top + 1) << 20) | static_cast<uint32_t>(__float2int_rn(cnt)) : 0u;
        }
    }
}

// TT = 1, 2 or 3: every problem of the launch has that unit kind (one tile,
// two tiles in one K block, two split tiles; the compiler specialises the MMA
// issue loop); TT = 0: read the kind per problem.
template <int TT>
__global__ void __launch_bounds__(kDirectThreads, 1) k_direct_fp8(const __grid_constant__ DirectLaunch dl) {
    constexpr int kStages = DirectCfg<TT>::stages;
    constexpr int kRedEntries = DirectCfg<TT>::red;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // red: one lane's result of one image row of one chunk (epi_read_rows)
    uint32_t* red = reinterpret_cast<uint32_t*>(base + kStages * kStageBytes);
    DirectSmemTail* tail = reinterpret_cast<DirectSmemTail*>(red + kRedEntries);
    volatile int* abort_flag = &tail->abort;
    const unsigned long long wait_ns = dl.wait_ns != 0ull ? dl.wait_ns : kWaitLimitNs;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&tail->full[s]), 1);
            mbar_init(smem_u32(&tail->empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tail->tfull[b]), 1);
            mbar_init(smem_u32(&tail->tempty[b]), 4);
        }
        for (int q = 0; q < kUnitQ; ++q) {
            mbar_init(smem_u32(&tail->ufull[q]), 1);
            mbar_init(smem_u32(&tail->uempty[q]), 2);
        }
        mbar_init(smem_u32(&tail->drain), 1);
        tail->abort = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(&tail->tmem_base), kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tail->tmem_base;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------ TMA producer
        const uint32_t full0 = smem_u32(&tail->full[0]), empty0 = smem_u32(&tail->empty[0]);
        const uint32_t ring0 = smem_u32(base);
        uint32_t it = 0;
        bool ok = true;
        // units: claimed from the launch's counter (direct_claim), or CTA b takes units b,
        // b + grid, ... where there is none; each is published to the MMA issuer and the
        // epilogue through the unit queue, and -1 ends their loops
        uint32_t uq = 0;
        long long t = dl.next_unit != nullptr ? direct_claim(dl, blockIdx.x) : static_cast<long long>(blockIdx.x);
        while (ok) {
            {
                const uint32_t qs = uq % kUnitQ, qph = (uq / kUnitQ) & 1u;
                if (!mbar_wait(smem_u32(&tail->uempty[qs]), qph ^ 1u, abort_flag, dl.err, wait_ns)) {
                    ok = false;
                    break;
                }
                if (t >= dl.total_tiles) t = -1;
                tail->unit[qs] = t;
                mbar_arrive(smem_u32(&tail->ufull[qs]));
                ++uq;
            }
            if (t < 0) break;
            const DirectProblemDev* P = direct_find(dl, t);
            if (dl.many != nullptr) {
                tma_fence_acquire_desc(&P->tmA);
                tma_fence_acquire_desc(&P->tmB);
            }
            const TileCoord tc = direct_tile(P, t);
            const DirectBand bd = direct_band(P, t);
            const int* rb = P->meta;
            const int* rows = P->meta + (P->n_pass + 1) + P->n_pass * 8;
            const int xw = tc.j0 - (P->kw - 1) + P->ox + P->shift;   // plane column of the K window (32-aligned)
            const int y0 = tc.i0 + P->oy, nk = P->nk, nb = P->nb, n_pass = P->n_pass;
            for (int p = 0; ok && p < n_pass; ++p) {
              const int nch = direct_pass_chunks(P, bd, p);
              for (int ch = 0; ok && ch < nch; ++ch) {
                // offset-group pass p, grey-level chunk ch (levels from `lev`, zero-filled by the copy
                // where they fall outside 0..L-1)
                const int lev = bd.hi - P->Lc * (ch + 1) + 1;
                const int q_end = rb[p + 1];
                for (int q = rb[p]; ok && q < q_end; ++q) {
                    const int y = y0 - rows[q];
                    for (int kc = 0; kc < nb; ++kc) {
                        const uint32_t s = it % kStages;
                        const uint32_t ph = (it / kStages) & 1u;
                        if (!mbar_wait(empty0 + 8u * s, ph ^ 1u, abort_flag, dl.err, wait_ns)) { ok = false; break; }
                        const uint32_t fb = full0 + 8u * s;
                        const bool with_a = kc < nk;   // split units stage one B block past the last A block
                        mbar_arrive_expect_tx(fb, with_a ? kStageBytes : kStageB);
                        const uint32_t sa = ring0 + s * kStageBytes;
                        if (with_a) tma_load_2d(sa, &P->tmA, 0, (q * nk + kc) * 128, fb);
                        tma_load_4d(sa + kStageA, &P->tmB, xw + 128 * kc, lev, y, tc.n, fb);
                        ++it;
                    }
                }
              }
            }
            t = dl.next_unit != nullptr
                    ? direct_claim(dl, static_cast<long long>(gridDim.x) + static_cast<long long>(atomicAdd(dl.next_unit, 1ull)))
                    : t + gridDim.x;
        }
        // drain, on every exit: the copies already issued land before the CTA may exit, also when
        // another role gave up while this loop ran to its end (in the normal course they have
        // landed already; older copies landed before their slot was refilled)
        {
            const uint32_t nd = it < static_cast<uint32_t>(kStages) ? it : static_cast<uint32_t>(kStages);
            for (uint32_t d = 0; d < nd; ++d) {
                const uint32_t k = it - 1 - d;
                mbar_wait_drain(smem_u32(&tail->full[k % kStages]), (k / kStages) & 1u);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // -------------------------------------------------------- MMA issuer
        const uint32_t idesc = idesc_e4m3_f32(kDirectM, kDirectN);
        // the issuing thread is on the critical path: stage barriers and descriptors are stepped
        // from slot 0's by plain additions, loop bounds are read once per pass
        const uint32_t full0 = smem_u32(&tail->full[0]), empty0 = smem_u32(&tail->empty[0]);
        const uint64_t desc0 = umma_desc_sw128(smem_u32(base));
        uint32_t it = 0;
        uint32_t use0 = 0u, use1 = 0u;   // completed claims of TMEM accumulator slots 0 and 1
        uint32_t next_slot = 0;
        unsigned long long n_mma = 0;    // MMAs this thread issued (measurement hook)
        bool ok = true;
        uint32_t uq = 0;                 // units read from the unit queue
        while (ok) {
            const uint32_t qs = uq % kUnitQ, qph = (uq / kUnitQ) & 1u;
            if (!mbar_wait(smem_u32(&tail->ufull[qs]), qph, abort_flag, dl.err, wait_ns)) {
                ok = false;
                break;
            }
            const long long t = tail->unit[qs];
            mbar_arrive(smem_u32(&tail->uempty[qs]));
            ++uq;
            if (t < 0) break;
            const DirectProblemDev* P = direct_find(dl, t);
            const int* rb = P->meta;
            const bool two = (TT == 0) ? (P->T == 2) : (TT >= 2);
            const bool split = (TT == 0) ? (P->split != 0) : (TT == 3);
            const uint64_t boff1 = static_cast<uint64_t>(P->J) >> 4;   // second tile: J bytes further along K
            const int sh1 = P->J >> 5;                                  // the same shift in 32-byte K steps
            const int ksteps = P->ksteps, nb = P->nb;
            const DirectBand bd = direct_band(P, t);
            for (int p = 0; ok && p < P->n_pass; ++p) {
              const int nch = direct_pass_chunks(P, bd, p);
              for (int ch = 0; ok && ch < nch; ++ch) {
                // a unit claims one slot (T = 1, alternating) or both (T = 2)
                const uint32_t s0 = two ? 0u : next_slot;
                next_slot = two ? 0u : (next_slot ^ 1u);
                if (two || s0 == 0u)
                    ok = mbar_wait(smem_u32(&tail->tempty[0]), (use0 & 1u) ^ 1u, abort_flag, dl.err, wait_ns);
                if (ok && (two || s0 == 1u))
                    ok = mbar_wait(smem_u32(&tail->tempty[1]), (use1 & 1u) ^ 1u, abort_flag, dl.err, wait_ns);
                if (!ok) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + s0 * kDirectN;
                uint32_t acc = 0, acc1 = 0;
                const int q_end = rb[p + 1];
                for (int q = rb[p]; ok && q < q_end; ++q) {
                    uint32_t s_prev = 0;
                    for (int kc = 0; kc < nb; ++kc) {
                        const uint32_t s = it % kStages;
                        const uint32_t ph = (it / kStages) & 1u;
                        if (!mbar_wait(full0 + 8u * s, ph, abort_flag, dl.err, wait_ns)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t adesc = desc0 + static_cast<uint64_t>(s * (kStageBytes >> 4));
                        const uint64_t bdesc = adesc + static_cast<uint64_t>(kStageA >> 4);
                        if (split) {
                            // K step ks of tile tt reads B byte 32 (ks + tt J / 32) of the unit's window,
                            // i.e. this block for the steps below; its A block is this stage's
                            // (ks / 4 == kc) or the previous stage's
                            const uint64_t adesc_prev = desc0 + static_cast<uint64_t>(s_prev * (kStageBytes >> 4));
                            {
                                const int lo = 4 * kc, hi = min(ksteps, 4 * kc + 4);
                                n_mma += static_cast<unsigned long long>(max(0, hi - lo));
                                for (int ks = lo; ks < hi; ++ks) {
                                    tc_mma_f8(d_tmem, adesc + 2ull * (ks & 3), bdesc + 2ull * (ks & 3), idesc, acc);
                                    acc = 1;
                                }
                            }
                            {
                                const int lo = max(0, 4 * kc - sh1), hi = min(ksteps, 4 * kc + 4 - sh1);
                                n_mma += static_cast<unsigned long long>(max(0, hi - lo));
                                for (int ks = lo; ks < hi; ++ks) {
                                    const uint64_t ad = ((ks >> 2) == kc ? adesc : adesc_prev) + 2ull * (ks & 3);
                                    tc_mma_f8(d_tmem + kDirectN, ad, bdesc + 2ull * ((ks + sh1) & 3), idesc, acc1);
                                    acc1 = 1;
                                }
                            }
                            // a stage's A block may still feed the next stage's tile-1 MMAs
                            if (kc > 0) tc_commit(empty0 + 8u * s_prev);
                            if (kc == nb - 1) tc_commit(empty0 + 8u * s);
                            s_prev = s;
                            ++it;
                            continue;
                        }
                        const int nks = min(4, ksteps - 4 * kc);
                        n_mma += static_cast<unsigned long long>(two ? 2 * nks : nks);
                        // advance the start addresses by 32 B of K inside the 128-B swizzled rows
                        if (two) {
                            for (int ks = 0; ks < nks; ++ks) {
                                tc_mma_f8(d_tmem, adesc + 2ull * ks, bdesc + 2ull * ks, idesc, acc);
                                tc_mma_f8(d_tmem + kDirectN, adesc + 2ull * ks, bdesc + boff1 + 2ull * ks, idesc, acc);
                                acc = 1;
                            }
                        } else {
#pragma unroll 4
                            for (int ks = 0; ks < nks; ++ks) {
                                tc_mma_f8(d_tmem, adesc + 2ull * ks, bdesc + 2ull * ks, idesc, acc);
                                acc = 1;
                            }
                        }
                        tc_commit(empty0 + 8u * s);
                        ++it;
                    }
                }
                if (ok) {
                    tc_commit(smem_u32(&tail->tfull[s0]));
                    if (two) tc_commit(smem_u32(&tail->tfull[1]));
                }
                if (two || s0 == 0u) ++use0;
                if (two || s0 == 1u) ++use1;
              }
            }
        }
        // drain, on every exit: every issued MMA completes before TMEM is freed, also when the
        // epilogue gave up and no longer waits for the accumulators
        tc_commit(smem_u32(&tail->drain));
        mbar_wait_drain(smem_u32(&tail->drain), 0);
        if (dl.mma_count != nullptr && n_mma != 0) atomicAdd(dl.mma_count, n_mma);
    } else if (warp >= 2) {
        // ----------------------------------------------------------- epilogue
        const int quarter = warp & 3;                 // TMEM lane quarter this warp may access
        const int m = quarter * 32 + lane;            // accumulator row = (group, column)
        const int et = threadIdx.x - 64;              // 0..127
        uint32_t use0 = 0u, use1 = 0u;   // same slot-claim sequence as the MMA issuer
        uint32_t next_slot = 0;
        unsigned long long band_wk = 0;  // band-limited multiply-adds of this CTA's units (measurement hook)
        uint32_t uq = 0;                 // units read from the unit queue
        // the running (degree, count) of this thread's pixels across a unit's accumulations (pixel
        // et + 128 k of the unit's T tiles in word k): packed (degree + 1) << 20 | count in 4-level
        // plans, whose degrees stay below L + max b <= kDirectNarrowMaxR, else an int2 in words
        // 2 k, 2 k + 1; thread-private memory, so the shared memory holds one more ring stage
        uint32_t runl[kRunWords];
        while (true) {
            const uint32_t qs = uq % kUnitQ, qph = (uq / kUnitQ) & 1u;
            const bool okq = mbar_wait(smem_u32(&tail->ufull[qs]), qph, abort_flag, dl.err, wait_ns);
            const long long t = okq ? tail->unit[qs] : -1;
            if (epi_any_failed(!okq)) break;           // also: every lane has read the slot
            if (et == 0) mbar_arrive(smem_u32(&tail->uempty[qs]));
            ++uq;
            if (t < 0) break;
            const DirectProblemDev* P = direct_find(dl, t);
            const TileCoord tc = direct_tile(P, t);
            const int J = P->J, G = P->G, rows_n = P->rows_n, Lc = P->Lc, T = (TT == 0) ? P->T : (TT == 3 ? 2 : TT);
            const int* gw = P->meta + (P->n_pass + 1);
            const DirectBand bd = direct_band(P, t);
            int n_units = 0;                              // accumulations of this unit, all passes
            for (int p = 0; p < P->n_pass; ++p) n_units += direct_pass_chunks(P, bd, p);
            if (et == 0 && dl.band_work != nullptr && P->band != nullptr) {
                // the contraction the unit needs: per pass, its taps x the levels of its band, per
                // pixel (taps unknown, -1, when the offsets are on the device: not counted)
                const int* pt = P->meta + P->pass_taps_off;
                unsigned long long wk = 0;
                bool known = true;
                for (int p = 0; p < P->n_pass; ++p) {
                    int wmax = 0;
                    for (int g = 0; g < G; ++g) wmax = max(wmax, gw[p * 8 + g]);
                    const int lo = bd.lb - wmax;
                    if (lo > bd.hi) continue;
                    if (pt[p] < 0) known = false;
                    wk += static_cast<unsigned long long>(max(pt[p], 0)) * static_cast<unsigned>(bd.hi - max(lo, 0) + 1);
                }
                const long long npx = static_cast<long long>(max(0, min(P->h, tc.i0 + rows_n) - max(0, tc.i0))) *
                                      max(0, min(P->w, tc.j0 + T * J) - max(0, tc.j0));
                if (known) band_wk += wk * static_cast<unsigned long long>(npx);
            }
            bool failed = false;
            int p = 0, ch = 0, nch = direct_pass_chunks(P, bd, 0);
            for (int u = 0; u < n_units; ++u, ++ch) {
                while (ch >= nch) {                       // next pass with chunks
                    ++p;
                    ch = 0;
                    nch = direct_pass_chunks(P, bd, p);
                }
                const int lev0 = bd.hi - Lc * (ch + 1) + 1;   // grey level of this chunk's first column
                const uint32_t s0 = (T == 2) ? 0u : next_slot;
                next_slot = (T == 2) ? 0u : (next_slot ^ 1u);
                bool ok = true;
                if (T == 2 || s0 == 0u) ok = mbar_wait(smem_u32(&tail->tfull[0]), use0 & 1u, abort_flag, dl.err, wait_ns);
                if (ok && (T == 2 || s0 == 1u))
                    ok = mbar_wait(smem_u32(&tail->tfull[1]), use1 & 1u, abort_flag, dl.err, wait_ns);
                if (epi_any_failed(!ok)) { failed = true; break; }
                tc_fence_after();
                // (max, sum-at-max) over the groups of tile tt, merged with the earlier unit passes;
                // group gg's degree of the chunk's level k is lev0 + k + its offset
                const int pairs = rows_n * J;
                // the groups' degree bases of this chunk, read once (not per pixel quad)
                int dbase[8];
#pragma unroll
                for (int gg = 0; gg < 8; ++gg) dbase[gg] = gg < G ? lev0 - 1 + gw[p * 8 + gg] : 0;
                const bool packed = Lc == kDirectLcNarrow;
                // quads of four pixels of one row per thread and step: one 16-byte shared load per
                // group, 16-byte output stores where the row allows them
                const int jsh = __ffs(J) - 1;                   // J is a power of two >= 16
                const int kq = (pairs + 511) >> 9;              // quads per thread per tile, at most
                const int h = P->h, w = P->w, outv = P->erode ? P->L - 1 : 0, sgn = P->erode ? -1 : 1;
                auto reduce = [&](int tt, int rbase) {
                    for (int qd = et, k = 0; qd < (pairs >> 2); qd += 128, ++k) {
                        const int p0 = qd << 2;
                        const int tr = p0 >> jsh, jl = p0 & (J - 1);
                        int best[4] = {-1, -1, -1, -1}, bc[4] = {0, 0, 0, 0};
#pragma unroll
                        for (int gg = 0; gg < 8; ++gg) {
                            if (gg >= G) break;
                            const uint4 e4 = *reinterpret_cast<const uint4*>(red + rbase + tr * 128 + gg * J + jl);
                            const uint32_t ev[4] = {e4.x, e4.y, e4.z, e4.w};
                            const int d0 = dbase[gg];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                if (ev[c] == 0u) continue;
                                const int deg = d0 + static_cast<int>(ev[c] >> 20);
                                const int cn = static_cast<int>(ev[c] & 0xFFFFFu);
                                if (deg > best[c]) { best[c] = deg; bc[c] = cn; }
                                else if (deg == best[c]) bc[c] += cn;
                            }
                        }
                        const int wq = (tt * kq + k) << 2;              // words of this quad in runl
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            if (u > 0) {
                                int2 prev;
                                if (packed) {
                                    const uint32_t e = runl[wq + c];
                                    prev = make_int2(static_cast<int>(e >> 20) - 1, static_cast<int>(e & 0xFFFFFu));
                                } else {
                                    prev = make_int2(static_cast<int>(runl[2 * (wq + c)]), static_cast<int>(runl[2 * (wq + c) + 1]));
                                }
                                if (prev.x > best[c]) { best[c] = prev.x; bc[c] = prev.y; }
                                else if (prev.x == best[c] && best[c] >= 0) bc[c] += prev.y;
                            }
                            if (u < n_units - 1) {
                                if (packed) {
                                    runl[wq + c] = best[c] < 0 ? 0u
                                                               : (static_cast<uint32_t>(best[c] + 1) << 20) | static_cast<uint32_t>(bc[c]);
                                } else {
                                    runl[2 * (wq + c)] = static_cast<uint32_t>(best[c]);
                                    runl[2 * (wq + c) + 1] = static_cast<uint32_t>(bc[c]);
                                }
                            }
                        }
                        if (u == n_units - 1) {
                            const int i = tc.i0 + tr, j = tc.j0 + tt * J + jl;
                            if (i < h) {
                                const long long o = (static_cast<long long>(tc.n) * h + i) * w + j;
                                int dv[4], cv[4];
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    dv[c] = outv + sgn * (best[c] < 0 ? 0 : best[c]) + P->out_add;
                                    cv[c] = best[c] < 0 ? 0 : bc[c];
                                }
                                int32_t* po = P->out + o;
                                int32_t* pc = P->out_cnt ? P->out_cnt + o : nullptr;
                                const int32_t* ps = P->out_sub ? P->out_sub + o : nullptr;
                                const bool vec = j >= 0 && j + 3 < w && (reinterpret_cast<uintptr_t>(po) & 15u) == 0 &&
                                                 (pc == nullptr || (reinterpret_cast<uintptr_t>(pc) & 15u) == 0) &&
                                                 (ps == nullptr || (reinterpret_cast<uintptr_t>(ps) & 15u) == 0);
                                if (vec) {
                                    if (ps) {
                                        const int4 sv = *reinterpret_cast<const int4*>(ps);
                                        dv[0] -= sv.x;
                                        dv[1] -= sv.y;
                                        dv[2] -= sv.z;
                                        dv[3] -= sv.w;
                                    }
                                    *reinterpret_cast<int4*>(po) = make_int4(dv[0], dv[1], dv[2], dv[3]);
                                    if (pc) *reinterpret_cast<int4*>(pc) = make_int4(cv[0], cv[1], cv[2], cv[3]);
                                } else {
#pragma unroll
                                    for (int c = 0; c < 4; ++c) {
                                        if (j + c < 0 || j + c >= w) continue;
                                        po[c] = dv[c] - (ps ? ps[c] : 0);
                                        if (pc) pc[c] = cv[c];
                                    }
                                }
                            }
                        }
                    }
                };
                // with two tiles whose lane results both fit `red`, read both accumulators and hand
                // them back before reducing, so the next unit's MMAs wait only for the TMEM reads
                const bool reads_first = T == 2 && 2 * rows_n * 128 <= kRedEntries;
                for (int tt = 0; tt < T; ++tt) {
                    const int rbase = reads_first ? tt * rows_n * 128 : 0;
                    const uint32_t trow =
                        tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + (s0 + tt) * kDirectN;
                    if (Lc == kDirectLcNarrow) epi_read_rows<kDirectLcNarrow>(trow, red + rbase + m);
                    else if (Lc == kDirectLcBand) epi_read_rows<kDirectLcBand>(trow, red + rbase + m);
                    else epi_read_rows<kDirectLc>(trow, red + rbase + m);
                    // this accumulator's TMEM reads are done: hand it back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&tail->tempty[s0 + tt]));
                    if (!reads_first) {
                        epi_bar();
                        reduce(tt, 0);
                        epi_bar();
                    }
                }
                if (reads_first) {
                    epi_bar();
                    reduce(0, 0);
                    reduce(1, rows_n * 128);
                    epi_bar();
                }
                if (T == 2 || s0 == 0u) ++use0;
                if (T == 2 || s0 == 1u) ++use1;
            }
            if (failed) break;
        }
        if (band_wk != 0ull) atomicAdd(dl.band_work, band_wk);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ---------------------------------------------------------------- Toeplitz
// blocks[(q * nk + kc)][m][k] = 1.0 (E4M3) iff the tap (r_q, c) with
// c = j + (kw - 1) - (128 kc + k), j = m mod J, lies in B and its offset is
// the level of group g = m / J of the pass that owns row index q.
// reflect: the offsets are in the original (unreflected) box order, read at
// kh kw - 1 - t (the erosion of a device-resident SE); err != nullptr: an
// offset of a tap outside [0, bound] is reported as a data error (the
// device-resident SE's declared bound).
__global__ void k_build_toeplitz(uint8_t* __restrict__ blocks, long long nbytes, const uint8_t* __restrict__ mask,
                                 const int* __restrict__ off, const int* __restrict__ meta, int n_pass, int nk, int J,
                                 int G, int kw, int nbox, int reflect, int bound, unsigned int* __restrict__ err) {
    if (err != nullptr) {
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nbox; t += (long long)gridDim.x * blockDim.x) {
            const int o = off[t];
            if (mask[reflect ? nbox - 1 - t : t] && (o < 0 || o > bound)) atomicOr(err, MORPH_DEVERR_RANGE);
        }
    }
    const int* rb = meta;
    const int* gw = meta + (n_pass + 1);
    const int* rows = gw + n_pass * 8;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nbytes;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(idx & 127);
        const int m = static_cast<int>((idx >> 7) & 127);
        const long long blk = idx >> 14;
        const int q = static_cast<int>(blk / nk);
        const int kc = static_cast<int>(blk % nk);
        int p = 0;
        while (p + 1 < n_pass && rb[p + 1] <= q) ++p;
        const int r = rows[q];
        const int g = m / J, j = m % J;
        const int c = j + (kw - 1) - (128 * kc + k);
        uint8_t v = 0;
        if (g < G && c >= 0 && c < kw) {
            const int t = r * kw + c;
            if (mask[t] && off[reflect ? nbox - 1 - t : t] == gw[p * 8 + g]) v = 0x38;
        }
        blocks[idx] = v;
    }
}

DirectPlan::~DirectPlan() {
    if (d_toeplitz) cudaFree(d_toeplitz);
    if (d_meta) cudaFree(d_meta);
    if (d_mask) cudaFree(d_mask);
}

// Host part of the plan: tiles, groups, passes, metadata and the issued FLOP.
int plan_direct_host(const morph_image* f, const morph_se* se, int erode, DirectPlan* p, int dev_bound) {
    // dev_bound >= 0: the offsets are in device memory (se->offset is not read); every level
    // 0..dev_bound is planned for, every SE row with a tap takes part in every pass, and the
    // band taps carry the tap's box index, -(t + 1), for the band kernel to look the offset up
    const bool dev = dev_bound >= 0;
    const int kh = se->kh, kw = se->kw;
    p->L = f->L;
    p->kh = kh;
    p->kw = kw;
    p->oy = se->oy;
    p->ox = se->ox;
    p->erode = erode;
    p->h = f->h;
    p->w = f->w;
    p->nimg = f->n;
    // plane pitch: a multiple of 32 bytes with room for any shift 0..31 (the planes' size
    // depends on the image only)
    p->w_pad = (f->w + 31 + 31) & ~31;
    // distinct offset levels among the taps
    std::vector<int> levels;
    int taps = 0, maxb = 0;
    for (int t = 0; t < kh * kw; ++t) {
        if (!se->mask[t]) continue;
        ++taps;
        if (dev) continue;
        maxb = std::max(maxb, static_cast<int>(se->offset[t]));
        levels.push_back(se->offset[t]);
    }
    if (dev) {
        maxb = dev_bound;
        for (int v = 0; v <= dev_bound; ++v) levels.push_back(v);
    }
    std::sort(levels.begin(), levels.end());
    levels.erase(std::unique(levels.begin(), levels.end()), levels.end());
    p->taps = taps;
    p->maxb = maxb;
    p->n_levels = static_cast<int>(levels.size());
    // N = rows_n image rows x Lc levels: one 16-level chunk holds every level up to L = 16.  For
    // 16 < L <= 64 a unit's band usually spans a few levels (uniform 2048^2 L = 64 content: at
    // most 4 in 95 % of 64-row units), so 4-level chunks of 64-row units contract about half the
    // levels of 8-level chunks of 32-row ones; their running results are packed into 32 bits,
    // which holds degrees below 4095 (L + max b beyond that takes the 8-level form).  Above
    // L = 64 bands span tens of levels, and on smooth content they widen with the unit's height,
    // so 16-row units with 16-level chunks cost less (4096^2 smooth L = 256: 22.4 vs 27.7 ms per
    // launch with 8-level chunks of 32-row units)
    if (f->L > kDirectLc && f->L <= 64)
        p->Lc = f->L + maxb <= kDirectNarrowMaxR ? kDirectLcNarrow : kDirectLcBand;
    else
        p->Lc = kDirectLc;
    p->rows_n = kDirectN / p->Lc;
    if (taps == 0) return MORPH_OK;
    // groups per pass: minimise passes x G x K-steps (the MMA work per output pixel)
    long long best = -1;
    for (int G = 1; G <= 8; G <<= 1) {
        const int J = 128 / G;
        const int ks = (J + kw - 1 + 31) / 32;
        const int passes = (p->n_levels + G - 1) / G;
        if (passes > kDirectMaxPasses) continue;
        const long long cost = static_cast<long long>(passes) * G * ks;
        // ties: with 4- or 8-level chunks (narrow bands) to smaller G -- with more passes of fewer
        // offset levels each, a unit whose lower bound lies above a pass's reach skips that pass,
        // e.g. the low-offset half of a 63x63 SE with offsets 0..7 on uniform content (measured
        // 1.06 -> 0.56 ms per 2048^2 launch); with 16-level chunks (wide bands, where passes
        // are rarely skipped) to larger G, fewer accumulations (4096^2 smooth L = 256: 22.4 vs
        // 26.4 ms)
        const bool take = p->Lc < kDirectLc ? cost < best : cost <= best;
        if (best < 0 || take) {
            best = cost;
            p->G = G;
        }
    }
    if (best < 0) return MORPH_E_UNSUPPORTED;
    p->J = 128 / p->G;
    p->ksteps = (p->J + kw - 1 + 31) / 32;
    p->nk = (p->J + kw - 1 + 127) / 128;
    p->n_pass = (p->n_levels + p->G - 1) / p->G;
    // two tiles per unit when both windows fit one 128-byte stage and the image is wide enough
    // (the second tile's K-steps read up to J + 32 ksteps bytes into the 128-byte rows)
    p->T = (2 * p->J + kw - 1 <= 128 && p->J + 32 * p->ksteps <= 128 && f->w > p->J) ? 2 : 1;
    if (p->Lc == kDirectLcNarrow) {
        // 64-row units halve the MMAs of a narrow band but double the epilogue's pixels per
        // accumulation and halve the units: keep them where an accumulation's MMAs outlast its
        // epilogue and the launch has two waves of units (64 x 1 x 128 x 128, 9 x 9 SE: 0.109 ms
        // with 32-row units, 0.135 ms with 64-row ones)
        int se_rows = 0;
        for (int r = 0; r < kh; ++r)
            for (int c = 0; c < kw; ++c)
                if (se->mask[r * kw + c]) {
                    ++se_rows;
                    break;
                }
        const long long units = static_cast<long long>(f->n) * ((f->h + 63) / 64) * ((f->w + p->T * p->J - 1) / (p->T * p->J));
        if (se_rows * p->ksteps * p->T < kDirectNarrowMinMmas || units < kDirectSplitMinUnits) p->Lc = kDirectLcBand;
        p->rows_n = kDirectN / p->Lc;
    }
    p->split = 0;
    p->nb = p->nk;
    // K windows start at image column j0 - (kw - 1 - ox): shifting the planes by that amount mod 32
    // puts every window of a tile grid starting at column 0 on a 32-byte boundary (TMA needs 16;
    // 32 keeps each 128-byte box row on four whole L2 sectors)
    p->shift = (((kw - 1 - se->ox) % 32) + 32) % 32;
    p->e = 0;
    p->tiles_y = (f->h + p->rows_n - 1) / p->rows_n;
    const int run_cap = p->Lc == kDirectLcNarrow ? kRunPacked : kRunEntries;
    if (p->T == 1 && p->J >= 32 && f->w > p->J && 2 * p->rows_n * p->J <= run_cap) {
        // split two-tile units: fewer staged blocks per SE row for both tiles; J a multiple of 32
        // keeps each K step inside one 128-byte row, both tiles' running results fit the epilogue
        // threads' run words
        const int nb = (p->J + 32 * p->ksteps + 127) / 128;
        const long long units = static_cast<long long>(f->n) * p->tiles_y * ((f->w + 2 * p->J - 1) / (2 * p->J));
        if (nb < 2 * p->nk && units >= kDirectSplitMinUnits) {
            p->T = 2;
            p->split = 1;
            p->nb = nb;
        }
    }
    p->tiles_x = (f->w + p->T * p->J - 1) / (p->T * p->J);
    p->tiles = static_cast<long long>(f->n) * p->tiles_x * p->tiles_y;
    // meta: pass_row_begin[n_pass + 1], group_w[n_pass * 8], rows[]
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
                if (!se->mask[t]) continue;
                if (dev) { any = true; break; }
                for (int g = 0; g < p->G; ++g)
                    if (gw[ps * 8 + g] == se->offset[t]) { any = true; break; }
            }
            if (any) rows.push_back(r);
        }
        if (static_cast<int>(rows.size()) == rb[ps]) return MORPH_E_UNSUPPORTED;   // every pass owns a tap
    }
    rb[p->n_pass] = static_cast<int>(rows.size());
    p->active_rows_total = static_cast<long long>(rows.size());
    p->meta.clear();
    p->meta.insert(p->meta.end(), rb.begin(), rb.end());
    p->meta.insert(p->meta.end(), gw.begin(), gw.end());
    p->meta.insert(p->meta.end(), rows.begin(), rows.end());
    // taps of the per-unit lower bound on the top degree: the SE box cut into up to 16 x 16 cells
    // (8 x 8 with 16-level chunks), from each the tap with the largest offset (ties: nearest
    // the cell centre), plus
    // the origin when it is a tap (valid at every pixel of the image); stored as the source
    // displacement (oy - r, ox - c) and b
    p->band_tap_off = static_cast<int>(p->meta.size());
    {
        // 16 x 16 cells wherever a band is computed (L <= 16 needs none: one chunk)
        const int cells = f->L > kDirectLc ? 16 : 8;
        const int ny = std::min(cells, kh), nx = std::min(cells, kw);
        std::vector<int> bt;
        bool has_origin = false;
        for (int a = 0; a < ny; ++a)
            for (int b2 = 0; b2 < nx; ++b2) {
                const int r0 = a * kh / ny, r1 = (a + 1) * kh / ny, c0 = b2 * kw / nx, c1 = (b2 + 1) * kw / nx;
                int best_t = -1;
                long long best_key = 0;
                for (int r = r0; r < r1; ++r)
                    for (int c = c0; c < c1; ++c) {
                        const int t = r * kw + c;
                        if (!se->mask[t]) continue;
                        const long long dr = 2 * r - (r0 + r1 - 1), dc = 2 * c - (c0 + c1 - 1);
                        const long long key = (dev ? 0LL : static_cast<long long>(se->offset[t]) * (1LL << 40)) -
                                              (dr * dr + dc * dc);
                        if (best_t < 0 || key > best_key) {
                            best_t = t;
                            best_key = key;
                        }
                    }
                if (best_t < 0) continue;
                const int r = best_t / kw, c = best_t % kw;
                if (r == se->oy && c == se->ox) has_origin = true;
                bt.insert(bt.end(), {se->oy - r, se->ox - c, dev ? -(best_t + 1) : static_cast<int>(se->offset[best_t])});
            }
        if (!has_origin && se->oy >= 0 && se->oy < kh && se->ox >= 0 && se->ox < kw && se->mask[se->oy * kw + se->ox]) {
            const int t0 = se->oy * kw + se->ox;
            bt.insert(bt.end(), {0, 0, dev ? -(t0 + 1) : static_cast<int>(se->offset[t0])});
        }
        p->n_band_taps = static_cast<int>(bt.size() / 3);
        p->n_band_segs = 0;
        if (!dev && p->n_band_taps > 0) {
            // taps in runs of equal offset (largest first): the band kernel takes each run's
            // maximum level and adds the run's offset once; segment ends follow the taps in meta
            std::vector<std::array<int, 3>> tv(p->n_band_taps);
            for (int k = 0; k < p->n_band_taps; ++k) tv[k] = {bt[3 * k], bt[3 * k + 1], bt[3 * k + 2]};
            std::stable_sort(tv.begin(), tv.end(), [](const auto& x, const auto& y) { return x[2] > y[2]; });
            for (int k = 0; k < p->n_band_taps; ++k)
                for (int e = 0; e < 3; ++e) bt[3 * k + e] = tv[k][e];
        }
        p->meta.insert(p->meta.end(), bt.begin(), bt.end());
        p->band_seg_off = static_cast<int>(p->meta.size());
        if (!dev)
            for (int k = 1; k <= p->n_band_taps; ++k)
                if (k == p->n_band_taps || bt[3 * k + 2] != bt[3 * (k - 1) + 2]) {
                    p->meta.push_back(k);
                    ++p->n_band_segs;
                }
    }
    // taps of each pass (the band-limited work count), -1 when the offsets are on the device
    p->pass_taps_off = static_cast<int>(p->meta.size());
    for (int ps = 0; ps < p->n_pass; ++ps) {
        int n = 0;
        for (int t = 0; !dev && t < kh * kw; ++t) {
            if (!se->mask[t]) continue;
            for (int g = 0; g < p->G; ++g)
                if (gw[ps * 8 + g] == se->offset[t]) { ++n; break; }
        }
        p->meta.push_back(dev ? -1 : n);
    }
    p->toeplitz_blocks = p->active_rows_total * p->nk;
    p->issued_flop = static_cast<double>(p->tiles) * p->T * static_cast<double>(p->active_rows_total) * p->ksteps * 2.0 *
                     kDirectM * kDirectN * 32.0 * ((p->L + p->Lc - 1) / p->Lc);

    return MORPH_OK;
}

int build_direct_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, int erode, DirectPlan* p) {
    int rc0 = plan_direct_host(f, se, erode, p);
    if (rc0 || p->taps == 0) return rc0;
    const int kh = se->kh, kw = se->kw;
    // device copies and the Toeplitz blocks
    const size_t tb = static_cast<size_t>(p->toeplitz_blocks) * 128 * 128;
    MORPH_CUDA_TRY(cudaMalloc(&p->d_toeplitz, tb));
    MORPH_CUDA_TRY(cudaMalloc(&p->d_meta, p->meta.size() * sizeof(int)));
    MORPH_CUDA_TRY(cudaMemcpy(p->d_meta, p->meta.data(), p->meta.size() * sizeof(int), cudaMemcpyHostToDevice));
    uint8_t* d_mask = nullptr;
    int* d_off = nullptr;
    MORPH_CUDA_TRY(cudaMalloc(&d_mask, kh * kw));
    MORPH_CUDA_TRY(cudaMalloc(&d_off, kh * kw * sizeof(int)));
    std::vector<int> offv(kh * kw);
    std::vector<uint8_t> maskv(kh * kw);
    for (int t = 0; t < kh * kw; ++t) {
        maskv[t] = se->mask[t] ? 1 : 0;
        offv[t] = se->offset[t];
    }
    MORPH_CUDA_TRY(cudaMemcpy(d_mask, maskv.data(), kh * kw, cudaMemcpyHostToDevice));
    MORPH_CUDA_TRY(cudaMemcpy(d_off, offv.data(), kh * kw * sizeof(int), cudaMemcpyHostToDevice));
    {
        long long blocks = (static_cast<long long>(tb) + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        k_build_toeplitz<<<static_cast<unsigned>(blocks), 256>>>(p->d_toeplitz, static_cast<long long>(tb), d_mask,
                                                                d_off, p->d_meta, p->n_pass, p->nk, p->J, p->G, kw,
                                                                kh * kw, 0, 0, nullptr);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
        MORPH_CUDA_TRY(cudaDeviceSynchronize());
    }
    cudaFree(d_mask);
    cudaFree(d_off);
    // tensor map of the Toeplitz blocks: rows of 128 B, boxes of 128 rows
    const uint64_t dims[2] = {128, static_cast<uint64_t>(p->toeplitz_blocks) * 128};
    const uint64_t strides[1] = {128};
    const uint32_t box[2] = {128, 128};
    return encode_tmap(&p->tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, p->d_toeplitz, dims, strides, box,
                       CU_TENSOR_MAP_SWIZZLE_128B);
}

// Plan of a device-resident SE: `se` holds the (reflected, for the erosion) mask
// and no offsets, which lie in [0, bound] in device memory.  The plan keeps its
// metadata and the mask on the device; the Toeplitz blocks depend on the
// offsets and are written by every call (launch_toeplitz_dev).
int build_direct_plan_dev(const morph_image* f, const morph_se* se, int bound, int erode, DirectPlan* p) {
    int rc = plan_direct_host(f, se, erode, p, bound);
    if (rc || p->taps == 0) return rc;
    const size_t nbox = static_cast<size_t>(se->kh) * se->kw;
    MORPH_CUDA_TRY(cudaMalloc(&p->d_meta, p->meta.size() * sizeof(int)));
    MORPH_CUDA_TRY(cudaMemcpy(p->d_meta, p->meta.data(), p->meta.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<uint8_t> m(nbox);
    for (size_t t = 0; t < nbox; ++t) m[t] = se->mask[t] ? 1 : 0;
    MORPH_CUDA_TRY(cudaMalloc(&p->d_mask, nbox));
    MORPH_CUDA_TRY(cudaMemcpy(p->d_mask, m.data(), nbox, cudaMemcpyHostToDevice));
    return MORPH_OK;
}

size_t direct_toeplitz_bytes(const DirectPlan& p) { return static_cast<size_t>(p.toeplitz_blocks) * 128 * 128; }

// The Toeplitz blocks of a device-resident SE's plan into `blocks` (stream-ordered;
// offsets outside [0, max b] raise the data error), and their tensor map.
int launch_toeplitz_dev(morph_ctx* ctx, const DirectPlan& p, const int32_t* dev_off, int reflect, uint8_t* blocks,
                        CUtensorMap* tmA, cudaStream_t st) {
    const long long tb = static_cast<long long>(direct_toeplitz_bytes(p));
    long long nblk = (tb + 255) / 256;
    if (nblk > ctx->num_sms * 8LL) nblk = ctx->num_sms * 8LL;
    if (nblk < 1) nblk = 1;
    prof_begin(ctx, st, "k_build_toeplitz");
    k_build_toeplitz<<<static_cast<unsigned>(nblk), 256, 0, st>>>(blocks, tb, p.d_mask, dev_off, p.d_meta, p.n_pass,
                                                                 p.nk, p.J, p.G, p.kw, p.kh * p.kw, reflect, p.maxb,
                                                                 ctx->d_err);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    const uint64_t dims[2] = {128, static_cast<uint64_t>(p.toeplitz_blocks) * 128};
    const uint64_t strides[1] = {128};
    const uint32_t box[2] = {128, 128};
    return encode_tmap(tmA, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, blocks, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_128B);
}

void direct_fill_problem(const DirectPlan& p, DirectProblemDev* d, const uint8_t* planes, int32_t* out,
                         int32_t* out_cnt, long long tile_base, int* status) {
    std::memset(static_cast<void*>(d), 0, sizeof(*d));
    d->tmA = p.tmA;
    const uint64_t dims[4] = {static_cast<uint64_t>(p.w + p.shift), static_cast<uint64_t>(p.L), static_cast<uint64_t>(p.h),
                              static_cast<uint64_t>(p.nimg)};
    const uint64_t strides[3] = {static_cast<uint64_t>(p.w_pad), static_cast<uint64_t>(p.w_pad) * p.L,
                                 static_cast<uint64_t>(p.w_pad) * p.L * p.h};
    const uint32_t box[4] = {128, static_cast<uint32_t>(p.Lc), static_cast<uint32_t>(p.rows_n), 1};
    *status = encode_tmap(&d->tmB, CU_TENSOR_MAP_DATA_TYPE_UINT8, 4, const_cast<uint8_t*>(planes), dims, strides, box,
                          CU_TENSOR_MAP_SWIZZLE_128B);
    d->out = out;
    d->out_cnt = out_cnt;
    d->out_add = 0;
    d->out_sub = nullptr;
    d->meta = p.d_meta;
    d->h = p.h;
    d->w = p.w;
    d->nimg = p.nimg;
    d->L = p.L;
    d->Lc = p.Lc;
    d->maxb = p.maxb;
    d->kh = p.kh;
    d->band_tap_off = p.band_tap_off;
    d->n_band_taps = p.n_band_taps;
    d->band_seg_off = p.band_seg_off;
    d->n_band_segs = p.n_band_segs;
    d->pass_taps_off = p.pass_taps_off;
    d->band = nullptr;
    d->lev_range = nullptr;
    d->dev_off = nullptr;
    d->dev_reflect = 0;
    d->rows_n = p.rows_n;
    d->J = p.J;
    d->G = p.G;
    d->n_pass = p.n_pass;
    d->nk = p.nk;
    d->ksteps = p.ksteps;
    d->kw = p.kw;
    d->oy = p.oy;
    d->ox = p.ox;
    d->e = p.e;
    d->shift = p.shift;
    d->erode = p.erode;
    d->T = p.T;
    d->split = p.split;
    d->nb = p.nb;
    d->tiles_x = p.tiles_x;
    d->tiles_y = p.tiles_y;
    d->tile_base = tile_base;
    d->tiles = p.tiles;
}

int direct_kind(const DirectProblemDev& d) { return d.split ? 3 : d.T; }

void direct_fill_band(DirectProblemDev* d, const morph_image* f, DirectBand* band) {
    // with L <= Lc one chunk holds every level: no band to compute
    d->band = f->L > d->Lc ? band : nullptr;
    d->lev_range = d->band != nullptr ? reinterpret_cast<int*>(direct_unit_counter(band, f) + 1) : nullptr;
    d->src = f->data;
    d->dtype = f->dtype;
    d->row_stride = f->row_stride;
    d->batch_stride = f->batch_stride;
}

static size_t band_entry_bytes(const morph_image* f) {
    // units are rows_n >= 16 image rows by at least 16 columns, with one entry per 32-row slab:
    // at most one entry per 16 image rows, or two for a 64-row unit over an image of <= 16 rows
    const size_t rows = std::max<size_t>((f->h + 15) / 16, 2);
    const size_t units = static_cast<size_t>(f->n) * rows * ((f->w + 15) / 16);
    return (units * sizeof(DirectBand) + 255) & ~size_t(255);
}

size_t direct_band_bytes(const morph_image* f) { return band_entry_bytes(f) + 256; }

unsigned long long* direct_unit_counter(DirectBand* band, const morph_image* f) {
    return reinterpret_cast<unsigned long long*>(reinterpret_cast<uint8_t*>(band) + band_entry_bytes(f));
}

// ------------------------------------------------------------ level bands
// Step 3 reads only the top nonzero degree D(x) of each pixel's count
// polynomial and its coefficient; every product f(x - y) + b(y) that reaches
// D(x) has f(x - y) >= D(x) - max b.  For a unit (rows_n x T J output pixels)
// the kernel below computes
//   hi = the largest level in the unit's input window (no tap reads a higher one),
//   lb = min over the unit's pixels x of max over a subset S of the taps valid
//        at x of level(f(x - y)) + b(y)     (<= D(x): a max over fewer taps),
// so the levels that can hold any top degree of the unit lie in
// [max(0, lb - max b), hi]; the direct kernel then contracts only those
// levels (chunks of Lc from the top), and the coefficients it computes are
// exactly those of the full polynomial at every degree >= lb.  A pixel with no
// valid tap of S makes lb = -1, i.e. every level from 0.
__device__ __forceinline__ int band_pixel(const void* src, int dtype, long long idx) {
    if (dtype == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (dtype == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

constexpr int kBandWinBytes = 96 * 1024;   // shared-memory window of a unit, 4 B per position
constexpr int kBandPairs = 8;              // pixel pairs per thread (32 rows x 128 columns / 2 / 256 threads)
constexpr int kBandCtasPerSm = 3;          // resident CTAs per SM the registers allow (80 per thread)
constexpr int kBandWMax = 1024;            // offsets above this are lowered to it for the bound (fp16-exact sums)

// Offset of a lower-bound tap: stored in the plan, or (v < 0) the device-resident
// offset of box entry -v - 1, clamped into [0, max b] (an offset outside it is
// reported by the Toeplitz build as a data error).
__device__ __forceinline__ int band_tap_offset(const DirectProblemDev* P, int v) {
    if (v >= 0) return v;
    const int t = -v - 1;
    const int o = P->dev_off[P->dev_reflect ? P->kh * P->kw - 1 - t : t];
    return min(max(o, 0), P->maxb);
}

// Level of pixel (i, j), flipped for the erosion and clamped into [0, L).
__device__ __forceinline__ int band_level(const DirectProblemDev* P, long long ibase, int i, int j) {
    int v = band_pixel(P->src, P->dtype, ibase + static_cast<long long>(i) * P->row_stride + j);
    v = min(max(v, 0), P->L - 1);          // out-of-range values are reported by the encoder
    return P->erode ? P->L - 1 - v : v;
}

// Pixel pairs and the staged window.  A thread takes pixel pairs (j, j + s) of a slab row,
// s = min(32, uw / 2): the first pixels of a row are the first s of each 2 s columns.  The
// window is staged as q[r][k] = (level(r, k), level(r, k + s)), k < WQ, so a pair reads a tap's
// two sources with one 4-byte load, and the lanes of a warp, which take consecutive first
// pixels, load consecutive words.  The row pitch WQ is s mod 32 when s < 32, so the rows one
// warp covers start on distinct banks.
__host__ __device__ __forceinline__ int band_pair_stride(int uw) { return uw >= 64 ? 32 : (uw >> 1); }
__host__ __device__ __forceinline__ int band_pitch(int uw, int kw) {
    const int s = band_pair_stride(uw);
    int wq = uw - s + kw - 1;                  // first pixels j <= uw - s - 1 read columns <= j + kw - 1
    if (s < 32) wq += ((s - wq) % 32 + 32) % 32;
    return wq;
}

// Warp `warp` stages window rows rr = warp, warp + nwarp, ...: its (row, 32-column
// group) items are taken a batch at a time, so each lane has several loads in flight
// before it stores their levels (the staging is bound by load latency otherwise).
// Columns WQ + s are staged (the highs of the last pairs); levels of the unit's true
// window, W = uw + kw - 1 columns, give the returned maximum.
constexpr int kBandStageBatch = 6;         // staging loads in flight per lane

template <typename Pix>
__device__ __forceinline__ int band_stage_rows(const DirectProblemDev* P, long long ibase, int wr0, int wc0, int WR,
                                               int WQ, int ps, int W, __half* qh, int warp, int nwarp, int lane) {
    const Pix* src = static_cast<const Pix*>(P->src);
    const int h = P->h, w = P->w, L = P->L, flip = P->erode;
    const int WS = WQ + ps;                                        // staged columns per row
    const int ng = (WS + 31) >> 5;                                 // 32-column groups per row
    const int my_rows = warp < WR ? (WR - warp + nwarp - 1) / nwarp : 0;
    const int items = my_rows * ng;
    int hi = -1;
    for (int base = 0; base < items; base += kBandStageBatch) {
        int v[kBandStageBatch], e[kBandStageBatch], cc[kBandStageBatch];
        bool in[kBandStageBatch];
        int r = base / ng, gcol = base - r * ng;
#pragma unroll
        for (int k = 0; k < kBandStageBatch; ++k) {
            const int rr = warp + r * nwarp;
            cc[k] = gcol * 32 + lane;
            e[k] = rr * WQ;
            const int i = wr0 + rr, j = wc0 + cc[k];
            in[k] = base + k < items && cc[k] < WS && i >= 0 && i < h && j >= 0 && j < w;
            v[k] = in[k] ? static_cast<int>(src[ibase + static_cast<long long>(i) * P->row_stride + j]) : 0;
            if (++gcol == ng) {
                gcol = 0;
                ++r;
            }
        }
#pragma unroll
        for (int k = 0; k < kBandStageBatch; ++k) {
            if (base + k >= items || cc[k] >= WS) continue;
            float fv = -4096.f;
            if (in[k]) {
                int lv = min(max(v[k], 0), L - 1);    // out-of-range values are reported by the encoder
                lv = flip ? L - 1 - lv : lv;
                if (cc[k] < W) hi = max(hi, lv);
                fv = static_cast<float>(lv);
            }
            const __half hv = __float2half_rn(fv);
            if (cc[k] < WQ) qh[2 * (e[k] + cc[k])] = hv;                   // low half of entry cc
            if (cc[k] >= ps) qh[2 * (e[k] + cc[k] - ps) + 1] = hv;         // high half of entry cc - s
        }
    }
    return hi;
}

union BandH2 {
    __half2 h;
    unsigned int u;
};

// The thread's minimum over its NP pixel pairs of the subset maximum: pair k of
// thread t is pair t + 256 k of the slab, row-major (uw / 2 pairs per row).
// With nseg > 0 the taps come in nseg runs of one offset (ends in s_seg): a run
// takes the maximum level over its taps and adds its offset once.  Otherwise
// (offsets on the device, in box order) each tap adds its own offset; two
// accumulators per pair take alternate taps, so consecutive taps do not wait
// on each other, and a tap pair's offsets and weights are read with one 8-byte
// load each.
template <int NP>
__device__ __forceinline__ int band_lower(const DirectProblemDev* P, const TileCoord& tc, const __half2* q,
                                          const int* s_toff, const __half2* s_tw, const int* s_seg, int nseg,
                                          int ntap, int WQ, int npair) {
    const int uw = P->T * P->J, half_w = uw >> 1, sh = __ffs(half_w) - 1;
    const int ps = band_pair_stride(uw), psh = __ffs(ps) - 1;
    if (static_cast<int>(threadIdx.x) >= npair) return 0x7fffffff;   // (NP == 1 with fewer pairs than threads)
    __half2 a0[NP], a1[NP];
    int base[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        a0[k] = __floats2half2_rn(-1.f, -1.f);
        a1[k] = a0[k];
        const int pp = threadIdx.x + k * 256;
        const int pr = pp >> sh, c = pp & (half_w - 1);
        const int j = ((c >> psh) << (psh + 1)) + (c & (ps - 1));
        base[k] = (pr + P->kh - 1 - P->oy) * WQ + j + P->kw - 1 - P->ox;
    }
    if (nseg > 0) {
        // a1 holds the result so far; a0 the current run's maximum level (-4096: no tap inside)
        int s = 0;
        for (int g = 0; g < nseg; ++g) {
            const int e = s_seg[g];
            const __half2 wg = s_tw[s];
#pragma unroll
            for (int k = 0; k < NP; ++k) a0[k] = __floats2half2_rn(-4096.f, -4096.f);
            for (; s + 1 < e; s += 2) {
                const int o0 = s_toff[s], o1 = s_toff[s + 1];
#pragma unroll
                for (int k = 0; k < NP; ++k) a0[k] = __hmax2(a0[k], __hmax2(q[base[k] + o0], q[base[k] + o1]));
            }
            if (s < e) {
                const int o0 = s_toff[s];
#pragma unroll
                for (int k = 0; k < NP; ++k) a0[k] = __hmax2(a0[k], q[base[k] + o0]);
                ++s;
            }
#pragma unroll
            for (int k = 0; k < NP; ++k) a1[k] = __hmax2(a1[k], __hadd2(a0[k], wg));
        }
    } else {
    const int2* toff2 = reinterpret_cast<const int2*>(s_toff);
    const uint2* tw2 = reinterpret_cast<const uint2*>(s_tw);
    int s = 0;
    for (; s + 1 < ntap; s += 2) {
        const int2 o = toff2[s >> 1];
        const uint2 wu = tw2[s >> 1];
        BandH2 w0, w1;
        w0.u = wu.x;
        w1.u = wu.y;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            a0[k] = __hmax2(a0[k], __hadd2(q[base[k] + o.x], w0.h));
            a1[k] = __hmax2(a1[k], __hadd2(q[base[k] + o.y], w1.h));
        }
    }
    if (s < ntap) {
        const int o0 = s_toff[s];
        const __half2 w0 = s_tw[s];
#pragma unroll
        for (int k = 0; k < NP; ++k) a0[k] = __hmax2(a0[k], __hadd2(q[base[k] + o0], w0));
    }
    }
    int lb = 0x7fffffff;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int pp = threadIdx.x + k * 256;
        const int c = pp & (half_w - 1);
        const int i = tc.i0 + (pp >> sh), j = tc.j0 + ((c >> psh) << (psh + 1)) + (c & (ps - 1));
        if (i >= P->h) continue;
        const float2 m = __half22float2(__hmax2(a0[k], a1[k]));
        if (j >= 0 && j < P->w) lb = min(lb, static_cast<int>(m.x));
        if (j + ps >= 0 && j + ps < P->w) lb = min(lb, static_cast<int>(m.y));
    }
    return lb;
}

__global__ void __launch_bounds__(256, kBandCtasPerSm) k_band(const __grid_constant__ DirectLaunch dl, int win_bytes, int slabs) {
    // One work item per unit slab (band_slab_rows image rows of a unit; item s T + t is slab s of
    // unit t, T units in the launch, and units with fewer slabs skip the items past theirs).
    // The slab's input window (rows i - r + oy, columns j - c + ox over the SE box, not clipped)
    // is staged as half2 pairs q[r][k] = (level(r, k), level(r, k + s)) (band_pitch), -4096
    // outside the image.  Sums level + min(b, 1024) <= 1279 and the sentinel -4096 + 1024 are
    // exact in fp16.
    extern __shared__ __align__(16) uint8_t s_raw[];
    __half* qh = reinterpret_cast<__half*>(s_raw);
    const __half2* q = reinterpret_cast<const __half2*>(s_raw);
    __shared__ int s_hi[8], s_lb[8];
    __shared__ __align__(8) int s_toff[kBandTapsMax];
    __shared__ __align__(8) __half2 s_tw[kBandTapsMax];
    __shared__ int s_seg[kBandTapsMax];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    if (dl.next_unit != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *dl.next_unit = 0ull;   // for the direct kernel
    for (long long it = blockIdx.x; it < slabs * dl.total_tiles; it += gridDim.x) {
        const int sl = static_cast<int>(it / dl.total_tiles);
        const long long t = it - sl * dl.total_tiles;
        const DirectProblemDev* P = direct_find(dl, t);
        if (P->band == nullptr || sl >= band_slabs(P->rows_n, P->T * P->J)) continue;   // block-uniform
        TileCoord tc = direct_tile(P, t);
        const int rows = band_slab_rows(P->rows_n, P->T * P->J);
        tc.i0 += sl * rows;
        const int h = P->h, w = P->w, uw = P->T * P->J, ntap = min(P->n_band_taps, kBandTapsMax);
        const long long ibase = static_cast<long long>(tc.n) * P->batch_stride;
        const int wr0 = tc.i0 - (P->kh - 1 - P->oy), wc0 = tc.j0 - (P->kw - 1 - P->ox);
        const int WR = rows + P->kh - 1, WQ = band_pitch(uw, P->kw);
        const bool fast = static_cast<long long>(WR) * WQ * 4 <= win_bytes &&
                          rows * (uw >> 1) <= 256 * kBandPairs;      // block-uniform
        __syncthreads();   // the previous item's readers of the shared arrays are done
        const int nseg = P->n_band_segs;
        for (int k = threadIdx.x; k < ntap; k += blockDim.x) {
            const int* tp = P->meta + P->band_tap_off + 3 * k;
            s_toff[k] = tp[0] * WQ + tp[1];
            const float wv = static_cast<float>(min(band_tap_offset(P, tp[2]), kBandWMax));
            s_tw[k] = __floats2half2_rn(wv, wv);
            if (k < nseg) s_seg[k] = P->meta[P->band_seg_off + k];
        }
        int hi = -1;
        int lb = 0x7fffffff;
        if (tc.i0 >= h) {
            // a slab below the image: no pixel, no window (hi -1, lb INT_MAX)
        } else if (fast) {
            const int ps = band_pair_stride(uw), W = uw + P->kw - 1;
            if (P->dtype == MORPH_U8)
                hi = band_stage_rows<uint8_t>(P, ibase, wr0, wc0, WR, WQ, ps, W, qh, warp, nwarp, lane);
            else if (P->dtype == MORPH_U16)
                hi = band_stage_rows<uint16_t>(P, ibase, wr0, wc0, WR, WQ, ps, W, qh, warp, nwarp, lane);
            else
                hi = band_stage_rows<int32_t>(P, ibase, wr0, wc0, WR, WQ, ps, W, qh, warp, nwarp, lane);
            __syncthreads();
            // pixel pairs of the slab: rows x uw / 2 pairs per row, npair / 256 per thread
            // (a power of two; with fewer pairs than threads, one pair for the first npair threads)
            const int npair = rows * (uw >> 1);
            if (npair <= 256) lb = band_lower<1>(P, tc, q, s_toff, s_tw, s_seg, nseg, ntap, WQ, npair);
            else if (npair <= 512) lb = band_lower<2>(P, tc, q, s_toff, s_tw, s_seg, nseg, ntap, WQ, npair);
            else if (npair <= 1024) lb = band_lower<4>(P, tc, q, s_toff, s_tw, s_seg, nseg, ntap, WQ, npair);
            else lb = band_lower<8>(P, tc, q, s_toff, s_tw, s_seg, nseg, ntap, WQ, npair);
        } else {
            // windows too large for shared memory (SE boxes of hundreds of rows): direct loads
            const int r0 = max(0, wr0), r1 = min(h, tc.i0 + rows + P->oy);
            const int c0 = max(0, wc0), c1 = min(w, tc.j0 + uw + P->ox);
            for (int i = r0 + warp; i < r1; i += nwarp)
                for (int j = c0 + lane; j < c1; j += 32) hi = max(hi, band_level(P, ibase, i, j));
            const int pi0 = max(0, tc.i0), pi1 = min(h, tc.i0 + rows);
            const int pj0 = max(0, tc.j0), pj1 = min(w, tc.j0 + uw);
            for (int i = pi0 + warp; i < pi1; i += nwarp)
                for (int j = pj0 + lane; j < pj1; j += 32) {
                    int m = -1;
                    for (int s = 0; s < ntap; ++s) {
                        const int* tp = P->meta + P->band_tap_off + 3 * s;
                        const int si = i + tp[0], sj = j + tp[1];
                        if (static_cast<unsigned>(si) < static_cast<unsigned>(h) &&
                            static_cast<unsigned>(sj) < static_cast<unsigned>(w))
                            m = max(m, band_level(P, ibase, si, sj) + min(band_tap_offset(P, tp[2]), kBandWMax));
                    }
                    lb = min(lb, m);
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            lb = min(lb, __shfl_xor_sync(0xffffffffu, lb, o));
        }
        if (lane == 0) {
            s_hi[warp] = hi;
            s_lb[warp] = lb;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < nwarp; ++k) {
                hi = max(hi, s_hi[k]);
                lb = min(lb, s_lb[k]);
            }
            DirectBand b;
            b.hi = hi;
            b.lb = lb;
            const_cast<DirectBand*>(P->band)[(t - P->tile_base) * band_slabs(P->rows_n, P->T * P->J) + sl] = b;
        }
    }
}

int direct_band_window(const DirectProblemDev& d) {
    if (d.band == nullptr) return 0;
    const long long b = static_cast<long long>(band_slab_rows(d.rows_n, d.T * d.J) + d.kh - 1) * band_pitch(d.T * d.J, d.kw) * 4;
    return static_cast<int>(std::min<long long>(kBandWinBytes, (b + 1023) & ~1023LL));
}

int direct_band_slabs(const DirectProblemDev& d) { return band_slabs(d.rows_n, d.T * d.J); }

int launch_band(morph_ctx* ctx, const DirectLaunch& dl, int win_bytes, int slabs, cudaStream_t st) {
    if (dl.total_tiles <= 0) return MORPH_OK;
    bool any = dl.many != nullptr || dl.single.band != nullptr;
    if (!any) return MORPH_OK;
    win_bytes = std::max(1024, std::min(win_bytes, kBandWinBytes));
    slabs = std::max(1, slabs);
    // resident CTAs per SM: kBandCtasPerSm by registers, fewer when their windows fill shared memory
    const long long per_sm = std::max(1, std::min(kBandCtasPerSm, (220 * 1024) / (win_bytes + 4 * 1024)));
    long long grid = slabs * dl.total_tiles;
    const long long cap = static_cast<long long>(ctx->num_sms) * per_sm;
    if (grid > cap) grid = cap;
    prof_begin(ctx, st, "k_band");
    if (!kernels_ready(ctx->device, kGroupBand)) {
        MORPH_CUDA_TRY(cudaFuncSetAttribute(k_band, cudaFuncAttributeMaxDynamicSharedMemorySize, kBandWinBytes));
        mark_kernels_ready(ctx->device, kGroupBand);
    }
    k_band<<<static_cast<unsigned>(grid), 256, win_bytes, st>>>(dl, win_bytes, slabs);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

// The levels the direct kernel reads for a problem: unit t's chunks cover at most
// [max(0, lb - max b) - (Lc - 1), hi] of its band (direct_band), so the union over the
// units is within [min_t (lb_t - max b - Lc + 1), max_t hi_t]; the encoder writes only those
// planes (levels outside 0..L-1 are the copy's zero fill).
__global__ void __launch_bounds__(1024) k_band_range(const __grid_constant__ DirectLaunch dl) {
    __shared__ int s_lo[32], s_hi[32];
    const DirectProblemDev* P = dl.many != nullptr ? &dl.many[blockIdx.x] : &dl.single;
    if (P->band == nullptr || P->lev_range == nullptr) return;      // block-uniform
    int lo = P->L, hi = -1;
    for (long long t = P->tile_base + threadIdx.x; t < P->tile_base + P->tiles; t += blockDim.x) {
        const DirectBand b = direct_band(P, t);
        lo = min(lo, max(0, b.lb - P->maxb - P->Lc + 1));
        hi = max(hi, b.hi);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < static_cast<int>(blockDim.x >> 5); ++k) {
            lo = min(lo, s_lo[k]);
            hi = max(hi, s_hi[k]);
        }
        P->lev_range[0] = lo;
        P->lev_range[1] = hi;
    }
}

int launch_band_range(morph_ctx* ctx, const DirectLaunch& dl, cudaStream_t st) {
    if (dl.total_tiles <= 0) return MORPH_OK;
    if (dl.many == nullptr && dl.single.band == nullptr) return MORPH_OK;
    const unsigned grid = dl.many != nullptr ? static_cast<unsigned>(dl.nprob) : 1u;
    prof_begin(ctx, st, "k_band_range");
    k_band_range<<<grid, 1024, 0, st>>>(dl);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

int launch_direct(morph_ctx* ctx, const DirectLaunch& dl, cudaStream_t st, int uniform_kind) {
    if (dl.total_tiles <= 0) return MORPH_OK;
    if (!kernels_ready(ctx->device, kGroupDirect)) {
        MORPH_CUDA_TRY(cudaFuncSetAttribute(k_direct_fp8<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_smem_bytes<0>()));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(k_direct_fp8<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_smem_bytes<1>()));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(k_direct_fp8<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_smem_bytes<2>()));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(k_direct_fp8<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, direct_smem_bytes<3>()));
        mark_kernels_ready(ctx->device, kGroupDirect);
    }
    const int kind = dl.many == nullptr ? direct_kind(dl.single) : (uniform_kind < 0 ? 0 : uniform_kind);
    long long grid = dl.total_tiles < ctx->num_sms ? dl.total_tiles : ctx->num_sms;
    prof_begin(ctx, st, "k_direct_fp8");
    if (kind == 1) k_direct_fp8<1><<<static_cast<unsigned>(grid), kDirectThreads, direct_smem_bytes<1>(), st>>>(dl);
    else if (kind == 2) k_direct_fp8<2><<<static_cast<unsigned>(grid), kDirectThreads, direct_smem_bytes<2>(), st>>>(dl);
    else if (kind == 3) k_direct_fp8<3><<<static_cast<unsigned>(grid), kDirectThreads, direct_smem_bytes<3>(), st>>>(dl);
    else k_direct_fp8<0><<<static_cast<unsigned>(grid), kDirectThreads, direct_smem_bytes<0>(), st>>>(dl);
    prof_end(ctx, st);
    ctx->launches += 1;
    MORPH_CUDA_TRY(cudaGetLastError());
    return MORPH_OK;
}

}  // namespace morph
