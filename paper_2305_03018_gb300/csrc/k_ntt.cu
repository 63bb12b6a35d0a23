// Step 2 of the method as an exact number-theoretic transform (NTT), followed
// by Step 3 (Eq. 9).  The paper points to modular transforms as the exact
// alternative to the floating-point FFT (Sec. 2.3): the count polynomial of
// Eq. Obs7 has integer coefficients in [0, |B|], so its convolution computed
// modulo a prime P > |B| is the exact count, with no round-off bound.
//
// P = 2^14 3^6 5^3 + 1 = 1492992001 (prime, < 2^31), so P - 1 is divisible by
// every transform length 2^a 3^b 5^c <= 2048 with c <= 3, and sums of two
// residues fit in 32 bits.  omega_N = g^((P-1)/N) with the primitive root
// g = 11 plays the part of exp(-2 pi i / N).  Products use the Montgomery
// form (REDC with 2^32): constants (twiddles, the SE spectrum) are stored
// pre-multiplied by 2^32 mod P, so one REDC of a plain residue by a stored
// constant gives the plain product.
//
// The data flow follows the FFT route: the grey axis of the umbra (Eq. 7) is
// one-hot, so its transform is the table omega_Rf^(k f(x)); for each grey
// frequency k (all Rf of them: residues have no conjugate symmetry) the
// spatial convolution with the SE spectrum runs on overlap-save tiles as 2-D
// NTTs; Step 3 inverts the grey axis per pixel and takes the highest degree
// with a nonzero count.  Inverse transforms are forward transforms read at
// index (N - n) mod N; the 1 / (Rf Ny Nx) scale is folded into the stored SE
// spectrum.
//
// Kernels (per wave of tiles):
//   k_ntt_rows_fwd : encode omega_Rf^(k f) for one input row, NTT along x, a
//                    group of k at a time;
//   k_ntt_cols     : NTT along y of C columns, multiply by the SE spectrum,
//                    inverse NTT along y, keep the output rows;
//   k_ntt_rows_inv : inverse NTT along x of output rows, keep the output columns;
//   k_ntt_range    : inverse NTT along the grey axis for a group of pixels,
//                    top nonzero degree and its count (one warp per pixel).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

constexpr uint32_t kP = 1492992001u;       // 2^14 3^6 5^3 + 1
constexpr uint32_t kPinv = 3372040191u;    // -P^-1 mod 2^32
constexpr uint64_t kG = 11u;               // primitive root mod P
constexpr int kNttMaxN = 2048;

static_assert(static_cast<uint32_t>(kP * kPinv) == 0xFFFFFFFFu, "kPinv must be -P^-1 mod 2^32");

constexpr uint64_t npow(uint64_t b, uint64_t e) {
    uint64_t r = 1;
    b %= kP;
    while (e) {
        if (e & 1) r = r * b % kP;
        b = b * b % kP;
        e >>= 1;
    }
    return r;
}
constexpr uint32_t to_mont(uint64_t x) { return static_cast<uint32_t>(((x % kP) << 32) % kP); }
constexpr uint64_t kInv2 = (kP + 1) / 2;

// radix roots (omega_r = g^((P-1)/r)) and the radix-5 combinations, Montgomery form
constexpr uint64_t kW3 = npow(kG, (kP - 1) / 3);
constexpr uint64_t kW4 = npow(kG, (kP - 1) / 4);
constexpr uint64_t kW5 = npow(kG, (kP - 1) / 5);
constexpr uint32_t kW3m = to_mont(kW3);
constexpr uint32_t kW4m = to_mont(kW4);
constexpr uint32_t kC1m = to_mont((kW5 + npow(kW5, 4)) % kP * kInv2 % kP);
constexpr uint32_t kC2m = to_mont((npow(kW5, 2) + npow(kW5, 3)) % kP * kInv2 % kP);
constexpr uint32_t kS1m = to_mont((kW5 + kP - npow(kW5, 4)) % kP * kInv2 % kP);
constexpr uint32_t kS2m = to_mont((npow(kW5, 2) + kP - npow(kW5, 3)) % kP * kInv2 % kP);

__device__ __forceinline__ uint32_t madd(uint32_t a, uint32_t b) {
    const uint32_t s = a + b;
    return s >= kP ? s - kP : s;
}
__device__ __forceinline__ uint32_t msub(uint32_t a, uint32_t b) {
    const uint32_t s = a + (kP - b);
    return s >= kP ? s - kP : s;
}
// a * bm * 2^-32 mod P for a, bm < P: with bm = b 2^32 mod P this is a b mod P.
// t = a bm, m = t mod 2^32 * (-P^-1); (t + m P) / 2^32 < 2P; the low words of
// t and m P sum to 0 or 2^32, a carry exactly when t mod 2^32 != 0.
__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t bm) {
    const uint64_t t = static_cast<uint64_t>(a) * bm;
    const uint32_t lo = static_cast<uint32_t>(t), hi = static_cast<uint32_t>(t >> 32);
    const uint32_t m = lo * kPinv;
    const uint32_t u = hi + __umulhi(m, kP) + (lo != 0u ? 1u : 0u);
    return u >= kP ? u - kP : u;
}

// Radix-r forward DFTs mod P, y_k = sum_j v_j omega_r^(jk), in registers.
__device__ __forceinline__ void ndft2(uint32_t* v) {
    const uint32_t a = v[0], b = v[1];
    v[0] = madd(a, b);
    v[1] = msub(a, b);
}
__device__ __forceinline__ void ndft4(uint32_t* v) {
    // omega_4^2 = -1
    const uint32_t s02 = madd(v[0], v[2]), d02 = msub(v[0], v[2]);
    const uint32_t s13 = madd(v[1], v[3]), d13 = mmul(msub(v[1], v[3]), kW4m);
    v[0] = madd(s02, s13);
    v[2] = msub(s02, s13);
    v[1] = madd(d02, d13);
    v[3] = msub(d02, d13);
}
__device__ __forceinline__ void ndft3(uint32_t* v) {
    // omega^2 = -1 - omega: y1 = (v0 - v2) + omega (v1 - v2), y2 = (v0 - v1) - omega (v1 - v2)
    const uint32_t t = mmul(msub(v[1], v[2]), kW3m);
    const uint32_t y0 = madd(madd(v[0], v[1]), v[2]);
    const uint32_t y1 = madd(msub(v[0], v[2]), t);
    const uint32_t y2 = msub(msub(v[0], v[1]), t);
    v[0] = y0;
    v[1] = y1;
    v[2] = y2;
}
__device__ __forceinline__ void ndft5(uint32_t* v) {
    // C_j = (w^j + w^-j) / 2, S_j = (w^j - w^-j) / 2 with w = omega_5
    const uint32_t b1 = madd(v[1], v[4]), b2 = madd(v[2], v[3]);
    const uint32_t d1 = msub(v[1], v[4]), d2 = msub(v[2], v[3]);
    const uint32_t a0 = v[0];
    const uint32_t A1 = madd(a0, madd(mmul(b1, kC1m), mmul(b2, kC2m)));
    const uint32_t B1 = madd(mmul(d1, kS1m), mmul(d2, kS2m));
    const uint32_t A2 = madd(a0, madd(mmul(b1, kC2m), mmul(b2, kC1m)));
    const uint32_t B2 = msub(mmul(d1, kS2m), mmul(d2, kS1m));
    v[0] = madd(a0, madd(b1, b2));
    v[1] = madd(A1, B1);
    v[4] = msub(A1, B1);
    v[2] = madd(A2, B2);
    v[3] = msub(A2, B2);
}

// One Stockham stage of radix R over `batch` interleaved transforms of length
// N (element p of transform c at p * batch + c).  tw[m] = omega_N^m, Montgomery.
template <int R>
__device__ __forceinline__ void ntt_stage(const uint32_t* __restrict__ x, uint32_t* __restrict__ y, int N, int Ns,
                                          const uint32_t* __restrict__ tw, int batch) {
    const int M = N / R;
    const int total = M * batch;
    const int tstep = N / (Ns * R);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int c = t % batch;
        const int j = t / batch;
        const int k = j % Ns;
        uint32_t v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[(j + r * M) * batch + c];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = mmul(v[r], tw[r * k * tstep]);
        }
        if (R == 2) ndft2(v);
        if (R == 3) ndft3(v);
        if (R == 4) ndft4(v);
        if (R == 5) ndft5(v);
        const int d = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[(d + r * Ns) * batch + c] = v[r];
    }
}

// Forward NTT of `batch` interleaved transforms in a (scratch b); returns the
// buffer holding the result.  Block-wide; ends with a barrier.
__device__ uint32_t* ntt_block(uint32_t* a, uint32_t* b, const FftAxis& ax, const uint32_t* tw, int batch) {
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s];
        if (R == 4) ntt_stage<4>(a, b, ax.N, Ns, tw, batch);
        else if (R == 2) ntt_stage<2>(a, b, ax.N, Ns, tw, batch);
        else if (R == 3) ntt_stage<3>(a, b, ax.N, Ns, tw, batch);
        else ntt_stage<5>(a, b, ax.N, Ns, tw, batch);
        __syncthreads();
        Ns *= R;
        uint32_t* t = a;
        a = b;
        b = t;
    }
    return a;
}

struct NttArgs {
    // image
    const void* src;
    int dtype, n, h, w;
    long long row_stride, batch_stride;
    int L, flip, erode;
    // method
    int R, Rf;                      // degrees, grey-axis length (= grey frequencies)
    FftAxis ar, ax, ay;
    int To_y, To_x, Rin_y, Win_x;   // output tile, input tile (To + k - 1)
    int ry, rx;                     // SE reach below / right: kh - 1 - oy, kw - 1 - ox
    int tiles_x, tiles_y;
    long long tile0;                // first global tile of this wave
    int wave_tiles;
    const uint32_t* tw_x;           // omega_Nx^m, Montgomery
    const uint32_t* tw_y;           // omega_Ny^m, Montgomery
    const uint32_t* tw_r;           // omega_Rf^m, Montgomery
    const uint32_t* wr;             // omega_Rf^m, plain (encoder table)
    const uint32_t* S;              // SE spectrum / (Rf Ny Nx), Montgomery, [Rf][Ny][Nx]
    uint32_t* buf;                  // [wave_tiles][Rf][Ny][Nx]
    int32_t* out;
    int32_t* out_cnt;
    unsigned int* err;
    int kgroup;                     // grey frequencies per pass in the row kernels
    int colgroup;                   // columns per CTA in k_ntt_cols
    int pixgroup;                   // pixels per CTA in k_ntt_range
};

__device__ __forceinline__ int ntt_load_px(const void* src, int dtype, long long idx) {
    if (dtype == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (dtype == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

__device__ __forceinline__ void ntt_tile_origin(const NttArgs& a, long long gt, int* n, int* y0, int* x0) {
    const long long per = static_cast<long long>(a.tiles_x) * a.tiles_y;
    *n = static_cast<int>(gt / per);
    const int rem = static_cast<int>(gt % per);
    *y0 = (rem / a.tiles_x) * a.To_y;
    *x0 = (rem % a.tiles_x) * a.To_x;
}

// grid (Rin_y, wave_tiles): input row rho of tile tl, every grey frequency
__global__ void __launch_bounds__(256) k_ntt_rows_fwd(const NttArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N, KB = a.kgroup;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Nx;
    uint32_t* b1 = b0 + KB * Nx;
    int* lev = reinterpret_cast<int*>(b1 + KB * Nx);
    const int rho = blockIdx.x, tl = blockIdx.y;
    int n, y0, x0;
    ntt_tile_origin(a, a.tile0 + tl, &n, &y0, &x0);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = a.tw_x[j];
    const int iy = y0 - a.ry + rho;
    bool bad = false;
    for (int p = threadIdx.x; p < Nx; p += blockDim.x) {
        const int ix = x0 - a.rx + p;
        int v = -1;
        if (p < a.Win_x && iy >= 0 && iy < a.h && ix >= 0 && ix < a.w) {
            const int f = ntt_load_px(a.src, a.dtype, n * a.batch_stride + iy * a.row_stride + ix);
            if (f < 0 || f >= a.L) bad = true;
            else v = a.flip ? a.L - 1 - f : f;
        }
        lev[p] = v;
    }
    if (bad) atomicOr(a.err, MORPH_DEVERR_RANGE);
    __syncthreads();
    const long long plane = static_cast<long long>(a.ay.N) * Nx;
    uint32_t* dst = a.buf + static_cast<long long>(tl) * a.Rf * plane + static_cast<long long>(rho) * Nx;
    for (int k0 = 0; k0 < a.Rf; k0 += KB) {
        const int kb = min(KB, a.Rf - k0);
        for (int t = threadIdx.x; t < kb * Nx; t += blockDim.x) {
            const int c = t % kb, p = t / kb;
            const int l = lev[p];
            b0[t] = l >= 0 ? a.wr[((k0 + c) * l) % a.Rf] : 0u;
        }
        __syncthreads();
        const uint32_t* res = ntt_block(b0, b1, a.ax, tw, kb);
        for (int t = threadIdx.x; t < kb * Nx; t += blockDim.x) {
            const int c = t / Nx, p = t % Nx;
            dst[(k0 + c) * plane + p] = res[p * kb + c];
        }
        __syncthreads();
    }
}

// grid (ceil(Nx / C), Rf, wave_tiles)
__global__ void __launch_bounds__(256) k_ntt_cols(const NttArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = a.ay.N, Nx = a.ax.N, C = a.colgroup;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Ny;
    uint32_t* b1 = b0 + Ny * C;
    const int u0 = blockIdx.x * C, k = blockIdx.y, tl = blockIdx.z;
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) tw[j] = a.tw_y[j];
    uint32_t* plane = a.buf + (static_cast<long long>(tl) * a.Rf + k) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t % C, rho = t / C;
        b0[t] = (rho < a.Rin_y && u0 + c < Nx) ? plane[static_cast<long long>(rho) * Nx + u0 + c] : 0u;
    }
    __syncthreads();
    uint32_t* res = ntt_block(b0, b1, a.ay, tw, C);
    uint32_t* other = (res == b0) ? b1 : b0;
    const uint32_t* S = a.S + static_cast<long long>(k) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t % C, v = t / C;
        if (u0 + c < Nx) res[t] = mmul(res[t], S[static_cast<long long>(v) * Nx + u0 + c]);
    }
    __syncthreads();
    const uint32_t* o = ntt_block(res, other, a.ay, tw, C);
    for (int t = threadIdx.x; t < a.To_y * C; t += blockDim.x) {
        const int c = t % C, q = t / C;
        // torus position of output row q is (q + ry) mod Ny (ry < 0 or >= Ny when the origin lies outside the box)
        const int pos = ((q + a.ry) % Ny + Ny) % Ny;
        const int idx = pos == 0 ? 0 : Ny - pos;
        if (u0 + c < Nx) plane[static_cast<long long>(q) * Nx + u0 + c] = o[idx * C + c];
    }
}

// grid (To_y, ceil(Rf / KB), wave_tiles): output row q, a group of grey frequencies
__global__ void __launch_bounds__(256) k_ntt_rows_inv(const NttArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N, KB = a.kgroup;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Nx;
    uint32_t* b1 = b0 + KB * Nx;
    const int q = blockIdx.x, k0 = blockIdx.y * KB, tl = blockIdx.z;
    const int kb = min(KB, a.Rf - k0);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = a.tw_x[j];
    const long long plane = static_cast<long long>(a.ay.N) * Nx;
    uint32_t* rows = a.buf + (static_cast<long long>(tl) * a.Rf + k0) * plane + static_cast<long long>(q) * Nx;
    for (int t = threadIdx.x; t < kb * Nx; t += blockDim.x) {
        const int c = t / Nx, p = t % Nx;
        b0[p * kb + c] = rows[c * plane + p];
    }
    __syncthreads();
    const uint32_t* res = ntt_block(b0, b1, a.ax, tw, kb);
    for (int t = threadIdx.x; t < kb * a.To_x; t += blockDim.x) {
        const int c = t / a.To_x, p = t % a.To_x;
        const int pos = ((p + a.rx) % Nx + Nx) % Nx;
        const int idx = pos == 0 ? 0 : Nx - pos;
        rows[c * plane + p] = res[idx * kb + c];
    }
}

// grid (ceil(To_x / C), To_y, wave_tiles): grey-axis inverse NTT of C pixels
// of output row q, then the top degree with a nonzero count (Eq. 9).
__global__ void __launch_bounds__(256) k_ntt_range(const NttArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Rf = a.Rf, C = a.pixgroup, Nx = a.ax.N, Ny = a.ay.N;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Rf;
    uint32_t* b1 = b0 + Rf * C;
    const int x0 = blockIdx.x * C, q = blockIdx.y, tl = blockIdx.z;
    int n, y0, tx0;
    ntt_tile_origin(a, a.tile0 + tl, &n, &y0, &tx0);
    for (int j = threadIdx.x; j < Rf; j += blockDim.x) tw[j] = a.tw_r[j];
    const long long kstride = static_cast<long long>(Ny) * Nx;
    const uint32_t* base = a.buf + static_cast<long long>(tl) * Rf * kstride + static_cast<long long>(q) * Nx;
    for (int t = threadIdx.x; t < Rf * C; t += blockDim.x) {
        const int c = t % C, k = t / C;
        b0[t] = (x0 + c < a.To_x) ? base[k * kstride + x0 + c] : 0u;
    }
    __syncthreads();
    const uint32_t* res = ntt_block(b0, b1, a.ar, tw, C);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int c = warp; c < C; c += nwarps) {
        const int xo = x0 + c;
        const int i = y0 + q, j = tx0 + xo;
        if (xo >= a.To_x || i >= a.h || j >= a.w) continue;          // warp-uniform
        int D = -1;
        uint32_t cnt = 0;
        for (int d0 = ((a.R - 1) / 32) * 32; d0 >= 0 && D < 0; d0 -= 32) {
            const int d = d0 + lane;
            uint32_t v = 0;
            if (d < a.R) {
                int idx = Rf - d;
                if (idx >= Rf) idx -= Rf;
                v = res[idx * C + c];
            }
            const unsigned m = __ballot_sync(0xffffffffu, v != 0u);
            if (m) {
                const int top = 31 - __clz(m);
                D = d0 + top;
                cnt = __shfl_sync(0xffffffffu, v, top);
            }
        }
        if (lane == 0) {
            const int dval = D < 0 ? 0 : D;
            const long long o = (static_cast<long long>(n) * a.h + i) * a.w + j;
            a.out[o] = a.erode ? (a.L - 1 - dval) : dval;
            if (a.out_cnt) a.out_cnt[o] = D < 0 ? 0 : static_cast<int32_t>(cnt);
        }
    }
}

// ----------------------------------------------------- SE spectrum
struct NttTap {
    int dy, dx, b;
};

// plane k: omega_Rf^(k b(y)) at (y mod Ny, y mod Nx) of the torus (planes zeroed)
__global__ void k_ntt_se_scatter(uint32_t* planes, int Rf, int Ny, int Nx, const NttTap* taps, int ntaps,
                                 const uint32_t* wr) {
    const long long per = static_cast<long long>(Ny) * Nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < static_cast<long long>(Rf) * ntaps;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(idx / ntaps), t = static_cast<int>(idx % ntaps);
        const NttTap tp = taps[t];
        const int py = ((tp.dy % Ny) + Ny) % Ny, px = ((tp.dx % Nx) + Nx) % Nx;
        planes[k * per + static_cast<long long>(py) * Nx + px] = wr[(static_cast<long long>(k) * tp.b) % Rf];
    }
}

// In-place forward NTT of every row of Rf planes (grid (Ny, Rf)).
__global__ void __launch_bounds__(256) k_ntt_plane_rows(uint32_t* planes, FftAxis ax, const uint32_t* gtw, int Ny) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = ax.N;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Nx;
    uint32_t* b1 = b0 + Nx;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = gtw[j];
    uint32_t* p = planes + (static_cast<long long>(blockIdx.y) * Ny + blockIdx.x) * Nx;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) b0[j] = p[j];
    __syncthreads();
    const uint32_t* res = ntt_block(b0, b1, ax, tw, 1);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) p[j] = res[j];
}

// In-place forward NTT of every column of Rf planes (grid (ceil(Nx / C), Rf)).
__global__ void __launch_bounds__(256) k_ntt_plane_cols(uint32_t* planes, FftAxis ay, const uint32_t* gtw, int Nx,
                                                        int C) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = ay.N;
    uint32_t* tw = reinterpret_cast<uint32_t*>(sm);
    uint32_t* b0 = tw + Ny;
    uint32_t* b1 = b0 + Ny * C;
    const int u0 = blockIdx.x * C;
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) tw[j] = gtw[j];
    uint32_t* p = planes + static_cast<long long>(blockIdx.y) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x)
        b0[t] = (u0 + t % C < Nx) ? p[static_cast<long long>(t / C) * Nx + u0 + t % C] : 0u;
    __syncthreads();
    const uint32_t* res = ntt_block(b0, b1, ay, tw, C);
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x)
        if (u0 + t % C < Nx) p[static_cast<long long>(t / C) * Nx + u0 + t % C] = res[t];
}

// S <- S * q * 2^-32: with q = (Rf Ny Nx)^-1 2^64 mod P, the Montgomery form of S / (Rf Ny Nx)
__global__ void k_ntt_to_mont(uint32_t* s, long long n, uint32_t q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = mmul(s[i], q);
}

}  // namespace morph

namespace morph {

NttPlan::~NttPlan() {
    for (void* q : {static_cast<void*>(tw_x), static_cast<void*>(tw_y), static_cast<void*>(tw_r),
                    static_cast<void*>(wr), static_cast<void*>(S)})
        if (q) cudaFree(q);
}

static uint64_t hpow(uint64_t b, uint64_t e) { return npow(b, e); }

// N = 2^a 3^b 5^c with c <= 3 (P - 1 = 2^14 3^6 5^3), stages 4, 2, 3, 5
static bool ntt_factor(int N, FftAxis* ax) {
    if (N < 1 || N > kNttMaxN) return false;
    ax->N = N;
    ax->nst = 0;
    int m = N, f4 = 0, f2 = 0, f3 = 0, f5 = 0;
    while (m % 4 == 0) { m /= 4; ++f4; }
    while (m % 2 == 0) { m /= 2; ++f2; }
    while (m % 3 == 0) { m /= 3; ++f3; }
    while (m % 5 == 0) { m /= 5; ++f5; }
    if (m != 1 || f5 > 3 || f3 > 6) return false;
    for (int i = 0; i < f4; ++i) ax->rad[ax->nst++] = 4;
    for (int i = 0; i < f2; ++i) ax->rad[ax->nst++] = 2;
    for (int i = 0; i < f3; ++i) ax->rad[ax->nst++] = 3;
    for (int i = 0; i < f5; ++i) ax->rad[ax->nst++] = 5;
    return ax->nst <= 16;
}

static int ntt_size_at_least(int n) {
    FftAxis t;
    for (int m = std::max(n, 1); m <= kNttMaxN; ++m)
        if (ntt_factor(m, &t)) return m;
    return 0;
}

// integer operations per element of one transform (Montgomery product ~6, add/sub ~2)
static double ntt_ops(const FftAxis& a) {
    double per = 0;
    for (int s = 0; s < a.nst; ++s) {
        const int r = a.rad[s];
        per += r == 2 ? 5.0 : r == 4 ? 8.0 : r == 3 ? 9.0 : 20.0;
    }
    return per * a.N;
}

static size_t ntt_smem_rows(int N, int kg) { return 4 * (static_cast<size_t>(N) * (1 + 2 * kg) + N); }
static size_t ntt_smem_cols(int N, int C) { return 4 * static_cast<size_t>(N) * (1 + 2 * C); }

constexpr double kNttIntOps = 1.2e13;     // sustained integer operations / s (estimate)
constexpr double kNttBytes = 4.0e12;      // sustained HBM bytes / s (estimate)

double ntt_time_estimate(const NttPlan& p) { return p.ops / kNttIntOps + p.bytes / kNttBytes; }

// Overlap-save tiling with the least estimated time.  Exact for every tiling:
// only the transform sizes limit it (each <= 2048).
int plan_ntt_tiles(const morph_image* f, const morph_se* se, NttPlan* p) {
    const int kh = se->kh, kw = se->kw;
    int taps = 0, maxb = 0;
    for (int t = 0; t < kh * kw; ++t)
        if (se->mask[t]) {
            ++taps;
            maxb = std::max(maxb, static_cast<int>(se->offset[t]));
        }
    p->taps = taps;
    p->R = f->L + maxb;
    p->Rf = ntt_size_at_least(p->R);
    if (p->Rf == 0 || !ntt_factor(p->Rf, &p->ar)) return MORPH_E_UNSUPPORTED;
    p->ry = kh - 1 - se->oy;
    p->rx = kw - 1 - se->ox;
    p->kh = kh;
    p->kw = kw;
    const double Rf = p->Rf;
    double best = -1.0;
    const int max_ty = std::min(f->h, 256), max_tx = std::min(f->w, 256);
    for (int nty = 1; nty <= max_ty; ++nty) {
        const int To_y = (f->h + nty - 1) / nty;
        if (nty > 1 && (f->h + nty - 2) / (nty - 1) == To_y) continue;      // same tiling as nty - 1
        const int Ny = ntt_size_at_least(To_y + kh - 1);
        if (Ny == 0) continue;
        FftAxis ay;
        ntt_factor(Ny, &ay);
        for (int ntx = 1; ntx <= max_tx; ++ntx) {
            const int To_x = (f->w + ntx - 1) / ntx;
            if (ntx > 1 && (f->w + ntx - 2) / (ntx - 1) == To_x) continue;
            const int Nx = ntt_size_at_least(To_x + kw - 1);
            if (Nx == 0) continue;
            FftAxis ax;
            ntt_factor(Nx, &ax);
            const int ty = (f->h + To_y - 1) / To_y, tx = (f->w + To_x - 1) / To_x;
            const double tiles = static_cast<double>(f->n) * ty * tx;
            const double Rin = To_y + kh - 1;
            const double ops = tiles * (Rf * ((Rin + To_y) * ntt_ops(ax) + 2.0 * Nx * ntt_ops(ay) + 6.0 * Nx * Ny) +
                                        static_cast<double>(To_y) * To_x * ntt_ops(p->ar));
            const double bytes = tiles * Rf * 4.0 *
                                 (2.0 * Rin * Nx + 2.0 * To_y * Nx + 2.0 * To_y * To_x + 0.5 * Nx * Ny);
            const double t = ops / kNttIntOps + bytes / kNttBytes;
            if (best < 0 || t < best) {
                best = t;
                p->ops = ops;
                p->bytes = bytes;
                p->To_y = To_y;
                p->To_x = To_x;
                p->ax = ax;
                p->ay = ay;
                p->tiles_y = ty;
                p->tiles_x = tx;
            }
        }
    }
    if (best < 0) return MORPH_E_UNSUPPORTED;
    p->Rin_y = p->To_y + kh - 1;
    p->Win_x = p->To_x + kw - 1;
    p->ntiles = static_cast<long long>(f->n) * p->tiles_y * p->tiles_x;
    const int Nx = p->ax.N, Ny = p->ay.N;
    p->kgroup = std::max(1, std::min(p->Rf, 4096 / Nx));
    p->colgroup = std::max(1, std::min(16, (51200 / Ny - 1) / 2));
    p->pixgroup = std::max(1, std::min(32, (51200 / p->Rf - 1) / 2));
    const size_t per_tile = static_cast<size_t>(p->Rf) * Nx * Ny * 4;
    const size_t budget = size_t(4) << 30;
    long long wt = static_cast<long long>(budget / std::max<size_t>(per_tile, 1));
    wt = std::max<long long>(1, std::min<long long>({wt, p->ntiles, 65535}));
    p->wave_tiles = static_cast<int>(wt);
    p->buf_bytes = per_tile * static_cast<size_t>(wt);
    p->ws_bytes = p->buf_bytes;
    return MORPH_OK;
}

static int set_ntt_smem() {
    static bool done = false;
    if (done) return MORPH_OK;
    const int big = 200 * 1024;
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_range, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_plane_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_plane_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    done = true;
    return MORPH_OK;
}

// omega_N^m for m < N: Montgomery form (mont = 1) or plain
static std::vector<uint32_t> ntt_table(int N, bool mont) {
    std::vector<uint32_t> t(N);
    const uint64_t w = hpow(kG, (kP - 1) / static_cast<uint64_t>(N));
    uint64_t x = 1;
    for (int m = 0; m < N; ++m) {
        t[m] = mont ? to_mont(x) : static_cast<uint32_t>(x);
        x = x * w % kP;
    }
    return t;
}

static int upload(uint32_t** d, const std::vector<uint32_t>& h) {
    MORPH_CUDA_TRY(cudaMalloc(d, h.size() * sizeof(uint32_t)));
    MORPH_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    return MORPH_OK;
}

// Tables and the SE spectrum S_k = 2-D NTT (Ny x Nx) of s_k, scaled by (Rf Ny Nx)^-1.
int build_ntt_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, NttPlan* p) {
    int rc = plan_ntt_tiles(f, se, p);
    if (rc) return rc;
    // the radix roots must have their exact orders (g primitive)
    if (npow(kW4, 2) != kP - 1 || kW3 == 1 || npow(kW3, 3) != 1 || kW5 == 1 || npow(kW5, 5) != 1)
        return MORPH_E_UNSUPPORTED;
    rc = set_ntt_smem();
    if (rc) return rc;
    const int Nx = p->ax.N, Ny = p->ay.N, Rf = p->Rf;
    if ((rc = upload(&p->tw_x, ntt_table(Nx, true)))) return rc;
    if ((rc = upload(&p->tw_y, ntt_table(Ny, true)))) return rc;
    if ((rc = upload(&p->tw_r, ntt_table(Rf, true)))) return rc;
    if ((rc = upload(&p->wr, ntt_table(Rf, false)))) return rc;
    std::vector<NttTap> taps;
    for (int r = 0; r < se->kh; ++r)
        for (int c = 0; c < se->kw; ++c) {
            const int t = r * se->kw + c;
            if (se->mask[t]) taps.push_back(NttTap{r - se->oy, c - se->ox, se->offset[t]});
        }
    const long long nS = static_cast<long long>(Rf) * Ny * Nx;
    MORPH_CUDA_TRY(cudaMalloc(&p->S, nS * sizeof(uint32_t)));
    MORPH_CUDA_TRY(cudaMemset(p->S, 0, nS * sizeof(uint32_t)));
    NttTap* d_taps = nullptr;
    MORPH_CUDA_TRY(cudaMalloc(&d_taps, taps.size() * sizeof(NttTap)));
    MORPH_CUDA_TRY(cudaMemcpy(d_taps, taps.data(), taps.size() * sizeof(NttTap), cudaMemcpyHostToDevice));
    {
        const long long n = static_cast<long long>(Rf) * static_cast<long long>(taps.size());
        const unsigned blocks = static_cast<unsigned>(std::min<long long>((n + 255) / 256, 4096));
        k_ntt_se_scatter<<<blocks, 256>>>(p->S, Rf, Ny, Nx, d_taps, static_cast<int>(taps.size()), p->wr);
    }
    k_ntt_plane_rows<<<dim3(Ny, Rf), 256, ntt_smem_rows(Nx, 1)>>>(p->S, p->ax, p->tw_x, Ny);
    const int C = p->colgroup;
    k_ntt_plane_cols<<<dim3((Nx + C - 1) / C, Rf), 256, ntt_smem_cols(Ny, C)>>>(p->S, p->ay, p->tw_y, Nx, C);
    const uint64_t scale = static_cast<uint64_t>(Rf) * Ny * Nx % kP;
    const uint64_t inv = hpow(scale, kP - 2);
    const uint64_t r32 = (uint64_t(1) << 32) % kP;
    const uint32_t q = static_cast<uint32_t>(inv * r32 % kP * r32 % kP);
    k_ntt_to_mont<<<static_cast<unsigned>(std::min<long long>((nS + 255) / 256, 8192)), 256>>>(p->S, nS, q);
    ctx->launches += 4;
    MORPH_CUDA_TRY(cudaGetLastError());
    MORPH_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(d_taps);
    return MORPH_OK;
}

int launch_ntt_in(morph_ctx* ctx, const NttPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                  void* buf, cudaStream_t st) {
    NttArgs a;
    std::memset(&a, 0, sizeof(a));
    a.src = f->data;
    a.dtype = f->dtype;
    a.n = f->n;
    a.h = f->h;
    a.w = f->w;
    a.row_stride = f->row_stride;
    a.batch_stride = f->batch_stride;
    a.L = f->L;
    a.flip = erode;
    a.erode = erode;
    a.R = p.R;
    a.Rf = p.Rf;
    a.ar = p.ar;
    a.ax = p.ax;
    a.ay = p.ay;
    a.To_y = p.To_y;
    a.To_x = p.To_x;
    a.Rin_y = p.Rin_y;
    a.Win_x = p.Win_x;
    a.ry = p.ry;
    a.rx = p.rx;
    a.tiles_x = p.tiles_x;
    a.tiles_y = p.tiles_y;
    a.tw_x = p.tw_x;
    a.tw_y = p.tw_y;
    a.tw_r = p.tw_r;
    a.wr = p.wr;
    a.S = p.S;
    a.buf = static_cast<uint32_t*>(buf);
    a.out = out;
    a.out_cnt = cnt;
    a.err = ctx->d_err;
    a.kgroup = p.kgroup;
    a.colgroup = p.colgroup;
    a.pixgroup = p.pixgroup;
    const int Nx = p.ax.N, Ny = p.ay.N;
    for (long long t0 = 0; t0 < p.ntiles; t0 += p.wave_tiles) {
        a.tile0 = t0;
        a.wave_tiles = static_cast<int>(std::min<long long>(p.wave_tiles, p.ntiles - t0));
        prof_begin(ctx, st, "k_ntt_rows_fwd");
        k_ntt_rows_fwd<<<dim3(p.Rin_y, a.wave_tiles), 256, ntt_smem_rows(Nx, p.kgroup), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_cols");
        k_ntt_cols<<<dim3((Nx + p.colgroup - 1) / p.colgroup, p.Rf, a.wave_tiles), 256,
                     ntt_smem_cols(Ny, p.colgroup), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_rows_inv");
        k_ntt_rows_inv<<<dim3(p.To_y, (p.Rf + p.kgroup - 1) / p.kgroup, a.wave_tiles), 256,
                         ntt_smem_rows(Nx, p.kgroup), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_range");
        k_ntt_range<<<dim3((p.To_x + p.pixgroup - 1) / p.pixgroup, p.To_y, a.wave_tiles), 256,
                      ntt_smem_cols(p.Rf, p.pixgroup), st>>>(a);
        prof_end(ctx, st);
        ctx->launches += 4;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    return MORPH_OK;
}

int launch_ntt(morph_ctx* ctx, const NttPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
               cudaStream_t st) {
    void* buf = nullptr;
    int rc = ctx_workspace(ctx, p.ws_bytes, &buf);
    if (rc) return rc;
    return launch_ntt_in(ctx, p, f, erode, out, cnt, buf, st);
}

}  // namespace morph
