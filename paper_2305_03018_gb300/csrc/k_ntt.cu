// Step 2 of the method as an exact number-theoretic transform (NTT), followed
// by Step 3 (Eq. 9).  The paper points to modular transforms as the exact
// alternative to the floating-point FFT (Sec. 2.2): the count polynomial of
// Eq. Obs7 has integer coefficients in [0, |B|], so its convolution computed
// modulo a prime P > |B| is the exact count, with no round-off bound.
//
// P = 2^13 3^6 5^3 + 1 = 746496001 (prime, < 2^30), so P - 1 is divisible by
// every transform length 2^a 3^b 5^c <= 2048 with c <= 3.  omega_N =
// g^((P-1)/N) with the primitive root g = 7 plays the part of exp(-2 pi i / N).
// Residues are kept lazily in [0, 2P) (sums of two stay below 4P < 2^32) and
// reduced once where a count is read.  Products by constants (twiddles, radix
// roots) use Shoup's precomputed quotient; products by the SE spectrum use the
// Montgomery form (REDC with 2^32), the spectrum being stored multiplied by
// 2^32 mod P.
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

constexpr uint32_t kP = 746496001u;        // 2^13 3^6 5^3 + 1
constexpr uint32_t kPinv = 1216258047u;    // -P^-1 mod 2^32
constexpr uint64_t kG = 7u;                // primitive root mod P
constexpr uint32_t k2P = 2u * kP;
static_assert(kP < (1u << 30), "lazy residues in [0, 2P) need 4P < 2^32");
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

// radix roots omega_r = g^((P-1)/r)
constexpr uint64_t kW3 = npow(kG, (kP - 1) / 3);
constexpr uint64_t kW4 = npow(kG, (kP - 1) / 4);
constexpr uint64_t kW5 = npow(kG, (kP - 1) / 5);

// [0, 4P) -> [0, 2P)
__device__ __forceinline__ uint32_t lz(uint32_t x) { return min(x, x - k2P); }
__device__ __forceinline__ uint32_t ladd(uint32_t a, uint32_t b) { return lz(a + b); }
__device__ __forceinline__ uint32_t lsub(uint32_t a, uint32_t b) { return lz(a + k2P - b); }
// [0, 2P) -> [0, P)
__device__ __forceinline__ uint32_t canon(uint32_t x) { return min(x, x - kP); }
// a * bm * 2^-32 mod P in [0, 2P) for a, bm < 2P (Montgomery REDC): with
// bm = b 2^32 mod P this is a b mod P.  t = a bm < 4P^2 < 2^62, m = (t mod
// 2^32) (-P^-1) mod 2^32; (t + m P) / 2^32 < P (4P / 2^32 + 1) < 2P.  The low
// words of t and m P sum to 0 or 2^32, a carry exactly when t mod 2^32 != 0.
__device__ __forceinline__ uint32_t mmul(uint32_t a, uint32_t bm) {
    const uint64_t t = static_cast<uint64_t>(a) * bm;
    const uint32_t lo = static_cast<uint32_t>(t), hi = static_cast<uint32_t>(t >> 32);
    const uint32_t m = lo * kPinv;
    return hi + __umulhi(m, kP) + (lo != 0u ? 1u : 0u);
}
// x w mod P in [0, 2P) for any 32-bit x and a constant w < P with
// wq = floor(w 2^32 / P) (Shoup): x w - floor(x wq / 2^32) P lies in [0, 2P).
__device__ __forceinline__ uint32_t lmul(uint32_t x, uint32_t w, uint32_t wq) {
    return x * w - __umulhi(x, wq) * kP;
}
constexpr uint32_t shoup_q(uint64_t w) { return static_cast<uint32_t>((w << 32) / kP); }

constexpr uint64_t kC1 = (kW5 + npow(kW5, 4)) % kP * kInv2 % kP;
constexpr uint64_t kC2 = (npow(kW5, 2) + npow(kW5, 3)) % kP * kInv2 % kP;
constexpr uint64_t kS1 = (kW5 + kP - npow(kW5, 4)) % kP * kInv2 % kP;
constexpr uint64_t kS2 = (npow(kW5, 2) + kP - npow(kW5, 3)) % kP * kInv2 % kP;
// (value, Shoup quotient) of the radix constants, as compile-time constants
struct NttConst {
    uint32_t w, q;
};
constexpr NttConst nconst(uint64_t c) { return NttConst{static_cast<uint32_t>(c), shoup_q(c)}; }
constexpr uint64_t kW16 = npow(kG, (kP - 1) / 16);
constexpr NttConst kW3c = nconst(kW3), kW4c = nconst(kW4);
// omega_16^m for the products m = n2 k1 (n2, k1 in 1..3) inside a radix-16 butterfly
constexpr NttConst kW16_1c = nconst(kW16), kW16_2c = nconst(npow(kW16, 2)), kW16_3c = nconst(npow(kW16, 3));
constexpr NttConst kW16_4c = nconst(npow(kW16, 4)), kW16_6c = nconst(npow(kW16, 6)), kW16_9c = nconst(npow(kW16, 9));
constexpr NttConst kC1c = nconst(kC1), kC2c = nconst(kC2), kS1c = nconst(kS1), kS2c = nconst(kS2);
#define NTT_K(x) x##c.w, x##c.q

// Radix-r forward DFTs mod P, y_k = sum_j v_j omega_r^(jk), in registers;
// inputs and outputs in [0, 2P).
__device__ __forceinline__ void ndft2(uint32_t* v) {
    const uint32_t a = v[0], b = v[1];
    v[0] = ladd(a, b);
    v[1] = lsub(a, b);
}
__device__ __forceinline__ void ndft4(uint32_t* v) {
    // omega_4^2 = -1
    const uint32_t s02 = ladd(v[0], v[2]), d02 = lsub(v[0], v[2]);
    const uint32_t s13 = ladd(v[1], v[3]), d13 = lmul(v[1] + k2P - v[3], NTT_K(kW4));
    v[0] = ladd(s02, s13);
    v[2] = lsub(s02, s13);
    v[1] = ladd(d02, d13);
    v[3] = lsub(d02, d13);
}
__device__ __forceinline__ void ndft3(uint32_t* v) {
    // omega^2 = -1 - omega: y1 = (v0 - v2) + omega (v1 - v2), y2 = (v0 - v1) - omega (v1 - v2)
    const uint32_t t = lmul(v[1] + k2P - v[2], NTT_K(kW3));
    const uint32_t y0 = ladd(ladd(v[0], v[1]), v[2]);
    const uint32_t y1 = ladd(lsub(v[0], v[2]), t);
    const uint32_t y2 = lsub(lsub(v[0], v[1]), t);
    v[0] = y0;
    v[1] = y1;
    v[2] = y2;
}
__device__ __forceinline__ void ndft5(uint32_t* v) {
    // C_j = (w^j + w^-j) / 2, S_j = (w^j - w^-j) / 2 with w = omega_5
    const uint32_t b1 = ladd(v[1], v[4]), b2 = ladd(v[2], v[3]);
    const uint32_t d1 = v[1] + k2P - v[4], d2 = v[2] + k2P - v[3];     // < 4P: Shoup inputs
    const uint32_t a0 = v[0];
    const uint32_t A1 = ladd(a0, ladd(lmul(b1, NTT_K(kC1)), lmul(b2, NTT_K(kC2))));
    const uint32_t B1 = ladd(lmul(d1, NTT_K(kS1)), lmul(d2, NTT_K(kS2)));
    const uint32_t A2 = ladd(a0, ladd(lmul(b1, NTT_K(kC2)), lmul(b2, NTT_K(kC1))));
    const uint32_t B2 = lsub(lmul(d1, NTT_K(kS2)), lmul(d2, NTT_K(kS1)));
    v[0] = ladd(a0, ladd(b1, b2));
    v[1] = ladd(A1, B1);
    v[4] = lsub(A1, B1);
    v[2] = ladd(A2, B2);
    v[3] = lsub(A2, B2);
}

// Radix 16 as 4 x 4: with n = 4 n1 + n2 and k = k1 + 4 k2,
// y_k = sum_n2 omega_16^(n2 k1) omega_4^(n2 k2) sum_n1 v_(4 n1 + n2) omega_4^(n1 k1):
// four radix-4 DFTs over n1, the nine twiddles omega_16^(n2 k1), four radix-4 DFTs over n2.
__device__ __forceinline__ void ndft16(uint32_t* v) {
    uint32_t u[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        uint32_t w[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
        ndft4(w);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) u[n2][k1] = w[k1];
    }
    u[1][1] = lmul(u[1][1], NTT_K(kW16_1));
    u[1][2] = lmul(u[1][2], NTT_K(kW16_2));
    u[1][3] = lmul(u[1][3], NTT_K(kW16_3));
    u[2][1] = lmul(u[2][1], NTT_K(kW16_2));
    u[2][2] = lmul(u[2][2], NTT_K(kW16_4));
    u[2][3] = lmul(u[2][3], NTT_K(kW16_6));
    u[3][1] = lmul(u[3][1], NTT_K(kW16_3));
    u[3][2] = lmul(u[3][2], NTT_K(kW16_6));
    u[3][3] = lmul(u[3][3], NTT_K(kW16_9));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        uint32_t w[4] = {u[0][k1], u[1][k1], u[2][k1], u[3][k1]};
        ndft4(w);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = w[k2];
    }
}

constexpr int ilog2c(int b) { return b <= 1 ? 0 : 1 + ilog2c(b / 2); }
// element p of transform c of a batch of B lives at p * pitch(B) + c; the odd
// pitch keeps column reads (fixed c, consecutive p) free of bank conflicts
constexpr int npitch(int B) { return B == 1 ? 1 : B + 1; }

// One Stockham stage of radix R over B interleaved transforms of length N.
// tw[m] = (omega_N^m, Shoup quotient).
template <int R, int B>
__device__ __forceinline__ void ntt_stage(const uint32_t* __restrict__ x, uint32_t* __restrict__ y, int N, int Ns,
                                          uint32_t nsm, int tstep, const uint2* __restrict__ tw) {
    constexpr int PB = npitch(B);
    constexpr int LB = ilog2c(B);
    const int M = N / R;
    const int total = M * B;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int c = t & (B - 1);
        const int j = t >> LB;
        const int g = Ns == 1 ? j : static_cast<int>(__umulhi(static_cast<uint32_t>(j), nsm));   // j / Ns
        const int k = j - g * Ns;
        uint32_t v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[(j + r * M) * PB + c];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const uint2 w = tw[r * k * tstep];
                v[r] = lmul(v[r], w.x, w.y);
            }
        }
        if (R == 2) ndft2(v);
        if (R == 3) ndft3(v);
        if (R == 4) ndft4(v);
        if (R == 5) ndft5(v);
        if (R == 16) ndft16(v);
        const int d = g * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[(d + r * Ns) * PB + c] = v[r];
    }
}

// Forward NTT of B interleaved transforms in a (scratch b); returns the buffer
// holding the result.  Block-wide; ends with a barrier.
template <int B>
__device__ __forceinline__ uint32_t* ntt_block(uint32_t* a, uint32_t* b, const NttAxis& ax, const uint2* tw) {
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s];
        if (R == 16) ntt_stage<16, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else if (R == 4) ntt_stage<4, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else if (R == 2) ntt_stage<2, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else if (R == 3) ntt_stage<3, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else ntt_stage<5, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
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
    uint32_t rfm;                   // ceil(2^32 / Rf)
    NttAxis ar, ax, ay;
    int To_y, To_x, Rin_y, Win_x;   // output tile, input tile (To + k - 1)
    int ry, rx;                     // SE reach below / right: kh - 1 - oy, kw - 1 - ox
    int tiles_x, tiles_y;
    long long tile0;                // first global tile of this wave
    int wave_tiles;
    const uint2* tw_x;              // (omega_Nx^m, Shoup quotient)
    const uint2* tw_y;
    const uint2* tw_r;
    const uint32_t* wr;             // omega_Rf^m (encoder table)
    const uint32_t* S;              // SE spectrum / (Rf Ny Nx), Montgomery form, [Rf][Ny][Nx]
    uint32_t* buf;                  // [wave_tiles][Rf][Ny][Nx]
    int32_t* out;
    int32_t* out_cnt;
    int out_add;                    // output adjustment of a composite's pass (OutAdjust)
    const int32_t* out_sub;
    unsigned int* err;
    int kper;                       // grey frequencies per CTA of k_ntt_rows_fwd (multiple of its batch)
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

__device__ __forceinline__ void ntt_copy_tw(uint2* dst, const uint2* src, int n) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
}

// grid (Rin_y, wave_tiles, ceil(Rf / kper)): input row rho of tile tl, grey
// frequencies [z kper, (z + 1) kper), B at a time
template <int B>
__global__ void __launch_bounds__(256) k_ntt_rows_fwd(const NttArgs a) {
    constexpr int PB = npitch(B);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N, Rf = a.Rf;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* wr = reinterpret_cast<uint32_t*>(tw + Nx);
    int* lev = reinterpret_cast<int*>(wr + Rf);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(lev + Nx);
    uint32_t* b1 = b0 + Nx * PB;
    const int rho = blockIdx.x, tl = blockIdx.y;
    int n, y0, x0;
    ntt_tile_origin(a, a.tile0 + tl, &n, &y0, &x0);
    ntt_copy_tw(tw, a.tw_x, Nx);
    for (int j = threadIdx.x; j < Rf; j += blockDim.x) wr[j] = a.wr[j];
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
    uint32_t* dst = a.buf + static_cast<long long>(tl) * Rf * plane + static_cast<long long>(rho) * Nx;
    const int kend = min(Rf, static_cast<int>(blockIdx.z + 1) * a.kper);
    for (int k0 = blockIdx.z * a.kper; k0 < kend; k0 += B) {
        for (int t = threadIdx.x; t < B * Nx; t += blockDim.x) {
            const int c = t & (B - 1), p = t >> ilog2c(B);
            const int l = lev[p];
            const uint32_t e = static_cast<uint32_t>(k0 + c) * static_cast<uint32_t>(l < 0 ? 0 : l);
            const uint32_t m = e - __umulhi(e, a.rfm) * static_cast<uint32_t>(Rf);       // e mod Rf
            b0[p * PB + c] = (l >= 0 && k0 + c < Rf) ? wr[m] : 0u;
        }
        __syncthreads();
        const uint32_t* res = ntt_block<B>(b0, b1, a.ax, tw);
        const int kb = min(B, Rf - k0);
        for (int c = 0; c < kb; ++c)
            for (int p = threadIdx.x; p < Nx; p += blockDim.x) dst[(k0 + c) * plane + p] = res[p * PB + c];
        __syncthreads();
    }
}

// grid (wave_tiles, ceil(Nx / C), Rf): the tiles of one (column group, k) run
// together, so they read that strip of the SE spectrum from L2
template <int C>
__global__ void __launch_bounds__(512) k_ntt_cols(const NttArgs a) {
    constexpr int PC = npitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = a.ay.N, Nx = a.ax.N;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(tw + Ny);
    uint32_t* b1 = b0 + Ny * PC;
    const int tl = blockIdx.x, u0 = blockIdx.y * C, k = blockIdx.z;
    ntt_copy_tw(tw, a.tw_y, Ny);
    uint32_t* plane = a.buf + (static_cast<long long>(tl) * a.Rf + k) * Ny * Nx;
    // four independent loads in flight per thread
    for (int t0 = threadIdx.x; t0 < Ny * C; t0 += 4 * blockDim.x) {
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * blockDim.x;
            const int c = t & (C - 1), rho = t >> ilog2c(C);
            v[u] = (rho < a.Rin_y && u0 + c < Nx) ? plane[static_cast<long long>(rho) * Nx + u0 + c] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < Ny * C) b0[(t >> ilog2c(C)) * PC + (t & (C - 1))] = v[u];
        }
    }
    __syncthreads();
    const uint32_t* S = a.S + static_cast<long long>(k) * Ny * Nx;
    // pull this CTA's strip of the SE spectrum towards L2 while the column transforms run
    for (int v = threadIdx.x; v < Ny; v += blockDim.x)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(S + static_cast<long long>(v) * Nx + u0));
    uint32_t* res = ntt_block<C>(b0, b1, a.ay, tw);
    uint32_t* other = (res == b0) ? b1 : b0;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), v = t >> ilog2c(C);
        if (u0 + c < Nx) res[v * PC + c] = mmul(res[v * PC + c], S[static_cast<long long>(v) * Nx + u0 + c]);
    }
    __syncthreads();
    const uint32_t* o = ntt_block<C>(res, other, a.ay, tw);
    // torus position of output row q is (q + ry) mod Ny (ry < 0 or >= Ny when the origin lies outside the box)
    const int base = ((a.ry % Ny) + Ny) % Ny;
    for (int t = threadIdx.x; t < a.To_y * C; t += blockDim.x) {
        const int c = t & (C - 1), q = t >> ilog2c(C);
        int pos = base + q;
        while (pos >= Ny) pos -= Ny;
        const int idx = pos == 0 ? 0 : Ny - pos;
        if (u0 + c < Nx) plane[static_cast<long long>(q) * Nx + u0 + c] = o[idx * PC + c];
    }
}

// grid (To_y, ceil(Rf / B), wave_tiles): output row q, B grey frequencies
template <int B>
__global__ void __launch_bounds__(256) k_ntt_rows_inv(const NttArgs a) {
    constexpr int PB = npitch(B);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(tw + Nx);
    uint32_t* b1 = b0 + Nx * PB;
    const int q = blockIdx.x, k0 = blockIdx.y * B, tl = blockIdx.z;
    const int kb = min(B, a.Rf - k0);
    ntt_copy_tw(tw, a.tw_x, Nx);
    const long long plane = static_cast<long long>(a.ay.N) * Nx;
    uint32_t* rows = a.buf + (static_cast<long long>(tl) * a.Rf + k0) * plane + static_cast<long long>(q) * Nx;
    for (int c = 0; c < B; ++c)
        for (int p0 = threadIdx.x; p0 < Nx; p0 += 4 * blockDim.x) {
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * blockDim.x;
                v[u] = (c < kb && p < Nx) ? rows[c * plane + p] : 0u;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * blockDim.x;
                if (p < Nx) b0[p * PB + c] = v[u];
            }
        }
    __syncthreads();
    const uint32_t* res = ntt_block<B>(b0, b1, a.ax, tw);
    const int base = ((a.rx % Nx) + Nx) % Nx;
    for (int c = 0; c < kb; ++c)
        for (int p = threadIdx.x; p < a.To_x; p += blockDim.x) {
            int pos = base + p;
            while (pos >= Nx) pos -= Nx;
            const int idx = pos == 0 ? 0 : Nx - pos;
            rows[c * plane + p] = res[idx * PB + c];
        }
}

// grid (ceil(To_x / C), To_y, wave_tiles): grey-axis inverse NTT of C pixels
// of output row q, then the top degree with a nonzero count (Eq. 9).
template <int C>
__global__ void __launch_bounds__(512) k_ntt_range(const NttArgs a) {
    constexpr int PC = npitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Rf = a.Rf, Nx = a.ax.N, Ny = a.ay.N;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(tw + Rf);
    uint32_t* b1 = b0 + Rf * PC;
    const int x0 = blockIdx.x * C, q = blockIdx.y, tl = blockIdx.z;
    int n, y0, tx0;
    ntt_tile_origin(a, a.tile0 + tl, &n, &y0, &tx0);
    ntt_copy_tw(tw, a.tw_r, Rf);
    const long long kstride = static_cast<long long>(Ny) * Nx;
    const uint32_t* base = a.buf + static_cast<long long>(tl) * Rf * kstride + static_cast<long long>(q) * Nx;
    for (int t0 = threadIdx.x; t0 < Rf * C; t0 += 4 * blockDim.x) {
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * blockDim.x;
            const int c = t & (C - 1), k = t >> ilog2c(C);
            v[u] = (t < Rf * C && x0 + c < a.To_x) ? base[k * kstride + x0 + c] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + u * blockDim.x;
            if (t < Rf * C) b0[(t >> ilog2c(C)) * PC + (t & (C - 1))] = v[u];
        }
    }
    __syncthreads();
    const uint32_t* res = ntt_block<C>(b0, b1, a.ar, tw);
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
            if (d < a.R) v = canon(res[(d == 0 ? 0 : Rf - d) * PC + c]);
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
            a.out[o] = (a.erode ? (a.L - 1 - dval) : dval) + a.out_add - (a.out_sub ? a.out_sub[o] : 0);
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
__global__ void __launch_bounds__(256) k_ntt_plane_rows(uint32_t* planes, NttAxis ax, const uint2* gtw, int Ny) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = ax.N;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(tw + Nx);
    uint32_t* b1 = b0 + Nx;
    ntt_copy_tw(tw, gtw, Nx);
    uint32_t* p = planes + (static_cast<long long>(blockIdx.y) * Ny + blockIdx.x) * Nx;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) b0[j] = p[j];
    __syncthreads();
    const uint32_t* res = ntt_block<1>(b0, b1, ax, tw);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) p[j] = res[j];
}

// In-place forward NTT of every column of Rf planes (grid (ceil(Nx / 8), Rf)).
__global__ void __launch_bounds__(256) k_ntt_plane_cols(uint32_t* planes, NttAxis ay, const uint2* gtw, int Nx) {
    constexpr int C = 8, PC = npitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = ay.N;
    uint2* tw = reinterpret_cast<uint2*>(sm);
    uint32_t* b0 = reinterpret_cast<uint32_t*>(tw + Ny);
    uint32_t* b1 = b0 + Ny * PC;
    const int u0 = blockIdx.x * C;
    ntt_copy_tw(tw, gtw, Ny);
    uint32_t* p = planes + static_cast<long long>(blockIdx.y) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), r = t >> ilog2c(C);
        b0[r * PC + c] = (u0 + c < Nx) ? p[static_cast<long long>(r) * Nx + u0 + c] : 0u;
    }
    __syncthreads();
    const uint32_t* res = ntt_block<C>(b0, b1, ay, tw);
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), r = t >> ilog2c(C);
        if (u0 + c < Nx) p[static_cast<long long>(r) * Nx + u0 + c] = res[r * PC + c];
    }
}

// S <- S * q * 2^-32: with q = (Rf Ny Nx)^-1 2^64 mod P, the Montgomery form of S / (Rf Ny Nx)
__global__ void k_ntt_to_mont(uint32_t* s, long long n, uint32_t q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s[i] = canon(mmul(s[i], q));
}

}  // namespace morph

namespace morph {

NttPlan::~NttPlan() {
    for (void* q : {static_cast<void*>(tw_x), static_cast<void*>(tw_y), static_cast<void*>(tw_r),
                    static_cast<void*>(wr), static_cast<void*>(S)})
        if (q) cudaFree(q);
}

static uint64_t hpow(uint64_t b, uint64_t e) { return npow(b, e); }

// N = 2^a 3^b 5^c with c <= 3 (P - 1 = 2^13 3^6 5^3), stages 16, 4, 2, 3, 5, with
// each stage's twiddle stride and the division magic for Ns
static bool ntt_factor(int N, NttAxis* ax) {
    if (N < 1 || N > kNttMaxN) return false;
    ax->N = N;
    ax->nst = 0;
    int m = N, f16 = 0, f4 = 0, f2 = 0, f3 = 0, f5 = 0;
    while (m % 16 == 0) { m /= 16; ++f16; }
    while (m % 4 == 0) { m /= 4; ++f4; }
    while (m % 2 == 0) { m /= 2; ++f2; }
    while (m % 3 == 0) { m /= 3; ++f3; }
    while (m % 5 == 0) { m /= 5; ++f5; }
    if (m != 1 || f5 > 3 || f3 > 6 || f16 + f4 + f2 + f3 + f5 > 16) return false;
    for (int i = 0; i < f16; ++i) ax->rad[ax->nst++] = 16;
    for (int i = 0; i < f4; ++i) ax->rad[ax->nst++] = 4;
    for (int i = 0; i < f2; ++i) ax->rad[ax->nst++] = 2;
    for (int i = 0; i < f3; ++i) ax->rad[ax->nst++] = 3;
    for (int i = 0; i < f5; ++i) ax->rad[ax->nst++] = 5;
    int Ns = 1;
    for (int s = 0; s < ax->nst; ++s) {
        ax->tstep[s] = N / (Ns * ax->rad[s]);
        // ceil(2^32 / Ns): floor(j * nsm / 2^32) = j / Ns exactly while j * Ns < 2^32
        ax->nsm[s] = Ns == 1 ? 0u : static_cast<uint32_t>(((uint64_t(1) << 32) + Ns - 1) / Ns);
        Ns *= ax->rad[s];
    }
    return true;
}

// smallest supported transform length >= n (0 if above 2048)
static int ntt_size_at_least(int n) {
    static std::vector<int> next;
    if (next.empty()) {
        next.assign(kNttMaxN + 2, 0);
        NttAxis t;
        for (int m = kNttMaxN; m >= 1; --m) next[m] = ntt_factor(m, &t) ? m : next[m + 1];
    }
    n = std::max(n, 1);
    return n > kNttMaxN ? 0 : next[n];
}

// integer instructions per element of one transform: per stage, the twiddle
// products (Shoup, ~5), the radix's own products and the modular sums (~3)
static double ntt_ops(const NttAxis& a) {
    double per = 0;
    for (int s = 0; s < a.nst; ++s) {
        const int r = a.rad[s];
        per += r == 2 ? 6.0 : r == 4 ? 11.0 : r == 16 ? 16.0 : r == 3 ? 12.0 : 24.0;
    }
    return per * a.N;
}

static int pow2_floor(int x) {
    int p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

// shared memory of each kernel (bytes): twiddle pairs, tables, two pitched buffers
static size_t smem_rows_fwd(int Nx, int Rf, int B) {
    return 8 * static_cast<size_t>(Nx) + 4 * static_cast<size_t>(Rf) + 4 * static_cast<size_t>(Nx) +
           8 * static_cast<size_t>(Nx) * npitch(B);
}
static size_t smem_pitched(int N, int B) { return 8 * static_cast<size_t>(N) + 8 * static_cast<size_t>(N) * npitch(B); }
constexpr size_t kNttSmemMax = 200 * 1024;
constexpr size_t kNttSmemHalf = 110 * 1024;

// rates of the time estimate, fitted to GB300 runs (2048^2 / 204^2, 4096^2 / 31^2 and
// 1024^2 / 102^2 at L = 256): the estimate lands within about 5 % of the measured time
constexpr double kNttIntOps = 1.6e13;     // model integer instructions / s
constexpr double kNttBytes = 4.0e12;      // HBM bytes / s
constexpr double kNttCta = 8.0e-9;        // s per CTA (start-up amortised over the SMs)

// grey frequencies per row-kernel pass: ~4096 elements, no more than the axis holds
static int ntt_kgroup(int Nx, int Rf) {
    int b = std::min(64, pow2_floor(std::max(1, 4096 / Nx)));
    while (b > 1 && b / 2 >= Rf) b /= 2;
    return b;
}

// pixels per k_ntt_range CTA: up to 128 (short grey axes), two CTAs per SM
static int ntt_pixgroup(int Rf) {
    int c = 128;
    while (c > 1 && smem_pitched(Rf, c) > kNttSmemHalf) c /= 2;
    return c;
}

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
        NttAxis ay;
        ntt_factor(Ny, &ay);
        for (int ntx = 1; ntx <= max_tx; ++ntx) {
            const int To_x = (f->w + ntx - 1) / ntx;
            if (ntx > 1 && (f->w + ntx - 2) / (ntx - 1) == To_x) continue;
            const int Nx = ntt_size_at_least(To_x + kw - 1);
            if (Nx == 0) continue;
            NttAxis ax;
            ntt_factor(Nx, &ax);
            const int ty = (f->h + To_y - 1) / To_y, tx = (f->w + To_x - 1) / To_x;
            const double tiles = static_cast<double>(f->n) * ty * tx;
            const double Rin = To_y + kh - 1;
            const double ops = tiles * (Rf * ((Rin + To_y) * ntt_ops(ax) + 2.0 * Nx * ntt_ops(ay) + 10.0 * Nx * Ny) +
                                        static_cast<double>(To_y) * To_x * ntt_ops(p->ar));
            const double bytes = tiles * Rf * 4.0 *
                                 (2.0 * Rin * Nx + 2.0 * To_y * Nx + 2.0 * To_y * To_x + 0.5 * Nx * Ny);
            // CTAs of the four kernels (each pays a fixed start-up: tables, barriers)
            const int kg = ntt_kgroup(Nx, p->Rf);
            const double ctas = tiles * (Rin + (Nx / 8.0) * Rf + To_y * std::ceil(Rf / kg) +
                                         std::ceil(To_x / static_cast<double>(ntt_pixgroup(p->Rf))) * To_y);
            const double t = ops / kNttIntOps + bytes / kNttBytes + ctas * kNttCta;
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
    // batch sizes (powers of two): ~4096 elements per row-kernel pass, the
    // widest column / pixel groups whose buffers fit in shared memory
    p->kgroup = ntt_kgroup(Nx, p->Rf);
    // column / pixel groups small enough for two CTAs per SM; 512 threads for big groups
    p->colgroup = 16;
    while (p->colgroup > 1 && smem_pitched(Ny, p->colgroup) > kNttSmemHalf) p->colgroup /= 2;
    // 8 columns instead of 16 where 8 fit a quarter of shared memory (five CTAs per SM instead
    // of two: the 576-point columns of a 512^2 image with a 64^2 filter ran 1.73 -> 1.60 ms);
    // fewer than two columns per CTA was slower (2048-point columns: 4.37 -> 4.93 ms)
    if (p->colgroup == 16 && smem_pitched(Ny, 8) <= 56 * 1024) p->colgroup = 8;
    p->pixgroup = ntt_pixgroup(p->Rf);
    p->col_threads = Ny * p->colgroup >= 8192 ? 512 : 256;
    p->pix_threads = p->Rf * p->pixgroup >= 8192 ? 512 : 256;
    const size_t per_tile = static_cast<size_t>(p->Rf) * Nx * Ny * 4;
    const size_t budget = size_t(4) << 30;
    long long wt = static_cast<long long>(budget / std::max<size_t>(per_tile, 1));
    wt = std::max<long long>(1, std::min<long long>({wt, p->ntiles, 65535}));
    p->wave_tiles = static_cast<int>(wt);
    p->buf_bytes = per_tile * static_cast<size_t>(wt);
    p->ws_bytes = p->buf_bytes;
    return MORPH_OK;
}

// ------------------------------------------------------- instantiations
typedef void (*NttKernel)(const NttArgs);

static NttKernel rows_fwd_for(int B) {
    switch (B) {
        case 1: return k_ntt_rows_fwd<1>;
        case 2: return k_ntt_rows_fwd<2>;
        case 4: return k_ntt_rows_fwd<4>;
        case 8: return k_ntt_rows_fwd<8>;
        case 16: return k_ntt_rows_fwd<16>;
        case 32: return k_ntt_rows_fwd<32>;
        default: return k_ntt_rows_fwd<64>;
    }
}
static NttKernel rows_inv_for(int B) {
    switch (B) {
        case 1: return k_ntt_rows_inv<1>;
        case 2: return k_ntt_rows_inv<2>;
        case 4: return k_ntt_rows_inv<4>;
        case 8: return k_ntt_rows_inv<8>;
        case 16: return k_ntt_rows_inv<16>;
        case 32: return k_ntt_rows_inv<32>;
        default: return k_ntt_rows_inv<64>;
    }
}
static NttKernel cols_for(int C) {
    switch (C) {
        case 1: return k_ntt_cols<1>;
        case 2: return k_ntt_cols<2>;
        case 4: return k_ntt_cols<4>;
        case 8: return k_ntt_cols<8>;
        default: return k_ntt_cols<16>;
    }
}
static NttKernel range_for(int C) {
    switch (C) {
        case 1: return k_ntt_range<1>;
        case 2: return k_ntt_range<2>;
        case 4: return k_ntt_range<4>;
        case 8: return k_ntt_range<8>;
        case 16: return k_ntt_range<16>;
        case 32: return k_ntt_range<32>;
        case 64: return k_ntt_range<64>;
        default: return k_ntt_range<128>;
    }
}

static int set_ntt_smem(int device) {
    if (kernels_ready(device, kGroupNtt)) return MORPH_OK;
    const int big = static_cast<int>(kNttSmemMax);
    for (int b = 1; b <= 64; b *= 2) {
        MORPH_CUDA_TRY(cudaFuncSetAttribute(rows_fwd_for(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(rows_inv_for(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        if (b <= 16) MORPH_CUDA_TRY(cudaFuncSetAttribute(cols_for(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    }
    for (int b = 1; b <= 128; b *= 2)
        MORPH_CUDA_TRY(cudaFuncSetAttribute(range_for(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_plane_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_ntt_plane_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    mark_kernels_ready(device, kGroupNtt);
    return MORPH_OK;
}

// omega_N^m for m < N, plain
static std::vector<uint32_t> ntt_powers(int N) {
    std::vector<uint32_t> t(N);
    const uint64_t w = hpow(kG, (kP - 1) / static_cast<uint64_t>(N));
    uint64_t x = 1;
    for (int m = 0; m < N; ++m) {
        t[m] = static_cast<uint32_t>(x);
        x = x * w % kP;
    }
    return t;
}

// (omega_N^m, Shoup quotient) pairs
static std::vector<uint2> ntt_twiddles(int N) {
    const std::vector<uint32_t> w = ntt_powers(N);
    std::vector<uint2> t(N);
    for (int m = 0; m < N; ++m) t[m] = make_uint2(w[m], shoup_q(w[m]));
    return t;
}

template <typename T>
static int upload(T** d, const std::vector<T>& h) {
    MORPH_CUDA_TRY(cudaMalloc(d, h.size() * sizeof(T)));
    MORPH_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return MORPH_OK;
}

// Tables and the SE spectrum S_k = 2-D NTT (Ny x Nx) of s_k, scaled by (Rf Ny Nx)^-1.
int build_ntt_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, NttPlan* p) {
    int rc = plan_ntt_tiles(f, se, p);
    if (rc) return rc;
    // the radix roots must have their exact orders (g primitive)
    if (npow(kW4, 2) != kP - 1 || kW3 == 1 || npow(kW3, 3) != 1 || kW5 == 1 || npow(kW5, 5) != 1)
        return MORPH_E_UNSUPPORTED;
    rc = set_ntt_smem(ctx->device);
    if (rc) return rc;
    const int Nx = p->ax.N, Ny = p->ay.N, Rf = p->Rf;
    if ((rc = upload(&p->tw_x, ntt_twiddles(Nx)))) return rc;
    if ((rc = upload(&p->tw_y, ntt_twiddles(Ny)))) return rc;
    if ((rc = upload(&p->tw_r, ntt_twiddles(Rf)))) return rc;
    if ((rc = upload(&p->wr, ntt_powers(Rf)))) return rc;
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
    if ((rc = upload(&d_taps, taps))) return rc;
    {
        const long long n = static_cast<long long>(Rf) * static_cast<long long>(taps.size());
        const unsigned blocks = static_cast<unsigned>(std::min<long long>((n + 255) / 256, 4096));
        k_ntt_se_scatter<<<blocks, 256>>>(p->S, Rf, Ny, Nx, d_taps, static_cast<int>(taps.size()), p->wr);
    }
    k_ntt_plane_rows<<<dim3(Ny, Rf), 256, smem_pitched(Nx, 1)>>>(p->S, p->ax, p->tw_x, Ny);
    k_ntt_plane_cols<<<dim3((Nx + 7) / 8, Rf), 256, smem_pitched(Ny, 8)>>>(p->S, p->ay, p->tw_y, Nx);
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
                  void* buf, cudaStream_t st, const OutAdjust* adj) {
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
    a.rfm = static_cast<uint32_t>(((uint64_t(1) << 32) + p.Rf - 1) / p.Rf);
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
    a.out_add = adj ? adj->add : 0;
    a.out_sub = adj ? adj->sub : nullptr;
    a.err = ctx->d_err;
    const int Nx = p.ax.N, Ny = p.ay.N;
    const NttKernel rf = rows_fwd_for(p.kgroup), ri = rows_inv_for(p.kgroup);
    const NttKernel cl = cols_for(p.colgroup), rg = range_for(p.pixgroup);
    for (long long t0 = 0; t0 < p.ntiles; t0 += p.wave_tiles) {
        a.tile0 = t0;
        a.wave_tiles = static_cast<int>(std::min<long long>(p.wave_tiles, p.ntiles - t0));
        prof_begin(ctx, st, "k_ntt_rows_fwd");
        // split the grey frequencies over CTAs when rows x tiles alone would leave SMs idle
        const int groups = (p.Rf + p.kgroup - 1) / p.kgroup;
        const long long rows = static_cast<long long>(p.Rin_y) * a.wave_tiles;
        const int ksplit = static_cast<int>(std::max<long long>(
            1, std::min<long long>(groups, (8LL * ctx->num_sms + rows - 1) / rows)));
        a.kper = ((groups + ksplit - 1) / ksplit) * p.kgroup;
        rf<<<dim3(p.Rin_y, a.wave_tiles, (p.Rf + a.kper - 1) / a.kper), 256, smem_rows_fwd(Nx, p.Rf, p.kgroup),
             st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_cols");
        cl<<<dim3(a.wave_tiles, (Nx + p.colgroup - 1) / p.colgroup, p.Rf), p.col_threads,
             smem_pitched(Ny, p.colgroup), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_rows_inv");
        ri<<<dim3(p.To_y, (p.Rf + p.kgroup - 1) / p.kgroup, a.wave_tiles), 256, smem_pitched(Nx, p.kgroup), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, "k_ntt_range");
        rg<<<dim3((p.To_x + p.pixgroup - 1) / p.pixgroup, p.To_y, a.wave_tiles), p.pix_threads,
             smem_pitched(p.Rf, p.pixgroup), st>>>(a);
        prof_end(ctx, st);
        ctx->launches += 4;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    return MORPH_OK;
}

int launch_ntt(morph_ctx* ctx, const NttPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
               cudaStream_t st, const OutAdjust* adj) {
    void* buf = nullptr;
    int rc = ctx_workspace(ctx, p.ws_bytes, &buf);
    if (rc) return rc;
    return launch_ntt_in(ctx, p, f, erode, out, cnt, buf, st, adj);
}

}  // namespace morph
