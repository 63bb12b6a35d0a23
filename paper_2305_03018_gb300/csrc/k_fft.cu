// Step 2 of the method with the FFT (Sec. 3, Step 2; Sec. 3.1 Eq. Obs3-Obs7),
// in FP32 or FP64, followed by Step 3 (Eq. 9).
//
// The umbra f_Um(x, v) = [f(x) = v] (Eq. 7) is one-hot along the grey axis,
// so its DFT along that axis (length R = L + max b, the number of degrees) is
// exactly a_k(x) = exp(-2 pi i k f(x) / Rf): the encoder writes it from a
// table, no forward grey-axis transform is run.  Rf is the smallest
// 2^a 3^b 5^c >= R; every degree lies in [0, R), so the length-Rf circular
// convolution along the grey axis never wraps.  Likewise the SE umbra
// (Eq. 8) gives s_k(y) = exp(-2 pi i k b(y) / Rf) on B.  For each grey
// frequency k = 0..Rf/2 (the count polynomial is real, so k and Rf-k are
// conjugate) the spatial full-mode convolution a_k (*) s_k runs as a 2-D FFT
// convolution on overlap-save tiles: an output tile of To_y x To_x pixels
// reads an input tile extended by the SE's reach, placed at buffer offset 0 of
// an Ny x Nx torus with Ny >= To_y + kh - 1, Nx >= To_x + kw - 1 (no wrap-around
// reaches an output).  Step 3 inverts the grey-axis DFT of each pixel with a
// length-Rf FFT (the Hermitian half extended), divides by Rf Nx Ny, rounds to
// the nearest integer and takes the highest d with C >= 1.
//
// Kernels (per wave of tiles):
//   k_fft_rows_fwd : encode a_k for one input row, FFT along x, a batch of k
//                    per pass;
//   k_fft_cols     : FFT along y of C columns, multiply by the SE spectrum,
//                    inverse FFT along y, keep the output rows;
//   k_fft_rows_inv : inverse FFT along x of one output row for a batch of k,
//                    keep the output columns;
//   k_fft_scan     : grey-axis inverse by direct evaluation, downward from a
//                    proven start degree, stopping at the top (short grey axes);
//   k_fft_range    : grey-axis inverse FFT of a group of pixels + rounding +
//                    top-degree scan (one warp per pixel, ballots over d).
// The FFTs are mixed-radix (2, 3, 4, 5) Stockham transforms in shared memory
// over power-of-two batches of interleaved transforms, with twiddle tables
// computed in FP64 (sincospi) and rounded to the working precision.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "morph_internal.h"
#include "ptx.cuh"

namespace morph {

template <typename T>
struct CxT;
template <>
struct CxT<float> {
    using type = float2;
};
template <>
struct CxT<double> {
    using type = double2;
};

template <typename cT>
__device__ __forceinline__ cT cx(decltype(cT().x) a, decltype(cT().x) b) {
    cT r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename cT>
__device__ __forceinline__ cT cadd(cT a, cT b) { return cx<cT>(a.x + b.x, a.y + b.y); }
template <typename cT>
__device__ __forceinline__ cT csub(cT a, cT b) { return cx<cT>(a.x - b.x, a.y - b.y); }
template <typename cT>
__device__ __forceinline__ cT cmul(cT a, cT b) { return cx<cT>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename cT>
__device__ __forceinline__ cT cconj(cT a) { return cx<cT>(a.x, -a.y); }
// multiply by -i
template <typename cT>
__device__ __forceinline__ cT cmul_mi(cT a) { return cx<cT>(a.y, -a.x); }

// Radix-r DFT (forward, exp(-2 pi i / r)) on r values in registers.
template <typename T, typename cT>
__device__ __forceinline__ void dft2(cT* v) {
    const cT a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <typename T, typename cT>
__device__ __forceinline__ void dft4(cT* v) {
    const cT s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const cT s13 = cadd(v[1], v[3]), d13 = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
template <typename T, typename cT>
__device__ __forceinline__ void dft3(cT* v) {
    // exp(-2 pi i / 3) = -1/2 - i sqrt(3)/2
    const T h = static_cast<T>(0.86602540378443864676372317075294);   // sqrt(3) / 2
    const cT t1 = cadd(v[1], v[2]);
    const cT t2 = cx<cT>(v[0].x - static_cast<T>(0.5) * t1.x, v[0].y - static_cast<T>(0.5) * t1.y);
    const cT t3 = cmul_mi(cx<cT>(h * (v[1].x - v[2].x), h * (v[1].y - v[2].y)));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
}
template <typename T, typename cT>
__device__ __forceinline__ void dft5(cT* v) {
    // cos(2 pi / 5) = (sqrt 5 - 1) / 4, cos(4 pi / 5) = -(sqrt 5 + 1) / 4,
    // sin(2 pi / 5), sin(4 pi / 5)
    const T c1 = static_cast<T>(0.30901699437494742410229341718282);
    const T c2 = static_cast<T>(-0.80901699437494742410229341718282);
    const T s1 = static_cast<T>(0.95105651629515357211643933337938);
    const T s2 = static_cast<T>(0.58778525229247312916870595463907);
    const cT b1 = cadd(v[1], v[4]), b2 = cadd(v[2], v[3]);
    const cT d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
    const cT a0 = v[0];
    const cT p1 = cx<cT>(a0.x + c1 * b1.x + c2 * b2.x, a0.y + c1 * b1.y + c2 * b2.y);
    const cT p2 = cx<cT>(a0.x + c2 * b1.x + c1 * b2.x, a0.y + c2 * b1.y + c1 * b2.y);
    const cT q1 = cmul_mi(cx<cT>(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const cT q2 = cmul_mi(cx<cT>(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(a0, cadd(b1, b2));
    v[1] = cadd(p1, q1);
    v[4] = csub(p1, q1);
    v[2] = cadd(p2, q2);
    v[3] = csub(p2, q2);
}

constexpr int kFftMaxStages = 16;   // FftAxis::rad capacity
constexpr int kFftMaxN = 2048;

constexpr int fft_ilog2(int b) { return b <= 1 ? 0 : 1 + fft_ilog2(b / 2); }
// element p of transform c of a batch of B interleaved transforms lives at
// p * pitch(B) + c; the odd pitch keeps column reads (fixed c, consecutive p)
// free of bank conflicts
constexpr int fpitch(int B) { return B == 1 ? 1 : B + 1; }

// One Stockham stage of radix R over B interleaved transforms of length N,
// forward direction; tw[m] = exp(-2 pi i m / N).  j / Ns by a precomputed
// magic multiplier (exact for j Ns < 2^32).
template <typename T, typename cT, int R, int B>
__device__ __forceinline__ void stockham_stage(const cT* __restrict__ x, cT* __restrict__ y, int N, int Ns,
                                               uint32_t nsm, int tstep, const cT* __restrict__ tw) {
    constexpr int PB = fpitch(B);
    constexpr int LB = fft_ilog2(B);
    const int M = N / R;
    const int total = M * B;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int c = t & (B - 1);
        const int j = t >> LB;
        const int g = Ns == 1 ? j : static_cast<int>(__umulhi(static_cast<uint32_t>(j), nsm));
        const int k = j - g * Ns;
        cT v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = x[(j + r * M) * PB + c];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * tstep]);
        }
        if (R == 2) dft2<T, cT>(v);
        if (R == 3) dft3<T, cT>(v);
        if (R == 4) dft4<T, cT>(v);
        if (R == 5) dft5<T, cT>(v);
        const int d = g * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) y[(d + r * Ns) * PB + c] = v[r];
    }
}

// Forward FFT of B interleaved transforms held in a (scratch b); returns the
// buffer holding the result.  Block-wide; ends with a barrier.
template <typename T, typename cT, int B>
__device__ __forceinline__ cT* fft_block(cT* a, cT* b, const FftAxis& ax, const cT* tw) {
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.rad[s];
        if (R == 4) stockham_stage<T, cT, 4, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else if (R == 2) stockham_stage<T, cT, 2, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else if (R == 3) stockham_stage<T, cT, 3, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        else stockham_stage<T, cT, 5, B>(a, b, ax.N, Ns, ax.nsm[s], ax.tstep[s], tw);
        __syncthreads();
        Ns *= R;
        cT* t = a;
        a = b;
        b = t;
    }
    return a;
}

struct FftArgs {
    // image
    const void* src;
    int dtype, n, h, w;
    long long row_stride, batch_stride;
    int L, flip, erode;
    // method
    int R, K;                 // degrees, grey frequencies (Rf/2 + 1)
    int Rf;                   // grey-axis DFT length (smooth, >= R)
    uint32_t rfm;             // ceil(2^32 / Rf): e mod Rf by a multiply for e < 2^21
    FftAxis ar;               // its factorisation
    int To_y, To_x, Rin_y, Win_x;   // output tile, input tile (To + k - 1)
    int ry, rx;               // SE reach below / right: kh - 1 - oy, kw - 1 - ox
    int tiles_x, tiles_y;
    long long tile0;          // first global tile of this wave
    int wave_tiles;           // tiles in this wave
    FftAxis ax, ay;
    const void* tw_x;         // Nx twiddles exp(-2 pi i j / Nx)
    const void* tw_y;
    const void* wr;           // Rf twiddles exp(-2 pi i m / Rf)
    const void* S;            // SE spectrum [K][Ny][Nx]
    void* buf;                // [wave_tiles][K][Ny][Nx]
    int32_t* out;
    int32_t* out_cnt;
    int out_add;              // output adjustment of a composite's pass (OutAdjust)
    const int32_t* out_sub;
    float* count_err;
    int validate;
    unsigned int* err;
    int* tilemax;             // [wave_tiles] largest grey level in each input tile (k_fft_scan start bound)
    int maxb;                 // largest SE offset
};

__device__ __forceinline__ int fft_load_px(const void* src, int dtype, long long idx) {
    if (dtype == MORPH_U8) return static_cast<const uint8_t*>(src)[idx];
    if (dtype == MORPH_U16) return static_cast<const uint16_t*>(src)[idx];
    return static_cast<const int32_t*>(src)[idx];
}

__device__ __forceinline__ void tile_origin(const FftArgs& a, long long gt, int* n, int* y0, int* x0) {
    const long long per = static_cast<long long>(a.tiles_x) * a.tiles_y;
    *n = static_cast<int>(gt / per);
    const int rem = static_cast<int>(gt % per);
    *y0 = (rem / a.tiles_x) * a.To_y;
    *x0 = (rem % a.tiles_x) * a.To_x;
}

// grid (Rin_y, wave_tiles): input row rho of tile tl; the K grey frequencies
// B at a time (B interleaved row transforms per pass)
template <typename T, int B>
__global__ void __launch_bounds__(512) k_fft_rows_fwd(const FftArgs a) {
    using cT = typename CxT<T>::type;
    constexpr int PB = fpitch(B);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N;
    cT* tw = reinterpret_cast<cT*>(sm);
    cT* b0 = tw + Nx;
    cT* b1 = b0 + Nx * PB;
    int* lev = reinterpret_cast<int*>(b1 + Nx * PB);
    const cT* gtw = static_cast<const cT*>(a.tw_x);
    const cT* wr = static_cast<const cT*>(a.wr);
    const int rho = blockIdx.x;                 // input row of the tile
    const int tl = blockIdx.y;                  // tile in wave
    int n, y0, x0;
    tile_origin(a, a.tile0 + tl, &n, &y0, &x0);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = gtw[j];
    const int iy = y0 - a.ry + rho;
    bool bad = false;
    for (int p = threadIdx.x; p < Nx; p += blockDim.x) {
        const int ix = x0 - a.rx + p;
        int v = -1;
        if (p < a.Win_x && iy >= 0 && iy < a.h && ix >= 0 && ix < a.w) {
            const int f = fft_load_px(a.src, a.dtype, n * a.batch_stride + iy * a.row_stride + ix);
            if (f < 0 || f >= a.L) bad = true;
            else v = a.flip ? a.L - 1 - f : f;
        }
        lev[p] = v;
    }
    if (bad) atomicOr(a.err, MORPH_DEVERR_RANGE);
    __syncthreads();
    if (a.tilemax) {
        int mx = -1;
        for (int p = threadIdx.x; p < Nx; p += blockDim.x) mx = max(mx, lev[p]);
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx >= 0) atomicMax(a.tilemax + tl, mx);
    }
    const long long plane = static_cast<long long>(a.ay.N) * Nx;
    cT* dst = static_cast<cT*>(a.buf) + static_cast<long long>(tl) * a.K * plane + static_cast<long long>(rho) * Nx;
    for (int k0 = 0; k0 < a.K; k0 += B) {
        for (int t = threadIdx.x; t < B * Nx; t += blockDim.x) {
            const int c = t & (B - 1), p = t >> fft_ilog2(B);
            const int l = lev[p];
            cT v = cx<cT>(0, 0);
            if (l >= 0 && k0 + c < a.K) {
                const uint32_t e = static_cast<uint32_t>((k0 + c) * l);
                v = wr[e - __umulhi(e, a.rfm) * static_cast<uint32_t>(a.Rf)];       // e mod Rf
            }
            b0[p * PB + c] = v;
        }
        __syncthreads();
        const cT* res = fft_block<T, cT, B>(b0, b1, a.ax, tw);
        const int kb = min(B, a.K - k0);
        for (int c = 0; c < kb; ++c)
            for (int p = threadIdx.x; p < Nx; p += blockDim.x) dst[(k0 + c) * plane + p] = res[p * PB + c];
        __syncthreads();
    }
}

// grid (wave_tiles, ceil(Nx / C), K): column FFT of C columns, multiply by the
// SE spectrum, inverse column FFT (conjugate, forward, conjugate), keep the
// output rows.  The tiles of one (column group, k) run together and share
// that strip of the SE spectrum through L2.
template <typename T, int C>
__global__ void __launch_bounds__(512) k_fft_cols(const FftArgs a) {
    using cT = typename CxT<T>::type;
    constexpr int PC = fpitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = a.ay.N, Nx = a.ax.N;
    cT* tw = reinterpret_cast<cT*>(sm);
    cT* b0 = tw + Ny;
    cT* b1 = b0 + Ny * PC;
    const cT* gtw = static_cast<const cT*>(a.tw_y);
    const int tl = blockIdx.x, u0 = blockIdx.y * C, k = blockIdx.z;
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) tw[j] = gtw[j];
    cT* plane = static_cast<cT*>(a.buf) + (static_cast<long long>(tl) * a.K + k) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), rho = t >> fft_ilog2(C);
        b0[rho * PC + c] = (rho < a.Rin_y && u0 + c < Nx) ? plane[static_cast<long long>(rho) * Nx + u0 + c]
                                                          : cx<cT>(0, 0);
    }
    __syncthreads();
    cT* res = fft_block<T, cT, C>(b0, b1, a.ay, tw);
    cT* other = (res == b0) ? b1 : b0;
    const cT* S = static_cast<const cT*>(a.S) + static_cast<long long>(k) * Ny * Nx;
    // multiply by the SE spectrum, conjugate for the inverse transform
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), v = t >> fft_ilog2(C);
        if (u0 + c < Nx) res[v * PC + c] = cconj(cmul(res[v * PC + c], S[static_cast<long long>(v) * Nx + u0 + c]));
    }
    __syncthreads();
    const cT* out = fft_block<T, cT, C>(res, other, a.ay, tw);
    // torus position of output row q is (q + ry) mod Ny (ry < 0 or >= Ny when the origin lies outside the box)
    const int base = ((a.ry % Ny) + Ny) % Ny;
    for (int t = threadIdx.x; t < a.To_y * C; t += blockDim.x) {
        const int c = t & (C - 1), q = t >> fft_ilog2(C);
        int pos = base + q;
        if (pos >= Ny) pos -= Ny;
        if (u0 + c < Nx) plane[static_cast<long long>(q) * Nx + u0 + c] = cconj(out[pos * PC + c]);
    }
}

// grid (To_y, ceil(K / B), wave_tiles): inverse row FFT of output row q for B
// grey frequencies, keep the output columns
template <typename T, int B>
__global__ void __launch_bounds__(512) k_fft_rows_inv(const FftArgs a) {
    using cT = typename CxT<T>::type;
    constexpr int PB = fpitch(B);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = a.ax.N;
    cT* tw = reinterpret_cast<cT*>(sm);
    cT* b0 = tw + Nx;
    cT* b1 = b0 + Nx * PB;
    const cT* gtw = static_cast<const cT*>(a.tw_x);
    const int q = blockIdx.x, k0 = blockIdx.y * B, tl = blockIdx.z;
    const int kb = min(B, a.K - k0);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = gtw[j];
    const long long plane = static_cast<long long>(a.ay.N) * Nx;
    cT* rows = static_cast<cT*>(a.buf) + (static_cast<long long>(tl) * a.K + k0) * plane + static_cast<long long>(q) * Nx;
    for (int c = 0; c < B; ++c)
        for (int p = threadIdx.x; p < Nx; p += blockDim.x)
            b0[p * PB + c] = c < kb ? cconj(rows[c * plane + p]) : cx<cT>(0, 0);
    __syncthreads();
    const cT* res = fft_block<T, cT, B>(b0, b1, a.ax, tw);
    const int base = ((a.rx % Nx) + Nx) % Nx;
    for (int c = 0; c < kb; ++c)
        for (int p = threadIdx.x; p < a.To_x; p += blockDim.x) {
            int pos = base + p;
            if (pos >= Nx) pos -= Nx;
            rows[c * plane + p] = cconj(res[pos * PB + c]);
        }
}


// Step 3 by direct evaluation, for grey axes short enough that a few
// evaluations per pixel beat a transform: C(x, d) = (1 / (Rf Nx Ny))
// sum_k w_k Re(c_k(x) exp(2 pi i k d / Rf)), evaluated for d downward from
// min(R - 1, largest level in the input tile + max b) -- no tap can exceed
// that, so C is exactly 0 above it -- and stopping at the first d with
// rint(C) >= 1.
template <typename T>
__global__ void __launch_bounds__(256) k_fft_scan(const FftArgs a) {
    using cT = typename CxT<T>::type;
    const int Nx = a.ax.N, Ny = a.ay.N, Rf = a.Rf;
    const long long per_tile = static_cast<long long>(a.To_y) * a.To_x;
    const long long total = per_tile * a.wave_tiles;
    const cT* tw = static_cast<const cT*>(a.wr);     // exp(-2 pi i m / Rf): conjugate for the inverse
    const T scale = static_cast<T>(1.0) / (static_cast<T>(Rf) * static_cast<T>(Nx) * static_cast<T>(Ny));
    const bool nyq = (Rf % 2) == 0;
    float emax = 0.f;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int tl = static_cast<int>(idx / per_tile);
        const int rem = static_cast<int>(idx % per_tile);
        const int q = rem / a.To_x, xo = rem % a.To_x;
        int n, y0, x0;
        tile_origin(a, a.tile0 + tl, &n, &y0, &x0);
        const int i = y0 + q, j = x0 + xo;
        if (i >= a.h || j >= a.w) continue;
        const cT* base = static_cast<const cT*>(a.buf) + (static_cast<long long>(tl) * a.K * Ny + q) * Nx + xo;
        const long long kstride = static_cast<long long>(Ny) * Nx;
        int dstart = a.R - 1;
        if (a.tilemax) dstart = min(dstart, a.tilemax[tl] + a.maxb);
        int D = -1, cnt = 0;
        for (int d = a.validate ? a.R - 1 : dstart; d >= 0; --d) {
            T s = base[0].x;
            int m = 0;
            for (int k = 1; k < a.K; ++k) {
                m += d;
                if (m >= Rf) m -= Rf;
                const cT c = base[k * kstride];
                const cT w = tw[m];
                const T re = c.x * w.x + c.y * w.y;       // Re(c * conj(w))
                s += (nyq && k == a.K - 1) ? re : static_cast<T>(2) * re;
            }
            const T C = s * scale;
            const T rc = rint(C);
            emax = fmaxf(emax, static_cast<float>(fabs(C - rc)));
            if (rc >= static_cast<T>(1) && D < 0) {
                D = d;
                cnt = static_cast<int>(rc);
                if (!a.validate) break;
            }
        }
        const int dval = D < 0 ? 0 : D;
        const long long o = (static_cast<long long>(n) * a.h + i) * a.w + j;
        a.out[o] = (a.erode ? (a.L - 1 - dval) : dval) + a.out_add - (a.out_sub ? a.out_sub[o] : 0);
        if (a.out_cnt) a.out_cnt[o] = D < 0 ? 0 : cnt;
    }
    if (a.count_err) {
        for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(a.count_err), __float_as_int(emax));
    }
}

// grid (ceil(To_x / C), To_y, wave_tiles): grey-axis inverse FFT + Step 3 for
// C consecutive output pixels of one tile row: C(x, d) = (1 / (Rf Nx Ny))
// sum_k c_k(x) exp(2 pi i k d / Rf) with c_{Rf-k} = conj(c_k); then each warp
// scans its pixels' degrees from R - 1 downward in chunks of 32 (ballot),
// keeping the top d with rint(C) >= 1 and its count.
template <typename T, int C>
__global__ void __launch_bounds__(512) k_fft_range(const FftArgs a) {
    using cT = typename CxT<T>::type;
    constexpr int PC = fpitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Rf = a.ar.N, Nx = a.ax.N, Ny = a.ay.N;
    cT* tw = reinterpret_cast<cT*>(sm);
    cT* b0 = tw + Rf;
    cT* b1 = b0 + Rf * PC;
    const cT* gtw = static_cast<const cT*>(a.wr);
    const int x0 = blockIdx.x * C, q = blockIdx.y, tl = blockIdx.z;
    int n, y0, tx0;
    tile_origin(a, a.tile0 + tl, &n, &y0, &tx0);
    for (int j = threadIdx.x; j < Rf; j += blockDim.x) tw[j] = gtw[j];
    const cT* base = static_cast<const cT*>(a.buf) + (static_cast<long long>(tl) * a.K * Ny + q) * Nx;
    const long long kstride = static_cast<long long>(Ny) * Nx;
    // Hermitian extension, conjugated for the inverse transform
    for (int t = threadIdx.x; t < Rf * C; t += blockDim.x) {
        const int c = t & (C - 1), k = t >> fft_ilog2(C);
        const int xo = x0 + c;
        cT v = cx<cT>(0, 0);
        if (xo < a.To_x) {
            if (k < a.K) v = cconj(base[k * kstride + xo]);
            else v = base[(Rf - k) * kstride + xo];
        }
        b0[k * PC + c] = v;
    }
    __syncthreads();
    const cT* res = fft_block<T, cT, C>(b0, b1, a.ar, tw);
    const T scale = static_cast<T>(1.0) / (static_cast<T>(Rf) * static_cast<T>(Nx) * static_cast<T>(Ny));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    float emax = 0.f;
    for (int c = warp; c < C; c += nwarps) {
        const int xo = x0 + c;
        const int i = y0 + q, j = tx0 + xo;
        if (xo >= a.To_x || i >= a.h || j >= a.w) continue;          // warp-uniform
        int D = -1, cnt = 0;
        for (int d0 = ((a.R - 1) / 32) * 32; d0 >= 0; d0 -= 32) {
            const int d = d0 + lane;
            T Cv = 0;
            bool hit = false;
            if (d < a.R) {
                Cv = res[d * PC + c].x * scale;          // real part of the conjugated result
                const T rc = rint(Cv);
                if (a.validate || D < 0) emax = fmaxf(emax, static_cast<float>(fabs(Cv - rc)));
                hit = rc >= static_cast<T>(1);
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (D < 0 && m) {
                const int top = 31 - __clz(m);
                D = d0 + top;
                cnt = static_cast<int>(rint(__shfl_sync(0xffffffffu, static_cast<double>(Cv), top)));
                if (!a.validate) break;
            }
        }
        if (lane == 0) {
            const int dval = D < 0 ? 0 : D;
            const long long o = (static_cast<long long>(n) * a.h + i) * a.w + j;
            a.out[o] = (a.erode ? (a.L - 1 - dval) : dval) + a.out_add - (a.out_sub ? a.out_sub[o] : 0);
            if (a.out_cnt) a.out_cnt[o] = D < 0 ? 0 : cnt;
        }
    }
    if (a.count_err) {
        for (int o = 16; o > 0; o >>= 1) emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
        if (lane == 0) atomicMax(reinterpret_cast<int*>(a.count_err), __float_as_int(emax));
    }
}

// ----------------------------------------------------- tables and SE spectrum
// tw[j] = exp(sign * 2 pi i j / N), computed in FP64 and rounded to T.
template <typename T>
__global__ void k_twiddles(typename CxT<T>::type* tw, int N, int sign) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * static_cast<double>(j) / static_cast<double>(N), &s, &c);
        tw[j].x = static_cast<T>(c);
        tw[j].y = static_cast<T>(sign * s);
    }
}

struct SeTap {
    int dy, dx, b;
};

// plane k of the SE umbra's grey-axis DFT, s_k(y) = exp(-2 pi i k b(y) / R),
// placed at (y mod Ny, y mod Nx) of the torus (planes zeroed beforehand)
__global__ void k_se_scatter(double2* planes, int K, int Ny, int Nx, const SeTap* taps, int ntaps, int R) {
    const long long per = static_cast<long long>(Ny) * Nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < static_cast<long long>(K) * ntaps;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = static_cast<int>(idx / ntaps), t = static_cast<int>(idx % ntaps);
        const SeTap tp = taps[t];
        const int py = ((tp.dy % Ny) + Ny) % Ny, px = ((tp.dx % Nx) + Nx) % Nx;
        const long long m = (static_cast<long long>(k) * tp.b) % R;
        double s, c;
        sincospi(2.0 * static_cast<double>(m) / static_cast<double>(R), &s, &c);
        planes[k * per + static_cast<long long>(py) * Nx + px] = make_double2(c, -s);
    }
}

// In-place forward FFT of every row (then every column) of K planes, FP64.
__global__ void __launch_bounds__(256) k_plane_rows(double2* planes, FftAxis ax, const double2* gtw, int Ny) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int Nx = ax.N;
    double2* tw = reinterpret_cast<double2*>(sm);
    double2* b0 = tw + Nx;
    double2* b1 = b0 + Nx;
    const int row = blockIdx.x, k = blockIdx.y;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) tw[j] = gtw[j];
    double2* p = planes + (static_cast<long long>(k) * Ny + row) * Nx;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) b0[j] = p[j];
    __syncthreads();
    const double2* res = fft_block<double, double2, 1>(b0, b1, ax, tw);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) p[j] = res[j];
}

constexpr int kPlaneCols = 4;   // columns per CTA of k_plane_cols, where they fit shared memory
constexpr int kPlaneSmem = 200 * 1024;   // dynamic shared memory opted into by the plane kernels

template <int C>
__global__ void __launch_bounds__(256) k_plane_cols(double2* planes, FftAxis ay, const double2* gtw, int Nx) {
    constexpr int PC = fpitch(C);
    extern __shared__ __align__(16) unsigned char sm[];
    const int Ny = ay.N;
    double2* tw = reinterpret_cast<double2*>(sm);
    double2* b0 = tw + Ny;
    double2* b1 = b0 + Ny * PC;
    const int u0 = blockIdx.x * C, k = blockIdx.y;
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) tw[j] = gtw[j];
    double2* p = planes + static_cast<long long>(k) * Ny * Nx;
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), r = t >> fft_ilog2(C);
        b0[r * PC + c] = (u0 + c < Nx) ? p[static_cast<long long>(r) * Nx + u0 + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const double2* res = fft_block<double, double2, C>(b0, b1, ay, tw);
    for (int t = threadIdx.x; t < Ny * C; t += blockDim.x) {
        const int c = t & (C - 1), r = t >> fft_ilog2(C);
        if (u0 + c < Nx) p[static_cast<long long>(r) * Nx + u0 + c] = res[r * PC + c];
    }
}

__global__ void k_to_float2(const double2* __restrict__ s, float2* __restrict__ d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        d[i] = make_float2(static_cast<float>(s[i].x), static_cast<float>(s[i].y));
}

// ------------------------------------------------------------------ planning
static bool factor_axis(int N, FftAxis* ax) {
    ax->N = N;
    ax->nst = 0;
    int m = N;
    int f4 = 0;
    while (m % 4 == 0) { m /= 4; ++f4; }
    int f2 = 0;
    while (m % 2 == 0) { m /= 2; ++f2; }
    int f3 = 0;
    while (m % 3 == 0) { m /= 3; ++f3; }
    int f5 = 0;
    while (m % 5 == 0) { m /= 5; ++f5; }
    if (m != 1) return false;
    auto push = [&](int r, int c) {
        for (int i = 0; i < c; ++i) {
            if (ax->nst >= kFftMaxStages) return false;
            ax->rad[ax->nst++] = r;
        }
        return true;
    };
    if (!(push(4, f4) && push(2, f2) && push(3, f3) && push(5, f5))) return false;
    int Ns = 1;
    for (int st = 0; st < ax->nst; ++st) {
        ax->tstep[st] = N / (Ns * ax->rad[st]);
        // ceil(2^32 / Ns): floor(j * nsm / 2^32) = j / Ns exactly while j * Ns < 2^32
        ax->nsm[st] = Ns == 1 ? 0u : static_cast<uint32_t>(((uint64_t(1) << 32) + Ns - 1) / Ns);
        Ns *= ax->rad[st];
    }
    return true;
}

static int smooth_at_least(int n) {
    for (int m = std::max(n, 1);; ++m) {
        int t = m;
        for (int p : {2, 3, 5})
            while (t % p == 0) t /= p;
        if (t == 1) return m;
    }
}

// Per-stage relative error (2-norm) of a radix-r Stockham stage with
// precomputed twiddles: the r-point sums, the constant multiplications of
// radix 3 and 5, the twiddle's own rounding and the complex multiply.
static double stage_eta(int r, double u) { return (r + 4) * u; }

double fft_error_bound(const FftAxis& ax, const FftAxis& ay, const FftAxis& ar, double sqrtP, int taps, double u) {
    double e1 = 0.0;
    for (int s = 0; s < ax.nst; ++s) e1 += stage_eta(ax.rad[s], u);
    for (int s = 0; s < ay.nst; ++s) e1 += stage_eta(ay.rad[s], u);
    // forward + inverse 2-D transforms, product and SE-spectrum rounding, input table rounding;
    // the grey-axis inverse averages the frequencies' errors (weights summing to 1)
    const double conv = 1.01 * (2.0 * e1 + 4.0 * u) * sqrtP * static_cast<double>(taps);
    // grey-axis inverse FFT of a vector of counts whose 2-norm is at most |B|
    double er = 0.0;
    for (int s = 0; s < ar.nst; ++s) er += stage_eta(ar.rad[s], u);
    const double range = 1.01 * (er + 4.0 * u) * static_cast<double>(taps);
    return conv + range;
}

}  // namespace morph

namespace morph {

FftPlan::~FftPlan() {
    for (void* q : {tw_x, tw_y, wr, S})
        if (q) cudaFree(q);
}

// shared memory (bytes): twiddles + two pitched buffers of B transforms (+ row levels)
static size_t smem_rows(int N, int B, int prec) {
    return static_cast<size_t>(N) * 2 * prec * (1 + 2 * fpitch(B)) + 4 * static_cast<size_t>(N);
}
static size_t smem_cols(int N, int C, int prec) { return static_cast<size_t>(N) * 2 * prec * (1 + 2 * fpitch(C)); }
constexpr size_t kFftSmemHalf = 110 * 1024;     // two CTAs per SM
constexpr size_t kFftSmemQuarter = 56 * 1024;   // four CTAs per SM

static int fft_pow2_floor(int x) {
    int p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

static double axis_flop(const FftAxis& a) {
    double lg = 0;
    for (int s = 0; s < a.nst; ++s) lg += std::log2(static_cast<double>(a.rad[s]));
    return 5.0 * a.N * lg;
}

// Choose the overlap-save tiling and the FFT sizes for one precision.  The
// a-priori bound (fft_error_bound) must stay below 0.5 unless `unproven` is
// set; among admissible tilings the one with the fewest FFT FLOPs wins.
int plan_fft_tiles(const morph_image* f, const morph_se* se, int prec, bool unproven, FftPlan* p) {
    const int kh = se->kh, kw = se->kw;
    int taps = 0, maxb = 0;
    for (int t = 0; t < kh * kw; ++t)
        if (se->mask[t]) {
            ++taps;
            maxb = std::max(maxb, static_cast<int>(se->offset[t]));
        }
    p->prec = prec;
    p->taps = taps;
    p->R = f->L + maxb;
    p->Rf = smooth_at_least(p->R);
    if (p->Rf > kFftMaxN || !factor_axis(p->Rf, &p->ar)) return MORPH_E_UNSUPPORTED;
    p->K = p->Rf / 2 + 1;
    p->ry = kh - 1 - se->oy;
    p->rx = kw - 1 - se->ox;
    p->kh = kh;
    p->kw = kw;
    const double u = prec == 4 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    double best = -1.0, best_bound = 0.0;
    const int max_ty = std::min(f->h, 256), max_tx = std::min(f->w, 256);
    for (int nty = 1; nty <= max_ty; ++nty) {
        const int To_y = (f->h + nty - 1) / nty;
        if (To_y + kh - 1 > kFftMaxN) continue;
        const int Ny = smooth_at_least(To_y + kh - 1);
        if (Ny > kFftMaxN) continue;
        FftAxis ay;
        if (!factor_axis(Ny, &ay)) continue;
        for (int ntx = 1; ntx <= max_tx; ++ntx) {
            const int To_x = (f->w + ntx - 1) / ntx;
            if (To_x + kw - 1 > kFftMaxN) continue;
            const int Nx = smooth_at_least(To_x + kw - 1);
            if (Nx > kFftMaxN) continue;
            FftAxis ax;
            if (!factor_axis(Nx, &ax)) continue;
            const double sqrtP = std::sqrt(static_cast<double>(std::min(To_y + kh - 1, f->h)) *
                                           static_cast<double>(std::min(To_x + kw - 1, f->w)));
            const double bound = fft_error_bound(ax, ay, p->ar, sqrtP, taps, u);
            if (!unproven && !(bound < 0.5)) continue;
            const double tiles = static_cast<double>(f->n) * nty * ntx;
            const double fl = tiles * p->K *
                              ((To_y + kh - 1 + To_y) * axis_flop(ax) + 2.0 * Nx * axis_flop(ay) + 6.0 * Nx * Ny);
            if (best < 0 || fl < best) {
                best = fl;
                best_bound = bound;
                p->To_y = To_y;
                p->To_x = To_x;
                p->ax = ax;
                p->ay = ay;
                p->tiles_y = nty;
                p->tiles_x = ntx;
            }
        }
    }
    if (best < 0) return MORPH_E_PRECISION;
    p->bound = best_bound;
    p->Rin_y = p->To_y + kh - 1;
    p->Win_x = p->To_x + kw - 1;
    p->ntiles = static_cast<long long>(f->n) * p->tiles_y * p->tiles_x;
    p->flop = best + static_cast<double>(f->n) * f->h * f->w * axis_flop(p->ar);
    // batches (powers of two): ~4096 elements per row-kernel pass, no more
    // frequencies than there are, row and column groups sized for four CTAs per
    // SM (the complex elements are 8 or 16 bytes), pixel groups for two
    p->kgroup = std::min(32, fft_pow2_floor(std::max(1, 4096 / p->ax.N)));
    while (p->kgroup > 1 && p->kgroup / 2 >= p->K) p->kgroup /= 2;
    while (p->kgroup > 1 && smem_rows(p->ax.N, p->kgroup, prec) > kFftSmemQuarter) p->kgroup /= 2;
    p->colgroup = 16;
    while (p->colgroup > 1 && smem_cols(p->ay.N, p->colgroup, prec) > kFftSmemQuarter) p->colgroup /= 2;
    p->pixgroup = 32;
    while (p->pixgroup > 1 && smem_cols(p->Rf, p->pixgroup, prec) > kFftSmemHalf) p->pixgroup /= 2;
    p->col_threads = p->ay.N * p->colgroup >= 2048 ? 512 : 256;
    p->pix_threads = p->Rf * p->pixgroup >= 4096 ? 512 : 256;
    p->row_threads = p->ax.N * p->kgroup >= 2048 ? 512 : 256;
    const size_t per_tile = static_cast<size_t>(p->K) * p->ax.N * p->ay.N * 2 * prec;
    const size_t budget = size_t(4) << 30;
    long long wt = static_cast<long long>(budget / std::max<size_t>(per_tile, 1));
    if (wt < 1) wt = 1;
    if (wt > p->ntiles) wt = p->ntiles;
    if (wt > 65535) wt = 65535;
    p->wave_tiles = static_cast<int>(wt);
    p->buf_bytes = per_tile * static_cast<size_t>(wt);
    // grey-axis inverse: a transform once the axis is long (a downward scan may
    // then evaluate many degrees per pixel); direct evaluation otherwise
    p->range_fft = p->Rf >= 128;
    p->ws_bytes = p->buf_bytes + (p->range_fft ? 0 : sizeof(int) * static_cast<size_t>(wt));
    return MORPH_OK;
}

typedef void (*FftKernel)(const FftArgs);

template <typename T>
static FftKernel rows_fwd_for(int B) {
    switch (B) {
        case 1: return k_fft_rows_fwd<T, 1>;
        case 2: return k_fft_rows_fwd<T, 2>;
        case 4: return k_fft_rows_fwd<T, 4>;
        case 8: return k_fft_rows_fwd<T, 8>;
        case 16: return k_fft_rows_fwd<T, 16>;
        default: return k_fft_rows_fwd<T, 32>;
    }
}
template <typename T>
static FftKernel rows_inv_for(int B) {
    switch (B) {
        case 1: return k_fft_rows_inv<T, 1>;
        case 2: return k_fft_rows_inv<T, 2>;
        case 4: return k_fft_rows_inv<T, 4>;
        case 8: return k_fft_rows_inv<T, 8>;
        case 16: return k_fft_rows_inv<T, 16>;
        default: return k_fft_rows_inv<T, 32>;
    }
}
template <typename T>
static FftKernel cols_for(int C) {
    switch (C) {
        case 1: return k_fft_cols<T, 1>;
        case 2: return k_fft_cols<T, 2>;
        case 4: return k_fft_cols<T, 4>;
        case 8: return k_fft_cols<T, 8>;
        default: return k_fft_cols<T, 16>;
    }
}
template <typename T>
static FftKernel range_for(int C) {
    switch (C) {
        case 1: return k_fft_range<T, 1>;
        case 2: return k_fft_range<T, 2>;
        case 4: return k_fft_range<T, 4>;
        case 8: return k_fft_range<T, 8>;
        case 16: return k_fft_range<T, 16>;
        default: return k_fft_range<T, 32>;
    }
}

template <typename T>
static int set_fft_smem(int device) {
    const KernelGroup grp = sizeof(T) == 4 ? kGroupFft32 : kGroupFft64;
    if (kernels_ready(device, grp)) return MORPH_OK;
    const int big = 200 * 1024;
    for (int b = 1; b <= 32; b *= 2) {
        MORPH_CUDA_TRY(cudaFuncSetAttribute(rows_fwd_for<T>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(rows_inv_for<T>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        MORPH_CUDA_TRY(cudaFuncSetAttribute(range_for<T>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        if (b <= 16) MORPH_CUDA_TRY(cudaFuncSetAttribute(cols_for<T>(b), cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    }
    mark_kernels_ready(device, grp);
    return MORPH_OK;
}

static int set_plane_smem(int device) {
    if (kernels_ready(device, kGroupFftPlane)) return MORPH_OK;
    const int big = kPlaneSmem;
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_plane_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_plane_cols<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    MORPH_CUDA_TRY(cudaFuncSetAttribute(k_plane_cols<kPlaneCols>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    mark_kernels_ready(device, kGroupFftPlane);
    return MORPH_OK;
}

// Device tables and the SE spectrum: S_k = 2-D DFT (Ny x Nx) of s_k, in FP64,
// rounded to the working precision.
int build_fft_plan(morph_ctx* ctx, const morph_image* f, const morph_se* se, int prec, bool unproven, FftPlan* p) {
    int rc = plan_fft_tiles(f, se, prec, unproven, p);
    if (rc) return rc;
    const int Nx = p->ax.N, Ny = p->ay.N, K = p->K, Rf = p->Rf;
    rc = set_plane_smem(ctx->device);
    if (rc) return rc;
    if (prec == 4) rc = set_fft_smem<float>(ctx->device);
    else rc = set_fft_smem<double>(ctx->device);
    if (rc) return rc;
    const size_t cbytes = 2 * static_cast<size_t>(prec);
    MORPH_CUDA_TRY(cudaMalloc(&p->tw_x, Nx * cbytes));
    MORPH_CUDA_TRY(cudaMalloc(&p->tw_y, Ny * cbytes));
    MORPH_CUDA_TRY(cudaMalloc(&p->wr, Rf * cbytes));
    if (prec == 4) {
        k_twiddles<float><<<(Nx + 255) / 256, 256>>>(static_cast<float2*>(p->tw_x), Nx, -1);
        k_twiddles<float><<<(Ny + 255) / 256, 256>>>(static_cast<float2*>(p->tw_y), Ny, -1);
        k_twiddles<float><<<(Rf + 255) / 256, 256>>>(static_cast<float2*>(p->wr), Rf, -1);
    } else {
        k_twiddles<double><<<(Nx + 255) / 256, 256>>>(static_cast<double2*>(p->tw_x), Nx, -1);
        k_twiddles<double><<<(Ny + 255) / 256, 256>>>(static_cast<double2*>(p->tw_y), Ny, -1);
        k_twiddles<double><<<(Rf + 255) / 256, 256>>>(static_cast<double2*>(p->wr), Rf, -1);
    }
    ctx->launches += 3;
    MORPH_CUDA_TRY(cudaGetLastError());
    // SE spectrum in FP64
    std::vector<SeTap> taps;
    for (int r = 0; r < se->kh; ++r)
        for (int c = 0; c < se->kw; ++c) {
            const int t = r * se->kw + c;
            if (se->mask[t]) taps.push_back(SeTap{r - se->oy, c - se->ox, se->offset[t]});
        }
    const size_t plane64 = static_cast<size_t>(K) * Ny * Nx * sizeof(double2);
    double2* s64 = nullptr;
    double2* tw64x = nullptr;
    double2* tw64y = nullptr;
    SeTap* d_taps = nullptr;
    MORPH_CUDA_TRY(cudaMalloc(&s64, plane64));
    MORPH_CUDA_TRY(cudaMalloc(&tw64x, Nx * sizeof(double2)));
    MORPH_CUDA_TRY(cudaMalloc(&tw64y, Ny * sizeof(double2)));
    MORPH_CUDA_TRY(cudaMalloc(&d_taps, taps.size() * sizeof(SeTap)));
    MORPH_CUDA_TRY(cudaMemcpy(d_taps, taps.data(), taps.size() * sizeof(SeTap), cudaMemcpyHostToDevice));
    MORPH_CUDA_TRY(cudaMemset(s64, 0, plane64));
    k_twiddles<double><<<(Nx + 255) / 256, 256>>>(tw64x, Nx, -1);
    k_twiddles<double><<<(Ny + 255) / 256, 256>>>(tw64y, Ny, -1);
    {
        const long long n = static_cast<long long>(K) * static_cast<long long>(taps.size());
        const unsigned blocks = static_cast<unsigned>(std::min<long long>((n + 255) / 256, 4096));
        k_se_scatter<<<blocks, 256>>>(s64, K, Ny, Nx, d_taps, static_cast<int>(taps.size()), Rf);
    }
    k_plane_rows<<<dim3(Ny, K), 256, smem_rows(Nx, 1, 8)>>>(s64, p->ax, tw64x, Ny);
    // four columns per CTA up to Ny = 1024 (180 KB); one at Ny = 2048 (four would need 360 KB)
    if (smem_cols(Ny, kPlaneCols, 8) <= static_cast<size_t>(kPlaneSmem))
        k_plane_cols<kPlaneCols><<<dim3((Nx + kPlaneCols - 1) / kPlaneCols, K), 256, smem_cols(Ny, kPlaneCols, 8)>>>(
            s64, p->ay, tw64y, Nx);
    else
        k_plane_cols<1><<<dim3(Nx, K), 256, smem_cols(Ny, 1, 8)>>>(s64, p->ay, tw64y, Nx);
    ctx->launches += 5;
    MORPH_CUDA_TRY(cudaGetLastError());
    if (prec == 4) {
        MORPH_CUDA_TRY(cudaMalloc(&p->S, static_cast<size_t>(K) * Ny * Nx * sizeof(float2)));
        const long long n = static_cast<long long>(K) * Ny * Nx;
        k_to_float2<<<static_cast<unsigned>(std::min<long long>((n + 255) / 256, 8192)), 256>>>(
            s64, static_cast<float2*>(p->S), n);
        ctx->launches += 1;
        MORPH_CUDA_TRY(cudaGetLastError());
        MORPH_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(s64);
    } else {
        MORPH_CUDA_TRY(cudaDeviceSynchronize());
        p->S = s64;
    }
    cudaFree(tw64x);
    cudaFree(tw64y);
    cudaFree(d_taps);
    return MORPH_OK;
}

template <typename T>
static int launch_fft_t(morph_ctx* ctx, const FftPlan& p, const morph_image* f, int erode, int32_t* out,
                        int32_t* cnt, float* count_err, int validate, void* buf, cudaStream_t st,
                        const OutAdjust* adj) {
    FftArgs a;
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
    a.K = p.K;
    a.Rf = p.Rf;
    a.rfm = static_cast<uint32_t>(((uint64_t(1) << 32) + p.Rf - 1) / p.Rf);
    a.ar = p.ar;
    a.maxb = p.R - f->L;
    a.tilemax = p.range_fft ? nullptr : reinterpret_cast<int*>(static_cast<unsigned char*>(buf) + p.buf_bytes);
    a.To_y = p.To_y;
    a.To_x = p.To_x;
    a.Rin_y = p.Rin_y;
    a.Win_x = p.Win_x;
    a.ry = p.ry;
    a.rx = p.rx;
    a.tiles_x = p.tiles_x;
    a.tiles_y = p.tiles_y;
    a.ax = p.ax;
    a.ay = p.ay;
    a.tw_x = p.tw_x;
    a.tw_y = p.tw_y;
    a.wr = p.wr;
    a.S = p.S;
    a.buf = buf;
    a.out = out;
    a.out_cnt = cnt;
    a.out_add = adj ? adj->add : 0;
    a.out_sub = adj ? adj->sub : nullptr;
    a.count_err = count_err;
    a.validate = validate;
    a.err = ctx->d_err;
    const int prec = static_cast<int>(sizeof(T));
    for (long long t0 = 0; t0 < p.ntiles; t0 += p.wave_tiles) {
        a.tile0 = t0;
        a.wave_tiles = static_cast<int>(std::min<long long>(p.wave_tiles, p.ntiles - t0));
        if (a.tilemax) MORPH_CUDA_TRY(cudaMemsetAsync(a.tilemax, 0xff, sizeof(int) * a.wave_tiles, st));
        prof_begin(ctx, st, prec == 4 ? "k_fft_rows_fwd<f32>" : "k_fft_rows_fwd<f64>");
        rows_fwd_for<T>(p.kgroup)<<<dim3(p.Rin_y, a.wave_tiles), p.row_threads, smem_rows(p.ax.N, p.kgroup, prec),
                                    st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, prec == 4 ? "k_fft_cols<f32>" : "k_fft_cols<f64>");
        cols_for<T>(p.colgroup)<<<dim3(a.wave_tiles, (p.ax.N + p.colgroup - 1) / p.colgroup, p.K), p.col_threads,
                                  smem_cols(p.ay.N, p.colgroup, prec), st>>>(a);
        prof_end(ctx, st);
        prof_begin(ctx, st, prec == 4 ? "k_fft_rows_inv<f32>" : "k_fft_rows_inv<f64>");
        rows_inv_for<T>(p.kgroup)<<<dim3(p.To_y, (p.K + p.kgroup - 1) / p.kgroup, a.wave_tiles), p.row_threads,
                                    smem_rows(p.ax.N, p.kgroup, prec), st>>>(a);
        prof_end(ctx, st);
        if (p.range_fft) {
            prof_begin(ctx, st, prec == 4 ? "k_fft_range<f32>" : "k_fft_range<f64>");
            range_for<T>(p.pixgroup)<<<dim3((p.To_x + p.pixgroup - 1) / p.pixgroup, p.To_y, a.wave_tiles),
                                       p.pix_threads, smem_cols(p.Rf, p.pixgroup, prec), st>>>(a);
            prof_end(ctx, st);
        } else {
            const long long px = static_cast<long long>(p.To_y) * p.To_x * a.wave_tiles;
            const unsigned blocks = static_cast<unsigned>(std::min<long long>((px + 255) / 256, ctx->num_sms * 16LL));
            prof_begin(ctx, st, prec == 4 ? "k_fft_scan<f32>" : "k_fft_scan<f64>");
            k_fft_scan<T><<<blocks, 256, 0, st>>>(a);
            prof_end(ctx, st);
        }
        ctx->launches += 4;
        MORPH_CUDA_TRY(cudaGetLastError());
    }
    return MORPH_OK;
}

int launch_fft_in(morph_ctx* ctx, const FftPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
                  float* count_err, int validate, void* buf, cudaStream_t st, const OutAdjust* adj) {
    if (p.prec == 4) return launch_fft_t<float>(ctx, p, f, erode, out, cnt, count_err, validate, buf, st, adj);
    return launch_fft_t<double>(ctx, p, f, erode, out, cnt, count_err, validate, buf, st, adj);
}

int launch_fft(morph_ctx* ctx, const FftPlan& p, const morph_image* f, int erode, int32_t* out, int32_t* cnt,
               float* count_err, int validate, cudaStream_t st, const OutAdjust* adj) {
    void* buf = nullptr;
    int rc = ctx_workspace(ctx, p.ws_bytes, &buf);
    if (rc) return rc;
    if (count_err) MORPH_CUDA_TRY(cudaMemsetAsync(count_err, 0, sizeof(float), st));
    return launch_fft_in(ctx, p, f, erode, out, cnt, count_err, validate, buf, st, adj);
}

}  // namespace morph
