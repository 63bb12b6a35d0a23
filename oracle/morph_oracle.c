/*
 * Brute-force CPU oracle for exact grey-value dilation and erosion with a
 * non-flat structuring element (SE), and for the tie-split backward pass of
 * dilation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the "Classical" sliding-max
 * reference of the paper (Sec. 4.1): only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may build, load or call it.  It shares no
 * code, header or table with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Conventions (all from Sec. 2.1 of the paper):
 *   image  f : F -> {0..L-1}, F = [0,H) x [0,W) per image, N images.
 *   SE     b : B -> {0,1,2,...}, B given as a kh x kw box with a mask; the
 *          box entry (r, c) is the SE offset y = (r - oy, c - ox), i.e. the
 *          origin (0,0) of Z^2 sits at box entry (oy, ox).
 *   dilation (Eq. 6new, cropped to F as in Eq. 6):
 *          (f (+) b)(x) = max{ f(x - y) + b(y) : x - y in F, y in B },
 *          and 0 when no y is valid (x not in F (+) B, Eq. 6).
 *   erosion (Eq. Erosion):
 *          (f (-) b)(x) = min{ f(x + y) - b(y) : x + y in F, y in B }.
 *          The paper leaves the no-valid-tap value unstated; this oracle
 *          returns L - 1 there, the value duality with Eq. 6 implies.
 *   count polynomial (Eq. Obs7): the coefficient of t^d at x is the number
 *          of valid pairs (x - y, y) with f(x - y) + b(y) = d.
 *
 * Nothing here is blocked, fused or reordered: each output is the plain
 * maximum / minimum / count over the SE taps in row-major box order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ERANGE 2

static int check_args(int N, int H, int W, int L, int kh, int kw, int oy, int ox,
                      const uint8_t *mask, const int32_t *off)
{
    if (N < 0 || H < 0 || W < 0 || L < 1 || kh < 1 || kw < 1) return ORC_EINVAL;
    (void)oy; (void)ox;
    for (int t = 0; t < kh * kw; ++t)
        if (mask[t] && off[t] < 0) return ORC_ERANGE; /* b >= 0, Sec. 2.1 */
    return ORC_OK;
}

static int check_image(const int32_t *f, int64_t n, int L)
{
    for (int64_t p = 0; p < n; ++p)
        if (f[p] < 0 || f[p] >= L) return ORC_ERANGE;
    return ORC_OK;
}

/* Largest SE value over B, 0 for an empty B (the range axis then has L
 * entries, Step 1 with the data-independent l_R = (L - 1) + max b). */
int orc_max_offset(int kh, int kw, const uint8_t *mask, const int32_t *off)
{
    int m = 0;
    for (int t = 0; t < kh * kw; ++t)
        if (mask[t] && off[t] > m) m = off[t];
    return m;
}

/*
 * Dilation, Eq. 6new / Eq. 6.  Outputs per pixel:
 *   D[x]  = (f (+) b)(x), 0 if no valid tap;
 *   cD[x] = number of valid taps attaining D[x] (the top coefficient of the
 *           count polynomial, Eq. 9 / Eq. Obs7), 0 if no valid tap;
 *   counts (optional, [N][H][W][R], R = L + max b): the full count
 *           polynomial of Eq. Obs7.
 * nthreads <= 0 uses the OpenMP default; 1 runs serially.
 * rows_begin/rows_end restrict the work to image rows [rows_begin, rows_end)
 * of every image (a bounded sample for timing); pass 0, H for all rows.
 */
int orc_dilate(const int32_t *f, int N, int H, int W, int L,
               int kh, int kw, int oy, int ox,
               const uint8_t *mask, const int32_t *off,
               int32_t *D, int32_t *cD, int32_t *counts,
               int rows_begin, int rows_end, int nthreads)
{
    int rc = check_args(N, H, W, L, kh, kw, oy, ox, mask, off);
    if (rc) return rc;
    rc = check_image(f, (int64_t)N * H * W, L);
    if (rc) return rc;
    if (rows_begin < 0) rows_begin = 0;
    if (rows_end > H) rows_end = H;
    const int R = L + orc_max_offset(kh, kw, mask, off);
    const int64_t nrows = (int64_t)N * (rows_end - rows_begin);
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < nrows; ++q) {
        const int n = (int)(q / (rows_end - rows_begin));
        const int i = rows_begin + (int)(q % (rows_end - rows_begin));
        const int32_t *fn = f + (int64_t)n * H * W;
        for (int j = 0; j < W; ++j) {
            const int64_t px = ((int64_t)n * H + i) * W + j;
            int32_t *cnt = counts ? counts + px * R : NULL;
            if (cnt) memset(cnt, 0, sizeof(int32_t) * (size_t)R);
            int best = -1, nbest = 0;
            for (int r = 0; r < kh; ++r) {
                for (int c = 0; c < kw; ++c) {
                    if (!mask[r * kw + c]) continue;
                    /* y = (r - oy, c - ox); source pixel x - y */
                    const int si = i - (r - oy), sj = j - (c - ox);
                    if (si < 0 || si >= H || sj < 0 || sj >= W) continue;
                    const int s = fn[(int64_t)si * W + sj] + off[r * kw + c];
                    if (cnt) cnt[s] += 1;
                    if (s > best) { best = s; nbest = 1; }
                    else if (s == best) nbest += 1;
                }
            }
            D[px] = best < 0 ? 0 : best;
            cD[px] = best < 0 ? 0 : nbest;
        }
    }
    return ORC_OK;
}

/*
 * Erosion, Eq. Erosion, computed directly (not through duality):
 *   E[x]  = min{ f(x + y) - b(y) : x + y in F, y in B }, L - 1 if no tap;
 *   cE[x] = number of valid taps attaining the minimum, 0 if no tap.
 */
int orc_erode(const int32_t *f, int N, int H, int W, int L,
              int kh, int kw, int oy, int ox,
              const uint8_t *mask, const int32_t *off,
              int32_t *E, int32_t *cE,
              int rows_begin, int rows_end, int nthreads)
{
    int rc = check_args(N, H, W, L, kh, kw, oy, ox, mask, off);
    if (rc) return rc;
    rc = check_image(f, (int64_t)N * H * W, L);
    if (rc) return rc;
    if (rows_begin < 0) rows_begin = 0;
    if (rows_end > H) rows_end = H;
    const int64_t nrows = (int64_t)N * (rows_end - rows_begin);
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < nrows; ++q) {
        const int n = (int)(q / (rows_end - rows_begin));
        const int i = rows_begin + (int)(q % (rows_end - rows_begin));
        const int32_t *fn = f + (int64_t)n * H * W;
        for (int j = 0; j < W; ++j) {
            const int64_t px = ((int64_t)n * H + i) * W + j;
            int have = 0, best = 0, nbest = 0;
            for (int r = 0; r < kh; ++r) {
                for (int c = 0; c < kw; ++c) {
                    if (!mask[r * kw + c]) continue;
                    /* y = (r - oy, c - ox); source pixel x + y */
                    const int si = i + (r - oy), sj = j + (c - ox);
                    if (si < 0 || si >= H || sj < 0 || sj >= W) continue;
                    const int s = fn[(int64_t)si * W + sj] - off[r * kw + c];
                    if (!have || s < best) { best = s; nbest = 1; have = 1; }
                    else if (s == best) nbest += 1;
                }
            }
            E[px] = have ? best : L - 1;
            cE[px] = have ? nbest : 0;
        }
    }
    return ORC_OK;
}

/*
 * Backward pass of dilation: the upstream gradient g(x) is routed to every
 * tap that attains the maximum at x, split equally among the cD(x) such taps
 * (one valid subgradient of the max).  In fp64, summed in a fixed order:
 *   grad_f(p) = sum over y in B (row-major box order) with p + y in F and
 *               f(p) + b(y) = D(p + y) of g(p + y) / cD(p + y);
 *   grad_b(y) = sum over x in F (image-major, row-major) with x - y in F and
 *               f(x - y) + b(y) = D(x) of g(x) / cD(x);  0 for y not in B.
 * D and cD are the forward outputs (orc_dilate).  grad_b is [kh][kw].
 */
int orc_dilate_backward(const int32_t *f, int N, int H, int W, int L,
                        int kh, int kw, int oy, int ox,
                        const uint8_t *mask, const int32_t *off,
                        const int32_t *D, const int32_t *cD, const double *g,
                        double *grad_f, double *grad_b)
{
    int rc = check_args(N, H, W, L, kh, kw, oy, ox, mask, off);
    if (rc) return rc;
    rc = check_image(f, (int64_t)N * H * W, L);
    if (rc) return rc;
    if (grad_f) {
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    const int64_t p = ((int64_t)n * H + i) * W + j;
                    double acc = 0.0;
                    for (int r = 0; r < kh; ++r)
                        for (int c = 0; c < kw; ++c) {
                            if (!mask[r * kw + c]) continue;
                            const int ti = i + (r - oy), tj = j + (c - ox);
                            if (ti < 0 || ti >= H || tj < 0 || tj >= W) continue;
                            const int64_t x = ((int64_t)n * H + ti) * W + tj;
                            if (f[p] + off[r * kw + c] == D[x] && cD[x] > 0)
                                acc += g[x] / (double)cD[x];
                        }
                    grad_f[p] = acc;
                }
    }
    if (grad_b) {
        for (int r = 0; r < kh; ++r)
            for (int c = 0; c < kw; ++c) {
                double acc = 0.0;
                if (mask[r * kw + c]) {
                    for (int n = 0; n < N; ++n)
                        for (int i = 0; i < H; ++i)
                            for (int j = 0; j < W; ++j) {
                                const int si = i - (r - oy), sj = j - (c - ox);
                                if (si < 0 || si >= H || sj < 0 || sj >= W) continue;
                                const int64_t x = ((int64_t)n * H + i) * W + j;
                                const int64_t s = ((int64_t)n * H + si) * W + sj;
                                if (f[s] + off[r * kw + c] == D[x] && cD[x] > 0)
                                    acc += g[x] / (double)cD[x];
                            }
                }
                grad_b[r * kw + c] = acc;
            }
    }
    return ORC_OK;
}

/*
 * Backward pass of erosion (Eq. Erosion): g(x) goes to every tap attaining
 * the minimum at x, split equally among the cE(x) such taps; b enters with a
 * minus sign.  In fp64, summed in a fixed order:
 *   grad_f(p) = sum over y in B (row-major box order) with p - y in F and
 *               f(p) - b(y) = E(p - y) of g(p - y) / cE(p - y);
 *   grad_b(y) = - sum over x in F (image-major, row-major) with x + y in F and
 *               f(x + y) - b(y) = E(x) of g(x) / cE(x);  0 for y not in B.
 */
int orc_erode_backward(const int32_t *f, int N, int H, int W, int L,
                       int kh, int kw, int oy, int ox,
                       const uint8_t *mask, const int32_t *off,
                       const int32_t *E, const int32_t *cE, const double *g,
                       double *grad_f, double *grad_b)
{
    int rc = check_args(N, H, W, L, kh, kw, oy, ox, mask, off);
    if (rc) return rc;
    rc = check_image(f, (int64_t)N * H * W, L);
    if (rc) return rc;
    if (grad_f) {
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < H; ++i)
                for (int j = 0; j < W; ++j) {
                    const int64_t p = ((int64_t)n * H + i) * W + j;
                    double acc = 0.0;
                    for (int r = 0; r < kh; ++r)
                        for (int c = 0; c < kw; ++c) {
                            if (!mask[r * kw + c]) continue;
                            const int ti = i - (r - oy), tj = j - (c - ox);
                            if (ti < 0 || ti >= H || tj < 0 || tj >= W) continue;
                            const int64_t x = ((int64_t)n * H + ti) * W + tj;
                            if (f[p] - off[r * kw + c] == E[x] && cE[x] > 0)
                                acc += g[x] / (double)cE[x];
                        }
                    grad_f[p] = acc;
                }
    }
    if (grad_b) {
        for (int r = 0; r < kh; ++r)
            for (int c = 0; c < kw; ++c) {
                double acc = 0.0;
                if (mask[r * kw + c]) {
                    for (int n = 0; n < N; ++n)
                        for (int i = 0; i < H; ++i)
                            for (int j = 0; j < W; ++j) {
                                const int si = i + (r - oy), sj = j + (c - ox);
                                if (si < 0 || si >= H || sj < 0 || sj >= W) continue;
                                const int64_t x = ((int64_t)n * H + i) * W + j;
                                const int64_t s = ((int64_t)n * H + si) * W + sj;
                                if (f[s] - off[r * kw + c] == E[x] && cE[x] > 0)
                                    acc += g[x] / (double)cE[x];
                            }
                }
                grad_b[r * kw + c] = -acc;
            }
    }
    return ORC_OK;
}

/*
 * 3-D volumes (the method is stated for N-D images, Sec. 2.1 and Sec. 3):
 * f on [0,Z) x [0,H) x [0,W) per volume, N volumes; SE on a kd x kh x kw box
 * with origin (oz, oy, ox), box entry (q, r, c) = offset (q-oz, r-oy, c-ox).
 *   op = 0: dilation  max{ f(x - y) + b(y) : x - y in F, y in B }, 0 if none;
 *   op = 1: erosion   min{ f(x + y) - b(y) : x + y in F, y in B }, L-1 if none;
 * out_c = number of taps attaining it (0 if none).
 */
int orc_morph3d(const int32_t *f, int N, int Z, int H, int W, int L,
                int kd, int kh, int kw, int oz, int oy, int ox,
                const uint8_t *mask, const int32_t *off, int op,
                int32_t *out, int32_t *out_c, int nthreads)
{
    if (N < 0 || Z < 0 || H < 0 || W < 0 || L < 1 || kd < 1 || kh < 1 || kw < 1) return ORC_EINVAL;
    for (int t = 0; t < kd * kh * kw; ++t)
        if (mask[t] && off[t] < 0) return ORC_ERANGE;
    if (check_image(f, (int64_t)N * Z * H * W, L)) return ORC_ERANGE;
    const int sgn = op ? 1 : -1;   /* source = x + sgn * y */
    const int64_t nrows = (int64_t)N * Z * H;
    (void)nthreads;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q0 = 0; q0 < nrows; ++q0) {
        const int n = (int)(q0 / ((int64_t)Z * H));
        const int z = (int)((q0 / H) % Z);
        const int i = (int)(q0 % H);
        const int32_t *fn = f + (int64_t)n * Z * H * W;
        for (int j = 0; j < W; ++j) {
            int have = 0, best = 0, nbest = 0;
            for (int q = 0; q < kd; ++q)
                for (int r = 0; r < kh; ++r)
                    for (int c = 0; c < kw; ++c) {
                        const int t = (q * kh + r) * kw + c;
                        if (!mask[t]) continue;
                        const int sz = z + sgn * (q - oz), si = i + sgn * (r - oy), sj = j + sgn * (c - ox);
                        if (sz < 0 || sz >= Z || si < 0 || si >= H || sj < 0 || sj >= W) continue;
                        const int v = fn[((int64_t)sz * H + si) * W + sj];
                        const int s = op ? v - off[t] : v + off[t];
                        const int better = op ? (s < best) : (s > best);
                        if (!have || better) { best = s; nbest = 1; have = 1; }
                        else if (s == best) nbest += 1;
                    }
            const int64_t px = ((int64_t)(n * (int64_t)Z + z) * H + i) * W + j;
            out[px] = have ? best : (op ? L - 1 : 0);
            out_c[px] = have ? nbest : 0;
        }
    }
    return ORC_OK;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
