/* Plain C use of the library (no Python, no PyTorch): read an image and an
 * SE, dilate and erode it on the GPU through include/morph.h, write the
 * results.
 *
 *   c_api_example IN OUT
 *   IN : int32 header n h w L kh kw oy ox, then n*h*w uint8 pixels, kh*kw
 *        uint8 mask, kh*kw int32 offsets (little-endian)
 *   OUT: n*h*w int32 dilation, n*h*w int32 counts, n*h*w int32 erosion,
 *        n*h*w int32 erosion counts
 * Exit status 0 on success; the library's status text on failure. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "morph.h"

static int fail(const char *what, int status) {
    fprintf(stderr, "%s: %s\n", what, status ? morph_strerror(status) : "I/O error");
    return 1;
}

int main(int argc, char **argv) {
    if (argc != 3) {
        fprintf(stderr, "usage: %s IN OUT\n", argv[0]);
        return 2;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return fail("open input", 0);
    int32_t hd[8];
    if (fread(hd, sizeof(int32_t), 8, in) != 8) return fail("read header", 0);
    const int n = hd[0], h = hd[1], w = hd[2], L = hd[3], kh = hd[4], kw = hd[5];
    const size_t npx = (size_t)n * h * w, ntap = (size_t)kh * kw;
    uint8_t *img = malloc(npx), *mask = malloc(ntap);
    int32_t *off = malloc(ntap * sizeof(int32_t)), *res = malloc(4 * npx * sizeof(int32_t));
    if (!img || !mask || !off || !res) return fail("allocate", 0);
    if (fread(img, 1, npx, in) != npx || fread(mask, 1, ntap, in) != ntap ||
        fread(off, sizeof(int32_t), ntap, in) != ntap)
        return fail("read body", 0);
    fclose(in);

    morph_ctx *ctx = NULL;
    int rc = morph_ctx_create(0, &ctx);
    if (rc) return fail("morph_ctx_create", rc);
    void *d_img = NULL;
    int32_t *d_out = NULL;
    if (cudaMalloc(&d_img, npx) != cudaSuccess || cudaMalloc((void **)&d_out, 4 * npx * sizeof(int32_t)) != cudaSuccess)
        return fail("cudaMalloc", MORPH_E_NOMEM);
    cudaStream_t st;
    cudaStreamCreate(&st);
    cudaMemcpyAsync(d_img, img, npx, cudaMemcpyHostToDevice, st);

    morph_image f = {d_img, MORPH_U8, n, h, w, w, (int64_t)h * w, L};
    morph_se se = {kh, kw, hd[6], hd[7], mask, off};
    morph_opts opts = {MORPH_AUTO, 0, NULL};
    rc = morph_dilate(ctx, &f, &se, d_out, d_out + npx, &opts, (morph_stream_t)st);
    if (rc) return fail("morph_dilate", rc);
    rc = morph_erode(ctx, &f, &se, d_out + 2 * npx, d_out + 3 * npx, &opts, (morph_stream_t)st);
    if (rc) return fail("morph_erode", rc);
    rc = morph_stream_check(ctx, (morph_stream_t)st);      /* syncs; reports data errors */
    if (rc) return fail("morph_stream_check", rc);
    cudaMemcpy(res, d_out, 4 * npx * sizeof(int32_t), cudaMemcpyDeviceToHost);

    FILE *out = fopen(argv[2], "wb");
    if (!out || fwrite(res, sizeof(int32_t), 4 * npx, out) != 4 * npx) return fail("write output", 0);
    fclose(out);
    cudaStreamDestroy(st);
    cudaFree(d_img);
    cudaFree(d_out);
    morph_ctx_destroy(ctx);
    free(img);
    free(mask);
    free(off);
    free(res);
    return 0;
}
