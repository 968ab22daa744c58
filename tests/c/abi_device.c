/* Device use of the C ABI from C99: one complex128 plan, host -> device copy,
 * lct_execute on the default stream, device -> host copy, status check.
 * Writes the input and the output (interleaved re, im doubles, count x N
 * each) to the file given as the only argument; the test compares them with
 * the oracle.  Returns 0 on success. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "lct.h"

int main(int argc, char** argv) {
    if (argc != 2) return 2;
    const int64_t N = 1024, count = 3;
    const double t = 0.9, s = 1.7;     /* (a, b, c, d) = (s cos t, s sin t, -sin t / s, cos t / s) */
    const double a = s * cos(t), b = s * sin(t), c = -sin(t) / s, d = cos(t) / s;
    double* x = malloc(sizeof(double) * N);
    double* f = malloc(sizeof(double) * 2 * N * count);
    double* g = malloc(sizeof(double) * 2 * N * count);
    if (!x || !f || !g) return 3;
    if (lct_input_grid(N, x) != LCT_OK) return 4;
    for (int64_t q = 0; q < count; ++q)
        for (int64_t k = 0; k < N; ++k) {
            const double w = 0.6 + 0.4 * (double)q, e = exp(-x[k] * x[k] / (2.0 * w * w));
            f[2 * (q * N + k)] = e * (1.0 + 0.3 * x[k]);
            f[2 * (q * N + k) + 1] = e * 0.2 * x[k] * x[k];
        }
    lct_plan p = NULL;
    if (lct_plan_create(&p, N, a, b, c, d, LCT_C128) != LCT_OK) return 5;
    void *din = NULL, *dout = NULL;
    const size_t bytes = sizeof(double) * 2 * N * count;
    if (cudaMalloc(&din, bytes) != cudaSuccess || cudaMalloc(&dout, bytes) != cudaSuccess) return 6;
    if (cudaMemcpy(din, f, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return 7;
    lct_status st = lct_execute(p, din, dout, count, NULL);
    if (st != LCT_OK) {
        fprintf(stderr, "lct_execute: %s\n", lct_status_string(st));
        return 8;
    }
    if (lct_device_status(p, NULL) != LCT_OK) return 9;
    if (cudaMemcpy(g, dout, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return 10;
    FILE* out = fopen(argv[1], "wb");
    if (!out) return 11;
    const double hdr[6] = {(double)N, (double)count, a, b, c, d};
    if (fwrite(hdr, sizeof(double), 6, out) != 6 || fwrite(f, 1, bytes, out) != bytes ||
        fwrite(g, 1, bytes, out) != bytes)
        return 12;
    fclose(out);
    cudaFree(din);
    cudaFree(dout);
    lct_plan_destroy(p);
    free(x);
    free(f);
    free(g);
    printf("ok\n");
    return 0;
}
