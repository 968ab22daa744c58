// Hermite-zero discrete fractional Fourier transform (Sec. 2, eq. (tmat)):
//   F_z = sqrt(2 pi) U^T D(z) U,   D(z) = diag(z^0, z^1, ..., z^{N-1}),
// with x_k the zeros of H_N -- the eigenvalues of the Jacobi matrix H (zero
// diagonal, off-diagonal sqrt(n/2), n = 1..N-1) -- and U's column k the
// normalised eigenvector u_k with the signs of eq. (ortvec).
//
//  * k_herm_nodes: one thread per eigenvalue, bisection on the Sturm count of
//    H - lambda I (the number of negative pivots of its LDL^T factorisation
//    is the number of eigenvalues below lambda), to the last bit.
//  * k_herm_vectors: one thread per node.  (u_k)_n is proportional to the
//    normalised Hermite polynomial p_n(x_k) = H_n(x_k) / sqrt(2^n n!), which
//    satisfies x p_n = sqrt((n+1)/2) p_{n+1} + sqrt(n/2) p_{n-1} (eq. (receqg)
//    divided by the normalisation) -- row n of H u_k = x_k u_k.  The forward
//    recurrence from p_0 = 1 gives component n the sign of H_n(x_k), which is
//    eq. (ortvec)'s sign; the column is then scaled to unit length.  The
//    values grow like e^{x^2/2} for edge nodes, so the column is rescaled by
//    2^-400 whenever a value passes 2^400.
//  * k_herm_gemm: out[b][j] = alpha_j sum_k A[b][k] B(k, j), A complex
//    (the signals), B real (U or U^T), one 32-signal x 64-column tile per
//    CTA; the first product T = f U^T takes alpha_n = sqrt(2 pi) z^n, the
//    second F_z f = T U takes alpha = 1.
#include "xft_common.cuh"

namespace {

// Number of eigenvalues of H below lam (Sturm count by the LDL^T pivots).
// A zero pivot is replaced by a tiny negative one before it is counted (the
// count of a lam perturbed by that much), so every pivot is counted with
// the sign the next step divides by.
__device__ int sturm_count(int n, double lam) {
    double q = -lam;
    if (q == 0.0) q = -1e-300;
    int c = q < 0.0;
    for (int i = 1; i < n; ++i) {
        q = -lam - (0.5 * (double)i) / q;
        if (q == 0.0) q = -1e-300;
        c += q < 0.0;
    }
    return c;
}

__global__ void k_herm_nodes(int n, double* __restrict__ x) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    // |lambda| <= max_i (sqrt(i/2) + sqrt((i+1)/2)) < sqrt(2n) (Gershgorin)
    double lo = -sqrt(2.0 * n) - 1.0, hi = sqrt(2.0 * n) + 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;          // interval at the last bit
        if (sturm_count(n, mid) <= k) lo = mid;
        else hi = mid;
    }
    x[k] = 0.5 * (lo + hi);
}

// Column k of U (row-major U[m][k], m = 0..n-1): the normalised recurrence
// vector at x_k.  Thread k writes U[m*n + k], so a warp's stores for one m
// are contiguous.
__global__ void k_herm_vectors(int n, const double* __restrict__ x, double* __restrict__ U) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double xk = x[k];
    const double s2x = 1.4142135623730951 * xk;
    constexpr double kBig = 0x1p400, kSmall = 0x1p-400;
    double pm = 0.0, p = 1.0;                       // p_{m-1}, p_m
    U[k] = p;
    for (int m = 0; m + 1 < n; ++m) {
        const double next = (s2x * p - sqrt((double)m) * pm) / sqrt((double)(m + 1));
        pm = p;
        p = next;
        U[(int64_t)(m + 1) * n + k] = p;
        if (fabs(p) > kBig) {
            pm *= kSmall;
            p *= kSmall;
            for (int j = 0; j <= m + 1; ++j) U[(int64_t)j * n + k] *= kSmall;
        }
    }
    double ss = 0.0;
    for (int m = 0; m < n; ++m) {
        const double v = U[(int64_t)m * n + k];
        ss = fma(v, v, ss);
    }
    const double inv = 1.0 / sqrt(ss);
    for (int m = 0; m < n; ++m) U[(int64_t)m * n + k] *= inv;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t count) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x)
        b[t] = (float)a[t];
}

// C[b][j] = alpha_j sum_k A[b][k] B(k, j) for b < batch, j < n, k < n.
// TRANSB = true: B(k, j) = Bm[j n + k] (the first product, B = U^T);
// TRANSB = false: B(k, j) = Bm[k n + j].  alpha: n complex values or null.
constexpr int kBM = 32, kBN = 64, kBK = 16, kGemmThreads = 256;

template <class R, bool TRANSB>
__global__ void __launch_bounds__(kGemmThreads)
k_herm_gemm(const cpx<R>* __restrict__ A, const R* __restrict__ Bm, cpx<R>* __restrict__ C,
            const cpx<R>* __restrict__ alpha, int64_t batch, int n) {
    __shared__ cpx<R> As[kBK][kBM + 1];
    __shared__ R Bs[kBK][kBN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;              // 16 x 16 threads
    const int64_t b0 = (int64_t)blockIdx.y * kBM;
    const int j0 = blockIdx.x * kBN;
    cpx<R> acc[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = {R(0), R(0)};
    for (int k0 = 0; k0 < n; k0 += kBK) {
        // A tile: 32 signals x 16 k (two elements per thread, k fastest)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int li = tid + e * kGemmThreads;
            const int kk = li & (kBK - 1), bb = li >> 4;
            const int64_t b = b0 + bb;
            const int k = k0 + kk;
            As[kk][bb] = (b < batch && k < n) ? A[b * n + k] : cpx<R>{R(0), R(0)};
        }
        // B tile: 16 k x 64 columns (four elements per thread)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int li = tid + e * kGemmThreads;
            int kk, jj;
            if (TRANSB) { kk = li & (kBK - 1); jj = li >> 4; }      // k fastest in memory
            else { jj = li & (kBN - 1); kk = li >> 6; }             // j fastest in memory
            const int k = k0 + kk, j = j0 + jj;
            R v = R(0);
            if (k < n && j < n) v = TRANSB ? Bm[(int64_t)j * n + k] : Bm[(int64_t)k * n + j];
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            cpx<R> a[2];
            R bv[4];
#pragma unroll
            for (int r = 0; r < 2; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c].x = madd(a[r].x, bv[c], acc[r][c].x);
                    acc[r][c].y = madd(a[r].y, bv[c], acc[r][c].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t b = b0 + ty + 16 * r;
        if (b >= batch) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + tx + 16 * c;
            if (j >= n) continue;
            cpx<R> v = acc[r][c];
            if (alpha) v = cmul(v, alpha[j]);
            C[b * n + j] = v;
        }
    }
}

template <class R>
cudaError_t herm_apply(int n, const void* in, void* out, void* work, const void* alpha,
                       const void* U, int64_t batch, cudaStream_t stream) {
    const dim3 grid((unsigned)((n + kBN - 1) / kBN), (unsigned)((batch + kBM - 1) / kBM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    k_herm_gemm<R, true><<<grid, kGemmThreads, 0, stream>>>(
        (const cpx<R>*)in, (const R*)U, (cpx<R>*)work, (const cpx<R>*)alpha, batch, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_herm_gemm<R, false><<<grid, kGemmThreads, 0, stream>>>(
        (const cpx<R>*)work, (const R*)U, (cpx<R>*)out, nullptr, batch, n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t lct_launch_hermite_basis(int n, double* x, double* U, float* Uf, cudaStream_t stream) {
    const int th = 128;
    const unsigned blocks = (unsigned)((n + th - 1) / th);
    k_herm_nodes<<<blocks, th, 0, stream>>>(n, x);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_herm_vectors<<<blocks, th, 0, stream>>>(n, x, U);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nn = (int64_t)n * n;
    k_to_float<<<(unsigned)((nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096), 256, 0, stream>>>(U, Uf, nn);
    return cudaGetLastError();
}

cudaError_t lct_launch_hermite_apply(int dtype, int n, const void* in, void* out, void* work,
                                     const void* alpha, const void* U, int64_t batch,
                                     cudaStream_t stream) {
    if (dtype == 0) return herm_apply<float>(n, in, out, work, alpha, U, batch, stream);
    return herm_apply<double>(n, in, out, work, alpha, U, batch, stream);
}
