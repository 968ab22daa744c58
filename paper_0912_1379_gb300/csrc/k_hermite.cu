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
//    second F_z f = T U takes alpha = 1 (FP64, and FP32 below N = 128).
//  * k_herm_umma: the same two products for complex64 on the tensor cores
//    (tcgen05.mma kind::tf32, accumulator in tensor memory), each operand
//    split into TF32 hi + lo parts and three products hi.hi + hi.lo + lo.hi
//    accumulated in FP32 (relative error about 1e-7).  A 128 x 256 output
//    tile per CTA: rows are 64 signals x (re, im) -- a complex-by-real
//    product is two real ones -- and columns 256 outputs; K runs over N in
//    chunks of 32 through two shared-memory stages, so one chunk's MMAs run
//    while the next chunk is staged.  B (U or U^T) is split and tiled once
//    per basis (k_umma_pack) and arrives by one bulk copy per chunk.
#include "xft_common.cuh"
#include "xft_umma.cuh"

__device__ int32_t g_herm_status;      // bounded waits of k_herm_umma that gave up

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

// alpha_m = sqrt(2 pi) z^m: |z|^m = e^{m log|z|}, and the angle m arg(z) in
// turns, reduced exactly: t = arg(z)/(2 pi) arrives as a double-double
// (t_hi + t_lo), m t_hi is split into a double-double by an FMA, and only
// the fractional part (to 2^-53 turns) reaches sincospi.  zero: z = 0
// (alpha = sqrt(2 pi) at m = 0, else 0).
template <class R>
__global__ void k_herm_alpha(int n, double t_hi, double t_lo, double log_r, int zero,
                             cpx<R>* __restrict__ alpha) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double s2pi = 2.5066282746310002;
    if (zero) {
        alpha[m] = {m == 0 ? (R)s2pi : R(0), R(0)};
        return;
    }
    const double p = (double)m * t_hi;
    const double pe = fma((double)m, t_hi, -p);        // m t_hi = p + pe exactly
    const double fp = p - rint(p);                      // exact
    double f = fp + (pe + (double)m * t_lo);
    f -= rint(f);                                       // turns in [-1/2, 1/2]
    double sn, cs;
    sincospi(2.0 * f, &sn, &cs);
    const double mag = m == 0 ? s2pi : s2pi * exp((double)m * log_r);
    alpha[m] = {(R)(mag * cs), (R)(mag * sn)};
}

// ---------------------------------------------------------------------------
// tensor-core form (complex64)
// ---------------------------------------------------------------------------
constexpr int kUM = 128, kUN = 256, kUK = 32, kUThreads = 256;
constexpr uint32_t kUASz = kUM * kUK * 4;            // one part (hi or lo) of an A chunk
constexpr uint32_t kUBSz = kUN * kUK * 4;            // one part of a B chunk
constexpr uint32_t kUStage = 2 * kUASz + 2 * kUBSz;  // A hi, A lo, B hi, B lo
constexpr uint32_t kUSmem = 2 * kUStage;
constexpr uint32_t kUTmemCols = 256;
constexpr uint64_t kUWaitNs = 2000000000ull;
constexpr uint32_t kULbo = 128, kUSbo = kUK * 32;    // core matrices along K / next 8 rows

// Split and tile B for the tensor-core product: block (jt, kc) of the output
// holds, for output columns j = 256 jt + r and inputs k = 32 kc + q, the TF32
// hi part of B(k, j) then its lo part, each in the K-major core-matrix
// layout of umma::tf32_offset.  trans = 1: B(k, j) = U[j][k] (first
// product); trans = 0: B(k, j) = U[k][j].  Zero outside n x n.
__global__ void k_umma_pack(const double* __restrict__ U, int n, int trans, int kc_count,
                            float* __restrict__ out, int64_t total) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(t % kUK);
        const int r = (int)((t / kUK) % kUN);
        const int64_t blk = t / (kUK * kUN);          // jt * kc_count + kc
        const int kc = (int)(blk % kc_count), jt = (int)(blk / kc_count);
        const int j = jt * kUN + r, k = kc * kUK + q;
        double v = 0.0;
        if (j < n && k < n) v = trans ? U[(int64_t)j * n + k] : U[(int64_t)k * n + j];
        const float hi = umma::to_tf32((float)v);
        const float lo = umma::to_tf32((float)(v - (double)hi));
        float* base = out + blk * (int64_t)(2 * kUBSz / 4);
        const uint32_t off = umma::tf32_offset((uint32_t)r, (uint32_t)q, kUK) / 4;
        base[off] = hi;
        base[kUBSz / 4 + off] = lo;
    }
}

__device__ __forceinline__ void record_umma_timeout() {
    atomicCAS(&g_herm_status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
}

// Accumulation: a tcgen05 accumulator that takes every K step of a long
// product loses accuracy (its FP32 additions measured as truncating: 1e-5
// relative at N = 1024 instead of 5e-7), so each 32-wide K chunk goes to a
// fresh accumulator, one of two in tensor memory (chunk c to accumulator
// c & 1, 2 x 256 columns), and is then added into FP32 register sums with
// round-to-nearest while the tensor cores fill the other accumulator.
// 8 warps: warp w reads TMEM lanes 32 (w & 3) .. + 31 (rows) and columns
// 128 (w >> 2) .. + 127, and keeps those 128 sums.
__device__ __forceinline__ void umma_drain(uint32_t taddr, float* sum) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float v[16];
        umma::tmem_ld16(taddr + 16 * q, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) sum[16 * q + i] += v[i];
    }
}

// The 8 complex inputs thread tid contributes to A chunk c: signal
// b0 + tid / 4, inputs 32 c + 8 (tid & 3) + 0..7 (zero outside).
__device__ __forceinline__ void load_a_chunk(const cpx<float>* __restrict__ A, int64_t batch, int n,
                                             int64_t b0, int c, int tid, cpx<float>* pre) {
    const int64_t b = b0 + (tid >> 2);
    const int k0 = c * kUK + (tid & 3) * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        pre[e] = (b < batch && k < n) ? A[b * n + k] : cpx<float>{0.f, 0.f};
    }
}

__global__ void __launch_bounds__(kUThreads, 1)
k_herm_umma(const cpx<float>* __restrict__ A, const float* __restrict__ Bblk,
            cpx<float>* __restrict__ C, const cpx<float>* __restrict__ alpha, int64_t batch, int n,
            int kc_count) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar_b[2], bar_mma[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int jt = blockIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * (kUM / 2);
    if (warp == 0) umma::tmem_alloc(&tmem_slot, 2 * kUTmemCols);
    if (tid == 0) {
        xasync::mbar_init(&bar_b[0], 1);
        xasync::mbar_init(&bar_b[1], 1);
        xasync::mbar_init(&bar_mma[0], 1);
        xasync::mbar_init(&bar_mma[1], 1);
        xasync::fence_mbar_init();
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    // this thread's view of accumulator a: lane 32 quad + lane, columns 128 half ..
    const uint32_t my_acc = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(128 * half);
    constexpr uint32_t idesc = umma::instr_desc(umma::kFmtTF32, umma::kFmtTF32, kUM, kUN);
    float sum[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) sum[i] = 0.f;
    cpx<float> pre[8];                        // this thread's A values of the next chunk
    load_a_chunk(A, batch, n, b0, 0, tid, pre);
    if (tid == 0) {                           // B of chunks 0 and 1 into the two free stages
        for (int c0 = 0; c0 < 2 && c0 < kc_count; ++c0) {
            float* b1 = reinterpret_cast<float*>(sm + c0 * kUStage + 2 * kUASz);
            xasync::mbar_arrive_expect_tx(&bar_b[c0], 2 * kUBSz);
            xasync::bulk_g2s(b1, Bblk + ((int64_t)jt * kc_count + c0) * (2 * kUBSz / 4), 2 * kUBSz,
                             &bar_b[c0]);
        }
    }
    bool ok = true;
    int c = 0;
    for (; c < kc_count; ++c) {
        const int s = c & 1;
        unsigned char* st = sm + s * kUStage;
        float* a_hi = reinterpret_cast<float*>(st);
        float* a_lo = reinterpret_cast<float*>(st + kUASz);
        // chunk c - 2 (stage s, accumulator s) is complete -- thread 0 waited
        // for it after issuing chunk c - 1, and issued chunk c's B copy --
        // so drain its accumulator and reuse the stage
        if (c >= 2) {
            if (!__syncthreads_and(ok)) break;
            umma::fence_after_sync();
            umma_drain(my_acc + (uint32_t)(s * kUTmemCols), sum);
            umma::fence_before_sync();
        }
        // A chunk c (loaded into registers one chunk ahead): signal bb =
        // tid / 4, inputs k = 32 c + 8 (tid & 3) + 0..7; row 2 bb holds the
        // real parts, row 2 bb + 1 the imaginary parts
        {
            const int bb = tid >> 2, kq = (tid & 3) * 8;
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const uint32_t o_re = umma::tf32_offset(2 * bb, kq + 4 * g, kUK) / 4;
                const uint32_t o_im = umma::tf32_offset(2 * bb + 1, kq + 4 * g, kUK) / 4;
                float4 h, l;
                h.x = umma::to_tf32(pre[4 * g + 0].x); l.x = umma::to_tf32(pre[4 * g + 0].x - h.x);
                h.y = umma::to_tf32(pre[4 * g + 1].x); l.y = umma::to_tf32(pre[4 * g + 1].x - h.y);
                h.z = umma::to_tf32(pre[4 * g + 2].x); l.z = umma::to_tf32(pre[4 * g + 2].x - h.z);
                h.w = umma::to_tf32(pre[4 * g + 3].x); l.w = umma::to_tf32(pre[4 * g + 3].x - h.w);
                *reinterpret_cast<float4*>(a_hi + o_re) = h;
                *reinterpret_cast<float4*>(a_lo + o_re) = l;
                h.x = umma::to_tf32(pre[4 * g + 0].y); l.x = umma::to_tf32(pre[4 * g + 0].y - h.x);
                h.y = umma::to_tf32(pre[4 * g + 1].y); l.y = umma::to_tf32(pre[4 * g + 1].y - h.y);
                h.z = umma::to_tf32(pre[4 * g + 2].y); l.z = umma::to_tf32(pre[4 * g + 2].y - h.z);
                h.w = umma::to_tf32(pre[4 * g + 3].y); l.w = umma::to_tf32(pre[4 * g + 3].y - h.w);
                *reinterpret_cast<float4*>(a_hi + o_im) = h;
                *reinterpret_cast<float4*>(a_lo + o_im) = l;
            }
            if (c + 1 < kc_count) load_a_chunk(A, batch, n, b0, c + 1, tid, pre);
        }
        xasync::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            ok = xasync::mbar_wait(&bar_b[s], (c >> 1) & 1, kUWaitNs);
            if (!ok) {
                // give up on this chunk, but let its copy land before leaving
                record_umma_timeout();
                xasync::mbar_wait(&bar_b[s], (c >> 1) & 1, kUWaitNs);
            } else {
                umma::fence_after_sync();
                const uint32_t ah = xasync::smem_addr(a_hi), al = ah + kUASz;
                const uint32_t bh = ah + 2 * kUASz, bl = bh + kUBSz;
                const uint32_t d = tmem + (uint32_t)(s * kUTmemCols);
#pragma unroll
                for (int ks = 0; ks < kUK / 8; ++ks) {
                    const uint32_t o = ks * 2 * kULbo;          // 8 K values = 2 core matrices
                    const uint64_t dah = umma::smem_desc(ah + o, kULbo, kUSbo);
                    const uint64_t dal = umma::smem_desc(al + o, kULbo, kUSbo);
                    const uint64_t dbh = umma::smem_desc(bh + o, kULbo, kUSbo);
                    const uint64_t dbl = umma::smem_desc(bl + o, kULbo, kUSbo);
                    umma::mma_tf32(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                    umma::mma_tf32(d, dah, dbl, idesc, 1u);
                    umma::mma_tf32(d, dal, dbh, idesc, 1u);
                }
                umma::commit(&bar_mma[s]);
                // stage 1 - s is free once chunk c - 1 completes: wait for it
                // and start chunk c + 1's B copy into that stage now
                if (c + 1 < kc_count) {
                    const int s1 = s ^ 1;
                    if (c >= 1) ok = xasync::mbar_wait(&bar_mma[s1], ((c - 1) >> 1) & 1, kUWaitNs);
                    if (ok && c >= 1) {
                        float* b1 = reinterpret_cast<float*>(sm + s1 * kUStage + 2 * kUASz);
                        xasync::mbar_arrive_expect_tx(&bar_b[s1], 2 * kUBSz);
                        xasync::bulk_g2s(b1, Bblk + ((int64_t)jt * kc_count + c + 1) * (2 * kUBSz / 4),
                                         2 * kUBSz, &bar_b[s1]);
                    }
                    if (!ok) record_umma_timeout();
                }
            }
        }
        if (!__syncthreads_and(ok)) break;          // chunk c was not issued
    }
    // chunks 0 .. c-1 were issued; the last two are still to be drained (all
    // issued MMAs complete before the CTA leaves; a failed wait skips the
    // epilogue)
    if (!ok && tid == 0) record_umma_timeout();
    for (int t = c - 2 < 0 ? 0 : c - 2; t < c; ++t) {
        bool w = true;
        if (tid == 0) {
            w = xasync::mbar_wait(&bar_mma[t & 1], (t >> 1) & 1, kUWaitNs);
            if (!w) record_umma_timeout();
        }
        ok = __syncthreads_and(w) && ok;
        umma::fence_after_sync();
        if (ok) umma_drain(my_acc + (uint32_t)((t & 1) * kUTmemCols), sum);
    }
    ok = ok && c == kc_count;
    if (ok) {
        // row m = 32 quad + lane = 2 bb + part of signal b0 + bb; the even lane
        // stores the first 64 of this warp's 128 columns, the odd lane the rest
        const int m = 32 * quad + lane;
        const int64_t b = b0 + (m >> 1);
        const bool odd = (m & 1) != 0;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            const float send0 = sum[i], send1 = sum[64 + i];
            const float got0 = __shfl_xor_sync(0xffffffffu, send0, 1);
            const float got1 = __shfl_xor_sync(0xffffffffu, send1, 1);
            // even lane: column i (re = own, im = partner); odd lane: column 64 + i
            const float re = odd ? got1 : send0;
            const float im = odd ? send1 : got0;
            const int j = jt * kUN + 128 * half + (odd ? 64 + i : i);
            if (b < batch && j < n) {
                cpx<float> r = {re, im};
                if (alpha) r = cmul(r, alpha[j]);
                C[b * n + j] = r;
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, 2 * kUTmemCols);
}

cudaError_t umma_apply(int n, const void* in, void* out, void* work, const void* alpha,
                       const float* B1, const float* B2, int64_t batch, cudaStream_t stream) {
    static int attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        e = cudaFuncSetAttribute(k_herm_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUSmem);
        if (e != cudaSuccess) return e;
        attr_set[dev] = 1;
    }
    const int kc = (n + kUK - 1) / kUK;
    const dim3 grid((unsigned)((n + kUN - 1) / kUN), (unsigned)((batch + kUM / 2 - 1) / (kUM / 2)));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    k_herm_umma<<<grid, kUThreads, kUSmem, stream>>>((const cpx<float>*)in, B1, (cpx<float>*)work,
                                                     (const cpx<float>*)alpha, batch, n, kc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_herm_umma<<<grid, kUThreads, kUSmem, stream>>>((const cpx<float>*)work, B2, (cpx<float>*)out,
                                                     nullptr, batch, n, kc);
    return cudaGetLastError();
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

// Bytes of one split, tiled B operand of the tensor-core product for N = n.
size_t lct_hermite_umma_bytes(int n) {
    const size_t jt = (size_t)((n + kUN - 1) / kUN), kc = (size_t)((n + kUK - 1) / kUK);
    return jt * kc * 2 * (size_t)kUBSz;
}

cudaError_t lct_launch_hermite_umma_pack(int n, const double* U, float* B1, float* B2,
                                         cudaStream_t stream) {
    const int kc = (n + kUK - 1) / kUK;
    const int64_t total = (int64_t)((n + kUN - 1) / kUN) * kc * kUN * kUK;
    const unsigned grid = (unsigned)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
    k_umma_pack<<<grid, 256, 0, stream>>>(U, n, 1, kc, B1, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_umma_pack<<<grid, 256, 0, stream>>>(U, n, 0, kc, B2, total);
    return cudaGetLastError();
}

cudaError_t lct_launch_hermite_apply_umma(int n, const void* in, void* out, void* work,
                                          const void* alpha, const float* B1, const float* B2,
                                          int64_t batch, cudaStream_t stream) {
    return umma_apply(n, in, out, work, alpha, B1, B2, batch, stream);
}

// Read and clear the status word of the tensor-core kernels (synchronises).
cudaError_t lct_hermite_read_status(int32_t* v) {
    cudaError_t e = cudaMemcpyFromSymbol(v, g_herm_status, sizeof(int32_t));
    if (e != cudaSuccess) return e;
    const int32_t zero = 0;
    return cudaMemcpyToSymbol(g_herm_status, &zero, sizeof(int32_t));
}

cudaError_t lct_launch_hermite_alpha(int dtype, int n, double t_hi, double t_lo, double log_r,
                                     int zero, void* alpha, cudaStream_t stream) {
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (dtype == 0)
        k_herm_alpha<float><<<grid, 256, 0, stream>>>(n, t_hi, t_lo, log_r, zero, (cpx<float>*)alpha);
    else
        k_herm_alpha<double><<<grid, 256, 0, stream>>>(n, t_hi, t_lo, log_r, zero, (cpx<double>*)alpha);
    return cudaGetLastError();
}
