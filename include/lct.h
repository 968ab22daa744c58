/*
 * lct.h -- C ABI of the GB300 library for the discrete linear canonical
 * transform (LCT) of Campos & Figueroa, "A fast algorithm for the linear
 * canonical transform" (the XFT).
 *
 * The transform (Sec. 3, eq. (lctdos), the matrix L = S1 F S2 and the
 * Algorithm).  For N = 2^p samples f_k of a function at the asymptotic
 * Hermite nodes of eq. (asymcer),
 *     x_k = (2k - N + 1) pi / (2 sqrt(2N)),   k = 0..N-1   (0-based),
 * with spacing dx = pi / sqrt(2N) (eq. (deltk)), the library returns, for
 * parameters (a, b, c, d) with ad - bc = 1 and b != 0,
 *     G_j = dx / sqrt(2 pi i b) * e^{i d y_j^2 / (2b)}
 *           * sum_k e^{-i x_k y_j / b} e^{i a x_k^2 / (2b)} f_k,
 *     y_j = 4 b x_j / pi,
 * computed in O(N log N) as chirp - DFT - chirp (the Algorithm of Sec. 3,
 * with the DFT taken with the forward sign e^{-2 pi i jk/N} and conjugated
 * centring phases, the reading under which it reproduces eq. (lctdos)).
 * For b == 0 (definition below eq. (lctuno)) it returns
 *     G_j = sqrt(d) e^{i c d y_j^2 / 2} f_j  on the output points y_j = x_j / d.
 * sqrt is the principal root.  For complex parameters (the fractional
 * transform with complex z, Sec. 1) the returned values are
 * Ghat_j = G_j e^{-rho_j}, rho_j = -Im(d y_j^2 / (2b)) (b != 0) or
 * -Im(c d y_j^2 / 2) (b == 0), which removes the real exponential of the
 * output chirp; lct_output_grid returns rho.  For real parameters rho = 0.
 *
 * Data layout.  Signals are complex, interleaved (re, im), row-major
 * [batch][N]: LCT_C64 = 2 x float (8 bytes per sample), LCT_C128 = 2 x
 * double (16 bytes).  Device pointers must be aligned to the sample size.
 *
 * Ownership.  The caller owns every buffer passed in.  A plan owns its
 * parameter descriptors, tables and workspace on the device, created on the
 * first execute on the current device and freed by lct_plan_destroy.
 *
 * Errors.  Every entry returns an lct_status; nothing traps.  Execution is
 * asynchronous on the given stream and performs no host synchronisation
 * (except lct_device_status, which synchronises).  Device-side per-item
 * errors are recorded in a status word read by lct_device_status.
 *
 * Streams are CUDA runtime streams (cudaStream_t); NULL is the legacy
 * default stream.
 *
 * Threads.  Entry points may be called from several host threads.  Calls
 * on one plan are serialised by the plan; the entry points that launch
 * kernels also hold one process-wide lock while they enqueue work (the
 * launchers cache per-device launch configurations on first use), so
 * concurrent calls on different plans are safe, and their kernels overlap
 * when they are given different streams.  lct_execute_host and
 * lct_plan_autotune wait for the device while they hold that lock.
 */
#ifndef LCT_H
#define LCT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The library is built with hidden symbol visibility; the declarations in
 * this header are its exported interface. */
#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

struct CUstream_st;
typedef struct CUstream_st* lct_stream_t;   /* == cudaStream_t */

typedef struct lct_plan_s* lct_plan;        /* opaque, owned by the library */

typedef enum { LCT_C64 = 0, LCT_C128 = 1 } lct_dtype;

/* Arithmetic of the transform.
 *  NATIVE      fused chirp-DFT-chirp kernel in the sample precision
 *              (FP32 for LCT_C64, FP64 for LCT_C128); phases exact (below).
 *  PLAIN64     unfused FP64 baseline: a chirp kernel, a library FFT (cuFFT
 *              Z2Z, forward sign) on an FP64 workspace, a chirp+scale kernel.
 *  PLAIN32     unfused FP32 baseline (complex64 plans of one N; else
 *              LCT_ERR_UNSUPPORTED): the same three steps in FP32 with cuFFT
 *              C2C on an FP32 workspace -- the fused kernel's arithmetic
 *              without the fusion.
 *  SPLIT_BF16, SPLIT_FP16, FP16
 *              tensor-core DFT (complex64 plans, one N in [16, 4096]): the
 *              radix-16 DFT passes run as real 32x32 DFT-matrix products
 *              (mma m16n8k16, FP32 accumulation); chirps and twiddles in FP32
 *              with the exact phases below.  SPLIT_*: operands split into
 *              hi + lo halves (BF16 or FP16), three products hi.hi + hi.lo +
 *              lo.hi; SPLIT_FP16 and FP16 scale each signal by a power of two
 *              so that the FP16 range holds.  FP16: one product of FP16
 *              operands (relative L2 error about 1e-3).  lct_plan_set_precision
 *              returns LCT_ERR_UNSUPPORTED for complex128 plans, ragged plans
 *              and other N.  b = 0 plans have no DFT and ignore the choice.
 *              lct_backward and the 2-D transform use NATIVE only.
 * Phases: every chirp phase is a turn fraction held as a fixed-point integer
 * (64 bits of fraction for FP32 paths, 128 for FP64 paths) and multiplied by
 * the integer m^2 (m = 2k - N + 1) with wrap-around, so no phase loses
 * accuracy as N or a/b grows. */
typedef enum {
    LCT_PREC_NATIVE = 0,
    LCT_PREC_SPLIT_BF16 = 1,
    LCT_PREC_SPLIT_FP16 = 2,
    LCT_PREC_FP16 = 3,
    LCT_PREC_PLAIN64 = 4,
    LCT_PREC_PLAIN32 = 5
} lct_precision;

typedef enum {
    LCT_OK = 0,
    LCT_ERR_ARG = 1,             /* null pointer, bad count/batch, bad z */
    LCT_ERR_N = 2,               /* N not a power of two in [2, 65536] */
    LCT_ERR_NOT_SYMPLECTIC = 3,  /* |ad - bc - 1| > 1e-9 max(1, |ad|, |bc|) */
    LCT_ERR_DTYPE = 4,
    LCT_ERR_ALIGN = 5,           /* pointer not aligned to the sample size */
    LCT_ERR_OOM = 6,
    LCT_ERR_CUDA = 7,            /* a CUDA runtime or cuFFT call failed */
    LCT_ERR_DEVICE = 8,          /* a kernel recorded a per-item error */
    LCT_ERR_TIMEOUT = 9,         /* a bounded device wait gave up */
    LCT_ERR_UNSUPPORTED = 10     /* combination not implemented */
} lct_status;

/* Plan for N-point transforms with real parameters (a, b, c, d), ad - bc = 1
 * (Sec. 1).  c is used only when b == 0.  Host-only: touches no GPU. */
lct_status lct_plan_create(lct_plan* out, int64_t N, double a, double b, double c, double d,
                           lct_dtype dtype);

/* Same with complex parameters: abcd_reim = {a_re, a_im, b_re, b_im, c_re,
 * c_im, d_re, d_im} (the fractional transform for complex z, Sec. 1). */
lct_status lct_plan_create_complex(lct_plan* out, int64_t N, const double abcd_reim[8],
                                   lct_dtype dtype);

/* Batch plan: `count` independent signals, signal s of length N[s] (power of
 * two) with parameters abcd_reim[8 s .. 8 s + 7] (layout as above), stored at
 * element offset offsets[s] of the in/out buffers.  All arrays are host
 * memory, copied by the plan.  Host-only.  A batch of mixed N, or of b = 0
 * signals mixed with b != 0 ones, is ragged: lct_execute runs it as one CUDA
 * graph -- one kernel per N for the b != 0 signals (the persistent two-pass
 * kernel from N = 32768), one launch for every b = 0 signal, on concurrent
 * branches -- captured on the first call for each (in, out) pair. */
lct_status lct_plan_create_batch(lct_plan* out, int64_t count, const int64_t* N,
                                 const double* abcd_reim, const int64_t* offsets,
                                 lct_dtype dtype);

lct_status lct_plan_set_precision(lct_plan plan, lct_precision precision);

/* Kernel variants of the fused path (LCT_PREC_NATIVE), chosen per plan:
 *  0  one CTA per group of signals, grid = number of groups (default);
 *  1  persistent CTAs that prefetch the next group into shared memory with
 *     bulk asynchronous copies while the current one is transformed
 *     (complex64, N = 256 .. 8192, 16-byte aligned signal starts; other
 *     plans fall back to variant 0), twiddles read from the table;
 *  2  as 1 with twiddles computed in registers;
 *  3  paired: every thread carries two signals in packed f32x2 registers,
 *     halving the arithmetic instructions (complex64, N = 32 .. 8192);
 *  4  paired and persistent, the next pair brought in by bulk asynchronous
 *     copy while the current one is written out (complex64, N = 4096,
 *     16-byte aligned signal starts; else variant 3);
 *  5  thread-block cluster of N/8192 CTAs per signal exchanging through
 *     distributed shared memory (N = 16384 .. 65536; with variant 0 it
 *     serves N = 16384 in complex128, where the fused kernel stops);
 *  6  paired with eight samples per thread (radix-8 passes), fewer
 *     registers and more resident warps (complex64, N = 64 .. 8192);
 *  7  two passes (four-step split N = N1 N2: column DFTs with the
 *     pre-chirp and inter-pass twiddles, then row DFTs with the post-chirp)
 *     in one persistent launch whose intermediate stays in a small ring of
 *     workspace slots (tens of MiB, owned by the plan), so it need not reach
 *     HBM (both dtypes, N = 8192 .. 65536; the default for N >= 32768);
 *  8  persistent CTAs whose input groups arrive by TMA tiled copies
 *     (cp.async.bulk.tensor) through a tensor map that views the batch as
 *     rows of 256 samples, one box per group of signals, completing on an
 *     mbarrier while the previous group is transformed (complex64, N = 256
 *     .. 8192, contiguous signals, 16-byte aligned input, batch N a multiple
 *     of 256; other launches fall back to variant 0);
 *  9  ragged batch plans (complex64, powers of two): the whole batch in one
 *     persistent launch that takes work items from one device queue,
 *     largest N first -- the two-pass tiles of every N >= 8192, then groups
 *     of signals of N <= 4096, then the b = 0 chunks -- instead of the CUDA
 *     graph of one kernel per N (other ragged plans keep the graph);
 * 10  schedule of variant 0 with radix-8 passes: eight samples per thread,
 *     N/8 threads per signal (N = 16 .. 8192), packed signals per CTA;
 * 11  schedule of variant 0 with one signal per CTA at any batch size
 *     (N = 32 .. 2048, where variant 0 packs several signals per CTA;
 *     complex128 with four samples per thread, radix-4 passes).
 * Variants 10 and 11 are the radix and signals-per-CTA choices the
 * autotuner times beside the others; a variant a plan cannot take falls
 * back to variant 0.  LCT_ERR_ARG for an unknown variant.  Host-only. */
lct_status lct_plan_set_variant(lct_plan plan, int variant);
/* The variant set on the plan, else the default for its N and dtype (7 for
 * N >= 32768; for complex64 10 at N = 32 .. 256 and 11 at N = 512 .. 2048,
 * the schedules that measured fastest there on GB300; else 0; a tuned
 * variant in the process cache overrides the default at execution). */
lct_status lct_plan_get_variant(lct_plan plan, int* variant);

/* Autotuner: run every variant that can execute this plan on the given
 * buffers (2 warm-up and 5 timed launches each, CUDA events on `stream`,
 * synchronising), keep the fastest in the plan and in a process-wide cache
 * keyed by (GPU name, dtype, N, precision).  If the environment variable
 * LCT_AUTOTUNE_CACHE names a file, it is read first (lines
 * "gpu|dtype|log2n|variant") and new results are appended.  `out` is
 * overwritten.  Plans created later with a cached key start with the cached
 * variant. */
lct_status lct_plan_autotune(lct_plan plan, const void* in, void* out, int64_t batch,
                             lct_stream_t stream);

/* Apply the plan.  in/out: device buffers in the plan's dtype.  For a plan
 * from lct_plan_create[_complex], `batch` signals of N samples, row-major.
 * For a batch plan, `batch` must equal its count.  in == out is allowed.
 * batch == 0 is a no-op.  Asynchronous on `stream`. */
lct_status lct_execute(lct_plan plan, const void* in, void* out, int64_t batch,
                       lct_stream_t stream);

/* lct_execute on host buffers: h_in/h_out are host memory (page-locked for
 * overlap; pageable memory works but each copy then blocks the host).  When
 * both are page-locked and mapped into the device's address space (memory
 * from cudaHostAlloc / cudaMallocHost, e.g. pinned torch tensors) and the
 * plan runs the native path with a plain-load kernel variant (not 1, 2, 4,
 * 8), the kernels read and write them directly over the host link, with no
 * staging.  Otherwise the batch is split into chunks of about 32 MiB that
 * are copied in, transformed and copied out on three plan-owned streams with
 * two plan-owned device staging pairs, so the copies in both directions
 * overlap each other and the kernels.  Ordered after the work already queued on `stream`; `stream`
 * waits for the last copy-out (the call itself returns after queueing).
 * Calls on one plan must be ordered (one stream).  Plans from
 * lct_plan_create[_complex] or batch plans of one N with offset[s] = s N;
 * LCT_ERR_UNSUPPORTED otherwise. */
lct_status lct_execute_host(lct_plan plan, const void* h_in, void* h_out, int64_t batch,
                            lct_stream_t stream);

/* Discrete fractional Fourier transform F_z with the normalisation of
 * eq. (eqifft): F_z = sqrt(2/(1 - z^2)) sqrt(2 pi i b) LCT(a, b, c, d) with
 * a = d = (z + 1/z)/2, b = (1/z - z)/(2i), c = i (1/z - z)/2, for
 * 0 < |z| <= 1 (|z| = 1, z != +-1: real-angle transform; z = +-1:
 * sqrt(2 pi) f on y_j = x_j / z).  Output points y_j = 4 b(z) x_j / pi;
 * the values are returned as G e^{-rho} (see above).  in/out as lct_execute. */
lct_status frft_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                        int64_t batch, lct_dtype dtype, lct_stream_t stream);

/* Fractional transform F_z for complex z on the real nodes, Sec. 2: the
 * matrix of eq. (fasy) applied to the samples, eq. (primcuad),
 *     g_j = sqrt(2/(1 - z^2)) dx sum_k e^{E_jk} f(x_k),
 *     E_jk = -[(1 + z^2)(x_j^2 + x_k^2) - 4 x_j x_k z] / (2 (1 - z^2)),
 * the Riemann sum of eq. (eqifft) at y_j = x_j (eq. (cuadtrfor)), x_k the
 * nodes of eq. (asymcer), dx of eq. (deltk).  Unlike frft_execute, whose
 * output points 4 b(z) x_j / pi are complex for complex z, the output here
 * is on the input's own real grid.  Computed exactly (up to rounding) in
 * O(N log N): E_jk = -B x_j^2 - A (x_j - x_k)^2 - B x_k^2 with
 * A = z/(1 - z^2), B = (1 - z)/(2(1 + z)), so g is a weighted circular
 * convolution of length M = 2^ceil(log2(2N - 1)); for Re z >= 0 neither
 * factor grows (Re A, Re B >= 0), and Re z < 0 is run as -z with the output
 * reversed (the kernel maps to itself under x_j -> -x_j, z -> -z).
 * in/out: `batch` signals of N samples at x_k (device memory, row-major
 * [batch][N], complex64 or complex128 computed in that precision, in == out
 * allowed).  N in [2, 8192] for complex64, [2, 4096] for complex128 (else
 * LCT_ERR_N); |z| <= 1 and z != +-1 (else LCT_ERR_ARG; on |z| = 1 the same
 * sum is the real-angle kernel, which aliases for small sin(arg z));
 * batch in [0, 2^31 - 1].  Two launches on `stream` (the lag kernel's
 * spectrum, one CTA; the transform) with a workspace of 256 + 8 M (16 M for
 * complex128) bytes from the stream-ordered allocator; asynchronous. */
lct_status frft_mehler_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                               int64_t batch, lct_dtype dtype, lct_stream_t stream);

/* Hermite-zero discrete fractional Fourier transform of Sec. 2, eq. (tmat):
 *     F_z = sqrt(2 pi) U^T D(z) U,   D(z) = diag(z^0, z^1, ..., z^{N-1}),
 * the exactly unitary (up to sqrt(2 pi), for |z| = 1) discrete transform
 * whose eigenvectors are the discrete Hermite functions.  Its nodes x_k are
 * the N zeros of H_N, the eigenvalues of the Jacobi matrix H (zero diagonal,
 * off-diagonal entries sqrt(n/2), n = 1..N-1); column k of the orthogonal U
 * is the normalised eigenvector u_k of x_k, with the signs of eq. (ortvec)
 * (component n has the sign of H_n(x_k)).  in/out: `batch` signals of N
 * samples at the nodes x_k (device memory, row-major [batch][N], complex
 * dtype as lct_execute, in == out allowed); out_j is the transform at x_j.
 * N in [2, 4096] (else LCT_ERR_N), |z| <= 1 (else LCT_ERR_ARG), batch <=
 * 2096960.  The basis (N nodes and U, N^2 doubles plus an FP32 copy) is
 * computed on the GPU at the first use of each N on a device -- nodes by
 * bisection on Sturm counts, vectors by the three-term recurrence -- and
 * cached for the life of the process; that first call synchronises.  Each
 * call takes a workspace of batch * N + N samples from the stream-ordered
 * allocator on `stream` and returns it there.  complex128: FP64 arithmetic
 * on the CUDA cores.  complex64: for N >= 128 the two products run on the
 * tensor cores (tcgen05, kind::tf32) with both operands split into TF32
 * hi + lo parts and three products accumulated in FP32 (relative error
 * about 1e-7; the split operands of U, 2 x 4 N^2 bytes rounded up to whole
 * tiles, are added to the cache at the first such call); below N = 128, FP32
 * CUDA-core arithmetic.  Asynchronous on `stream` after the first call for
 * an N. */
lct_status frft_hermite_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                                int64_t batch, lct_dtype dtype, lct_stream_t stream);
/* The nodes x_k (ascending, N doubles into host memory x) and, if U is not
 * NULL, U (N x N doubles into host memory, row-major: U[n N + k] =
 * component n of u_k) of the Hermite-zero transform above, computed on the
 * current device (built there if needed; synchronises). */
lct_status frft_hermite_basis(int64_t N, double* x, double* U);
/* Synchronise `stream`, then read and clear the status word of the
 * Hermite-zero tensor-core kernels: LCT_ERR_TIMEOUT if one of their bounded
 * waits (bulk copy or MMA completion, 2 s) gave up since the last call (its
 * output is then not written), else LCT_OK. */
lct_status frft_hermite_status(lct_stream_t stream);

/* Backward pass of lct_execute (spec differentiation; the chain rule
 * on L = S1 F S2 of Sec. 3).  grad_out: cotangent g = dl/dRe G + i dl/dIm G
 * (PyTorch's convention for a real loss l); writes grad_in = L^H g, the
 * adjoint transform (conjugated chirps, inverse-sign DFT).  If grad_abd is
 * not NULL it also writes the parameter gradients (dl/da, dl/db, dl/dd) --
 * c is not a free parameter when b != 0 -- computed from the dense-matrix
 * derivative with the output points y_j = 4 b x_j / pi moving with b:
 * 3 doubles per signal for batch plans, 3 doubles summed over `batch` for
 * single plans; `in` (f) and `out` (G) of the forward call are then
 * required.  All pointers are device memory.  Supported: uniform N <= 4096,
 * b != 0; parameter gradients for real parameters only.  The input gradient
 * alone (grad_abd NULL) is also computed for every other plan of one N the
 * forward path takes -- N = 8192 .. 65536, N that is not a power of two,
 * b = 0 -- with real parameters and signals at s N: as conj(L' conj(g)), L'
 * the forward transform with its two chirps exchanged (the DFT part of the
 * factorisation is symmetric), i.e. two conjugation passes around one
 * forward launch in grad_in (descriptors for L' kept by the plan).
 * LCT_ERR_UNSUPPORTED otherwise.  The plan keeps a workspace of 3 doubles
 * per signal for the reductions. */
lct_status lct_backward(lct_plan plan, const void* grad_out, const void* in, const void* out,
                        void* grad_in, double* grad_abd, int64_t batch, lct_stream_t stream);

/* Separable 2-D LCT (fields [batch][ny][nx], row-major): the 1-D transform
 * with abcd_x (4 reals) along every row (length nx), then with abcd_y along
 * every column (length ny).  Output points: the 1-D grids of each axis.
 * nx, ny powers of two in [128 (256 for complex128), 4096]; b != 0 on both
 * axes.  Host-only creation. */
typedef struct lct2d_plan_s* lct2d_plan;
lct_status lct2d_plan_create(lct2d_plan* out, int64_t ny, int64_t nx, const double abcd_y[4],
                             const double abcd_x[4], lct_dtype dtype);
/* mid receives the row-transformed fields (kept for lct2d_backward; mid ==
 * out is allowed when no backward pass follows). */
lct_status lct2d_execute(lct2d_plan plan, const void* in, void* mid, void* out, int64_t batch,
                         lct_stream_t stream);
/* Backward of lct2d_execute: grad_in = (L_y (x) L_x)^H grad_out, using the
 * caller's scratch field grad_mid; grad_abd (may be NULL) receives 6 doubles
 * summed over the batch: (dl/da, dl/db, dl/dd) of the x axis, then of the
 * y axis.  in, mid, out: the buffers of the forward call. */
lct_status lct2d_backward(lct2d_plan plan, const void* grad_out, const void* in, const void* mid,
                          const void* out, void* grad_mid, void* grad_in, double* grad_abd,
                          int64_t batch, lct_stream_t stream);
lct_status lct2d_plan_destroy(lct2d_plan plan);

/* No counterpart in the paper: the data movement of a separable 2-D
 * transform of one field sharded over several GPUs (rows on each GPU, an
 * all-to-all exchange, then the columns as rows; see the Python binding's
 * lct2d_sharded).  Transposes `batch` arrays of rows x cols vectors of `vec`
 * complex samples: in [batch][rows][cols][vec] -> out [batch][cols][rows][vec]
 * (device memory, dtype as lct_execute, in != out, else LCT_ERR_ARG; empty
 * sizes are a no-op).  Asynchronous on `stream`. */
lct_status lct_transpose(lct_dtype dtype, const void* in, void* out, int64_t rows, int64_t cols,
                         int64_t vec, int64_t batch, lct_stream_t stream);

/* Output points and rho of signal `index` of the plan (0 for single plans):
 * y_reim receives N complex points (2N doubles), rho N doubles (may be
 * NULL).  Host-only. */
lct_status lct_output_grid(lct_plan plan, int64_t index, double* y_reim, double* rho);

/* Input nodes x_k of eq. (asymcer), N doubles.  Host-only. */
lct_status lct_input_grid(int64_t N, double* x);

/* Fixed-point phase constants of signal `index` (for inspection and tests):
 * out[0..1] = Re(beta_in)/(2 pi) as a 128-bit turn fraction (hi, lo words),
 * out[2..3] = Re(beta_out)/(2 pi) likewise, out[4] = constant output turn
 * offset (64-bit fraction), where the pre-chirp is e^{i beta_in m^2} and the
 * post-chirp e^{i beta_out m^2}, m = 2k - N + 1.  Host-only. */
lct_status lct_plan_phase_turns(lct_plan plan, int64_t index, uint64_t out[5]);

/* Synchronise `stream`, read and clear the plan's device status word. */
lct_status lct_device_status(lct_plan plan, lct_stream_t stream);

lct_status lct_plan_destroy(lct_plan plan);

/* No counterpart in the paper: an extra entry point for callers that cannot
 * call cudaMalloc -- a process whose device memory is fully reserved up front
 * by its own pool allocator, or a latency-critical caller that must not hit
 * the implicit device synchronisation of cudaMalloc/cudaFree.
 * Computes the same transform as a plan from lct_plan_create(N, a, b, c, d,
 * dtype) with LCT_PREC_PLAIN64 (FP64 chirp, FP64 DFT, FP64 chirp + scale;
 * complex64 or complex128 samples in and out), but allocates nothing: no
 * plan, no cudaMalloc/cudaFree, no cuFFT plan, no other allocating library
 * call.  The FP64 intermediate lives in one static device array of
 * LCT_NOALLOC_MAX_POINTS complex128 samples (32 MiB) that every GPU which
 * loads the library holds until the process exits.
 * Limits: N a power of two in [2, LCT_NOALLOC_MAX_N], else LCT_ERR_N;
 * batch * N <= LCT_NOALLOC_MAX_POINTS, else LCT_ERR_ARG (nothing is run).
 * The first call on a device (batch 0 is enough) looks up the array's device
 * address, sets the DFT kernel's shared-memory limit and reads the
 * multiprocessor count, once per device.  Under CUDA's lazy module loading
 * that first call is also when the 32 MiB array is committed on the device,
 * so make it before the caller's pool reserves the device memory, and before
 * any stream capture.  The per-device set-up is not redone after
 * cudaDeviceReset: do not use this entry point across a device reset.  If a
 * CUDA error is already pending on the calling thread, the call returns
 * LCT_ERR_CUDA without launching and leaves that error pending.  All calls
 * share the array: calls whose kernels overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.  No state
 * carries over between calls.  in/out as lct_execute (device buffers, in ==
 * out allowed); asynchronous on `stream`. */
#define LCT_NOALLOC_MAX_N 4096
#define LCT_NOALLOC_MAX_POINTS (1 << 21)
lct_status lct_execute_noalloc(int64_t N, double a, double b, double c, double d,
                               lct_dtype dtype, const void* in, void* out, int64_t batch,
                               lct_stream_t stream);

const char* lct_status_string(lct_status status);

/* Debug mode (also enabled by the environment variable LCT_DEBUG=1, read
 * once): every lct_execute (its output) and lct_backward (its grad_in) then
 * synchronises its stream, scans those signals for NaN or infinite samples
 * and returns LCT_ERR_DEVICE if one is
 * found or a kernel recorded a per-item error (LCT_ERR_TIMEOUT for a timed-
 * out wait), clearing the device status word.  on = 0 turns it off. */
lct_status lct_set_debug(int on);

/* Test support, no counterpart in the paper: runs one kernel whose single
 * thread waits on purpose for an event that never happens -- which = 0: an
 * mbarrier phase (the wait of the bulk-copy kernels), 1: a global counter
 * (the wait of the two-pass kernel) -- bounded by limit_ms milliseconds (at
 * most 1000), then synchronises `stream`.  Returns LCT_ERR_TIMEOUT when the
 * wait gave up as designed (the kernel returned normally and the context
 * stays usable), LCT_OK if it completed, LCT_ERR_ARG for a bad argument,
 * LCT_ERR_CUDA / LCT_ERR_OOM on runtime errors. */
lct_status lct_selftest_timeout(int which, double limit_ms, lct_stream_t stream);

/* Multi-GPU sharding of a batch (one process per GPU; the signals are
 * independent, so no collective is needed on the data path).  Assigns each
 * of `count` signals to one of `world` ranks by cost, largest first, each to
 * the currently least-loaded rank (ties: the lowest rank): the cost of a
 * signal is N log2 N (its DFT), or N when b == 0 (diagonal only, from
 * abcd_reim in the layout of lct_plan_create_batch; abcd_reim may be NULL:
 * every signal then costs N log2 N).  Signals of equal cost keep their
 * order.  Deterministic: every rank computes the same assignment.
 * owner[s] (count entries) receives the rank of signal s; load (world
 * entries, may be NULL) each rank's total cost.  Host-only, O(count log
 * count). */
lct_status lct_partition(int64_t count, const int64_t* N, const double* abcd_reim, int32_t world,
                         int32_t* owner, double* load);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* LCT_H */
