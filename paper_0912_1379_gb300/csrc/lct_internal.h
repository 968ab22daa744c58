// Internal definitions shared by the host library and the CUDA kernels.
//
// Per-signal descriptor.  The transform of one signal (Sec. 3, Algorithm,
// with the forward-sign DFT) is, for k, j = 0..N-1 and m = 2k - N + 1:
//
//   u_k = e^{2 pi i [phi_in m_k^2 + (N-1) k / (2N)]} e^{-decay m_k^2} f_k
//   U   = DFT_N(u)          (forward sign e^{-2 pi i jk/N})
//   G_j = scale * e^{2 pi i [phi_out m_j^2 + (N-1) j / (2N) + c_out]} U_j
//
// with phi_in  = Re(beta_in)/(2 pi),  beta_in  = a pi^2 / (16 b N)   (= a x_k^2/(2b) / m_k^2)
//      phi_out = Re(beta_out)/(2 pi), beta_out = b d / N            (= d y_j^2/(2b) / m_j^2)
//      decay   = Im(beta_in)
//      scale * e^{2 pi i c_out} = dx e^{-i pi (N-1)^2 / (2N)} / sqrt(2 pi i b),  dx = pi/sqrt(2N).
// phi_in and phi_out are 128-bit turn fractions (hi, lo words): the phase of
// element m is the wrapped product phi * m^2 (m^2 < 2^32), which is exact to
// 2^-96 turns; FP32 kernels use the top 64 bits only (error <= 2^-32 turns).
// c_out is a 64-bit turn fraction.  The centring phases (N-1)k/(2N) are exact
// dyadic fractions and are formed in the kernels from k and N.
//
// kind == LCT_KIND_DIAG (b == 0): G_j = scale e^{2 pi i [phi_out m_j^2 + c_out]} f_j
// with phi_out = Re(c/d) pi / (32 N) (the phase c x_j^2/(2d)), scale e^{2 pi i c_out} = sqrt(d).
//
// N not a power of two.  The DFT kernel of the factorisation is a chirp
// convolution: with m_j - m_k = 2 (j - k),
//   e^{-i pi m_j m_k / (2N)} = e^{-i pi m_j^2/(4N)} e^{-i pi m_k^2/(4N)} e^{i pi (j-k)^2 / N},
// so  G_j = scale e^{2 pi i [phi_out' m_j^2 + c_out]} sum_k h_{j-k} e^{2 pi i phi_in' m_k^2} f_k
// with h_n = e^{i pi n^2 / N}, phi_in' = phi_in - 1/(8N), phi_out' = phi_out - 1/(8N) and
// scale e^{2 pi i c_out} = dx / sqrt(2 pi i b) (no centring phases).  The
// convolution runs as a circular one of length M = 2^log2n >= 2N - 1
// (Bluestein's algorithm): kind LCT_KIND_BLUE, n = N.  b == 0 signals of such
// N are kind LCT_KIND_DIAGN (the diagonal above, log2n unused).
//
// N = 2^a 3^b 5^c 7^d that is not a power of two: the direct form above with
// a mixed-radix DFT (k_mixed.cu), kind LCT_KIND_MIXED, log2n = ceil(log2 N)
// (group order only): phi_in,
// phi_out, decay and scale as for LCT_KIND_XFT (N in place of 2^log2n), the
// centring phases (N-1) k/(2N) formed in the kernel, and
// scale e^{2 pi i c_out} = dx e^{-i pi (N-1)^2/(2N)} / sqrt(2 pi i b).  Other N
// keep the chirp-convolution form (LCT_KIND_BLUE).
//
// Fractional transform for complex z on the real nodes (Sec. 2, eqs. (fasy),
// (primcuad)): the kernel e^{-[(1+z^2)(x_j^2+x_k^2) - 4 x_j x_k z]/(2(1-z^2))}
// is exactly e^{-B x_j^2} e^{-A (x_j - x_k)^2} e^{-B x_k^2} with
// A = z/(1 - z^2), B = (1 - z)/(2 (1 + z)), so with x = pi m/(2 sqrt(2N)) the
// same convolution form holds with real weights:
//   G_j = e^{2 pi i phi m_j^2} e^{-decay m_j^2} sum_k h_{j-k} e^{2 pi i phi m_k^2} e^{-decay m_k^2} f_k,
//   phi = -Im(B) pi/(16N) turns (in_hi/lo = out_hi/lo), decay = Re(B) pi^2/(8N),
//   h_n = e^{-A pi^2 n^2/(2N)} times sqrt(2/(1 - z^2)) dx,
// kind LCT_KIND_MEHLER, flags DECAY and OUT_DECAY.  For Re z >= 0, Re A >= 0
// and Re B >= 0, so no factor grows; Re z < 0 runs -z and reverses the output
// (the kernel is odd in z through x_j -> -x_j: flag REVERSE).
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

enum { LCT_KIND_XFT = 0, LCT_KIND_DIAG = 1, LCT_KIND_BLUE = 2, LCT_KIND_DIAGN = 3, LCT_KIND_MEHLER = 4,
       LCT_KIND_MIXED = 5 };
// DECAY: the input weight carries e^{-decay m^2}; OUT_DECAY: the output
// weight too (kind LCT_KIND_MEHLER); REVERSE: sample j is stored at N-1-j.
enum { LCT_FLAG_DECAY = 1, LCT_FLAG_OUT_DECAY = 2, LCT_FLAG_REVERSE = 4 };

struct __align__(16) lct_desc {
    uint64_t in_hi, in_lo;    // phi_in  (128-bit turn fraction)
    uint64_t out_hi, out_lo;  // phi_out (128-bit turn fraction)
    uint64_t out_c;           // constant output turn offset (64-bit fraction)
    int64_t offset;           // element offset of the signal in in/out
    double scale;             // |prefactor|
    double decay;             // Im(beta_in) (pre-chirp magnitude e^{-decay m^2})
    int32_t log2n;            // log2 N; for LCT_KIND_BLUE log2 M (M >= 2N - 1)
    int32_t kind;
    int32_t flags;
    int32_t n;                // N (every kind)
};
static_assert(sizeof(lct_desc) == 80, "descriptor layout");

// Device status word values (first error wins).
enum { LCT_DEV_OK = 0, LCT_DEV_BAD_DESC = 1, LCT_DEV_TIMEOUT = 2, LCT_DEV_NONFINITE = 3 };

// Host: the descriptor of one N-point signal with parameters
// p = {a_re, a_im, b_re, b_im, c_re, c_im, d_re, d_im} (validates like
// lct_plan_create; returns an lct_status value).
int lct_make_desc_host(int64_t N, const double* p, int64_t offset, lct_desc* D);

// Host: device twiddle table of the Stockham engine for N = 2^log2n on the
// current device (built once per device, dtype and N; owned by the library
// for the life of the process).  Layout [pass p = 1..P-1][j = 1..15][k < Ns_p]:
// entry e^{-2 pi i j k / (16 Ns_p)}, Ns_p = R0 16^(p-1), R0 the first radix.
// Returns nullptr on failure (and for N < 32, which needs no table).
const void* lct_twiddle_table(int dtype, int log2n);
// Complex64 table of the radix-8 engine (8 samples per thread), same
// layout with radix 8: the column kernels' twiddles.
const void* lct_twiddle_table_r8(int log2n);
// Broadcast form of the complex64 table for the paired kernels (radix
// 2^le passes, le = 4 or 3): every entry (wx, wy) stored as
// {(wx, wx), (wy, wy)} (16 bytes).
const void* lct_twiddle_table_pair(int log2n, int le = 4);
// Table of the engine with radix 2^le passes (le = 2, 3 or 4) in the dtype's
// precision, same layout.
const void* lct_twiddle_table_le(int dtype, int log2n, int le);

// ---- kernel launchers (defined in the .cu files) ---------------------------
// Fused chirp-DFT-chirp on N = 2^log2n, one or several signals per CTA.
// desc_step = 0: one descriptor for all `count` signals (signal s at s*N);
// desc_step = 1: desc[s] for signal s (its own offset).
// dtype: 0 = complex64 (FP32 arithmetic), 1 = complex128 (FP64 arithmetic).
// tw: the twiddle table of lct_twiddle_table(dtype, log2n).
// idx (may be null): ragged mode, signal s of the launch is descriptor
// idx[s] (desc_step must be 1); descriptors that do not match the kernel's N
// or kind are skipped and LCT_DEV_BAD_DESC is recorded in *status.
cudaError_t lct_launch_fused(int dtype, int log2n, const void* in, void* out,
                             const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                             const int32_t* idx, int32_t* status, cudaStream_t stream);
bool lct_fused_supported(int dtype, int log2n);

// Large-N fused kernel (N = 16384 .. 65536, both dtypes): a thread-block
// cluster of N/8192 CTAs per signal exchanging through distributed shared
// memory.  tw_local: lct_twiddle_table(dtype, lct_cluster_local_log2(...)).
int lct_cluster_local_log2(int dtype, int log2n);     // -1 if unsupported
cudaError_t lct_launch_cluster(int dtype, int log2n, const void* in, void* out,
                               const lct_desc* desc, int desc_step, int64_t count,
                               const void* tw_local, const int32_t* idx, int32_t* status,
                               cudaStream_t stream);

// Persistent variant of the fused kernel with bulk-async prefetch of the next
// signal group (complex64, N = 256 .. 8192).  Signal starts must be 16-byte
// aligned.  status: device status word (a timed-out wait records LCT_DEV_TIMEOUT).
// twiddle_compute: 1 = compute twiddles in registers, 0 = read the table.
cudaError_t lct_launch_fused_tma(int dtype, int log2n, const void* in, void* out,
                                 const lct_desc* desc, int desc_step, int64_t count,
                                 const void* tw, int32_t* status, int twiddle_compute,
                                 cudaStream_t stream);
bool lct_fused_tma_supported(int dtype, int log2n);

// Variant 8: the persistent fused kernel with its input staged by TMA tiled
// copies through a tensor map (complex64, N = 256 .. 8192, signal s at
// element s N of `in`, count N a multiple of 256, 16-byte aligned `in`;
// cudaErrorInvalidValue otherwise).
bool lct_fused_tmat_supported(int dtype, int log2n);
cudaError_t lct_launch_fused_tmat(int log2n, const void* in, void* out, const lct_desc* desc,
                                  int desc_step, int64_t count, const void* tw, int32_t* status,
                                  cudaStream_t stream);

// Paired variant (complex64, N = 32 .. 8192): two signals per thread in
// packed f32x2 registers.  tw_pair: lct_twiddle_table_pair(log2n).
cudaError_t lct_launch_fused_pair(int dtype, int log2n, const void* in, void* out,
                                  const lct_desc* desc, int desc_step, int64_t count,
                                  const void* tw_pair, cudaStream_t stream);
bool lct_fused_pair_supported(int dtype, int log2n);
// Paired variant with eight samples per thread (radix-8 passes), complex64,
// N = 64 .. 8192.  tw_pair8: lct_twiddle_table_pair(log2n, 3).
cudaError_t lct_launch_fused_pair8(int dtype, int log2n, const void* in, void* out,
                                   const lct_desc* desc, int desc_step, int64_t count,
                                   const void* tw_pair8, cudaStream_t stream);
bool lct_fused_pair8_supported(int dtype, int log2n);

// Persistent paired variant with bulk-async refill of its single shared
// buffer (complex64, N = 4096, 16-byte aligned signal starts).
cudaError_t lct_launch_fused_pair_tma(int dtype, int log2n, const void* in, void* out,
                                      const lct_desc* desc, int desc_step, int64_t count,
                                      const void* tw_pair, int32_t* status, cudaStream_t stream);
bool lct_fused_pair_tma_supported(int dtype, int log2n);

// Two-pass large-N XFT (k_twopass.cu), one persistent launch: N = N1 N2
// with log2 N1 = log2n / 2 (lct_twopass_split); tw1, tw2:
// lct_twiddle_table(dtype, log2 N1), (dtype, log2 N2).  work: `slots` ring
// slots of N samples (lct_twopass_ring); sync: the queue, abort flag and
// counters (4 + 2 slots int32, 8-byte aligned), zeroed by the launch.
// Signal s of the launch is descriptor idx[s] when idx is not null
// (desc_step must then be 1).  A timed-out wait records LCT_DEV_TIMEOUT.
bool lct_twopass_supported(int dtype, int log2n);
void lct_twopass_split(int log2n, int* l1, int* l2);
cudaError_t lct_twopass_ring(int dtype, int log2n, int64_t count, int64_t* slots);
cudaError_t lct_launch_twopass(int dtype, int log2n, const void* in, void* out, void* work,
                               int32_t* sync, const lct_desc* desc, int desc_step, int64_t count,
                               const int32_t* idx, int32_t* status, const void* tw1,
                               const void* tw2, cudaStream_t stream);

// Persistent ragged kernel (k_ragged.cu, complex64): one launch over a work
// queue of int4 items -- {LCT_RG_TP, group, p >> 32, p & 0xffffffff}: tile p
// of the two-pass group; {LCT_RG_FUSED, log2n, position in idx, count}: up
// to lct_ragged_fused_spc(log2n) signals of N <= 4096; {LCT_RG_DIAG, chunk
// index, position of the b = 0 index list, 0}.  groups: the two-pass groups
// (ring workspace at work + work_off samples, counters at sync + 2 +
// sync_off int32); sync: the queue word (2 int32) then the counters, zeroed
// by the launch (sync_bytes in all); tw[L]: lct_twiddle_table(0, L).
enum { LCT_RG_TP = 0, LCT_RG_FUSED = 1, LCT_RG_DIAG = 2 };
struct lct_rg_group {
    int64_t count, lag, slots, idx_off, work_off, sync_off;
    int32_t log2n, pad;
};
void lct_twopass_tiles(int log2n, int* cb, int* rb);
int lct_ragged_fused_spc(int log2n);
size_t lct_ragged_smem_bytes();
cudaError_t lct_launch_ragged(const void* in, void* out, const lct_desc* desc, const int32_t* idx,
                              const int4* items, int64_t n_items, const lct_rg_group* groups,
                              const int4* chunks, void* work, int32_t* sync, size_t sync_bytes,
                              const void* const* tw, int32_t* status, cudaStream_t stream);

// Self-test of the bounded waits (k_selftest.cu): word[0..2] zeroed device
// int32; which 0 = mbarrier wait, 1 = counter wait.
cudaError_t lct_launch_selftest_wait(int which, uint64_t limit_ns, int32_t* word,
                                     cudaStream_t stream);

// Split-precision XFT on the tensor cores (complex64, N = 16 .. 4096; a CTA
// transforms 4096/N signals).  mode: 1 = split BF16 (three products),
// 2 = split FP16 (three products, per-signal power-of-two scaling), 3 = FP16
// (one product).  tw: lct_twiddle_table(0, log2n) (unused for N = 16).
// async_ok: every signal start is 16-byte aligned, so inputs may arrive by
// bulk-async copies (a timed-out wait records LCT_DEV_TIMEOUT in *status);
// contiguous: signal s of the launch starts at element s N of `in` (one
// copy per tile).
// The three modes on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory), N = 4096: persistent CTAs, one signal at a
// time; a timed-out wait records LCT_DEV_TIMEOUT.  prec: the mode numbers
// above.  tw: lct_twiddle_table(0, 12).
bool lct_split_umma_supported(int dtype, int log2n);
cudaError_t lct_launch_split_umma(int prec, int log2n, const void* in, void* out, const lct_desc* desc,
                                  int desc_step, int64_t count, const void* tw, int32_t* status,
                                  cudaStream_t stream);
cudaError_t lct_launch_split(int mode, int log2n, const void* in, void* out, const lct_desc* desc,
                             int desc_step, int64_t count, const void* tw, int async_ok,
                             int contiguous, int32_t* status, cudaStream_t stream);
bool lct_split_supported(int dtype, int log2n);

// Diagonal branch (b == 0) for `count` signals of N = 2^log2n; idx as for
// lct_launch_fused (may be null).
cudaError_t lct_launch_diag(int dtype, int log2n, const void* in, void* out,
                            const lct_desc* desc, int desc_step, int64_t count,
                            const int32_t* idx, int32_t* status, cudaStream_t stream);

// Diagonal branch (b == 0) for every diagonal signal of a ragged batch in
// one launch.  chunks: nchunks int32 quadruples {pos, start, log2n, nsig}
// (16-byte aligned): elements start .. start + kDiagChunk - 1 of signal
// idx[pos] (nsig == 1) or the nsig whole signals idx[pos ..] of equal N
// (nsig N <= kDiagChunk).  Mismatching descriptors set LCT_DEV_BAD_DESC.
constexpr int kDiagChunk = 2048;
cudaError_t lct_launch_diag_chunks(int dtype, const void* in, void* out, const lct_desc* desc,
                                   const int32_t* idx, const int32_t* chunks, int64_t nchunks,
                                   int32_t* status, cudaStream_t stream);

// General single-CTA kernel (k_general.cu): forward or adjoint, rows
// (cols = 0) or interleaved columns (cols = 1), optional gradient sums
// (SA, SR, SG) per signal into partial[3 s ..].  Signal s starts at D.offset
// (desc_step = 1) or (s / P) * big + (s % P); element stride es.
// host_desc (may be null): a host copy of desc[0]; with it, complex64
// columns of uniform parameters run the persistent kernel that stages the
// next strip in shared memory (P a power of two, whole groups of columns,
// 16-byte aligned strips), else the one-strip-per-CTA kernel.  tw: the
// table of lct_twiddle_table(dtype, log2n), except for complex64 columns:
// lct_twiddle_table_r8(log2n) (or null: twiddles computed in registers).
bool lct_gen_supported(int dtype, int log2n, int cols);
cudaError_t lct_launch_gen(int dtype, int log2n, int cols, int adjoint, int grad, const void* in,
                           void* out, const lct_desc* desc, int desc_step, int64_t count,
                           const void* tw, int64_t es, int64_t P, int64_t big,
                           const void* fwd_out, const void* fwd_in, double* partial,
                           const lct_desc* host_desc, cudaStream_t stream);
// grad[3 s + {0,1,2}] = (dl/da, dl/db, dl/dd) from the sums; coef: 5 doubles
// per signal (coef_step 1) or shared (coef_step 0); shared != 0 sums over
// the signals into grad[0..2].
cudaError_t lct_launch_grad_finalize(const double* partial, const double* coef, int coef_step,
                                     int64_t count, int shared, double* grad, double* scratch,
                                     cudaStream_t stream);
// Bytes of the finalize scratch (slice totals and a ticket counter that must
// be zero before the first launch; the kernel leaves it zero).
size_t lct_grad_finalize_scratch_bytes();

// Debug scan: records LCT_DEV_NONFINITE in *status if any sample of the
// `count` output signals is NaN or infinite.  desc_step = 0: signal s is
// elements [s n, (s + 1) n); desc_step = 1: desc[s].offset and desc[s].n.
cudaError_t lct_launch_scan(int dtype, const void* out, const lct_desc* desc, int desc_step,
                            int64_t count, int64_t n, int32_t* status, cudaStream_t stream);

// ---- N not a power of two (k_bluestein.cu, lct_phase.cpp) ------------------
// Largest such N per dtype (the convolution of length M <= 16384 complex64 /
// 8192 complex128 fits one CTA's shared memory).
constexpr int64_t kBlueMaxN64 = 8192, kBlueMaxN128 = 4096;
// log2 M, M the smallest power of two >= 2N - 1.
int lct_blue_log2m(int64_t n);
bool lct_blue_supported(int dtype, int64_t n);
// Host: device table of the kernel spectrum H_j / M, j < M, H = DFT_M of the
// circularly placed chirp h_n = e^{i pi n^2/N} (|n| < N), for this N on the
// current device, in the dtype's precision (cached for the process).
const void* lct_blue_spectrum(int dtype, int64_t n);
// Chirp - FFT_M - spectrum - inverse FFT_M - chirp for `count` signals of one
// N (kind LCT_KIND_BLUE), one CTA per signal or group of signals.  tw:
// lct_twiddle_table(dtype, log2 M); spec: lct_blue_spectrum(dtype, n).
// idx as for lct_launch_fused (descriptors of another N or kind are flagged).
cudaError_t lct_launch_blue(int dtype, int64_t n, const void* in, void* out, const lct_desc* desc,
                            int desc_step, int64_t count, const void* tw, const void* spec,
                            const int32_t* idx, int32_t* status, cudaStream_t stream);
// The same kernel for kind LCT_KIND_MEHLER descriptors (any N = 2 ..
// kBlueMaxN64 / kBlueMaxN128, powers of two included) with the spectrum of
// lct_launch_mehler_spectrum.
cudaError_t lct_launch_mehler(int dtype, int64_t n, const void* in, void* out, const lct_desc* desc,
                              int64_t count, const void* tw, const void* spec, int32_t* status,
                              cudaStream_t stream);
// One CTA: spec[t] = c/M DFT_M(h)[t] for h_l = e^{-a_h l^2} e^{2 pi i phi_h l^2}
// placed circularly (|l| < n, zero elsewhere), M = 2^lct_blue_log2m(n),
// phi_h a 128-bit turn fraction, c = (c_re, c_im); also stores `D` at
// d_desc and zeroes *status (all in device memory).
cudaError_t lct_launch_mehler_spectrum(int dtype, int64_t n, double a_h, uint64_t phi_hi,
                                       uint64_t phi_lo, double c_re, double c_im,
                                       const lct_desc& D, lct_desc* d_desc, void* spec,
                                       int32_t* status, const void* tw, cudaStream_t stream);
// Fused kernel with an explicit schedule (autotuner variants 10 and 11):
// le = 3 (radix-8 passes, N/8 threads per signal, packed signals per CTA),
// or one signal per CTA with le = 4 (radix-16 passes) or, complex128 up to
// N = 2048, le = 2 (radix-4 passes).  tw: lct_twiddle_table_le(dtype,
// log2n, le).
bool lct_fused_sched_supported(int dtype, int log2n, int le, int one);
cudaError_t lct_launch_fused_sched(int dtype, int log2n, int le, int one, const void* in, void* out,
                                   const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                                   const int32_t* idx, int32_t* status, cudaStream_t stream);
// out[e] = conj(in[e]) for e < n (in == out allowed).
cudaError_t lct_launch_conj(int dtype, const void* in, void* out, int64_t n, cudaStream_t stream);
// Mixed-radix plan of one N (kind LCT_KIND_MIXED): the passes' radices
// (16, 8, 4, 2, 7, 5, 3), Ns_p (product of the earlier radices), the exact
// divisor magic floor(2^32 / Ns_p) + 1 (b / Ns_p = umulhi(b, magic) for
// b < 2^32 / Ns_p), each pass's offset into the twiddle table, the 128-bit
// turn fraction 1/(2N), and the threads per signal (>= N / (R K_R) for every
// pass, K_R = 16 / R butterflies a thread, a multiple of 32).
constexpr int kMixedMaxPasses = 16;
struct __align__(16) lct_mixed_plan {
    int n, npass, threads, pad;
    int radix[kMixedMaxPasses];
    int ns[kMixedMaxPasses];
    uint32_t magic[kMixedMaxPasses];
    int twoff[kMixedMaxPasses];
    uint64_t inv_hi, inv_lo;
};
static_assert(sizeof(lct_mixed_plan) <= 512, "plan header");
// Host: is N a non-power-of-two 7-smooth size in [3, 8192]?
bool lct_mixed_ok(int64_t n);
// Host: the plan of such an N (false otherwise).
bool lct_mixed_make_plan(int64_t n, int dtype, lct_mixed_plan* pl);
// Host: device buffer of that plan (cached per device, dtype and N): the
// lct_mixed_plan itself, then at byte kMixedPlanBytes the twiddle table in
// the dtype's precision: for pass p >= 1, entry [twoff_p + (r - 1) Ns_p + j]
// = e^{-2 pi i j r / (Ns_p R_p)}.
constexpr size_t kMixedPlanBytes = 512;
const void* lct_mixed_twiddles(int dtype, int64_t n);
// Threads per CTA of the mixed-radix kernel for a plan (several signals per
// CTA below 256 threads per signal).
int lct_mixed_threads_per_cta(const lct_mixed_plan& pl);
cudaError_t lct_launch_mixed(int dtype, const lct_mixed_plan& pl, const void* in, void* out,
                             const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                             const int32_t* idx, int32_t* status, cudaStream_t stream);
// b == 0 signals of one N that is not a power of two (kind LCT_KIND_DIAGN).
cudaError_t lct_launch_diag_any(int dtype, int64_t n, const void* in, void* out,
                                const lct_desc* desc, int desc_step, int64_t count,
                                const int32_t* idx, int32_t* status, cudaStream_t stream);

// Plain FP64 baseline pieces.  work: complex128 [count][N].
cudaError_t lct_launch_plain_pre(int dtype, int log2n, const void* in, void* work,
                                 const lct_desc* desc, int desc_step, int64_t count,
                                 cudaStream_t stream);
cudaError_t lct_launch_plain_post(int dtype, int log2n, const void* work, void* out,
                                  const lct_desc* desc, int desc_step, int64_t count,
                                  cudaStream_t stream);
// Batched transpose (k_transpose.cu): in [batch][rows][cols][vec] ->
// out [batch][cols][rows][vec], complex samples of the dtype.
cudaError_t lct_launch_transpose(int dtype, const void* in, void* out, int64_t rows, int64_t cols,
                                 int64_t vec, int64_t batch, cudaStream_t stream);

// Plain FP32 baseline pieces (complex64 in/out).  work: complex64 [count][N].
cudaError_t lct_launch_plain32_pre(const void* in, void* work, const lct_desc* desc, int log2n,
                                   int desc_step, int64_t count, cudaStream_t stream);
cudaError_t lct_launch_plain32_post(const void* work, void* out, const lct_desc* desc, int log2n,
                                    int desc_step, int64_t count, cudaStream_t stream);
