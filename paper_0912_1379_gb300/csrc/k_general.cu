// General single-CTA XFT kernel: forward or adjoint transform, rows or
// columns, with optional parameter-gradient sums.  Used by lct_backward
// (adjoint + gradients) and by the separable 2-D transform (columns).
//
// Adjoint (Sec. 3: L = S1 F S2, so L^H = S2^H F^H S1^H): the input is
// multiplied by conj(post-chirp) * scale, the DFT runs with the inverse sign
// e^{+2 pi i jk/N}, and the output by conj(pre-chirp) (including the real
// factor e^{-decay m^2} of complex parameters).
//
// Gradient sums (real parameters, b != 0), per signal, with g the cotangent
// dl/dRe G + i dl/dIm G, G the forward output, f the forward input and
// h = L^H g:
//   SA = sum_k m_k^2 Im(conj(h_k) f_k)
//   SR = sum_j Re(conj(g_j) G_j)
//   SG = sum_j m_j^2 Im(conj(g_j) G_j)
// from which dl/da, dl/db, dl/dd follow linearly (lct_grad_finalize): with
// x^2 = pi^2 m^2 / (8N) the derivatives of
//   L_jk = dx (2 pi i b)^{-1/2} e^{i 8 b d x_j^2/pi^2} e^{-i 4 x_j x_k / pi} e^{i a x_k^2/(2b)}
// give dl/da = -pi^2/(16 b N) SA,  dl/dd = -(b/N) SG,
//      dl/db = a pi^2/(16 b^2 N) SA - SR/(2b) - (d/N) SG.
//
// Layout: signal s starts at D.offset (batch plans) or at
// (s / P) * big + (s % P), with element stride es.  Rows: P = 1, big = N,
// es = 1.  Columns of a [fields][N][W] array: P = W, big = N W, es = W; then
// G = 4 (complex64) or 2 (complex128) adjacent columns share a CTA with
// interleaved lanes so that every warp access covers whole 32-byte sectors.
#include "xft_engine.cuh"
#include "xft_chirp.cuh"

namespace {

using namespace xft;

template <int L, class R>
__device__ __forceinline__ cpx<R> pre_g(const lct_desc& D, int n, bool decay) {
    if constexpr (sizeof(R) == 4) return pre_chirp<L>(D, n, decay);
    else return pre_chirp64<L>(D, n, decay);
}
template <int L, class R>
__device__ __forceinline__ cpx<R> post_g(const lct_desc& D, int n) {
    if constexpr (sizeof(R) == 4) return post_chirp<L>(D, n);
    else return post_chirp64<L>(D, n);
}
template <class R>
__device__ __forceinline__ cpx<R> conj_of(cpx<R> a) { return {a.x, -a.y}; }

// Signals per CTA: interleaved columns (G) or, for rows, enough signals to
// fill 256 threads.
template <int L, int G, int LE = 4>
struct gen_shape {
    static constexpr int T = shape<L, LE>::T;
    static constexpr int SPC = G > 1 ? G : (T >= 256 ? 1 : 256 / T);
    static constexpr int THREADS = T * SPC;
    // per-signal shared-memory stride: interleaved columns are offset by
    // 16 / G samples so that the G columns of a half-warp fall on different
    // banks (a multiple of 16 put them all on the same bank pairs)
    static constexpr int STR = shape<L, LE>::NP + (G > 1 ? 16 / G : 0);
};

// 768 resident threads (complex64, <= 85 registers) / 512 (complex128, 128).
// LE = 3 (8 samples per thread, complex64 columns): 1024 resident threads
// at <= 64 registers.
template <int L, class R, int G, int LE = 4>
constexpr int gen_min_blocks() {
    constexpr int per_sm = sizeof(R) == 4 ? (LE == 3 ? 1024 : 768) : 512;
    constexpr int b = per_sm / gen_shape<L, G, LE>::THREADS;
    return b < 1 ? 1 : (b > 16 ? 16 : b);
}

// LE: log2 of the samples per thread (4: radix-16 passes with the twiddle
// table; 3: radix-8 passes with twiddles computed in registers, used for
// complex64 columns to halve the registers per thread).
template <int L, class R, int G, bool ADJ, bool GRAD, int LE = 4>
__global__ void __launch_bounds__(gen_shape<L, G, LE>::THREADS, (gen_min_blocks<L, R, G, LE>()))
k_xft_gen(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
          const lct_desc* __restrict__ desc, int desc_step, int64_t count,
          const cpx<R>* __restrict__ tw, int64_t es, int64_t P, int64_t big,
          const cpx<R>* __restrict__ fwd_out, const cpx<R>* __restrict__ fwd_in,
          double* __restrict__ partial) {
    using S = shape<L, LE>;
    using F = gen_shape<L, G, LE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int sl = G > 1 ? tid % G : tid / S::T;
    const int i = G > 1 ? tid / G : tid - sl * S::T;
    const int64_t sig = (int64_t)blockIdx.x * F::SPC + sl;
    const bool active = sig < count;
    const lct_desc D = desc[desc_step && active ? sig : 0];
    // rows: unit stride, signal s at s * big; columns: (s / P) * big + (s % P), stride es
    const int64_t base = desc_step ? D.offset : (G > 1 ? (sig / P) * big + (sig % P) : sig * big);
    const int64_t est = G > 1 ? es : 1;
    cpx<R>* buf = smem + sl * F::STR;
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
    const R sc = (R)D.scale;

    R sa = 0, sr = 0, sg = 0;                 // sums in the sample precision
    cpx<R> v[S::E];
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int n = i + e * S::T;
        const int64_t at = base + (int64_t)n * est;
        cpx<R> x = {R(0), R(0)};
        if (active) x = ld_stream(in + at);
        if (ADJ) {
            if (GRAD && active) {
                const cpx<R> Gv = fwd_out[at];
                sr += x.x * Gv.x + x.y * Gv.y;                              // Re(conj(g) G)
                sg += (R)m_squared(n, S::N) * (x.x * Gv.y - x.y * Gv.x);     // m^2 Im(conj(g) G)
            }
            v[e] = cscale(cmul(x, conj_of(post_g<L, R>(D, n))), sc);
        } else {
            v[e] = cmul(x, pre_g<L, R>(D, n, decay));
        }
    }
    dft_signal<L, ADJ ? 1 : -1, LE == 3, LE>(v, buf, i, tw);
    if (active) {
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            const int64_t at = base + (int64_t)n * est;
            cpx<R> y;
            if (ADJ) {
                y = cmul(v[e], conj_of(pre_g<L, R>(D, n, decay)));
                if (GRAD) {
                    const cpx<R> fv = fwd_in[at];
                    sa += (R)m_squared(n, S::N) * (y.x * fv.y - y.y * fv.x);  // m^2 Im(conj(h) f)
                }
            } else {
                y = cscale(cmul(v[e], post_g<L, R>(D, n)), sc);
            }
            out[at] = y;
        }
    }
    if (GRAD) {
        // Reduce (sa, sr, sg) over the threads of each signal: shuffles
        // within a warp (sample precision), then the warps' partials in double.
        constexpr int SEG = G > 1 ? 32 : (S::T < 32 ? S::T : 32);   // lanes of one signal per warp
        if (G > 1) {
#pragma unroll
            for (int o = 16; o >= G; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                sg += __shfl_xor_sync(0xffffffffu, sg, o);
            }
        } else {
#pragma unroll
            for (int o = SEG / 2; o >= 1; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                sg += __shfl_xor_sync(0xffffffffu, sg, o);
            }
        }
        const int lane = tid & 31, warp = tid >> 5;
        if (G == 1 && S::T <= 32) {
            // every signal lies inside one warp: its first lane holds the total
            if (i == 0 && active) {
                partial[3 * sig + 0] = sa;
                partial[3 * sig + 1] = sr;
                partial[3 * sig + 2] = sg;
            }
        } else {
            __syncthreads();                   // shared memory free for the partials
            double* red = reinterpret_cast<double*>(smem_raw);
            constexpr int NW = F::THREADS / 32;
            if (G > 1) {
                if (lane < G) {
                    red[3 * (warp * G + lane) + 0] = sa;
                    red[3 * (warp * G + lane) + 1] = sr;
                    red[3 * (warp * G + lane) + 2] = sg;
                }
            } else if (lane == 0) {
                red[3 * warp + 0] = sa;
                red[3 * warp + 1] = sr;
                red[3 * warp + 2] = sg;
            }
            __syncthreads();
            if (i == 0 && active) {
                double a = 0, r = 0, g = 0;
                if (G > 1) {
                    for (int w = 0; w < NW; ++w) {
                        a += red[3 * (w * G + sl) + 0];
                        r += red[3 * (w * G + sl) + 1];
                        g += red[3 * (w * G + sl) + 2];
                    }
                } else {
                    const int w0 = (sl * S::T) >> 5, nw = S::T >> 5;
                    for (int w = w0; w < w0 + nw; ++w) {
                        a += red[3 * w + 0];
                        r += red[3 * w + 1];
                        g += red[3 * w + 2];
                    }
                }
                partial[3 * sig + 0] = a;
                partial[3 * sig + 1] = r;
                partial[3 * sig + 2] = g;
            }
        }
    }
}

template <int L, class R, int G, bool ADJ, bool GRAD, int LE = 4>
cudaError_t launch_gen(const void* in, void* out, const lct_desc* desc, int desc_step,
                       int64_t count, const void* tw, int64_t es, int64_t P, int64_t big,
                       const void* fwd_out, const void* fwd_in, double* partial,
                       cudaStream_t stream) {
    using S = shape<L, LE>;
    using F = gen_shape<L, G, LE>;
    size_t smem = S::P > 1 ? (size_t)F::SPC * F::STR * sizeof(cpx<R>) : 0;
    constexpr size_t red_bytes = (size_t)F::THREADS / 32 * (G > 1 ? G : 1) * 3 * sizeof(double) + 64;
    if (GRAD && smem < red_bytes) smem = red_bytes;
    auto kern = k_xft_gen<L, R, G, ADJ, GRAD, LE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (count + F::SPC - 1) / F::SPC;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, F::THREADS, smem, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)out, desc, desc_step, count, (const cpx<R>*)tw, es, P, big,
        (const cpx<R>*)fwd_out, (const cpx<R>*)fwd_in, partial);
    return cudaGetLastError();
}

// Complex64 columns: radix-8 engine, 4 interleaved columns per CTA (2 at
// N = 4096, so that a CTA stays within 1024 threads).
template <bool ADJ, bool GRAD>
cudaError_t gen_cols8(int log2n, const void* in, void* out, const lct_desc* desc, int desc_step,
                      int64_t count, int64_t es, int64_t P, int64_t big, const void* fo,
                      const void* fi, double* partial, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE8(L, G)                                                                          \
    case L:                                                                                      \
        return launch_gen<L, float, G, ADJ, GRAD, 3>(in, out, desc, desc_step, count, nullptr, es, \
                                                     P, big, fo, fi, partial, stream);
        LCT_CASE8(7, 4) LCT_CASE8(8, 4) LCT_CASE8(9, 4) LCT_CASE8(10, 4) LCT_CASE8(11, 4)
        LCT_CASE8(12, 2)
#undef LCT_CASE8
        default: return cudaErrorInvalidValue;
    }
}

template <class R, int G, bool ADJ, bool GRAD>
cudaError_t gen_dispatch(int log2n, const void* in, void* out, const lct_desc* desc, int desc_step,
                         int64_t count, const void* tw, int64_t es, int64_t P, int64_t big,
                         const void* fo, const void* fi, double* partial, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE(L)                                                                           \
    case L:                                                                                   \
        return launch_gen<L, R, G, ADJ, GRAD>(in, out, desc, desc_step, count, tw, es, P, big, \
                                             fo, fi, partial, stream);
        LCT_CASE(1) LCT_CASE(2) LCT_CASE(3) LCT_CASE(4) LCT_CASE(5) LCT_CASE(6)
        LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10) LCT_CASE(11) LCT_CASE(12)
#undef LCT_CASE
        default: return cudaErrorInvalidValue;
    }
}

template <class R, int G>
cudaError_t gen_mode(int log2n, bool adj, bool grad, const void* in, void* out,
                     const lct_desc* desc, int desc_step, int64_t count, const void* tw, int64_t es,
                     int64_t P, int64_t big, const void* fo, const void* fi, double* partial,
                     cudaStream_t stream) {
    if (!adj)
        return gen_dispatch<R, G, false, false>(log2n, in, out, desc, desc_step, count, tw, es, P,
                                                big, fo, fi, partial, stream);
    if (!grad)
        return gen_dispatch<R, G, true, false>(log2n, in, out, desc, desc_step, count, tw, es, P,
                                               big, fo, fi, partial, stream);
    return gen_dispatch<R, G, true, true>(log2n, in, out, desc, desc_step, count, tw, es, P, big,
                                          fo, fi, partial, stream);
}

// dl/da, dl/db, dl/dd from the sums (SA, SR, SG); coef: per signal
// (cA_a, cA_b, cR_b, cG_b, cG_d).  shared != 0: one parameter set for all
// signals, the sums are added first and grad has 3 entries.
constexpr int kFinalizeThreads = 1024;
constexpr int kFinalizeBlocks = 64;

__global__ void k_grad_finalize(const double* __restrict__ partial, const double* __restrict__ coef,
                                int coef_step, int64_t count, int shared, double* __restrict__ grad,
                                double* __restrict__ scratch) {
    if (!shared) {
        for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < count;
             s += (int64_t)gridDim.x * blockDim.x) {
            const double* c = coef + 5 * (coef_step ? s : 0);
            const double SA = partial[3 * s], SR = partial[3 * s + 1], SG = partial[3 * s + 2];
            grad[3 * s + 0] = c[0] * SA;
            grad[3 * s + 1] = c[1] * SA + c[2] * SR + c[3] * SG;
            grad[3 * s + 2] = c[4] * SG;
        }
        return;
    }
    // Shared parameters: CTA b sums its slice of the signals (four chains per
    // thread, then a tree), stores the slice total in scratch[3 b ..]; the
    // last CTA to finish adds the slice totals in slice order (deterministic)
    // and resets the ticket counter for the next launch.
    __shared__ double red[3][kFinalizeThreads];
    __shared__ bool last;
    const int64_t slice = (count + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = blockIdx.x * slice;
    const int64_t s1 = s0 + slice < count ? s0 + slice : count;
    double a[4] = {0, 0, 0, 0}, r[4] = {0, 0, 0, 0}, g[4] = {0, 0, 0, 0};
    int64_t s = s0 + threadIdx.x;
    for (; s + 3 * (int64_t)blockDim.x < s1; s += 4 * (int64_t)blockDim.x) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = s + u * (int64_t)blockDim.x;
            a[u] += partial[3 * t];
            r[u] += partial[3 * t + 1];
            g[u] += partial[3 * t + 2];
        }
    }
    for (; s < s1; s += blockDim.x) {
        a[0] += partial[3 * s];
        r[0] += partial[3 * s + 1];
        g[0] += partial[3 * s + 2];
    }
    red[0][threadIdx.x] = (a[0] + a[1]) + (a[2] + a[3]);
    red[1][threadIdx.x] = (r[0] + r[1]) + (r[2] + r[3]);
    red[2][threadIdx.x] = (g[0] + g[1]) + (g[2] + g[3]);
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + 3 * kFinalizeBlocks);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) scratch[3 * blockIdx.x + q] = red[q][0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const volatile double* v = scratch;
        double SA = 0, SR = 0, SG = 0;
        for (unsigned int b = 0; b < gridDim.x; ++b) {
            SA += v[3 * b];
            SR += v[3 * b + 1];
            SG += v[3 * b + 2];
        }
        grad[0] = coef[0] * SA;
        grad[1] = coef[1] * SA + coef[2] * SR + coef[3] * SG;
        grad[2] = coef[4] * SG;
        atomicExch(ticket, 0u);
    }
}

}  // namespace

// Interleaved columns need a CTA of at least one full warp (T G >= 32).
bool lct_gen_supported(int dtype, int log2n, int cols) {
    if (log2n < 1 || log2n > 12) return false;
    if (!cols) return true;
    return dtype == 0 ? log2n >= 7 : log2n >= 8;
}

// cols: 0 = rows (signals contiguous), 1 = interleaved columns.
cudaError_t lct_launch_gen(int dtype, int log2n, int cols, int adjoint, int grad, const void* in,
                           void* out, const lct_desc* desc, int desc_step, int64_t count,
                           const void* tw, int64_t es, int64_t P, int64_t big,
                           const void* fwd_out, const void* fwd_in, double* partial,
                           cudaStream_t stream) {
    if (dtype == 0) {
        if (cols) {
            if (!adjoint)
                return gen_cols8<false, false>(log2n, in, out, desc, desc_step, count, es, P, big,
                                               fwd_out, fwd_in, partial, stream);
            if (!grad)
                return gen_cols8<true, false>(log2n, in, out, desc, desc_step, count, es, P, big,
                                              fwd_out, fwd_in, partial, stream);
            return gen_cols8<true, true>(log2n, in, out, desc, desc_step, count, es, P, big,
                                         fwd_out, fwd_in, partial, stream);
        }
        return gen_mode<float, 1>(log2n, adjoint, grad, in, out, desc, desc_step, count, tw, es, P,
                                  big, fwd_out, fwd_in, partial, stream);
    }
    if (cols)
        return gen_mode<double, 2>(log2n, adjoint, grad, in, out, desc, desc_step, count, tw, es, P,
                                   big, fwd_out, fwd_in, partial, stream);
    return gen_mode<double, 1>(log2n, adjoint, grad, in, out, desc, desc_step, count, tw, es, P, big,
                               fwd_out, fwd_in, partial, stream);
}

cudaError_t lct_launch_grad_finalize(const double* partial, const double* coef, int coef_step,
                                     int64_t count, int shared, double* grad, double* scratch,
                                     cudaStream_t stream) {
    if (shared) {
        int64_t blocks = (count + 4095) / 4096;                 // at least 4096 signals per CTA
        if (blocks > kFinalizeBlocks) blocks = kFinalizeBlocks;
        if (blocks < 1) blocks = 1;
        k_grad_finalize<<<(unsigned)blocks, kFinalizeThreads, 0, stream>>>(
            partial, coef, coef_step, count, 1, grad, scratch);
    } else {
        k_grad_finalize<<<(unsigned)((count + 255) / 256 < 4096 ? (count + 255) / 256 : 4096), 256, 0,
                          stream>>>(partial, coef, coef_step, count, 0, grad, scratch);
    }
    return cudaGetLastError();
}

size_t lct_grad_finalize_scratch_bytes() { return (3 * kFinalizeBlocks + 1) * sizeof(double); }
