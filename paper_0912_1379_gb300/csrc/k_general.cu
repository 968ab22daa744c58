// General single-CTA XFT kernel (k_xft_gen): forward or adjoint transform,
// rows or columns, with optional parameter-gradient sums.  Used by
// lct_backward (adjoint + gradients) and by the separable 2-D transform.
// Complex64 columns of uniform parameters run the persistent form
// k_xft_cols (strips staged by cp.async, diagonal factors tabulated once per
// CTA); the gradient finalisation is k_grad_finalize.
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
#include "xft_async.cuh"

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
            // the warps' partials added in double by a shuffle tree (a fixed
            // order: deterministic).  Columns: warp 0, lane c + G r takes
            // column c's partials of warps r, r + 32/G, ...  Rows: the
            // signal's first warp, lane w its warp w (T/32 <= 32 warps).
            if (G > 1) {
                if (warp == 0) {
                    constexpr int SL = 32 / G;
                    const int c = lane % G, r = lane / G;
                    double a = 0, rs = 0, g = 0;
                    for (int w = r; w < NW; w += SL) {
                        a += red[3 * (w * G + c) + 0];
                        rs += red[3 * (w * G + c) + 1];
                        g += red[3 * (w * G + c) + 2];
                    }
#pragma unroll
                    for (int o = G; o < 32; o <<= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, o);
                        rs += __shfl_xor_sync(0xffffffffu, rs, o);
                        g += __shfl_xor_sync(0xffffffffu, g, o);
                    }
                    const int64_t sc = (int64_t)blockIdx.x * F::SPC + c;
                    if (r == 0 && sc < count) {
                        partial[3 * sc + 0] = a;
                        partial[3 * sc + 1] = rs;
                        partial[3 * sc + 2] = g;
                    }
                }
            } else if (i < 32) {
                constexpr int NWS = S::T / 32;             // warps per signal
                const int w0 = (sl * S::T) >> 5;
                double a = 0, rs = 0, g = 0;
                if (lane < NWS) {
                    a = red[3 * (w0 + lane) + 0];
                    rs = red[3 * (w0 + lane) + 1];
                    g = red[3 * (w0 + lane) + 2];
                }
#pragma unroll
                for (int o = 1; o < NWS; o <<= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    rs += __shfl_xor_sync(0xffffffffu, rs, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (i == 0 && active) {
                    partial[3 * sig + 0] = a;
                    partial[3 * sig + 1] = rs;
                    partial[3 * sig + 2] = g;
                }
            }
        }
    }
}

// Persistent form of the complex64 column kernel (radix-8 engine, G
// interleaved columns of one field per work item, uniform parameters).  With
// one 1024-thread CTA per SM the one-strip-per-CTA kernel cannot overlap an
// item's loads with another's arithmetic, so here each CTA copies the strip
// of its next item (N rows x G columns) into shared memory by cp.async while
// it transforms the current one.  The two diagonal factors, which are the
// same for every column, are tabulated once per CTA in shared memory.  With
// gradients the forward output and input are read directly.  Requires count
// and P = 2^lp to be multiples of G and 16-byte aligned strips (checked by
// the launcher).  The descriptor is passed by value: its words stay in the
// constant bank instead of registers.
template <int L, int G, bool GRAD>
struct cols_shape {
    static constexpr int LE = 3;
    using S = shape<L, LE>;
    using F = gen_shape<L, G, LE>;
    static constexpr int NT = F::THREADS, NW = NT / 32;
    // exchange buffers: one padding slot every 2^PS samples and column
    // buffers CO samples apart, chosen by enumerating the bank of every
    // lane's access in every exchange so that the G interleaved columns
    // exchange without bank conflicts (N = 1024: one 2-way store remains)
    static constexpr int PS = L == 11 ? 2 : 3;
    static constexpr int CO = L == 12 ? 8 : 4;
    static constexpr int STRC = S::N + (S::N >> PS) + CO;
    static constexpr size_t STAGE = (size_t)S::N * G;                // samples
    static constexpr size_t WORK = (size_t)G * STRC;
    static constexpr size_t CTAB = 2 * (size_t)S::N;
    static constexpr size_t SMEM = (STAGE + WORK + CTAB) * sizeof(cpx<float>) +
                                   (GRAD ? (size_t)NW * G * 3 * sizeof(double) : 0);
    static constexpr int MIN_BLOCKS = 1024 / NT > 0 ? 1024 / NT : 1;
};

// TWT: twiddles from the engine's table tw (else computed in registers).
template <int L, int G, bool ADJ, bool GRAD, bool TWT>
__global__ void __launch_bounds__(gen_shape<L, G, 3>::THREADS, (cols_shape<L, G, GRAD>::MIN_BLOCKS))
k_xft_cols(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out, const lct_desc D,
           int64_t count, int64_t es, int lp, int64_t big, const cpx<float>* __restrict__ tw,
           const cpx<float>* __restrict__ fwd_out, const cpx<float>* __restrict__ fwd_in,
           double* __restrict__ partial) {
    using C = cols_shape<L, G, GRAD>;
    using S = typename C::S;
    constexpr int NT = C::NT, NW = C::NW;
    constexpr int CPR = G / 2;                                // 16-byte chunks per strip row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* stage = reinterpret_cast<cpx<float>*>(smem_raw);     // [N][G]
    cpx<float>* work = stage + C::STAGE;                            // [G][STRC]
    cpx<float>* ctab = work + C::WORK;                              // [2][N]
    double* red = reinterpret_cast<double*>(ctab + C::CTAB);        // [NW][G][3] (gradients)
    const int tid = threadIdx.x;
    const int sl = tid % G, i = tid / G;
    const int64_t groups = count / G;
    const int64_t pm = ((int64_t)1 << lp) - 1;

    auto issue = [&](int64_t q) {
        const int64_t s0 = q * G;
        const int64_t b0 = (s0 >> lp) * big + (s0 & pm);
        for (int j = tid; j < S::N * CPR; j += NT) {
            const int n = j / CPR, h = j - n * CPR;
            xasync::cp_async16(stage + n * G + 2 * h, in + b0 + (int64_t)n * es + 2 * h);
        }
        xasync::cp_async_commit();
    };

    int64_t q = blockIdx.x;
    if (q < groups) issue(q);
    {
        // input-side and output-side factors of every sample index n
        const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
        const float sc = (float)D.scale;
        for (int n = tid; n < S::N; n += NT) {
            if (ADJ) {
                ctab[n] = cscale(conj_of(post_g<L, float>(D, n)), sc);
                ctab[S::N + n] = conj_of(pre_g<L, float>(D, n, decay));
            } else {
                ctab[n] = pre_g<L, float>(D, n, decay);
                ctab[S::N + n] = cscale(post_g<L, float>(D, n), sc);
            }
        }
    }
    for (; q < groups; q += gridDim.x) {
        xasync::cp_async_wait_all();
        __syncthreads();                  // strip q landed; the previous item is done with smem
        const int64_t sig = q * G + sl;
        const int64_t base = (sig >> lp) * big + (sig & pm);
        float sa = 0, sr = 0, sg = 0;
        cpx<float> v[S::E];
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            const int64_t at = base + (int64_t)n * es;
            const cpx<float> x = stage[n * G + sl];
            if (GRAD) {
                const cpx<float> Gv = fwd_out[at];
                sr += x.x * Gv.x + x.y * Gv.y;                                // Re(conj(g) G)
                sg += (float)m_squared(n, S::N) * (x.x * Gv.y - x.y * Gv.x);  // m^2 Im(conj(g) G)
            }
            v[e] = cmul(x, ctab[n]);
        }
        __syncthreads();                  // strip consumed: refill it with the next item
        if (q + gridDim.x < groups) {
            issue(q + gridDim.x);
            if (GRAD) {
                // the next item's rows of the forward output and input into L2
                const int64_t s1 = (q + gridDim.x) * G;
                const int64_t b1 = (s1 >> lp) * big + (s1 & pm);
                for (int n = tid; n < S::N; n += NT) {
                    xasync::prefetch_l2(fwd_out + b1 + (int64_t)n * es);
                    xasync::prefetch_l2(fwd_in + b1 + (int64_t)n * es);
                }
            }
        }
        dft_signal<L, ADJ ? 1 : -1, !TWT, 3, C::PS>(v, work + sl * C::STRC, i, tw);
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            const int64_t at = base + (int64_t)n * es;
            const cpx<float> y = cmul(v[e], ctab[S::N + n]);
            if (GRAD) {
                const cpx<float> fv = fwd_in[at];
                sa += (float)m_squared(n, S::N) * (y.x * fv.y - y.y * fv.x);      // m^2 Im(conj(h) f)
            }
            out[at] = y;
        }
        if (GRAD) {
            // per-column sums: shuffles over the lanes of a column, then the
            // warps' partials in double, in warp order
#pragma unroll
            for (int o = 16; o >= G; o >>= 1) {
                sa += __shfl_xor_sync(0xffffffffu, sa, o);
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                sg += __shfl_xor_sync(0xffffffffu, sg, o);
            }
            const int lane = tid & 31, warp = tid >> 5;
            if (lane < G) {
                red[3 * (warp * G + lane) + 0] = sa;
                red[3 * (warp * G + lane) + 1] = sr;
                red[3 * (warp * G + lane) + 2] = sg;
            }
            __syncthreads();
            if (warp == 0) {
                // warp 0 adds the warps' partials in double: lane c + G r
                // takes column c's partials of warps r, r + 32/G, ..., then
                // a shuffle tree over r (a fixed order: deterministic)
                constexpr int SL = 32 / G;
                const int c = lane % G, r = lane / G;
                double a = 0, rs = 0, g = 0;
                for (int w = r; w < NW; w += SL) {
                    a += red[3 * (w * G + c) + 0];
                    rs += red[3 * (w * G + c) + 1];
                    g += red[3 * (w * G + c) + 2];
                }
#pragma unroll
                for (int o = G; o < 32; o <<= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, o);
                    rs += __shfl_xor_sync(0xffffffffu, rs, o);
                    g += __shfl_xor_sync(0xffffffffu, g, o);
                }
                if (r == 0) {
                    const int64_t sc = q * G + c;
                    partial[3 * sc + 0] = a;
                    partial[3 * sc + 1] = rs;
                    partial[3 * sc + 2] = g;
                }
            }
        }
    }
    xasync::cp_async_wait_all();          // no copy left in flight at exit
}

template <int L, int G, bool ADJ, bool GRAD>
cudaError_t launch_cols(const void* in, void* out, const lct_desc& desc, int64_t count,
                        int64_t es, int lp, int64_t big, const void* tw, const void* fwd_out,
                        const void* fwd_in, double* partial, cudaStream_t stream) {
    using C = cols_shape<L, G, GRAD>;
    auto kern = tw ? k_xft_cols<L, G, ADJ, GRAD, true> : k_xft_cols<L, G, ADJ, GRAD, false>;
    static int per_sm[2][64] = {}, sms[64] = {};
    const int t = tw ? 1 : 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!per_sm[t][dev]) {
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)C::SMEM)) != cudaSuccess)
            return e;
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, C::NT, C::SMEM)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        per_sm[t][dev] = nb > 0 ? nb : 1;
    }
    const int64_t groups = count / G;
    const int64_t slots = (int64_t)per_sm[t][dev] * sms[dev];
    const int64_t grid = groups < slots ? groups : slots;
    if (grid <= 0) return cudaSuccess;
    kern<<<(unsigned)grid, C::NT, C::SMEM, stream>>>(
        (const cpx<float>*)in, (cpx<float>*)out, desc, count, es, lp, big, (const cpx<float>*)tw,
        (const cpx<float>*)fwd_out, (const cpx<float>*)fwd_in, partial);
    return cudaGetLastError();
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
                      int64_t count, const void* tw8, int64_t es, int64_t P, int64_t big,
                      const void* fo, const void* fi, double* partial, const lct_desc* host_desc,
                      cudaStream_t stream) {
    // the persistent staged kernel: uniform parameters known on the host,
    // whole groups of columns, P a power of two, 16-byte aligned strips
    const int G = log2n == 12 ? 2 : 4;
    int lp = 0;
    while (lp < 62 && ((int64_t)1 << lp) < P) ++lp;
    const bool staged = host_desc && desc_step == 0 && log2n >= 9 && ((int64_t)1 << lp) == P &&
                        count % G == 0 && P % G == 0 && es % 2 == 0 && big % 2 == 0 &&
                        ((uintptr_t)in) % 16 == 0;
    if (staged) {
        const lct_desc& hd = *host_desc;
        // twiddles: computed in registers without gradients (measured faster),
        // read from the radix-8 table with them (fewer registers)
        const void* tw8k = GRAD ? tw8 : nullptr;
        switch (log2n) {
            case 9: return launch_cols<9, 4, ADJ, GRAD>(in, out, hd, count, es, lp, big, tw8k, fo, fi, partial, stream);
            case 10: return launch_cols<10, 4, ADJ, GRAD>(in, out, hd, count, es, lp, big, tw8k, fo, fi, partial, stream);
            case 11: return launch_cols<11, 4, ADJ, GRAD>(in, out, hd, count, es, lp, big, tw8k, fo, fi, partial, stream);
            case 12: return launch_cols<12, 2, ADJ, GRAD>(in, out, hd, count, es, lp, big, tw8k, fo, fi, partial, stream);
            default: break;
        }
    }
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
                           const lct_desc* host_desc, cudaStream_t stream) {
    if (dtype == 0) {
        if (cols) {
            if (!adjoint)
                return gen_cols8<false, false>(log2n, in, out, desc, desc_step, count, tw, es, P,
                                               big, fwd_out, fwd_in, partial, host_desc, stream);
            if (!grad)
                return gen_cols8<true, false>(log2n, in, out, desc, desc_step, count, tw, es, P,
                                              big, fwd_out, fwd_in, partial, host_desc, stream);
            return gen_cols8<true, true>(log2n, in, out, desc, desc_step, count, tw, es, P, big,
                                         fwd_out, fwd_in, partial, host_desc, stream);
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
