// XFT for N = 2^a 3^b 5^c 7^d that is not a power of two: the Algorithm of
// Sec. 3 with its DFT ("any FFT") as a mixed-radix Stockham transform in one
// CTA, so each sample is read from HBM once and written once and no padding
// to a power of two (nor a second transform, as in the chirp convolution) is
// paid.
//
// The factorisation's kernel e^{-i pi m_j m_k / (2N)} (m = 2k - N + 1) is the
// DFT kernel e^{-2 pi i jk/N} times the centring phases e^{i pi (N-1) k/N},
// e^{i pi (N-1) j/N} and the constant e^{-i pi (N-1)^2/(2N)}, so
//   u_k = e^{2 pi i [phi_in m_k^2 + (N-1) k/(2N)]} e^{-decay m_k^2} f_k
//   U   = DFT_N(u)
//   G_j = scale e^{2 pi i [phi_out m_j^2 + (N-1) j/(2N) + c_out]} U_j
// (kind LCT_KIND_MIXED, lct_internal.h).  The centring turn (N-1)k/(2N) is
// r/(2N) with r = ((N-1) k) mod 2N = (N (k mod 2) - k) mod 2N, formed from a
// 128-bit fixed-point 1/(2N).
//
// DFT: passes p = 0..P-1 of radix R_p (16, 8, 4, 2, 7, 5, 3), Ns_p the
// product of the earlier radices; butterfly b < N/R_p of pass p reads
// x[b + r N/R_p] (r < R_p), multiplies by e^{-2 pi i j r/(Ns_p R_p)}
// (j = b mod Ns_p, from a table), takes the R_p-point DFT and writes
// y[(b - j) R_p + j + s Ns_p] (s < R_p): Stockham's self-sorting order, so
// the last pass writes U_j in natural order.  Pass 0 reads HBM (with the
// input chirp), the last pass writes HBM (with the output chirp), the
// others run in shared memory in place (one pad slot per 16 samples): each
// thread loads all of its butterflies' inputs into registers, the CTA
// synchronises, then stores.
// A thread owns K_R = 16/R butterflies of a pass (at most 16 samples in
// registers), so T >= N/14 threads per signal cover every pass.
#include "xft_engine.cuh"

namespace {

using namespace xft;

// ---- small DFTs of odd prime radix, forward sign: pair form ----------------
// y_k = x_0 + sum_{n=1}^{(R-1)/2} [cos(2 pi k n/R)(x_n + x_{R-n})
//                                 - i sin(2 pi k n/R)(x_n - x_{R-n})]
template <class R>
__device__ __forceinline__ void dft3f(cpx<R>* a) {
    const R h = kconst<R>(-0.5), s = kconst<R>(0.86602540378443864676);   // sin(2 pi/3)
    const cpx<R> p = a[1] + a[2], d = a[1] - a[2];
    const cpx<R> t = {madd(h, p.x, a[0].x), madd(h, p.y, a[0].y)};
    a[0] = a[0] + p;
    // -i s d = (s d.y, -s d.x)
    a[1] = {madd(s, d.y, t.x), madd(-s, d.x, t.y)};
    a[2] = {madd(-s, d.y, t.x), madd(s, d.x, t.y)};
}

template <class R>
__device__ __forceinline__ void dft5f(cpx<R>* a) {
    const R c1 = kconst<R>(0.30901699437494742410), c2 = kconst<R>(-0.80901699437494742410);
    const R s1 = kconst<R>(0.95105651629515357212), s2 = kconst<R>(0.58778525229247312917);
    const cpx<R> p1 = a[1] + a[4], d1 = a[1] - a[4], p2 = a[2] + a[3], d2 = a[2] - a[3];
    const cpx<R> x0 = a[0];
    // real-coefficient parts
    const cpx<R> t1 = {madd(c1, p1.x, madd(c2, p2.x, x0.x)), madd(c1, p1.y, madd(c2, p2.y, x0.y))};
    const cpx<R> t2 = {madd(c2, p1.x, madd(c1, p2.x, x0.x)), madd(c2, p1.y, madd(c1, p2.y, x0.y))};
    // sine parts: q1 = s1 d1 + s2 d2, q2 = s2 d1 - s1 d2
    const cpx<R> q1 = {madd(s1, d1.x, s2 * d2.x), madd(s1, d1.y, s2 * d2.y)};
    const cpx<R> q2 = {madd(s2, d1.x, -s1 * d2.x), madd(s2, d1.y, -s1 * d2.y)};
    a[0] = x0 + p1 + p2;
    // y1 = t1 - i q1, y4 = t1 + i q1, y2 = t2 - i q2, y3 = t2 + i q2
    a[1] = {t1.x + q1.y, t1.y - q1.x};
    a[4] = {t1.x - q1.y, t1.y + q1.x};
    a[2] = {t2.x + q2.y, t2.y - q2.x};
    a[3] = {t2.x - q2.y, t2.y + q2.x};
}

template <class R>
__device__ __forceinline__ void dft7f(cpx<R>* a) {
    // cos / sin of 2 pi n / 7, n = 1, 2, 3
    const double C[3] = {0.62348980185873353053, -0.22252093395631440429, -0.90096886790241912624};
    const double S[3] = {0.78183148246802980871, 0.97492791218182360702, 0.43388373911755812048};
    cpx<R> p[3], d[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        p[n] = a[n + 1] + a[6 - n];
        d[n] = a[n + 1] - a[6 - n];
    }
    const cpx<R> x0 = a[0];
    a[0] = x0 + p[0] + p[1] + p[2];
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        cpx<R> t = x0, q = {R(0), R(0)};
#pragma unroll
        for (int n = 1; n <= 3; ++n) {
            const int kn = (k * n) % 7;                 // cos(2 pi kn/7) = C[min(kn, 7-kn)-1]
            const int idx = kn <= 3 ? kn : 7 - kn;
            const R c = kconst<R>(C[idx - 1]);
            const R s = kconst<R>(kn <= 3 ? S[idx - 1] : -S[idx - 1]);
            t = {madd(c, p[n - 1].x, t.x), madd(c, p[n - 1].y, t.y)};
            q = {madd(s, d[n - 1].x, q.x), madd(s, d[n - 1].y, q.y)};
        }
        a[k] = {t.x + q.y, t.y - q.x};                  // t - i q
        a[7 - k] = {t.x - q.y, t.y + q.x};              // t + i q
    }
}

template <int RAD, class R>
__device__ __forceinline__ void dft_fwd(cpx<R>* a) {
    if constexpr (RAD == 3) dft3f(a);
    else if constexpr (RAD == 5) dft5f(a);
    else if constexpr (RAD == 7) dft7f(a);
    else dft<RAD, -1>(a);
}

template <int RAD>
struct mx_k {
    static constexpr int K = 16 / RAD;         // butterflies per thread and pass
};

// Shared-memory position of sample e: one pad slot per 16 samples, so that
// the stride-R stores of the early passes (R up to 16) fall on distinct
// banks within each half-warp.
__device__ __forceinline__ int mx_pad(int e) { return e + (e >> 4); }

// Exchange barrier: a signal of 32 threads is one warp (slices start at
// multiples of T), which then synchronises alone; wider signals use the CTA
// barrier.  T is the same for every thread of the launch.
__device__ __forceinline__ void mx_sync(int T) {
    if (T == 32) __syncwarp();
    else __syncthreads();
}

// Exact turn of the chirp and centring at sample k (m = 2k - n + 1).
template <class R>
__device__ __forceinline__ cpx<R> mx_chirp(uint64_t phi_hi, uint64_t phi_lo, uint64_t inv_hi,
                                           uint64_t inv_lo, uint64_t off, int k, int n) {
    const uint32_t m2 = m_squared(k, n);
    int r = ((k & 1) ? n : 0) - k;
    if (r < 0) r += 2 * n;
    if constexpr (sizeof(R) == 4) {
        const uint32_t t = phase32(phi_hi, m2) + phase32(inv_hi, (uint32_t)r) +
                           (uint32_t)((off + 0x80000000ull) >> 32);
        return expi_turn32<true>(t);
    } else {
        return expi_turn64(phase64(phi_hi, phi_lo, m2) + phase64(inv_hi, inv_lo, (uint32_t)r) + off);
    }
}

// One pass p of radix RAD: reads HBM (with the input chirp) when it is the
// first pass, else shared memory; writes HBM (with the output chirp and
// scale) when it is the last, else shared memory.
template <int RAD, class R>
__device__ __forceinline__ void mx_pass(const lct_mixed_plan& pl, int p, cpx<R>* buf, int i, int T,
                                        const cpx<R>* __restrict__ gin, cpx<R>* __restrict__ gout,
                                        const lct_desc* Dp, bool active,
                                        const cpx<R>* __restrict__ tw) {
    constexpr int K = mx_k<RAD>::K;
    const bool first = p == 0, last = p == pl.npass - 1;
    const int n = pl.n;
    const int nb = n / RAD;
    const int ns = pl.ns[p];
    const uint32_t magic = pl.magic[p];
    const cpx<R>* twp = tw + pl.twoff[p];
    cpx<R> v[K][RAD];
    if (first) {
        const uint64_t phi_hi = Dp->in_hi, phi_lo = Dp->in_lo;
        const bool decay = (Dp->flags & LCT_FLAG_DECAY) != 0;
        const double dec = Dp->decay;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = i + k * T;
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                const int src = b + r * nb;
                cpx<R> x = {R(0), R(0)};
                if (active && b < nb) {
                    x = ld_stream(gin + src);
                    cpx<R> w = mx_chirp<R>(phi_hi, phi_lo, pl.inv_hi, pl.inv_lo, 0, src, n);
                    if (decay) {
                        const uint32_t m2 = m_squared(src, n);
                        if constexpr (sizeof(R) == 4) w = cscale(w, expf(-(float)dec * (float)m2));
                        else w = cscale(w, exp(-dec * (double)m2));
                    }
                    x = cmul(x, w);
                }
                v[k][r] = x;
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = i + k * T;
            const int q = (int)__umulhi((uint32_t)b, magic);
            const int j = b - q * ns;
#pragma unroll
            for (int r = 0; r < RAD; ++r) {
                cpx<R> x = {R(0), R(0)};
                if (b < nb) {
                    x = buf[mx_pad(b + r * nb)];
                    if (r > 0) x = cmul(x, ld_tw<R>(twp + (r - 1) * ns + j));
                }
                v[k][r] = x;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) dft_fwd<RAD>(v[k]);
    if (!last) {
        if (!first) mx_sync(T);                      // every input read before any output
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = i + k * T;
            if (b < nb) {
                const int q = ns > 1 ? (int)__umulhi((uint32_t)b, magic) : b;
                const int j = b - q * ns;
                const int o = q * ns * RAD + j;
#pragma unroll
                for (int s = 0; s < RAD; ++s) buf[mx_pad(o + s * ns)] = v[k][s];
            }
        }
        mx_sync(T);
    } else if (active) {
        // last pass: ns * RAD = n, so b < ns and the output index is b + s ns
        const uint64_t out_hi = Dp->out_hi, out_lo = Dp->out_lo, out_c = Dp->out_c;
        const R sc = (R)Dp->scale;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int b = i + k * T;
            if (b < nb) {
#pragma unroll
                for (int s = 0; s < RAD; ++s) {
                    const int jo = b + s * nb;
                    const cpx<R> w = mx_chirp<R>(out_hi, out_lo, pl.inv_hi, pl.inv_lo, out_c, jo, n);
                    gout[jo] = cscale(cmul(v[k][s], w), sc);
                }
            }
        }
    }
}

// SPC slices of pl.threads threads, one signal each; buffer of n samples per slice.
template <class R>
__global__ void __launch_bounds__(sizeof(R) == 4 ? 1024 : 512)
k_xft_mixed(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, const lct_desc* __restrict__ desc,
            int desc_step, int64_t count, const lct_mixed_plan* __restrict__ plp,
            const int32_t* __restrict__ idx, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the plan sits in device memory at the head of the twiddle buffer (its
    // arrays are indexed by the pass number, which kernel parameters are not
    // cheaply)
    __shared__ lct_mixed_plan pl;                       // the plan, read once per CTA
    if (threadIdx.x < sizeof(lct_mixed_plan) / 4)
        reinterpret_cast<uint32_t*>(&pl)[threadIdx.x] = reinterpret_cast<const uint32_t*>(plp)[threadIdx.x];
    __syncthreads();
    const cpx<R>* __restrict__ tw =
        reinterpret_cast<const cpx<R>*>(reinterpret_cast<const char*>(plp) + kMixedPlanBytes);
    const int T = pl.threads;
    const int spc = blockDim.x / T;
    const int sl = threadIdx.x / T, i = threadIdx.x - sl * T;
    const int64_t sig = (int64_t)blockIdx.x * spc + sl;
    bool active = sig < count;
    const int64_t gsig = idx ? (active ? idx[sig] : 0) : sig;
    const lct_desc* Dp = desc + (desc_step && active ? gsig : 0);
    if (active && (Dp->kind != LCT_KIND_MIXED || Dp->n != pl.n || Dp->offset < 0)) {
        if (i == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        active = false;
    }
    const int64_t base = desc_step ? Dp->offset : sig * (int64_t)pl.n;
    cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw) + (size_t)sl * (pl.n + (pl.n >> 4) + 1);
    const cpx<R>* gin = in + (active ? base : 0);
    cpx<R>* gout = out + (active ? base : 0);
    // the plan lists the passes as 16s, one 8, 4 or 2, then 7s, 5s, 3s: one
    // loop per radix, so that every loop body is a single pass kind (a loop
    // over a switch of all of them kept the sample arrays out of registers)
    int p = 0;
    const int P = pl.npass;
#define MX_LOOP(RR)                                                        \
    while (p < P && pl.radix[p] == RR) {                                   \
        mx_pass<RR>(pl, p, buf, i, T, gin, gout, Dp, active, tw);          \
        ++p;                                                               \
    }
    MX_LOOP(16) MX_LOOP(8) MX_LOOP(4) MX_LOOP(2) MX_LOOP(7) MX_LOOP(5) MX_LOOP(3)
#undef MX_LOOP
}

}  // namespace

int lct_mixed_threads_per_cta(const lct_mixed_plan& pl) {
    const int spc = pl.threads >= 256 ? 1 : 256 / pl.threads;
    return spc * pl.threads;
}

cudaError_t lct_launch_mixed(int dtype, const lct_mixed_plan& pl, const void* in, void* out,
                             const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                             const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if (!tw || pl.npass < 1 || pl.threads < 32 || pl.threads > (dtype == 0 ? 1024 : 512))
        return cudaErrorInvalidValue;
    const int threads = lct_mixed_threads_per_cta(pl);
    const int spc = threads / pl.threads;
    const size_t es = dtype == 0 ? sizeof(cpx<float>) : sizeof(cpx<double>);
    const size_t smem = (size_t)spc * (pl.n + (pl.n >> 4) + 1) * es;
    const int64_t blocks = (count + spc - 1) / spc;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (dtype == 0) {
        auto kern = k_xft_mixed<float>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(unsigned)blocks, threads, smem, stream>>>((const cpx<float>*)in, (cpx<float>*)out, desc,
                                                          desc_step, count, (const lct_mixed_plan*)tw, idx,
                                                          status);
    } else {
        auto kern = k_xft_mixed<double>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<(unsigned)blocks, threads, smem, stream>>>((const cpx<double>*)in, (cpx<double>*)out, desc,
                                                          desc_step, count, (const lct_mixed_plan*)tw, idx,
                                                          status);
    }
    return cudaGetLastError();
}
