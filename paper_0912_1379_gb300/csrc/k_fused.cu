// Fused XFT kernel: pre-chirp -> N-point DFT -> post-chirp + scale, with the
// whole signal resident in registers and shared memory, so each sample is
// read from HBM once and written once (Sec. 3, Algorithm, steps 1-3; the DFT
// with the forward sign, see include/lct.h).  The DFT is the Stockham engine
// of xft_engine.cuh; one CTA holds SPC signals (several for small N).
// Sizes: N = 2 .. 16384 (complex64), N = 2 .. 8192 (complex128).
#include "xft_engine.cuh"
#include "xft_async.cuh"
#include "xft_chirp.cuh"

namespace {

using namespace xft;

// ONE = false: several signals per CTA for small N (256 threads);
// ONE = true: one signal per CTA, for batches too small to give every SM a
// CTA of packed signals (latency: FP64 work spread over more SMs).
// LE: log2 of the samples per thread (4: radix-16 passes; 2: radix-4 passes
// with four times the threads per signal, for latency).
template <int L, bool ONE = false, int LE = 4>
struct fused_shape {
    static constexpr int T = shape<L, LE>::T;
    static constexpr int SPC = (T >= 256 || ONE) ? 1 : 256 / T;     // signals per CTA
    static constexpr int THREADS = T * SPC;
};

// Minimum resident CTAs per SM for __launch_bounds__: keeps FP32 kernels at
// <= 64 registers (1024 resident threads fill the 64K register file) and
// FP64 kernels at <= 128 (512 resident threads).
template <int L, class R, bool ONE = false, int LE = 4>
constexpr int min_blocks() {
    constexpr int per_sm = sizeof(R) == 4 ? 1024 : 512;
    constexpr int th = fused_shape<L, ONE, LE>::THREADS;
    constexpr int b = per_sm / th > 0 ? per_sm / th : 1;
    return b > 32 ? 32 : b;
}

template <int L, class R, bool ONE, int LE>
__global__ void __launch_bounds__(fused_shape<L, ONE, LE>::THREADS, (min_blocks<L, R, ONE, LE>()))
k_xft_fused(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
            const lct_desc* __restrict__ desc, int desc_step, int64_t count,
            const cpx<R>* __restrict__ tw, const int32_t* __restrict__ idx,
            int32_t* __restrict__ status) {
    using S = shape<L, LE>;
    using F = fused_shape<L, ONE, LE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x;
    const int sl = tid / S::T;
    const int i = tid - sl * S::T;
    const int64_t sig = (int64_t)blockIdx.x * F::SPC + sl;
    bool active = sig < count;
    // idx (ragged batches): this launch's signal s is descriptor idx[s]; a
    // descriptor that does not match the kernel is flagged, not transformed.
    const int64_t gsig = idx ? (active ? idx[sig] : 0) : sig;
    const lct_desc D = desc[desc_step && active ? gsig : 0];
    if (idx && active && (D.log2n != L || D.kind != LCT_KIND_XFT || D.offset < 0)) {
        if (i == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        active = false;
    }
    const int64_t base = desc_step ? D.offset : sig * (int64_t)S::N;
    cpx<R>* buf = smem + sl * S::NP;
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;

    cpx<R> v[S::E];
    // global load (coalesced: sample i + e T) with the pre-chirp
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int n = i + e * S::T;
        cpx<R> f = {R(0), R(0)};
        if (active) f = ld_stream(in + base + n);
        v[e] = cmul(f, pre_w<L, R>(D, n, decay));
    }
    // signals of at most 32 consecutive threads synchronise their warp only
    // (CTAs of whole warps; a CTA smaller than a warp keeps the CTA barrier)
    if constexpr (S::T <= 32 && F::THREADS % 32 == 0) dft_signal_warp<L, -1, false, LE>(v, buf, i, tw);
    else dft_signal<L, -1, false, LE>(v, buf, i, tw);
    // global store (sample i + e T) with the post-chirp and scale
    if (active) {
        const R sc = (R)D.scale;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            out[base + n] = cscale(cmul(v[e], post_w<L, R>(D, n)), sc);
        }
    }
}

// Persistent variant (complex64): each CTA loops over groups of SPC signals.
// The next group's samples are brought into a shared-memory stage by bulk
// asynchronous copies (cp.async.bulk, completing on an mbarrier) while the
// current group is transformed, so HBM latency is hidden behind compute.
// Requires 16-byte aligned signal starts (checked on the host).
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s

template <int L>
__device__ __forceinline__ void issue_group(const cpx<float>* in, const lct_desc* desc,
                                            int desc_step, int64_t count, int64_t g,
                                            cpx<float>* stage, uint64_t* bar) {
    using S = shape<L>;
    using F = fused_shape<L>;
    uint32_t bytes = 0;
    for (int s = 0; s < F::SPC; ++s)
        if (g * F::SPC + s < count) bytes += S::N * (uint32_t)sizeof(cpx<float>);
    xasync::mbar_arrive_expect_tx(bar, bytes);
    for (int s = 0; s < F::SPC; ++s) {
        const int64_t sig = g * F::SPC + s;
        if (sig >= count) break;
        const int64_t base = desc_step ? desc[sig].offset : sig * (int64_t)S::N;
        xasync::bulk_g2s(stage + s * S::N, in + base, S::N * (uint32_t)sizeof(cpx<float>), bar);
    }
}

// 3 CTAs fit per SM by shared memory (about 67 KB each) up to N = 4096.
// TWC: compute twiddles instead of reading the table (with ~200 KB of shared
// memory per SM the L1 left over may not hold the table).
template <int L, bool TWC>
__global__ void __launch_bounds__(fused_shape<L>::THREADS, (L <= 12 ? 3 : 1))
k_xft_fused_tma(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                const cpx<float>* __restrict__ tw, int32_t* __restrict__ status) {
    using S = shape<L>;
    using F = fused_shape<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* stage = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* work = stage + F::SPC * S::N;
    uint64_t* bar = reinterpret_cast<uint64_t*>(work + F::SPC * S::NP);
    const int64_t groups = (count + F::SPC - 1) / F::SPC;
    int64_t g = blockIdx.x;
    if (g >= groups) return;
    const int tid = threadIdx.x;
    const int sl = tid / S::T;
    const int i = tid - sl * S::T;
    cpx<float>* buf = work + sl * S::NP;
    if (tid == 0) {
        xasync::mbar_init(bar, 1);
        xasync::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) issue_group<L>(in, desc, desc_step, count, g, stage, bar);
    uint32_t parity = 0;
    for (; g < groups; g += gridDim.x) {
        bool ok = true;
        if (tid == 0) ok = xasync::mbar_wait(bar, parity, kWaitLimitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
                xasync::mbar_wait(bar, parity, kWaitLimitNs);   // let the copy in flight land
            }
            return;
        }
        parity ^= 1u;
        const int64_t sig = g * F::SPC + sl;
        const bool active = sig < count;
        const lct_desc D = desc[desc_step && active ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * (int64_t)S::N;
        const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
        cpx<float> v[S::E];
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            cpx<float> f = {0.f, 0.f};
            if (active) f = stage[sl * S::N + n];
            v[e] = cmul(f, pre_w<L, float>(D, n, decay));
        }
        __syncthreads();                       // stage fully read
        if (tid == 0 && g + gridDim.x < groups) {
            xasync::fence_proxy_async_smem();
            issue_group<L>(in, desc, desc_step, count, g + gridDim.x, stage, bar);
        }
        dft_signal<L, -1, TWC>(v, buf, i, tw);
        if (active) {
            const float sc = (float)D.scale;
#pragma unroll
            for (int e = 0; e < S::E; ++e) {
                const int n = i + e * S::T;
                out[base + n] = cscale(cmul(v[e], post_w<L, float>(D, n)), sc);
            }
        }
    }
}

template <int L, bool TWC>
cudaError_t launch_tma(const void* in, void* out, const lct_desc* desc, int desc_step,
                       int64_t count, const void* tw, int32_t* status, cudaStream_t stream) {
    using S = shape<L>;
    using F = fused_shape<L>;
    const size_t smem = (size_t)F::SPC * (S::N + S::NP) * sizeof(cpx<float>) + 16;
    auto kern = k_xft_fused_tma<L, TWC>;
    static int blocks_per_sm[64] = {};
    static int sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!blocks_per_sm[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, F::THREADS, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        blocks_per_sm[dev] = nb > 0 ? nb : 1;
    }
    const int64_t groups = (count + F::SPC - 1) / F::SPC;
    int64_t grid = (int64_t)blocks_per_sm[dev] * sms[dev];
    if (grid > groups) grid = groups;
    kern<<<(unsigned)grid, F::THREADS, smem, stream>>>(
        (const cpx<float>*)in, (cpx<float>*)out, desc, desc_step, count, (const cpx<float>*)tw, status);
    return cudaGetLastError();
}

template <int L, class R, bool ONE, int LE = 4>
cudaError_t launch_shape(const void* in, void* out, const lct_desc* desc, int desc_step,
                         int64_t count, const void* tw, const int32_t* idx, int32_t* status,
                         cudaStream_t stream) {
    using S = shape<L, LE>;
    using F = fused_shape<L, ONE, LE>;
    const size_t smem = S::P > 1 ? (size_t)F::SPC * S::NP * sizeof(cpx<R>) : 0;
    auto kern = k_xft_fused<L, R, ONE, LE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (count + F::SPC - 1) / F::SPC;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, F::THREADS, smem, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)out, desc, desc_step, count, (const cpx<R>*)tw, idx, status);
    return cudaGetLastError();
}

// Multiprocessors of the current device (cached per device).
int sm_count() {
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!sms[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        sms[dev] = n;
    }
    return sms[dev];
}

// Packed signals per CTA, unless that leaves SMs idle: then one signal per
// CTA, so that a small batch (the 12-signal FP64 case, say) runs on as many
// SMs as it has signals.  FP64 signals then also take four samples per
// thread (radix-4 passes, four times the threads), which shortens each
// thread's chain of FP64 phase and butterfly arithmetic (uniform plans; the
// radix-4 twiddle table is created here, outside any graph capture).
template <int L, class R>
cudaError_t launch_one(const void* in, void* out, const lct_desc* desc, int desc_step,
                       int64_t count, const void* tw, const int32_t* idx, int32_t* status,
                       cudaStream_t stream) {
    if constexpr (fused_shape<L>::SPC > 1) {
        const int64_t packed = (count + fused_shape<L>::SPC - 1) / fused_shape<L>::SPC;
        if (packed < sm_count()) {
            if constexpr (sizeof(R) == 8 && L >= 5) {
                if (!idx) {
                    const void* tw4 = lct_twiddle_table_le(1, L, 2);
                    if (!tw4) return cudaErrorMemoryAllocation;
                    return launch_shape<L, R, true, 2>(in, out, desc, desc_step, count, tw4, idx,
                                                       status, stream);
                }
            }
            return launch_shape<L, R, true>(in, out, desc, desc_step, count, tw, idx, status,
                                            stream);
        }
    }
    return launch_shape<L, R, false>(in, out, desc, desc_step, count, tw, idx, status, stream);
}

template <class R>
cudaError_t launch_dispatch(int log2n, const void* in, void* out, const lct_desc* desc,
                            int desc_step, int64_t count, const void* tw, const int32_t* idx,
                            int32_t* status, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_one<L, R>(in, out, desc, desc_step, count, tw, idx, status, stream);
        LCT_CASE(1) LCT_CASE(2) LCT_CASE(3) LCT_CASE(4) LCT_CASE(5) LCT_CASE(6)
        LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10) LCT_CASE(11) LCT_CASE(12)
        LCT_CASE(13)
#undef LCT_CASE
        case 14:
            if constexpr (sizeof(R) == 4)
                return launch_one<14, R>(in, out, desc, desc_step, count, tw, idx, status, stream);
            return cudaErrorInvalidValue;
        default: return cudaErrorInvalidValue;
    }
}

// Explicit schedules for the autotuner: radix-8 passes (LE = 3, twice the
// threads of the radix-16 schedule, packed signals per CTA), or one signal
// per CTA with radix-16 passes (LE = 4) or, FP64, radix-4 passes (LE = 2).
template <class R>
cudaError_t sched_dispatch(int log2n, int le, bool one, const void* in, void* out,
                           const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                           const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (le == 3 && !one) {
        switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_shape<L, R, false, 3>(in, out, desc, desc_step, count, tw, idx, status, stream);
            LCT_CASE(4) LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10)
            LCT_CASE(11) LCT_CASE(12) LCT_CASE(13)
#undef LCT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    if (le == 2 && one) {
        switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_shape<L, R, true, 2>(in, out, desc, desc_step, count, tw, idx, status, stream);
            LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10) LCT_CASE(11)
#undef LCT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    if (le == 4 && one) {
        switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_shape<L, R, true, 4>(in, out, desc, desc_step, count, tw, idx, status, stream);
            LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10) LCT_CASE(11)
#undef LCT_CASE
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool lct_fused_sched_supported(int dtype, int log2n, int le, int one) {
    if (le == 3 && !one) return log2n >= 4 && log2n <= 13;
    if (le == 2 && one) return dtype == 1 && log2n >= 5 && log2n <= 11;
    // from N = 4096 the packed shape already holds one signal per CTA
    if (le == 4 && one) return log2n >= 5 && log2n <= 11;
    return false;
}

cudaError_t lct_launch_fused_sched(int dtype, int log2n, int le, int one, const void* in, void* out,
                                   const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                                   const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (!lct_fused_sched_supported(dtype, log2n, le, one)) return cudaErrorInvalidValue;
    if (dtype == 0)
        return sched_dispatch<float>(log2n, le, one != 0, in, out, desc, desc_step, count, tw, idx,
                                     status, stream);
    return sched_dispatch<double>(log2n, le, one != 0, in, out, desc, desc_step, count, tw, idx,
                                  status, stream);
}

bool lct_fused_tma_supported(int dtype, int log2n) {
    return dtype == 0 && log2n >= 8 && log2n <= 13;
}

template <bool TWC>
cudaError_t tma_dispatch(int log2n, const void* in, void* out, const lct_desc* desc,
                         int desc_step, int64_t count, const void* tw, int32_t* status,
                         cudaStream_t stream) {
    switch (log2n) {
        case 8: return launch_tma<8, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        case 9: return launch_tma<9, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        case 10: return launch_tma<10, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        case 11: return launch_tma<11, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        case 12: return launch_tma<12, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        case 13: return launch_tma<13, TWC>(in, out, desc, desc_step, count, tw, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t lct_launch_fused_tma(int dtype, int log2n, const void* in, void* out,
                                 const lct_desc* desc, int desc_step, int64_t count,
                                 const void* tw, int32_t* status, int twiddle_compute,
                                 cudaStream_t stream) {
    if (dtype != 0) return cudaErrorInvalidValue;
    if (twiddle_compute)
        return tma_dispatch<true>(log2n, in, out, desc, desc_step, count, tw, status, stream);
    return tma_dispatch<false>(log2n, in, out, desc, desc_step, count, tw, status, stream);
}

bool lct_fused_supported(int dtype, int log2n) {
    return log2n >= 1 && log2n <= (dtype == 0 ? 14 : 13);
}

cudaError_t lct_launch_fused(int dtype, int log2n, const void* in, void* out,
                             const lct_desc* desc, int desc_step, int64_t count, const void* tw,
                             const int32_t* idx, int32_t* status, cudaStream_t stream) {
    if (dtype == 0)
        return launch_dispatch<float>(log2n, in, out, desc, desc_step, count, tw, idx, status,
                                      stream);
    return launch_dispatch<double>(log2n, in, out, desc, desc_step, count, tw, idx, status, stream);
}
