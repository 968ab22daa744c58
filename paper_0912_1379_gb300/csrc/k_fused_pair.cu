// Paired fused XFT kernel (complex64): every thread transforms the same
// sample positions of TWO signals at once, holding the real parts of both in
// one packed FP32 register pair and the imaginary parts in another, so that
// each butterfly addition, twiddle product and scaling of the DFT is a single
// f32x2 instruction for two samples.  The chirp phases stay exact per signal
// (integer turn fractions, one sine/cosine each).  Same data flow as
// k_xft_fused: one HBM read and one HBM write per sample, Stockham passes of
// xft_engine.cuh on cpx<pf> values, shared-memory exchanges of 16-byte pairs.
// The twiddle table is the broadcast form of the FP32 table: entry
// {(wx, wx), (wy, wy)} (lct_twiddle_table_pair).
#include "xft_engine.cuh"
#include "xft_chirp.cuh"
#include "xft_async.cuh"

namespace {

using namespace xft;

template <int L, int LE = 4>
struct pair_shape {
    static constexpr int T = shape<L, LE>::T;
    static constexpr int PPC = T >= 256 ? 1 : 256 / T;     // signal pairs per CTA
    static constexpr int THREADS = T * PPC;
    static constexpr int PS = LE == 3 ? 3 : 4;              // padding shift (16-byte samples)
    static constexpr int NP = padded_len<L, PS>();
};

__device__ __forceinline__ cpx<pf> pack(cpx<float> a, cpx<float> b) {
    return {pf_make(a.x, b.x), pf_make(a.y, b.y)};
}

template <int L, int MINB, int LE = 4>
__global__ void __launch_bounds__(pair_shape<L, LE>::THREADS, MINB)
k_xft_pair(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
           const lct_desc* __restrict__ desc, int desc_step, int64_t count,
           const cpx<pf>* __restrict__ tw) {
    using S = shape<L, LE>;
    using F = pair_shape<L, LE>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<pf>* smem = reinterpret_cast<cpx<pf>*>(smem_raw);
    const int tid = threadIdx.x;
    const int sl = tid / S::T;
    const int i = tid - sl * S::T;
    const int64_t sa = ((int64_t)blockIdx.x * F::PPC + sl) * 2;   // signal A; B = A + 1
    const bool act_a = sa < count, act_b = sa + 1 < count;
    const lct_desc DA = desc[desc_step && act_a ? sa : 0];
    const lct_desc DB = desc[desc_step && act_b ? sa + 1 : 0];
    const int64_t base_a = desc_step ? DA.offset : sa * (int64_t)S::N;
    const int64_t base_b = desc_step ? DB.offset : (sa + 1) * (int64_t)S::N;
    cpx<pf>* buf = smem + sl * F::NP;
    const bool dec_a = (DA.flags & LCT_FLAG_DECAY) != 0, dec_b = (DB.flags & LCT_FLAG_DECAY) != 0;

    cpx<pf> v[S::E];
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int n = i + e * S::T;
        cpx<float> fa = {0.f, 0.f}, fb = {0.f, 0.f};
        if (act_a) fa = ld_stream(in + base_a + n);
        if (act_b) fb = ld_stream(in + base_b + n);
        const cpx<float> ca = pre_chirp<L>(DA, n, dec_a), cb = pre_chirp<L>(DB, n, dec_b);
        v[e] = cmul(pack(fa, fb), pack(ca, cb));
    }
    dft_signal<L, -1, false, LE, F::PS>(v, buf, i, tw);
    const pf sc = pf_make((float)DA.scale, (float)DB.scale);
#pragma unroll
    for (int e = 0; e < S::E; ++e) {
        const int n = i + e * S::T;
        const cpx<float> ca = post_chirp<L>(DA, n), cb = post_chirp<L>(DB, n);
        const cpx<pf> g = cscale(cmul(v[e], pack(ca, cb)), sc);
        if (act_a) out[base_a + n] = {g.x.v.x, g.y.v.x};
        if (act_b) out[base_b + n] = {g.x.v.y, g.y.v.y};
    }
}

// Persistent paired kernel: each CTA (one signal pair at a time, N >= 256)
// loops over pairs.  One shared buffer serves both roles: it receives the
// pair's samples by bulk asynchronous copy (A then B, unpadded), is read
// into registers, and then holds the padded Stockham exchanges.  As soon as
// the last exchange has been read, the next pair's copy is issued into it,
// so the copy overlaps the post-chirp, the global stores and the other
// resident CTA's work.
constexpr uint64_t kPairWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ void issue_pair(const cpx<float>* in, const lct_desc* desc,
                                           int desc_step, int64_t count, int64_t pair,
                                           int n, cpx<float>* dst, uint64_t* bar) {
    const int64_t sa = 2 * pair;
    const uint32_t bytes = (uint32_t)n * (uint32_t)sizeof(cpx<float>);
    const int nsig = sa + 1 < count ? 2 : 1;
    xasync::mbar_arrive_expect_tx(bar, bytes * nsig);
    for (int s = 0; s < nsig; ++s) {
        const int64_t base = desc_step ? desc[sa + s].offset : (sa + s) * (int64_t)n;
        xasync::bulk_g2s(dst + s * n, in + base, bytes, bar);
    }
}

template <int L>
__global__ void __launch_bounds__(shape<L>::T, 2)
k_xft_pair_tma(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
               const lct_desc* __restrict__ desc, int desc_step, int64_t count,
               const cpx<pf>* __restrict__ tw, int32_t* __restrict__ status) {
    using S = shape<L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<pf>* buf = reinterpret_cast<cpx<pf>*>(smem_raw);
    cpx<float>* stage = reinterpret_cast<cpx<float>*>(smem_raw);
    constexpr size_t BUF_BYTES = (size_t)S::NP * sizeof(cpx<pf>);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + BUF_BYTES);
    const int64_t pairs = (count + 1) / 2;
    int64_t g = blockIdx.x;
    if (g >= pairs) return;
    const int i = threadIdx.x;
    if (i == 0) {
        xasync::mbar_init(bar, 1);
        xasync::fence_mbar_init();
    }
    __syncthreads();
    if (i == 0) issue_pair(in, desc, desc_step, count, g, S::N, stage, bar);
    uint32_t parity = 0;
    for (; g < pairs; g += gridDim.x) {
        bool ok = true;
        if (i == 0) ok = xasync::mbar_wait(bar, parity, kPairWaitNs);
        if (__syncthreads_or(!ok)) {
            if (i == 0) {
                atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
                xasync::mbar_wait(bar, parity, kPairWaitNs);
            }
            return;
        }
        parity ^= 1u;
        const int64_t sa = 2 * g;
        const bool act_b = sa + 1 < count;
        const lct_desc DA = desc[desc_step ? sa : 0];
        const lct_desc DB = desc[desc_step && act_b ? sa + 1 : 0];
        const int64_t base_a = desc_step ? DA.offset : sa * (int64_t)S::N;
        const int64_t base_b = desc_step ? DB.offset : (sa + 1) * (int64_t)S::N;
        const bool dec_a = (DA.flags & LCT_FLAG_DECAY) != 0, dec_b = (DB.flags & LCT_FLAG_DECAY) != 0;
        cpx<pf> v[S::E];
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            const cpx<float> fa = stage[n];
            const cpx<float> fb = act_b ? stage[S::N + n] : cpx<float>{0.f, 0.f};
            const cpx<float> ca = pre_chirp<L>(DA, n, dec_a), cb = pre_chirp<L>(DB, n, dec_b);
            v[e] = cmul(pack(fa, fb), pack(ca, cb));
        }
        __syncthreads();                      // stage read: the buffer now serves the exchanges
        dft_signal<L, -1>(v, buf, i, tw);
        __syncthreads();                      // last exchange read: refill for the next pair
        if (i == 0 && g + gridDim.x < pairs) {
            xasync::fence_proxy_async_smem();
            issue_pair(in, desc, desc_step, count, g + gridDim.x, S::N, stage, bar);
        }
        const pf sc = pf_make((float)DA.scale, (float)DB.scale);
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            const cpx<float> ca = post_chirp<L>(DA, n), cb = post_chirp<L>(DB, n);
            const cpx<pf> gg = cscale(cmul(v[e], pack(ca, cb)), sc);
            out[base_a + n] = {gg.x.v.x, gg.y.v.x};
            if (act_b) out[base_b + n] = {gg.x.v.y, gg.y.v.y};
        }
    }
}

template <int L>
cudaError_t launch_pair_tma(const void* in, void* out, const lct_desc* desc, int desc_step,
                            int64_t count, const void* tw, int32_t* status, cudaStream_t stream) {
    using S = shape<L>;
    const size_t smem = (size_t)S::NP * sizeof(cpx<pf>) + 16;
    auto kern = k_xft_pair_tma<L>;
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
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, S::T, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        blocks_per_sm[dev] = nb > 0 ? nb : 1;
    }
    const int64_t pairs = (count + 1) / 2;
    int64_t grid = (int64_t)blocks_per_sm[dev] * sms[dev];
    if (grid > pairs) grid = pairs;
    kern<<<(unsigned)grid, S::T, smem, stream>>>((const cpx<float>*)in, (cpx<float>*)out, desc,
                                                 desc_step, count, (const cpx<pf>*)tw, status);
    return cudaGetLastError();
}

template <int L, int MINB, int LE = 4>
cudaError_t launch_pair(const void* in, void* out, const lct_desc* desc, int desc_step,
                        int64_t count, const void* tw, cudaStream_t stream) {
    using F = pair_shape<L, LE>;
    const size_t smem = (size_t)F::PPC * F::NP * sizeof(cpx<pf>);
    auto kern = k_xft_pair<L, MINB, LE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t pairs = (count + 1) / 2;
    const int64_t blocks = (pairs + F::PPC - 1) / F::PPC;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, F::THREADS, smem, stream>>>(
        (const cpx<float>*)in, (cpx<float>*)out, desc, desc_step, count, (const cpx<pf>*)tw);
    return cudaGetLastError();
}

template <int MINB>
cudaError_t pair_dispatch(int log2n, const void* in, void* out, const lct_desc* desc,
                          int desc_step, int64_t count, const void* tw, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_pair<L, MINB>(in, out, desc, desc_step, count, tw, stream);
        LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10)
        LCT_CASE(11) LCT_CASE(12)
#undef LCT_CASE
        case 13: return launch_pair<13, 1>(in, out, desc, desc_step, count, tw, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool lct_fused_pair_supported(int dtype, int log2n) { return dtype == 0 && log2n >= 5 && log2n <= 13; }
// Eight samples per thread (radix-8 passes): half the registers of the
// 16-sample kernel, so two CTAs of up to 512 threads stay resident at <= 64
// registers (complex64, N = 64 .. 8192).
bool lct_fused_pair8_supported(int dtype, int log2n) { return dtype == 0 && log2n >= 6 && log2n <= 13; }

cudaError_t lct_launch_fused_pair8(int dtype, int log2n, const void* in, void* out,
                                   const lct_desc* desc, int desc_step, int64_t count,
                                   const void* tw_pair8, cudaStream_t stream) {
    if (dtype != 0) return cudaErrorInvalidValue;
    switch (log2n) {
#define LCT_CASE(L, MB) \
    case L: return launch_pair<L, MB, 3>(in, out, desc, desc_step, count, tw_pair8, stream);
        LCT_CASE(6, 4) LCT_CASE(7, 4) LCT_CASE(8, 4) LCT_CASE(9, 4) LCT_CASE(10, 4)
        LCT_CASE(11, 4) LCT_CASE(12, 2) LCT_CASE(13, 1)
#undef LCT_CASE
        default: return cudaErrorInvalidValue;
    }
}

// One pair per CTA needs T = N/16 >= 256 threads to keep the SM busy: N = 4096.
bool lct_fused_pair_tma_supported(int dtype, int log2n) { return dtype == 0 && log2n == 12; }

cudaError_t lct_launch_fused_pair_tma(int dtype, int log2n, const void* in, void* out,
                                      const lct_desc* desc, int desc_step, int64_t count,
                                      const void* tw_pair, int32_t* status, cudaStream_t stream) {
    if (dtype != 0) return cudaErrorInvalidValue;
    if (log2n != 12) return cudaErrorInvalidValue;
    return launch_pair_tma<12>(in, out, desc, desc_step, count, tw_pair, status, stream);
}

// Two resident CTAs of 256 threads per SM (register budget 128).
cudaError_t lct_launch_fused_pair(int dtype, int log2n, const void* in, void* out,
                                  const lct_desc* desc, int desc_step, int64_t count,
                                  const void* tw_pair, cudaStream_t stream) {
    if (dtype != 0) return cudaErrorInvalidValue;
    return pair_dispatch<2>(log2n, in, out, desc, desc_step, count, tw_pair, stream);
}
