// Split-precision XFT on the 5th-generation tensor cores (tcgen05), N = 4096
// complex64: the three radix-16 passes of the Stockham plan run as products
// of the real 32 x 32 DFT matrix on the tcgen05.mma pipe (kind::f16 with
// BF16 operands, FP32 accumulators in tensor memory); chirps, twiddles and
// the exchanges between passes stay on the CUDA cores, with the exact
// fixed-point chirp phases of the native path.
//
// One radix-16 DFT y_j = sum_e u_e e^{-2 pi i j e / 16} of a group of 16
// samples is the real product  D[g][n] = sum_k A[g][k] B[k][n]  with
//   A[g][2e + c]  = (Re, Im)_c u_e             (the group's 32 inputs)
//   B[2e][2j] = Re F_je,  B[2e+1][2j] = -Im F_je,
//   B[2e][2j+1] = Im F_je, B[2e+1][2j+1] = Re F_je   (F_je = e^{-2 pi i je/16})
// so D[g][2j + c] = (Re, Im)_c y_j.  A signal's 256 groups are two M = 128
// tiles; N = 32, K = 32 (two K = 16 steps); each operand is split into BF16
// hi + lo parts and the product taken as hi.hi + hi.lo + lo.hi: 12 MMAs per
// pass, issued by one thread and committed to an mbarrier.
//
// Data flow of one CTA (256 threads, one signal at a time, persistent):
// thread t owns TMEM lane t, i.e. row t of the accumulator.  Pass 0: thread t
// loads samples t + 256 e with the pre-chirp, splits them and writes A row t.
// After the MMAs of pass p, thread t reads its row -- the 16 outputs of its
// group -- and, for p < 2, applies the twiddle of pass p + 1 to each output,
// splits it and writes it straight into the A row of the group that takes it
// in pass p + 1 (the Stockham exchange, without an FP32 buffer); after pass 2
// thread t holds X[t + 256 j] and stores it with the post-chirp.  The A rows
// of pass 1 are permuted (16 x 16 index transpose) so that these scattered
// 4-byte stores meet at most 2 lanes per bank; thread t then owns group
// transpose(t) in pass 1.
//
// Operand layout (umma_desc.h): K-major, no swizzle, core matrices of 8 rows
// x 8 16-bit values (16 bytes per row), LBO = 128 bytes along K, SBO = 512
// bytes per 8 rows (32 K values per row).
//
// The same kernel takes FP16 operands (kind::f16, both A and B FP16): split
// hi + lo with three products, or hi alone with one product (TERMS = 1).
// FP16 signals are scaled by a power of two after the pre-chirp so that
// their largest component is below 1 (each radix-16 pass grows it at most
// 16-fold: below 4096 after the three, inside the FP16 range), and the
// output by the inverse.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "xft_engine.cuh"
#include "xft_chirp.cuh"
#include "xft_umma.cuh"

namespace {

using namespace xft;

constexpr int kSL = 12, kSN = 1 << kSL, kST = 256;        // N, threads = groups
constexpr uint32_t kPlane = 256 * 32 * 2;                  // one A plane: 256 rows x 32 BF16
constexpr uint32_t kBPlane = 32 * 32 * 2;                  // one B plane
constexpr uint32_t kOffAlo = kPlane, kOffBhi = 2 * kPlane, kOffBlo = 2 * kPlane + kBPlane;
constexpr uint32_t kSmem = 2 * kPlane + 2 * kBPlane;       // 36 KB
constexpr uint32_t kSLbo = 128, kSSbo = 512, kTmemCols = 64;
constexpr uint64_t kSWaitNs = 2000000000ull;

// Byte offset of element (row, k) of a 32-wide K-major 16-bit operand.
__host__ __device__ constexpr uint32_t boff(uint32_t r, uint32_t k) {
    return (r >> 3) * kSSbo + (k >> 3) * kSLbo + (r & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ int transpose16(int g) { return ((g & 15) << 4) | (g >> 4); }

// A pair of 16-bit operand values (a low, b high) in BF16 or FP16, and back.
template <int FMT>
__device__ __forceinline__ uint32_t pk2(float a, float b) {
    if constexpr (FMT == umma::kFmtBF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <int FMT>
__device__ __forceinline__ float2 upk2(uint32_t v) {
    if constexpr (FMT == umma::kFmtBF16) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
}
// hi = rn(re, im), lo = rn((re, im) - hi) (TERMS = 3), each a pair (re low, im high)
template <int FMT, int TERMS>
__device__ __forceinline__ void split_c(cpx<float> v, uint32_t& hi, uint32_t& lo) {
    hi = pk2<FMT>(v.x, v.y);
    if constexpr (TERMS == 3) {
        const float2 h = upk2<FMT>(hi);
        lo = pk2<FMT>(v.x - h.x, v.y - h.y);
    } else {
        lo = 0;
    }
}
// One 16-bit value at p (B operand set-up), and its rounded value.
template <int FMT>
__device__ __forceinline__ float st16(unsigned char* p, float v) {
    if constexpr (FMT == umma::kFmtBF16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16*>(p) = h;
        return __bfloat162float(h);
    } else {
        const __half h = __float2half_rn(v);
        *reinterpret_cast<__half*>(p) = h;
        return __half2float(h);
    }
}
// 2^-ex (DOWN) or 2^ex for m the bit pattern of max |component| = f 2^ex,
// f in [0.5, 1) (1 for a zero signal); ex clamped to [-125, 125] so that both
// factors are normal numbers.
template <bool DOWN>
__device__ __forceinline__ float exp2_of_max(uint32_t m) {
    int ex = 0;
    if (m) frexpf(__uint_as_float(m), &ex);
    ex = min(max(ex, -125), 125);
    return ldexpf(1.f, DOWN ? -ex : ex);
}

__constant__ float kCosT16[16] = {
    1.0f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f,
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128676f,
    -1.0f, -0.92387953251128676f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128676f};

__device__ __forceinline__ bool bar_wait_all(uint64_t* bar, uint32_t parity) {
    return xasync::mbar_wait(bar, parity, kSWaitNs);
}

template <int FMT, int TERMS>
__global__ void __launch_bounds__(kST, 4)
k_xft_split_umma(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                 const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                 const cpx<float>* __restrict__ tw, int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    __shared__ uint32_t s_amax[kST / 32];                   // FP16: per-warp max |component|
    const int t = threadIdx.x, warp = t >> 5;
    if (warp == 0) umma::tmem_alloc(&tmem_slot, kTmemCols);
    if (t == 0) {
        xasync::mbar_init(&bar, 1);
        xasync::fence_mbar_init();
    }
    // the DFT matrix, split: thread t writes 4 entries of B (row n = output
    // index 2j + c', column k = input index 2e + c)
    for (int q = t; q < 32 * 32; q += kST) {
        const int n = q >> 5, k = q & 31;
        const int j = n >> 1, cp = n & 1, e = k >> 1, c = k & 1;
        const int m = (j * e) & 15;
        const float re = kCosT16[m], im = -kCosT16[(m + 12) & 15];      // F_je = re + i im
        const float v = cp == 0 ? (c == 0 ? re : -im) : (c == 0 ? im : re);
        const float h = st16<FMT>(sm + kOffBhi + boff(n, k), v);
        if (TERMS == 3) st16<FMT>(sm + kOffBlo + boff(n, k), v - h);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    // this thread's accumulator row: tile warp >> 2 (columns 32 tile ..), lane t
    const uint32_t my_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
    constexpr uint32_t idesc = umma::instr_desc(FMT, FMT, 128, 32);       // A and B of one type
    const uint32_t a_base = xasync::smem_addr(sm);
    uint32_t phase = 0;
    bool ok = true;

    for (int64_t sig = blockIdx.x; sig < count && ok; sig += gridDim.x) {
        const lct_desc D = desc[desc_step ? sig : 0];
        const int64_t base = desc_step ? D.offset : sig * (int64_t)kSN;
        const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
        // pass 0 input: samples t + 256 e with the pre-chirp, into A row t
        float inv_scale = 1.f;                              // FP16: undoes the input scale
        {
            cpx<float> f[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n = t + kST * e;
                f[e] = cmul(ld_stream(in + base + n), pre_w<kSL, float>(D, n, decay));
            }
            if constexpr (FMT == umma::kFmtF16) {
                uint32_t m = 0;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    m = max(m, __float_as_uint(fmaxf(fabsf(f[e].x), fabsf(f[e].y))));
                m = __reduce_max_sync(0xffffffffu, m);
                if ((t & 31) == 0) s_amax[warp] = m;
                __syncthreads();
#pragma unroll
                for (int w = 0; w < kST / 32; ++w) m = max(m, s_amax[w]);
                const float sc_in = exp2_of_max<true>(m);
                inv_scale = exp2_of_max<false>(m);
#pragma unroll
                for (int e = 0; e < 16; ++e) f[e] = cscale(f[e], sc_in);
            }
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) split_c<FMT, TERMS>(f[e], hi[e], lo[e]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                *reinterpret_cast<uint4*>(sm + boff(t, 8 * q)) =
                    make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
                if (TERMS == 3)
                    *reinterpret_cast<uint4*>(sm + kOffAlo + boff(t, 8 * q)) =
                        make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
            }
        }
#pragma unroll 1
        for (int p = 0; p < 3; ++p) {
            xasync::fence_proxy_async_smem();
            umma::fence_before_sync();
            __syncthreads();
            if (t == 0) {
                umma::fence_after_sync();
#pragma unroll
                for (int tile = 0; tile < 2; ++tile) {
                    const uint32_t d = tmem + 32 * tile;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t o = tile * (16 * kSSbo) + ks * 2 * kSLbo;
                        const uint64_t ah = umma::smem_desc(a_base + o, kSLbo, kSSbo);
                        const uint64_t al = umma::smem_desc(a_base + kOffAlo + o, kSLbo, kSSbo);
                        const uint64_t bh = umma::smem_desc(a_base + kOffBhi + ks * 2 * kSLbo, kSLbo, kSSbo);
                        const uint64_t bl = umma::smem_desc(a_base + kOffBlo + ks * 2 * kSLbo, kSLbo, kSSbo);
                        umma::mma_f16(d, ah, bh, idesc, ks > 0 ? 1u : 0u);
                        if (TERMS == 3) {
                            umma::mma_f16(d, ah, bl, idesc, 1u);
                            umma::mma_f16(d, al, bh, idesc, 1u);
                        }
                    }
                }
                umma::commit(&bar);
            }
            if (!bar_wait_all(&bar, phase)) {
                ok = false;
                atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
            }
            phase ^= 1u;
            if (!__syncthreads_and(ok)) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            float v[32];
            umma::tmem_ld16(my_row, v);
            umma::tmem_ld16(my_row + 16, v + 16);
            umma::fence_before_sync();
            if (p == 2) {
                // thread t holds X[t + 256 j]: post-chirp, scale, store
                const float sc = (float)D.scale * inv_scale;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = t + kST * j;
                    const cpx<float> y = {v[2 * j], v[2 * j + 1]};
                    out[base + n] = cscale(cmul(y, post_w<kSL, float>(D, n)), sc);
                }
                break;
            }
            // Stockham exchange into pass p + 1: output j of group g goes to
            // position pos = (g - k) 16 + k + j NS_p (k = g mod NS_p), i.e.
            // group pos mod 256, element e' = pos / 256 = g / 16 (the same for
            // all j), twiddled by e^{-2 pi i e' k' / (16 NS_{p+1})} with
            // k' = group mod NS_{p+1} = j (p = 0) or k + 16 j (p = 1): the
            // powers w0 w1^j of w1 = e^{-2 pi i e'/256}, w0 = 1 or
            // e^{-2 pi i e' k/4096}, formed in registers (one or two sincospi
            // and a running product) instead of table loads.  The A row of
            // output j is 16 j + g mod 16 in both exchanges (transpose16 of
            // group g1 = 16 (g mod 16) + j for p = 0; g1 = g mod 16 + 16 j for
            // p = 1), so a thread's 16 stores step by 16 rows = 2 SBO bytes
            // from the offset of j = 0.
            const int g = p == 0 ? t : transpose16(t);
            const int k = p == 0 ? 0 : (g & 15);
            const int e1 = g >> 4;
            const cpx<float> w1 = twiddle_exact<float, -1>(e1, 256);
            cpx<float> u = p == 0 ? cpx<float>{1.f, 0.f} : twiddle_exact<float, -1>(e1 * k, 4096);
            const uint32_t o0 = boff((uint32_t)(g & 15), (uint32_t)(2 * e1));
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                cpx<float> y = {v[2 * j], v[2 * j + 1]};
                y = cmul(y, u);                             // u = 1 exactly when e' = 0
                u = cmul(u, w1);
                uint32_t hi, lo;
                split_c<FMT, TERMS>(y, hi, lo);
                const uint32_t o = o0 + (uint32_t)j * (2 * kSSbo);
                *reinterpret_cast<uint32_t*>(sm + o) = hi;
                if (TERMS == 3) *reinterpret_cast<uint32_t*>(sm + kOffAlo + o) = lo;
            }
        }
    }
    // every MMA issued has been waited on (or the wait gave up and the CTA
    // stops); release the tensor memory
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

bool lct_split_umma_supported(int dtype, int log2n) { return dtype == 0 && log2n == kSL; }

namespace {
template <int FMT, int TERMS>
cudaError_t launch_umma(const void* in, void* out, const lct_desc* desc, int desc_step, int64_t count,
                        const void* tw, int32_t* status, cudaStream_t stream) {
    auto kern = k_xft_split_umma<FMT, TERMS>;
    static int blocks_per_sm[64] = {}, sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!blocks_per_sm[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
        // resident CTAs per SM from the kernel's own registers and shared
        // memory (and 8 by tensor memory: 64 of 512 columns each); more CTAs
        // than fit only wait for a slot, as the CTAs never wait on each other
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int regs_sm = 0, smem_sm = 0;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess)
            return e;
        const int by_regs = regs_sm / ((fa.numRegs > 0 ? fa.numRegs : 1) * kST);
        const int by_smem = smem_sm / (int)(kSmem + fa.sharedSizeBytes + 1024);
        int nb = by_regs < by_smem ? by_regs : by_smem;
        nb = nb < 1 ? 1 : (nb > 8 ? 8 : nb);
        blocks_per_sm[dev] = nb;
    }
    if (count <= 0) return cudaSuccess;
    int64_t grid = (int64_t)blocks_per_sm[dev] * sms[dev];
    if (grid > count) grid = count;
    kern<<<(unsigned)grid, kST, kSmem, stream>>>((const cpx<float>*)in, (cpx<float>*)out, desc, desc_step,
                                                count, (const cpx<float>*)tw, status);
    return cudaGetLastError();
}
}  // namespace

cudaError_t lct_launch_split_umma(int prec, int log2n, const void* in, void* out, const lct_desc* desc,
                                  int desc_step, int64_t count, const void* tw, int32_t* status,
                                  cudaStream_t stream) {
    if (log2n != kSL || !tw) return cudaErrorInvalidValue;
    switch (prec) {
        case 1: return launch_umma<umma::kFmtBF16, 3>(in, out, desc, desc_step, count, tw, status, stream);
        case 2: return launch_umma<umma::kFmtF16, 3>(in, out, desc, desc_step, count, tw, status, stream);
        case 3: return launch_umma<umma::kFmtF16, 1>(in, out, desc, desc_step, count, tw, status, stream);
        default: return cudaErrorInvalidValue;
    }
}
