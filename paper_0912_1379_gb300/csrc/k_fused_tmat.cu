// Fused XFT kernel, variant 8: the persistent form of the fused kernel whose
// input arrives through the TMA engine's tiled copies described by a tensor
// map (cp.async.bulk.tensor), instead of per-thread loads.
//
// The batch of contiguous complex64 signals is viewed as a 2-D tensor of
// rows of 256 samples (2048 bytes): a group of signals that one CTA
// transforms (SPC signals, SPC N = max(4096, N) samples) is one box of 256 x
// (SPC N / 256) rows, brought into a shared-memory stage by one
// cp.async.bulk.tensor.2d that completes on an mbarrier -- while the CTA
// transforms the previous group (Sec. 3, Algorithm, steps 1-3; the same
// chirps and Stockham engine as the fused kernel).  The output is written
// by the threads directly (coalesced).
// Requirements (checked on the host): complex64, N = 256 .. 8192, signal s at
// element s N, count N a multiple of 256, 16-byte aligned input.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "xft_engine.cuh"
#include "xft_async.cuh"
#include "xft_chirp.cuh"

namespace {

using namespace xft;

template <int L>
struct tm_shape {
    static constexpr int T = shape<L>::T;
    static constexpr int SPC = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = T * SPC;
    static constexpr int ROWS = SPC * (1 << L) / 256;          // tensor rows per group
};

constexpr uint64_t kTmWaitNs = 2000000000ull;

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(xasync::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(xasync::smem_addr(bar))
        : "memory");
}

template <int L>
__global__ void __launch_bounds__(tm_shape<L>::THREADS, (L <= 12 ? 3 : 1))
k_xft_fused_tmat(const __grid_constant__ CUtensorMap map, cpx<float>* __restrict__ out,
                 const lct_desc* __restrict__ desc, int desc_step, int64_t count,
                 const cpx<float>* __restrict__ tw, int32_t* __restrict__ status) {
    using S = shape<L>;
    using F = tm_shape<L>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
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
    constexpr uint32_t kBytes = (uint32_t)F::SPC * S::N * 8u;
    if (tid == 0) {
        xasync::mbar_init(bar, 1);
        xasync::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        xasync::mbar_arrive_expect_tx(bar, kBytes);
        tma_load_2d(stage, &map, 0, (int)(g * F::ROWS), bar);
    }
    uint32_t parity = 0;
    for (; g < groups; g += gridDim.x) {
        bool ok = true;
        if (tid == 0) ok = xasync::mbar_wait(bar, parity, kTmWaitNs);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
                xasync::mbar_wait(bar, parity, kTmWaitNs);   // let the copy in flight land
            }
            return;
        }
        parity ^= 1u;
        const int64_t sig = g * F::SPC + sl;
        const bool active = sig < count;
        const lct_desc D = desc[desc_step && active ? sig : 0];
        const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
        cpx<float> v[S::E];
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            v[e] = cmul(stage[sl * S::N + n], pre_w<L, float>(D, n, decay));
        }
        __syncthreads();                       // stage fully read
        if (tid == 0 && g + gridDim.x < groups) {
            xasync::fence_proxy_async_smem();
            xasync::mbar_arrive_expect_tx(bar, kBytes);
            tma_load_2d(stage, &map, 0, (int)((g + gridDim.x) * F::ROWS), bar);
        }
        dft_signal<L, -1>(v, buf, i, tw);
        if (active) {
            const float sc = (float)D.scale;
            const int64_t base = sig * (int64_t)S::N;
#pragma unroll
            for (int e = 0; e < S::E; ++e) {
                const int n = i + e * S::T;
                out[base + n] = cscale(cmul(v[e], post_w<L, float>(D, n)), sc);
            }
        }
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <int L>
cudaError_t launch_tmat(const void* in, void* out, const lct_desc* desc, int desc_step,
                        int64_t count, const void* tw, int32_t* status, cudaStream_t stream) {
    using S = shape<L>;
    using F = tm_shape<L>;
    const int64_t total = count * (int64_t)S::N;
    if (total % 256 != 0 || ((uintptr_t)in) % 16 != 0) return cudaErrorInvalidValue;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[2] = {256, (cuuint64_t)(total / 256)};
    const cuuint64_t strides[1] = {2048};
    const cuuint32_t box[2] = {256, (cuuint32_t)F::ROWS};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(in), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const size_t smem = (size_t)F::SPC * (S::N + S::NP) * sizeof(cpx<float>) + 16;
    auto kern = k_xft_fused_tmat<L>;
    static int blocks_per_sm[64] = {}, sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!blocks_per_sm[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, F::THREADS, smem)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        blocks_per_sm[dev] = nb > 0 ? nb : 1;
    }
    const int64_t groups = (count + F::SPC - 1) / F::SPC;
    int64_t grid = (int64_t)blocks_per_sm[dev] * sms[dev];
    if (grid > groups) grid = groups;
    kern<<<(unsigned)grid, F::THREADS, smem, stream>>>(map, (cpx<float>*)out, desc, desc_step, count,
                                                       (const cpx<float>*)tw, status);
    return cudaGetLastError();
}

}  // namespace

bool lct_fused_tmat_supported(int dtype, int log2n) { return dtype == 0 && log2n >= 8 && log2n <= 13; }

cudaError_t lct_launch_fused_tmat(int log2n, const void* in, void* out, const lct_desc* desc,
                                  int desc_step, int64_t count, const void* tw, int32_t* status,
                                  cudaStream_t stream) {
    switch (log2n) {
        case 8: return launch_tmat<8>(in, out, desc, desc_step, count, tw, status, stream);
        case 9: return launch_tmat<9>(in, out, desc, desc_step, count, tw, status, stream);
        case 10: return launch_tmat<10>(in, out, desc, desc_step, count, tw, status, stream);
        case 11: return launch_tmat<11>(in, out, desc, desc_step, count, tw, status, stream);
        case 12: return launch_tmat<12>(in, out, desc, desc_step, count, tw, status, stream);
        case 13: return launch_tmat<13>(in, out, desc, desc_step, count, tw, status, stream);
        default: return cudaErrorInvalidValue;
    }
}
