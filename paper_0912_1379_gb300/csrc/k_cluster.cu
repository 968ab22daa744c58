// Large-N XFT (N = 16384 .. 65536): one thread-block cluster of C CTAs per
// signal, samples exchanged through distributed shared memory, so each
// sample still crosses HBM once in and once out, with coalesced accesses.
//
// Decomposition (N = C M, decimation in time across the cluster):
//   n = c + C n2 (c < C), k = k2 + M k1 (k1 < C)
//   X[k2 + M k1] = sum_c W_C^{c k1} W_N^{c k2} [ sum_{n2} x[c + C n2] W_M^{n2 k2} ]
// 1. CTA r loads the contiguous chunk [r M, (r+1) M) with the pre-chirp and
//    scatters sample n to CTA n mod C, position n div C (DSMEM stores; each
//    thread reads runs of C consecutive samples, one for every CTA).
// 2. Each CTA c runs the M-point Stockham DFT (xft_engine.cuh) of its
//    stride-C subsequence and multiplies by W_N^{c k2}.
// 3. CTA d takes k2 in [d M/C, (d+1) M/C): gathers the C values Z_c[k2],
//    applies the C-point DFT and writes X[k2 + M k1] (contiguous in k2)
//    with the post-chirp.
// Cluster barriers separate the phases; the last one follows the final
// gather, so no CTA exits while its shared memory may still be read.
#include <cooperative_groups.h>

#include "xft_engine.cuh"
#include "xft_chirp.cuh"

namespace cg = cooperative_groups;

namespace {

using namespace xft;

template <int LN, class R>
__device__ __forceinline__ cpx<R> pre_n(const lct_desc& D, int n, bool decay) {
    if constexpr (sizeof(R) == 4) return pre_chirp<LN>(D, n, decay);
    else return pre_chirp64<LN>(D, n, decay);
}
template <int LN, class R>
__device__ __forceinline__ cpx<R> post_n(const lct_desc& D, int n) {
    if constexpr (sizeof(R) == 4) return post_chirp<LN>(D, n);
    else return post_chirp64<LN>(D, n);
}

// Input load of one sample of a run of consecutive samples read by one
// thread: L1-allocating, so the run's neighbours come from the same lines.
template <class R>
__device__ __forceinline__ cpx<R> ld_run(const cpx<R>* p) { return *p; }

// Resident CTAs per SM: 4 x 256 threads (complex64, 4096-point rows),
// 1 x 512 threads (complex128, 8192-point rows).
template <int LM, class R>
constexpr int cluster_min_blocks() { return sizeof(R) == 4 ? (LM <= 12 ? 4 : 2) : 1; }

template <int LM, int LC, class R>
__global__ void __launch_bounds__(shape<LM>::T, (cluster_min_blocks<LM, R>()))
k_xft_cluster(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
              const lct_desc* __restrict__ desc, int desc_step, int64_t count,
              const cpx<R>* __restrict__ tw, const int32_t* __restrict__ idx,
              int32_t* __restrict__ status) {
    using S = shape<LM>;
    constexpr int C = 1 << LC, M = S::N, LN = LM + LC, N = 1 << LN;
    constexpr int Q = S::E / C;              // step-A positions per thread
    static_assert(Q >= 1, "cluster larger than 16");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const int64_t sig = blockIdx.x / C;
    const int i = threadIdx.x;
    bool active = sig < count;
    const int64_t gsig = idx ? (active ? idx[sig] : 0) : sig;
    const lct_desc D = desc[desc_step && active ? gsig : 0];
    if (idx && active && (D.log2n != LN || D.kind != LCT_KIND_XFT || D.offset < 0)) {
        if (i == 0 && c == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        active = false;                       // uniform over the cluster: every CTA reads D
    }
    const int64_t base = desc_step ? D.offset : sig * (int64_t)N;
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;

    // 1. contiguous chunk c, pre-chirped, scattered into stride-C subsequences:
    //    thread i takes the runs of C consecutive samples n0 + j (n0 = c M +
    //    C (i + q T)) and writes sample j to CTA j at position n0 / C, so each
    //    remote store instruction covers consecutive positions of one CTA.
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int pos = c * (M / C) + i + q * S::T;        // n0 / C
        const int n0 = pos * C;
        cpx<R> f[C];
#pragma unroll
        for (int j = 0; j < C; ++j) f[j] = {R(0), R(0)};
        if (active) {
#pragma unroll
            for (int j = 0; j < C; ++j) f[j] = ld_run(in + base + n0 + j);
        }
#pragma unroll
        for (int j = 0; j < C; ++j) {
            cpx<R>* rb = cl.map_shared_rank(buf, j);
            rb[pos] = cmul(f[j], pre_n<LN, R>(D, n0 + j, decay));
        }
    }
    cl.sync();

    // 2. local M-point DFT of x[c + C n2], then the twiddle W_N^{c k2}, k2 = i + e T
    cpx<R> v[S::E];
#pragma unroll
    for (int e = 0; e < S::E; ++e) v[e] = buf[i + e * S::T];
    __syncthreads();                          // subsequence read before the engine reuses buf
    dft_signal<LM, -1>(v, buf, i, tw);
    if (c != 0) {
        const cpx<R> step = twiddle_exact<R, -1>(c * S::T, N);   // W_N^{c T}
        cpx<R> w = twiddle_exact<R, -1>(c * i, N);               // W_N^{c i}
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            v[e] = cmul(v[e], w);
            w = cmul(w, step);
        }
    }
    __syncthreads();                          // engine's last exchange read
#pragma unroll
    for (int e = 0; e < S::E; ++e) buf[i + e * S::T] = v[e];
    cl.sync();

    // 3. gather Z_c[k2] over the cluster, C-point DFT, contiguous stores
    cpx<R> a[Q][C];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int k2 = c * (M / C) + q * S::T + i;
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
            const cpx<R>* rb = cl.map_shared_rank(buf, cc);
            a[q][cc] = rb[k2];
        }
    }
    cl.sync();                                // no shared memory is read after this
    if (active) {
        const R sc = (R)D.scale;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int k2 = c * (M / C) + q * S::T + i;
            dft<C, -1>(a[q]);
#pragma unroll
            for (int k1 = 0; k1 < C; ++k1) {
                const int k = k2 + M * k1;
                out[base + k] = cscale(cmul(a[q][k1], post_n<LN, R>(D, k)), sc);
            }
        }
    }
}

template <int LM, int LC, class R>
cudaError_t launch_cluster(const void* in, void* out, const lct_desc* desc, int desc_step,
                           int64_t count, const void* tw, const int32_t* idx, int32_t* status,
                           cudaStream_t stream) {
    using S = shape<LM>;
    constexpr int C = 1 << LC;
    const size_t smem = (size_t)S::NP * sizeof(cpx<R>);
    auto kern = k_xft_cluster<LM, LC, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = count * C;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(S::T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, (const cpx<R>*)in, (cpx<R>*)out, desc, desc_step, count,
                              (const cpx<R>*)tw, idx, status);
}

}  // namespace

// Local length M = 8192 for both precisions; C = N / 8192 CTAs per cluster.
// (Measured on GB300: 4096-point rows with C = 8 / 16 were slower -- the
// distributed shared-memory exchange, not the row transform, dominates.)
int lct_cluster_local_log2(int dtype, int log2n) {
    (void)dtype;
    return (log2n >= 14 && log2n <= 16) ? 13 : -1;
}

cudaError_t lct_launch_cluster(int dtype, int log2n, const void* in, void* out,
                               const lct_desc* desc, int desc_step, int64_t count,
                               const void* tw_local, const int32_t* idx, int32_t* status,
                               cudaStream_t stream) {
    if (dtype == 0) {
        switch (log2n) {
            case 14: return launch_cluster<13, 1, float>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
            case 15: return launch_cluster<13, 2, float>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
            case 16: return launch_cluster<13, 3, float>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (log2n) {
        case 14: return launch_cluster<13, 1, double>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
        case 15: return launch_cluster<13, 2, double>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
        case 16: return launch_cluster<13, 3, double>(in, out, desc, desc_step, count, tw_local, idx, status, stream);
        default: return cudaErrorInvalidValue;
    }
}
