// Ragged batch in one persistent launch (complex64): every signal of a batch
// of mixed N and kinds -- the XFT of Sec. 3 for N = 2 .. 65536 and the b = 0
// diagonal -- transformed by one grid of 256-thread CTAs that take work
// items from a single device queue.  The host lays the queue out largest N
// first:
//   1. the two-pass tiles (pass A / pass B, xft_twopass.cuh) of every group
//      of N = 8192 .. 65536, group by group, each group in the order of the
//      two-pass kernel ("A tiles of signal t, then B tiles of signal t - lag")
//      with its own ring of workspace slots and counters;
//   2. the fused items of N <= 4096: one CTA's worth of signals of one N
//      (4096 / N signals, or one), the chirp-DFT-chirp of the fused kernel;
//   3. the chunks of the b = 0 signals (2048 samples, or several small
//      signals of equal N).
// A pass-B tile waits for its signal's A tiles, a pass-A tile for the B
// tiles of the slot's previous occupant; both were taken from the queue
// earlier, by CTAs that are running, so every wait ends (bounded anyway: a
// timeout records LCT_DEV_TIMEOUT and raises the group's abort flag).
// Descriptors that do not match an item's N or kind are skipped and flagged.
#include "xft_twopass.cuh"

namespace {

using namespace xft;
using namespace xtp;

constexpr int RG_THREADS = 256;

// the fused item: up to SPC signals of N = 2^L from the index list ids
template <int L>
__device__ __forceinline__ void fused_item(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                                           const lct_desc* __restrict__ desc,
                                           const int32_t* __restrict__ ids, int cnt,
                                           const cpx<float>* __restrict__ tw, int32_t* __restrict__ status,
                                           cpx<float>* smem) {
    using S = shape<L>;
    constexpr int SPC = S::T >= RG_THREADS ? 1 : RG_THREADS / S::T;
    const int tid = threadIdx.x;
    const int sl = tid / S::T, i = tid - sl * S::T;
    bool active = sl < SPC && sl < cnt;
    const lct_desc D = desc[active ? ids[sl] : ids[0]];
    if (active && (D.log2n != L || D.kind != LCT_KIND_XFT || D.offset < 0)) {
        if (i == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        active = false;
    }
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
    cpx<float> v[S::E];
    if (sl < SPC) {
        cpx<float>* buf = smem + sl * S::NP;
#pragma unroll
        for (int e = 0; e < S::E; ++e) {
            const int n = i + e * S::T;
            cpx<float> f = {0.f, 0.f};
            if (active) f = ld_stream(in + D.offset + n);
            v[e] = cmul(f, pre_w<L, float>(D, n, decay));
        }
        if constexpr (S::T <= 32) dft_signal_warp<L, -1>(v, buf, i, tw);   // signal within a warp
        else dft_signal<L, -1>(v, buf, i, tw);
        if (active) {
            const float sc = (float)D.scale;
#pragma unroll
            for (int e = 0; e < S::E; ++e) {
                const int n = i + e * S::T;
                out[D.offset + n] = cscale(cmul(v[e], post_w<L, float>(D, n)), sc);
            }
        }
    }
    __syncthreads();                   // shared memory free for the next item
}

// a chunk of the diagonal (b = 0) signals: {pos, start, log2n, nsig}
__device__ __forceinline__ void diag_item(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
                                          const lct_desc* __restrict__ desc,
                                          const int32_t* __restrict__ ids, int4 ch,
                                          int32_t* __restrict__ status) {
    const int L = ch.z, N = 1 << L;
    const int len = ch.w > 1 ? (ch.w << L) : min(N - ch.y, kDiagChunk);
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const int j = ch.w > 1 ? (e >> L) : 0;
        const int n = ch.w > 1 ? (e & (N - 1)) : ch.y + e;
        const lct_desc& D = desc[ids[ch.x + j]];
        if (D.kind != LCT_KIND_DIAG || D.log2n != L || D.offset < 0) {
            if (n == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
            continue;
        }
        const uint32_t m2 = m_squared(n, N);
        const uint32_t off = (uint32_t)((D.out_c + 0x80000000ull) >> 32);
        const cpx<float> w = expi_turn32<true>(phase32(D.out_hi, m2) + off);
        out[D.offset + n] = cscale(cmul(in[D.offset + n], w), (float)D.scale);
    }
}

}  // namespace

// Tables of the persistent ragged kernel (k_ragged.cu).
struct lct_rg_tables {
    const void* tw[17];          // lct_twiddle_table(0, L)
};

namespace {

__global__ void __launch_bounds__(RG_THREADS, 3)
k_xft_ragged(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
             const lct_desc* __restrict__ desc, const int32_t* __restrict__ idx,
             const int4* __restrict__ items, int64_t n_items, const lct_rg_group* __restrict__ groups,
             const int4* __restrict__ chunks, cpx<float>* __restrict__ work,
             int32_t* __restrict__ sync, unsigned long long* __restrict__ queue,
             const lct_rg_tables tabs, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* smem = reinterpret_cast<cpx<float>*>(smem_raw);
    __shared__ long long s_item;
    const cpx<float>* const* tw = reinterpret_cast<const cpx<float>* const*>(tabs.tw);
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(queue, 1ull);
        __syncthreads();
        const int64_t it = s_item;
        if (it >= n_items) break;
        const int4 w = items[it];
        if (w.x == LCT_RG_TP) {
            const lct_rg_group g = groups[w.y];
            const int64_t p = ((int64_t)(uint32_t)w.z << 32) | (int64_t)(uint32_t)w.w;
            cpx<float>* gw = work + g.work_off;
            int32_t* gs = sync + g.sync_off;
            const int32_t* gi = idx + g.idx_off;
            switch (g.log2n) {
                case 13: tp_item<6, 7, float>(p, in, out, gw, gs, desc, 1, g.count, g.lag, g.slots, gi, status, tw[6], tw[7], smem); break;
                case 14: tp_item<7, 7, float>(p, in, out, gw, gs, desc, 1, g.count, g.lag, g.slots, gi, status, tw[7], tw[7], smem); break;
                case 15: tp_item<7, 8, float>(p, in, out, gw, gs, desc, 1, g.count, g.lag, g.slots, gi, status, tw[7], tw[8], smem); break;
                case 16: tp_item<8, 8, float>(p, in, out, gw, gs, desc, 1, g.count, g.lag, g.slots, gi, status, tw[8], tw[8], smem); break;
                default: if (threadIdx.x == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC); __syncthreads();
            }
        } else if (w.x == LCT_RG_FUSED) {
            const int32_t* ids = idx + w.z;
            switch (w.y) {
#define LCT_RG_CASE(L) case L: fused_item<L>(in, out, desc, ids, w.w, tw[L], status, smem); break;
                LCT_RG_CASE(1) LCT_RG_CASE(2) LCT_RG_CASE(3) LCT_RG_CASE(4) LCT_RG_CASE(5)
                LCT_RG_CASE(6) LCT_RG_CASE(7) LCT_RG_CASE(8) LCT_RG_CASE(9) LCT_RG_CASE(10)
                LCT_RG_CASE(11) LCT_RG_CASE(12)
#undef LCT_RG_CASE
                default: if (threadIdx.x == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC); __syncthreads();
            }
        } else {
            diag_item(in, out, desc, idx + w.z, chunks[w.y], status);
            __syncthreads();
        }
    }
}

}  // namespace

size_t lct_ragged_smem_bytes() {
    size_t m = (size_t)(4096 + 256) * sizeof(cpx<float>);          // fused items
    m = m > pt_shape<6, 7, float>::SMEM ? m : pt_shape<6, 7, float>::SMEM;
    m = m > pt_shape<7, 7, float>::SMEM ? m : pt_shape<7, 7, float>::SMEM;
    m = m > pt_shape<7, 8, float>::SMEM ? m : pt_shape<7, 8, float>::SMEM;
    m = m > pt_shape<8, 8, float>::SMEM ? m : pt_shape<8, 8, float>::SMEM;
    return m;
}

void lct_twopass_tiles(int log2n, int* cb, int* rb) {
    switch (log2n) {
        case 13: *cb = pt_shape<6, 7, float>::CB; *rb = pt_shape<6, 7, float>::RB; return;
        case 14: *cb = pt_shape<7, 7, float>::CB; *rb = pt_shape<7, 7, float>::RB; return;
        case 15: *cb = pt_shape<7, 8, float>::CB; *rb = pt_shape<7, 8, float>::RB; return;
        case 16: *cb = pt_shape<8, 8, float>::CB; *rb = pt_shape<8, 8, float>::RB; return;
        default: *cb = *rb = 0;
    }
}

int lct_ragged_fused_spc(int log2n) {
    const int t = log2n >= 4 ? (1 << (log2n - 4)) : 1;
    return t >= RG_THREADS ? 1 : RG_THREADS / t;
}

cudaError_t lct_launch_ragged(const void* in, void* out, const lct_desc* desc, const int32_t* idx,
                              const int4* items, int64_t n_items, const lct_rg_group* groups,
                              const int4* chunks, void* work, int32_t* sync, size_t sync_bytes,
                              const void* const* tw, int32_t* status, cudaStream_t stream) {
    static int per_sm[64] = {}, sms[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const size_t smem = lct_ragged_smem_bytes();
    if (!per_sm[dev]) {
        if ((e = cudaFuncSetAttribute(k_xft_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        int nb = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_xft_ragged, RG_THREADS, smem)) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return e;
        per_sm[dev] = nb > 0 ? nb : 1;
    }
    // the queue word and every group's counters start at zero
    if ((e = cudaMemsetAsync(sync, 0, sync_bytes, stream)) != cudaSuccess) return e;
    int64_t grid = (int64_t)per_sm[dev] * sms[dev];
    if (grid > n_items) grid = n_items;
    if (grid < 1) return cudaSuccess;
    lct_rg_tables tabs;
    for (int l = 0; l < 17; ++l) tabs.tw[l] = tw[l];
    k_xft_ragged<<<(unsigned)grid, RG_THREADS, smem, stream>>>(
        (const cpx<float>*)in, (cpx<float>*)out, desc, idx, items, n_items, groups, chunks,
        (cpx<float>*)work, sync + 2, reinterpret_cast<unsigned long long*>(sync), tabs, status);
    return cudaGetLastError();
}
