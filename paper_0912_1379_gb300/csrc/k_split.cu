// Split-precision XFT (complex64 in/out, N = 16 .. 4096): the radix-16 DFT
// passes of the Stockham plan run as matrix products on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation); chirps, twiddles and a leading
// radix-2/4/8 pass (when log2 N is not a multiple of 4) stay on the CUDA
// cores.  Chirp phases are the exact fixed-point phases of the native path.
//
// One radix-16 DFT of a vector u (16 complex) is the real product
//   [Re y; Im y] (32) = Freal (32 x 32) [Re u_0, Im u_0, Re u_1, ...] (32)
// with, for F_jn = e^{-2 pi i j n / 16},
//   Freal[j][2n] = Re F_jn,       Freal[j][2n+1] = -Im F_jn,
//   Freal[16+j][2n] = Im F_jn,    Freal[16+j][2n+1] = Re F_jn.
// A warp multiplies Freal by 8 vectors at a time: 2 row tiles (the real and
// the imaginary outputs) x 2 k tiles, each one m16n8k16 product.  Operands
// are split u = u_hi + u_lo, Freal = F_hi + F_lo, with hi = rn(x) and
// lo = rn(x - hi) in FP16 or BF16, and the product is taken as
// F_hi u_hi + F_hi u_lo + F_lo u_hi (TERMS = 3; the dropped F_lo u_lo is
// below the FP32 accumulation error for FP16 halves) or F_hi u_hi (TERMS = 1).
// FP16 operands are scaled per signal by a power of two (max |component| < 1
// after the pre-chirp), which keeps every pass inside the FP16 range
// (|value| < 16^3 sqrt 2 after three passes) and the low halves mostly normal.
//
// A CTA of 256 threads transforms a tile of 4096 samples (4096/N signals).
// Pass structure: every pass first gathers its operands from shared memory
// into registers (twiddled and split), synchronises, then multiplies and
// scatters to the Stockham output positions of the same buffer, so a single
// 32 KB buffer serves all passes.  Fragment layouts (PTX ISA, m16n8k16 with
// 16-bit operands, lane = 4 g + t):
//   A reg q: rows g + 8 (q & 1), columns 2t + 8 (q >> 1) + {0, 1}
//   B reg h: rows 2t + 8 h + {0, 1}, column g
//   D elem q: row g + 8 (q >> 1), column 2t + (q & 1)
// Shared memory is XOR-swizzled on 8-byte slots: slot a is stored at
// a ^ x(a), x(a) = M * bits(a >> 4 & 255) over GF(2) with the 4 x 8 matrix
// rows {223, 25, 117, 170}; for every access pattern of every N this puts the
// 16 lanes of each half-warp on 16 different bank pairs.  Because the map is
// linear, an address whose pieces (signal, vector, element) occupy disjoint
// bits is swizzled piecewise: swz(a + c) = swz(a) ^ swz(c), with swz of the
// compile-time pieces folded by the compiler.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "xft_engine.cuh"
#include "xft_chirp.cuh"
#include "xft_async.cuh"

namespace {

using namespace xft;

constexpr int TILE_L = 12, TILE = 1 << TILE_L, T = 256;

// Swizzle: 16-entry nibble tables for address bits 4..7 and 8..11.
constexpr int kSwzRows[4] = {223, 25, 117, 170};
constexpr uint64_t swz_table(int shift) {
    uint64_t t = 0;
    for (int v = 0; v < 16; ++v) {
        int x = 0;
        for (int r = 0; r < 4; ++r) {
            int bits = (v << shift) & kSwzRows[r];
            int par = 0;
            while (bits) { par ^= bits & 1; bits >>= 1; }
            x |= par << r;
        }
        t |= (uint64_t)x << (4 * v);
    }
    return t;
}
constexpr uint64_t kSwzLo = swz_table(0), kSwzHi = swz_table(4);

__device__ __forceinline__ int swz(int a) {
    const int lo = (int)(kSwzLo >> (4 * ((a >> 4) & 15))) & 15;
    const int hi = (int)(kSwzHi >> (4 * ((a >> 8) & 15))) & 15;
    return a ^ lo ^ hi;
}

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool BF>
__device__ __forceinline__ float2 unpack2(uint32_t v) {
    if constexpr (BF) {
        __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
        return __bfloat1622float2(h);
    } else {
        __half2 h = *reinterpret_cast<__half2*>(&v);
        return __half22float2(h);
    }
}

// hi = rn(a, b), lo = rn((a, b) - hi)
template <bool BF>
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pack2<BF>(a, b);
    const float2 h = unpack2<BF>(hi);
    lo = pack2<BF>(a - h.x, b - h.y);
}

template <bool BF>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    if constexpr (BF) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
            "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// cos(2 pi k / 16), k = 0..15, rounded to FP32 (cos pi/8, sin pi/8, 1/sqrt 2).
__constant__ float kCos16[16] = {
    1.0f, 0.92387953251128676f, 0.70710678118654752f, 0.38268343236508977f,
    0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128676f,
    -1.0f, -0.92387953251128676f, -0.70710678118654752f, -0.38268343236508977f,
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128676f};

// Freal[rho][kappa] (rho, kappa < 32): F_jn = cos(theta) - i sin(theta),
// theta = 2 pi (j n mod 16) / 16, sin(theta) = cos(theta - pi/2).
__device__ __forceinline__ float freal(int rho, int kappa) {
    const int k = ((rho & 15) * (kappa >> 1)) & 15;
    const float c = kCos16[k], s = -kCos16[(k + 12) & 15];    // F = c + i s
    if (rho < 16) return (kappa & 1) ? -s : c;
    return (kappa & 1) ? c : s;
}

// 2^ex (UP) or 2^-ex for the bit pattern m of max |component| = f 2^ex,
// f in [0.5, 1) (1 when the signal is zero).  ex is clamped to [-125, 125]
// so that both factors are normal numbers; a clamped signal's scaled maximum
// stays below 8, inside the FP16 range through every pass.
template <bool UP>
__device__ __forceinline__ float exp2_of_max(uint32_t m) {
    int ex = 0;
    if (m) frexpf(__uint_as_float(m), &ex);
    ex = min(max(ex, -125), 125);
    return ldexpf(1.f, UP ? ex : -ex);
}

// Signal s of the CTA's tile: its descriptor and first element.
struct sig_ref {
    const lct_desc* D;
    int64_t base;
    bool valid;
};
template <int L>
__device__ __forceinline__ sig_ref signal_of(const lct_desc* __restrict__ desc, int desc_step,
                                             int64_t count, int64_t tile, int s) {
    const int64_t sig = tile * (TILE >> L) + s;
    sig_ref r;
    r.valid = sig < count;
    r.D = desc + (desc_step ? (r.valid ? sig : 0) : 0);
    r.base = desc_step ? r.D->offset : sig << L;
    return r;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s bound on every mbarrier wait

// Bulk-async copy of tile `tile`'s input into the linear stage (one copy when
// the tile's signals are contiguous, else one per signal issued by the lanes
// of warp 0).  Called by all of warp 0.
template <int L>
__device__ __forceinline__ void issue_tile(const cpx<float>* in, const lct_desc* desc,
                                           int desc_step, int contiguous, int64_t count,
                                           int64_t tile, cpx<float>* stage, uint64_t* bar,
                                           int lane) {
    constexpr int N = 1 << L, S = TILE >> L;
    const int64_t first = tile * S;
    const int64_t left = count - first;
    const int ns = left < S ? (int)left : S;
    const uint32_t bytes = (uint32_t)ns * N * (uint32_t)sizeof(cpx<float>);
    if (lane == 0) xasync::mbar_arrive_expect_tx(bar, bytes);
    __syncwarp();
    if (contiguous) {
        if (lane == 0) {
            const int64_t base = desc_step ? desc[first].offset : first * (int64_t)N;
            xasync::bulk_g2s(stage, in + base, bytes, bar);
        }
    } else {
        for (int s = lane; s < ns; s += 32)
            xasync::bulk_g2s(stage + s * N, in + desc[first + s].offset,
                             N * (uint32_t)sizeof(cpx<float>), bar);
    }
}

// ASYNC: inputs arrive by bulk-async copies into a linear stage, the next
// tile's copy overlapping this tile's DFT passes (signal starts 16-byte
// aligned, checked on the host); otherwise plain streaming loads.
template <int L, bool BF, int TERMS, bool ASYNC>
__global__ void __launch_bounds__(T, 2)
k_xft_split(const cpx<float>* __restrict__ in, cpx<float>* __restrict__ out,
            const lct_desc* __restrict__ desc, int desc_step, int64_t count,
            const cpx<float>* __restrict__ tw, int64_t ntiles, int contiguous,
            int32_t* __restrict__ status) {
    constexpr int N = 1 << L, S = TILE >> L;      // signals per tile
    constexpr int R0L = L & 3;                     // leading CUDA-core pass radix 2^R0L (0: none)
    constexpr int PT = L >> 2;                     // tensor-core passes
    constexpr int VS = N / 16;                     // radix-16 vectors per signal
    constexpr int FR = R0L > 0 ? (1 << R0L) : 16;   // first radix of the Stockham plan
    constexpr bool SCALED = !BF;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* buf = reinterpret_cast<cpx<float>*>(smem_raw);
    cpx<float>* stage = buf + TILE;                        // ASYNC only
    __shared__ uint32_t s_amax[S];
    __shared__ __align__(8) uint64_t bar[1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;

    // constant A fragments of Freal: [row tile][k tile][reg], hi and lo halves
    uint32_t ahi[2][2][4], alo[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int kt = 0; kt < 2; ++kt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = 16 * mt + g + ((q & 1) ? 8 : 0);
                const int kk = 16 * kt + 2 * t + ((q & 2) ? 8 : 0);
                split2<BF>(freal(r, kk), freal(r, kk + 1), ahi[mt][kt][q], alo[mt][kt][q]);
            }

    if (ASYNC) {
        if (blockIdx.x >= ntiles) return;
        if (tid == 0) {
            xasync::mbar_init(bar, 1);
            xasync::fence_mbar_init();
        }
        __syncthreads();
        if (warp == 0)
            issue_tile<L>(in, desc, desc_step, contiguous, count, blockIdx.x, stage, bar, lane);
    }
    uint32_t parity = 0;

    // persistent loop over tiles of 4096 samples
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (SCALED)
        for (int s = tid; s < S; s += T) s_amax[s] = 0u;
    if (ASYNC) {
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
    } else if (SCALED) {
        __syncthreads();
    }

    // load + pre-chirp (tile position n = tid + e T; signal n >> L), and the
    // signals' max |component| (FP16 modes)
#pragma unroll 4
    for (int e = 0; e < 16; ++e) {
        const int n = tid + e * T, s = n >> L, nl = n & (N - 1);
        const sig_ref r = signal_of<L>(desc, desc_step, count, tile, s);
        cpx<float> f = {0.f, 0.f};
        if (r.valid) {
            const bool decay = (r.D->flags & LCT_FLAG_DECAY) != 0;
            const cpx<float> x = ASYNC ? stage[n] : ld_stream(in + r.base + nl);
            f = cmul(x, pre_chirp<L>(*r.D, nl, decay));
        }
        buf[swz(tid) ^ swz(e * T)] = f;
        if (SCALED) {
            uint32_t m = __float_as_uint(fmaxf(fabsf(f.x), fabsf(f.y)));
            if (L >= 5) {                   // the warp's 32 samples share one signal
                m = __reduce_max_sync(0xffffffffu, m);
                if (lane == 0 && m) atomicMax(&s_amax[s], m);
            } else if (m) {
                atomicMax(&s_amax[s], m);
            }
        }
    }
    __syncthreads();                     // work written, stage fully read
    if (ASYNC && warp == 0 && tile + gridDim.x < ntiles) {
        xasync::fence_proxy_async_smem();
        issue_tile<L>(in, desc, desc_step, contiguous, count, tile + gridDim.x, stage, bar, lane);
    }

    // leading radix 2^R0L pass on the CUDA cores (no twiddles: Ns = 1)
    if constexpr (R0L > 0) {
        constexpr int R0 = 1 << R0L, NV = N / R0, C = 16 / R0;
        cpx<float> u[C][R0];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int ivg = tid + c * T, s = ivg / NV, iv = ivg % NV;
#pragma unroll
            for (int j = 0; j < R0; ++j) u[c][j] = buf[swz(s * N + iv) ^ swz(j * NV)];
            if (SCALED) {
                const float sc = exp2_of_max<false>(s_amax[s]);
#pragma unroll
                for (int j = 0; j < R0; ++j) u[c][j] = cscale(u[c][j], sc);
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int ivg = tid + c * T, s = ivg / NV, iv = ivg % NV;
            dft<R0, -1>(u[c]);
#pragma unroll
            for (int j = 0; j < R0; ++j) buf[swz(s * N + iv * R0) ^ j] = u[c][j];
        }
        __syncthreads();
    }

    // radix-16 passes on the tensor cores
#pragma unroll
    for (int p = 0; p < PT; ++p) {
        const int pe = p + (R0L > 0 ? 1 : 0);                       // engine pass index
        const int NS = pe == 0 ? 1 : FR << (4 * (pe - 1));   // sub-length Ns of the pass
        const int TW_OFF = NS - FR;                           // its offset in the table
        uint32_t bh[4][2][2], bl[4][2][2];
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
            const int ivg = warp * 32 + grp * 8 + g, s = ivg / VS, iv = ivg % VS;
            const int k = iv & (NS - 1);
            const int rbase = swz(s * N + iv);
            const float sc = (SCALED && R0L == 0 && p == 0) ? exp2_of_max<false>(s_amax[s]) : 1.f;
#pragma unroll
            for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int n = 8 * kt + t + 4 * h;
                    cpx<float> u = buf[rbase ^ swz(n * VS)];
                    if (NS > 1 && n > 0) u = cmul(u, ld_tw<float>(tw + TW_OFF + (n - 1) * NS + k));
                    if (SCALED && R0L == 0 && p == 0) u = cscale(u, sc);
                    if (TERMS == 3) split2<BF>(u.x, u.y, bh[grp][kt][h], bl[grp][kt][h]);
                    else bh[grp][kt][h] = pack2<BF>(u.x, u.y);
                }
        }
        __syncthreads();
        const int xg = swz(g * NS);       // output j = g + 8 (q >> 1): pieces g NS and 8 NS
#pragma unroll
        for (int grp = 0; grp < 4; ++grp) {
            float d[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int q = 0; q < 4; ++q) d[mt][q] = 0.f;
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) {
                    mma16816<BF>(d[mt], ahi[mt][kt], bh[grp][kt][0], bh[grp][kt][1]);
                    if (TERMS == 3) {
                        mma16816<BF>(d[mt], ahi[mt][kt], bl[grp][kt][0], bl[grp][kt][1]);
                        mma16816<BF>(d[mt], alo[mt][kt], bh[grp][kt][0], bh[grp][kt][1]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ovg = warp * 32 + grp * 8 + 2 * t + (q & 1);
                const int s = ovg / VS, ov = ovg % VS, ok = ov & (NS - 1);
                buf[swz(s * N + (ov - ok) * 16 + ok) ^ xg ^ swz((q & 2) ? 8 * NS : 0)] =
                    {d[0][q], d[1][q]};
            }
        }
        __syncthreads();
    }

    // post-chirp, scale, store (natural order)
#pragma unroll 4
    for (int e = 0; e < 16; ++e) {
        const int n = tid + e * T, s = n >> L, nl = n & (N - 1);
        const sig_ref r = signal_of<L>(desc, desc_step, count, tile, s);
        if (!r.valid) continue;
        float sc = (float)r.D->scale;
        if (SCALED) sc *= exp2_of_max<true>(s_amax[s]);
        out[r.base + nl] = cscale(cmul(buf[swz(tid) ^ swz(e * T)], post_chirp<L>(*r.D, nl)), sc);
    }
    __syncthreads();                     // buf and s_amax are reused by the next tile
    }
}

template <int L, bool BF, int TERMS, bool ASYNC>
cudaError_t launch_t(const void* in, void* out, const lct_desc* desc, int desc_step,
                     int64_t count, const void* tw, int contiguous, int32_t* status,
                     cudaStream_t stream) {
    constexpr int S = TILE >> L;
    const size_t smem = (ASYNC ? 2 : 1) * (size_t)TILE * sizeof(cpx<float>);
    auto kern = k_xft_split<L, BF, TERMS, ASYNC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = (count + S - 1) / S;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem)) != cudaSuccess)
        return e;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)sms * std::max(per_sm, 1));
    kern<<<(unsigned)grid, T, smem, stream>>>((const cpx<float>*)in, (cpx<float>*)out, desc,
                                              desc_step, count, (const cpx<float>*)tw, ntiles,
                                              contiguous, status);
    return cudaGetLastError();
}

template <int L, bool ASYNC>
cudaError_t launch_mode(int mode, const void* in, void* out, const lct_desc* desc, int desc_step,
                        int64_t count, const void* tw, int contiguous, int32_t* status,
                        cudaStream_t stream) {
    switch (mode) {
        case 1: return launch_t<L, true, 3, ASYNC>(in, out, desc, desc_step, count, tw, contiguous, status, stream);
        case 2: return launch_t<L, false, 3, ASYNC>(in, out, desc, desc_step, count, tw, contiguous, status, stream);
        case 3: return launch_t<L, false, 1, ASYNC>(in, out, desc, desc_step, count, tw, contiguous, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int L>
cudaError_t launch_l(int mode, const void* in, void* out, const lct_desc* desc, int desc_step,
                     int64_t count, const void* tw, int async_ok, int contiguous, int32_t* status,
                     cudaStream_t stream) {
    if (async_ok)
        return launch_mode<L, true>(mode, in, out, desc, desc_step, count, tw, contiguous, status, stream);
    return launch_mode<L, false>(mode, in, out, desc, desc_step, count, tw, 0, status, stream);
}

}  // namespace

bool lct_split_supported(int dtype, int log2n) { return dtype == 0 && log2n >= 4 && log2n <= 12; }

cudaError_t lct_launch_split(int mode, int log2n, const void* in, void* out, const lct_desc* desc,
                             int desc_step, int64_t count, const void* tw, int async_ok,
                             int contiguous, int32_t* status, cudaStream_t stream) {
    switch (log2n) {
#define LCT_CASE(L) \
    case L: return launch_l<L>(mode, in, out, desc, desc_step, count, tw, async_ok, contiguous, status, stream);
        LCT_CASE(4) LCT_CASE(5) LCT_CASE(6) LCT_CASE(7) LCT_CASE(8) LCT_CASE(9) LCT_CASE(10)
        LCT_CASE(11) LCT_CASE(12)
#undef LCT_CASE
        default: return cudaErrorInvalidValue;
    }
}
