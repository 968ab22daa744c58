// The persistent two-pass form of the large-N XFT (k_twopass.cu), factored
// as one work item: the shapes, the descriptor lookup and tp_item, which
// runs pass-A or pass-B tile p of a launch's queue order.  Shared by the
// two-pass kernel and the persistent ragged kernel (k_ragged.cu).
#pragma once
#include "xft_engine.cuh"
#include "xft_chirp.cuh"
#include "xft_async.cuh"

namespace xtp {

using namespace xft;


template <int LN, class R>
__device__ __forceinline__ cpx<R> pre_tp(const lct_desc& D, int n, bool decay) {
    if constexpr (sizeof(R) == 4) return pre_chirp<LN>(D, n, decay);
    else return pre_chirp64<LN>(D, n, decay);
}
template <int LN, class R>
__device__ __forceinline__ cpx<R> post_tp(const lct_desc& D, int n) {
    if constexpr (sizeof(R) == 4) return post_chirp<LN>(D, n);
    else return post_chirp64<LN>(D, n);
}

// Descriptor of signal `sig` of the launch (through idx for ragged
// batches); a descriptor that does not match the kernel is flagged, and the
// signal skipped.
template <int LN>
__device__ __forceinline__ bool tp_signal(const lct_desc* __restrict__ desc, int desc_step,
                                          int64_t sig, const int32_t* __restrict__ idx,
                                          int32_t* status, lct_desc& D, int64_t& base) {
    const int64_t gsig = idx ? idx[sig] : sig;
    D = desc[desc_step ? gsig : 0];
    base = desc_step ? D.offset : gsig << LN;
    if (idx && (D.log2n != LN || D.kind != LCT_KIND_XFT || D.offset < 0)) {
        if (threadIdx.x == 0) atomicCAS(status, LCT_DEV_OK, LCT_DEV_BAD_DESC);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Persistent single-launch form: one grid of PT_THREADS-thread CTAs takes
// work items from a queue, pass-A tiles (GA columns) and pass-B tiles (GB
// rows) in the order
//   step t: the A tiles of signal t, then the B tiles of signal t - D,
// and keeps the intermediate of W = D + 2 signals in a ring of workspace
// slots (signal t in slot t mod W), small enough to stay in L2.  Per-slot
// counters (monotone over the launch) order the two passes: a B tile of
// signal s waits until all CB A tiles of s are stored; an A tile of signal
// t >= W waits until the RB B tiles of signal t - W have read the slot.
// Every wait is on items taken from the queue earlier, so it always ends;
// waits are bounded anyway (a timeout is recorded, never a hang).
// ---------------------------------------------------------------------------
constexpr int PT_THREADS = 256;
constexpr uint64_t kPtWaitNs = 2000000000ull;   // 2 s

template <int L1, int L2, class R>
struct pt_shape {
    static constexpr int LN = L1 + L2, N = 1 << LN, N1 = 1 << L1, N2 = 1 << L2;
    static constexpr int T1 = shape<L1>::T, T2 = shape<L2>::T;
    static constexpr int GA = PT_THREADS / T1;            // columns per A tile
    static constexpr int GB = PT_THREADS / T2;            // rows per B tile
    static constexpr int CB = N2 / GA, RB = N1 / GB;      // A and B tiles per signal
    static constexpr int STR = padded_len<L1>() + 1;      // odd: column buffers on distinct banks
    static constexpr int NPB = padded_len<L2>();
    static constexpr int TS = GB + 16 / T2;               // transpose row stride (conflict-free)
    static constexpr size_t SA = (size_t)GA * STR, SB1 = (size_t)GB * NPB, SB2 = (size_t)N2 * TS;
    static constexpr size_t ELEMS = SA > SB1 ? (SA > SB2 ? SA : SB2) : (SB1 > SB2 ? SB1 : SB2);
    static constexpr size_t SMEM = ELEMS * sizeof(cpx<R>);
    static_assert(CB >= 1 && RB >= 1, "tile larger than the signal");
};

template <class R>
__device__ __forceinline__ cpx<R> ld_l2(const cpx<R>* p);
template <>
__device__ __forceinline__ cpx<float> ld_l2<float>(const cpx<float>* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
template <>
__device__ __forceinline__ cpx<double> ld_l2<double>(const cpx<double>* p) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}

// Work item p (0 <= p < count (CB + RB)) of a two-pass launch over `count`
// signals: in the order "A tiles of signal t, then B tiles of signal t - lag",
// pass A or B of one tile.  Every thread of the CTA calls it (it
// synchronises); smem: P::SMEM bytes.  sync: abort flag at sync[2],
// counters at sync[4 ..] (the queue word sync[0..1] is the caller's).
template <int L1, int L2, class R>
__device__ __forceinline__ void tp_item(int64_t p, const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out,
                                        cpx<R>* __restrict__ work, int32_t* __restrict__ sync,
                                        const lct_desc* __restrict__ desc, int desc_step,
                                        int64_t count, int64_t lag, int64_t slots,
                                        const int32_t* __restrict__ idx, int32_t* __restrict__ status,
                                        const cpx<R>* __restrict__ tw1, const cpx<R>* __restrict__ tw2,
                                        cpx<R>* smem) {
    using P = pt_shape<L1, L2, R>;
    constexpr int LN = P::LN, N = P::N, N1 = P::N1, N2 = P::N2, T1 = P::T1, T2 = P::T2;
    constexpr int GA = P::GA, GB = P::GB, CB = P::CB, RB = P::RB;
    (void)N1;
    int32_t* abort_flag = sync + 2;
    int32_t* cnt_a = sync + 4;
    int32_t* cnt_b = cnt_a + slots;
    const int tid = threadIdx.x;
    const int64_t a_head = lag * CB, mid = (count - lag) * (CB + RB);
    // decode: pass, signal, tile
    bool is_a;
    int64_t sig;
    int tile;
    if (p < a_head) {
        is_a = true; sig = p / CB; tile = (int)(p % CB);
    } else if ((p -= a_head) < mid) {
        const int64_t t = lag + p / (CB + RB);
        const int r = (int)(p % (CB + RB));
        is_a = r < CB;
        sig = is_a ? t : t - lag;
        tile = is_a ? r : r - CB;
    } else {
        p -= mid;
        is_a = false; sig = count - lag + p / RB; tile = (int)(p % RB);
    }
    const int64_t slot = sig % slots;
    const int32_t round = (int32_t)(sig / slots);       // earlier occupants of the slot
    cpx<R>* y = work + slot * (int64_t)N;
    lct_desc D;
    int64_t base;
    const bool active = tp_signal<LN>(desc, desc_step, sig, idx, status, D, base);

    if (is_a) {
        const int s = tid % GA, i = tid / GA;
        const int n2 = tile * GA + s;
        const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;
        cpx<R> v[shape<L1>::E];
#pragma unroll
        for (int e = 0; e < shape<L1>::E; ++e) {
            const int n = n2 + N2 * (i + e * T1);
            cpx<R> f = {R(0), R(0)};
            if (active) f = ld_stream(in + base + n);
            v[e] = cmul(f, pre_tp<LN, R>(D, n, decay));
        }
        dft_signal<L1, -1>(v, smem + s * P::STR, i, tw1);
        const cpx<R> w0 = twiddle_exact<R, -1>((n2 * i) & (N - 1), N);
        cpx<R> ws[shape<L1>::E];
        twiddle_powers<shape<L1>::E>(twiddle_exact<R, -1>((n2 * T1) & (N - 1), N), ws);
        // the slot is free once the previous occupant's B tiles have read it
        if (tid == 0 && round > 0 && !xasync::wait_geq(cnt_b + slot, round * RB, abort_flag, kPtWaitNs))
            atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
        __syncthreads();
#pragma unroll
        for (int e = 0; e < shape<L1>::E; ++e)
            y[(i + e * T1) * N2 + n2] = cmul(v[e], cmul(w0, ws[e]));
        __syncthreads();                             // stores issued, shared memory free
        if (tid == 0) {
            __threadfence();
            atomicAdd(cnt_a + slot, 1);
        }
    } else {
        const int r = tid / T2, i = tid % T2;
        if (tid == 0 && !xasync::wait_geq(cnt_a + slot, (round + 1) * CB, abort_flag, kPtWaitNs))
            atomicCAS(status, LCT_DEV_OK, LCT_DEV_TIMEOUT);
        __syncthreads();
        const int k1b = tile * GB;
        cpx<R> v[shape<L2>::E];
        const cpx<R>* row = y + (int64_t)(k1b + r) * N2;
#pragma unroll
        for (int e = 0; e < shape<L2>::E; ++e) v[e] = ld_l2<R>(row + i + e * T2);
        dft_signal<L2, -1>(v, smem + r * P::NPB, i, tw2);
        __syncthreads();                             // slot read, engine buffers free
        if (tid == 0) atomicAdd(cnt_b + slot, 1);
#pragma unroll
        for (int e = 0; e < shape<L2>::E; ++e) smem[(i + e * T2) * P::TS + r] = v[e];
        __syncthreads();
        if (active) {
            const R sc = (R)D.scale;
            const int rr = tid % GB, q = tid / GB;   // row k1b + rr, k2 = q + e T2
#pragma unroll
            for (int e = 0; e < shape<L2>::E; ++e) {
                const int k2 = q + e * T2;
                const int k = k1b + rr + N1 * k2;
                out[base + k] = cscale(cmul(smem[k2 * P::TS + rr], post_tp<LN, R>(D, k)), sc);
            }
        }
        __syncthreads();                             // shared memory free for the next item
    }
}

}  // namespace xtp
