// Large-N XFT in two passes over memory (four-step factorisation of the
// N-point DFT of Sec. 3, N = N1 N2):
//   n = n2 + N2 n1, k = k1 + N1 k2,
//   X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_N^{n2 k1} sum_{n1} W_{N1}^{n1 k1} u[n2 + N2 n1]
// with u the pre-chirped input and W_M = e^{-2 pi i / M} (forward sign).
//
// Pass A (a CTA per signal and group of G consecutive columns n2): loads u
// (pre-chirp on the fly; each row n1 of the group is G consecutive samples),
// runs the N1-point DFT down every column with the Stockham engine, multiplies
// by W_N^{n2 k1} and stores Y[k1][n2] row-major in a workspace.
// Pass B (a CTA per signal and group of G consecutive rows k1): N2-point DFT
// along every row (contiguous loads), a transpose through shared memory, then
// X[k1 + N1 k2] with the post-chirp and scale (G consecutive k1 per k2).
//
// Every sample is read and written twice (32 B/point for complex64); the
// host runs the passes over chunks of signals to bound the workspace.
#include "xft_engine.cuh"
#include "xft_chirp.cuh"

namespace {

using namespace xft;

constexpr int G = 16;                  // columns (pass A) or rows (pass B) per CTA

template <int L1, class R>
struct pass_a_shape {
    static constexpr int T = shape<L1>::T;                      // threads per column
    static constexpr int THREADS = G * T;
    // per-column shared-memory stride: the engine's padded length plus one, an
    // odd number of samples, so the G columns of a half-warp hit distinct banks
    static constexpr int STR = padded_len<L1>() + 1;
    static constexpr size_t SMEM = (size_t)G * STR * sizeof(cpx<R>);
};

template <int L2, class R>
struct pass_b_shape {
    static constexpr int T = shape<L2>::T;                      // threads per row
    static constexpr int THREADS = G * T;
    static constexpr int NP = padded_len<L2>();
    // the transpose tile [N2][G + 1] reuses the engine buffers
    static constexpr size_t ENGINE = (size_t)G * NP;
    static constexpr size_t TILE = (size_t)(1 << L2) * (G + 1);
    static constexpr size_t SMEM = (ENGINE > TILE ? ENGINE : TILE) * sizeof(cpx<R>);
};

// Resident threads per SM for the register budget: 1024 (complex64, <= 64
// registers), 512 (complex128, <= 128).
template <class R, int THREADS>
constexpr int tp_min_blocks() {
    constexpr int per_sm = sizeof(R) == 4 ? 1024 : 512;
    return per_sm / THREADS > 0 ? per_sm / THREADS : 1;
}

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

// Descriptor of signal `first + j` of the launch (through idx for ragged
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

template <int L1, int L2, class R>
__global__ void __launch_bounds__(pass_a_shape<L1, R>::THREADS,
                                  (tp_min_blocks<R, pass_a_shape<L1, R>::THREADS>()))
k_xft_pass_a(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ work,
             const lct_desc* __restrict__ desc, int desc_step, int64_t first,
             const int32_t* __restrict__ idx, int32_t* __restrict__ status,
             const cpx<R>* __restrict__ tw1) {
    using S1 = shape<L1>;
    using A = pass_a_shape<L1, R>;
    constexpr int LN = L1 + L2, N = 1 << LN, N2 = 1 << L2, CB = N2 / G, T1 = S1::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x, s = tid % G, i = tid / G;
    const int64_t j = blockIdx.x / CB;                  // signal within the chunk
    const int n2 = (int)(blockIdx.x % CB) * G + s;      // this thread's column
    lct_desc D;
    int64_t base;
    const bool active = tp_signal<LN>(desc, desc_step, first + j, idx, status, D, base);
    const bool decay = (D.flags & LCT_FLAG_DECAY) != 0;

    cpx<R> v[S1::E];
#pragma unroll
    for (int e = 0; e < S1::E; ++e) {
        const int n = n2 + N2 * (i + e * T1);
        cpx<R> f = {R(0), R(0)};
        if (active) f = ld_stream(in + base + n);
        v[e] = cmul(f, pre_tp<LN, R>(D, n, decay));
    }
    dft_signal<L1, -1>(v, smem + s * A::STR, i, tw1);
    // inter-pass twiddle W_N^{n2 k1}, k1 = i + e T1: W_N^{n2 i} times the
    // powers of W_N^{n2 T1} (product tree, a few roundings deep)
    const cpx<R> w0 = twiddle_exact<R, -1>((n2 * i) & (N - 1), N);
    cpx<R> ws[S1::E];
    twiddle_powers<S1::E>(twiddle_exact<R, -1>((n2 * T1) & (N - 1), N), ws);
    if (active) {
        cpx<R>* y = work + j * (int64_t)N + n2;
#pragma unroll
        for (int e = 0; e < S1::E; ++e) y[(i + e * T1) * N2] = cmul(v[e], cmul(w0, ws[e]));
    }
}

template <int L1, int L2, class R>
__global__ void __launch_bounds__(pass_b_shape<L2, R>::THREADS,
                                  (tp_min_blocks<R, pass_b_shape<L2, R>::THREADS>()))
k_xft_pass_b(const cpx<R>* __restrict__ work, cpx<R>* __restrict__ out,
             const lct_desc* __restrict__ desc, int desc_step, int64_t first,
             const int32_t* __restrict__ idx, int32_t* __restrict__ status,
             const cpx<R>* __restrict__ tw2) {
    using S2 = shape<L2>;
    using B = pass_b_shape<L2, R>;
    constexpr int LN = L1 + L2, N = 1 << LN, N1 = 1 << L1, N2 = S2::N, RB = N1 / G, T2 = S2::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* smem = reinterpret_cast<cpx<R>*>(smem_raw);
    const int tid = threadIdx.x, r = tid / T2, i = tid % T2;
    const int64_t j = blockIdx.x / RB;
    const int k1b = (int)(blockIdx.x % RB) * G;          // first row of the group
    lct_desc D;
    int64_t base;
    const bool active = tp_signal<LN>(desc, desc_step, first + j, idx, status, D, base);

    cpx<R> v[S2::E];
    const cpx<R>* y = work + j * (int64_t)N + (int64_t)(k1b + r) * N2;
#pragma unroll
    for (int e = 0; e < S2::E; ++e) v[e] = ld_stream(y + i + e * T2);
    dft_signal<L2, -1>(v, smem + r * B::NP, i, tw2);
    __syncthreads();                                     // engine buffers free
#pragma unroll
    for (int e = 0; e < S2::E; ++e) smem[(i + e * T2) * (G + 1) + r] = v[e];
    __syncthreads();
    if (!active) return;
    const R sc = (R)D.scale;
    const int rr = tid % G, q = tid / G;                 // row k1b + rr, k2 = q + e T2
#pragma unroll
    for (int e = 0; e < S2::E; ++e) {
        const int k2 = q + e * T2;
        const int k = k1b + rr + N1 * k2;
        out[base + k] = cscale(cmul(smem[k2 * (G + 1) + rr], post_tp<LN, R>(D, k)), sc);
    }
}

template <int L1, int L2, class R>
cudaError_t launch_tp(const void* in, void* out, void* work, const lct_desc* desc, int desc_step,
                      int64_t first, int64_t count, const int32_t* idx, int32_t* status,
                      const void* tw1, const void* tw2, cudaStream_t stream) {
    using A = pass_a_shape<L1, R>;
    using B = pass_b_shape<L2, R>;
    constexpr int N1 = 1 << L1, N2 = 1 << L2;
    auto ka = k_xft_pass_a<L1, L2, R>;
    auto kb = k_xft_pass_b<L1, L2, R>;
    cudaError_t e;
    if (A::SMEM > 48 * 1024 &&
        (e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)A::SMEM)) != cudaSuccess)
        return e;
    if (B::SMEM > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM)) != cudaSuccess)
        return e;
    const int64_t blocks_a = count * (N2 / G), blocks_b = count * (N1 / G);
    if (blocks_a > 0x7fffffffLL || blocks_b > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    ka<<<(unsigned)blocks_a, A::THREADS, A::SMEM, stream>>>(
        (const cpx<R>*)in, (cpx<R>*)work, desc, desc_step, first, idx, status, (const cpx<R>*)tw1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kb<<<(unsigned)blocks_b, B::THREADS, B::SMEM, stream>>>(
        (const cpx<R>*)work, (cpx<R>*)out, desc, desc_step, first, idx, status, (const cpx<R>*)tw2);
    return cudaGetLastError();
}

template <class R>
cudaError_t tp_dispatch(int log2n, const void* in, void* out, void* work, const lct_desc* desc,
                        int desc_step, int64_t first, int64_t count, const int32_t* idx,
                        int32_t* status, const void* tw1, const void* tw2, cudaStream_t stream) {
    switch (log2n) {
        case 13: return launch_tp<6, 7, R>(in, out, work, desc, desc_step, first, count, idx, status, tw1, tw2, stream);
        case 14: return launch_tp<7, 7, R>(in, out, work, desc, desc_step, first, count, idx, status, tw1, tw2, stream);
        case 15: return launch_tp<7, 8, R>(in, out, work, desc, desc_step, first, count, idx, status, tw1, tw2, stream);
        case 16: return launch_tp<8, 8, R>(in, out, work, desc, desc_step, first, count, idx, status, tw1, tw2, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool lct_twopass_supported(int dtype, int log2n) {
    (void)dtype;
    return log2n >= 13 && log2n <= 16;
}

void lct_twopass_split(int log2n, int* l1, int* l2) {
    *l1 = log2n / 2;
    *l2 = log2n - log2n / 2;
}

cudaError_t lct_launch_twopass(int dtype, int log2n, const void* in, void* out, void* work,
                               const lct_desc* desc, int desc_step, int64_t first, int64_t count,
                               const int32_t* idx, int32_t* status, const void* tw1,
                               const void* tw2, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if (dtype == 0)
        return tp_dispatch<float>(log2n, in, out, work, desc, desc_step, first, count, idx, status,
                                  tw1, tw2, stream);
    return tp_dispatch<double>(log2n, in, out, work, desc, desc_step, first, count, idx, status,
                               tw1, tw2, stream);
}
