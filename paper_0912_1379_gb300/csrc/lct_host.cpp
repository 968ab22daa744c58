// Host side of the LCT library: parameter validation, exact phase constants,
// plans, and dispatch to the kernels.  Implements include/lct.h.
//
// Phase constants.  The chirp coefficients (Sec. 3, Algorithm, steps 1-2)
//   Re(beta_in)/(2 pi)  = Re(a/b) pi / (32 N)
//   Re(beta_out)/(2 pi) = Re(b d) / (2 pi N)
// are evaluated in double-double arithmetic (about 106 significant bits)
// from the exact FP64 parameters and reduced modulo one turn into 128-bit
// fixed-point fractions.  The output constant e^{-i pi (N-1)^2/(2N)} is an
// exact dyadic turn fraction; the argument of dx/sqrt(2 pi i b) is added to
// it in double precision.
#include "lct_internal.h"
#include "../../include/lct.h"

#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <map>
#include <numeric>
#include <queue>
#include <string>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// double-double arithmetic (Dekker / Knuth error-free transformations)
// ---------------------------------------------------------------------------
struct dd { double hi, lo; };

dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul(b, {q1, 0.0}));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul(b, {q2, 0.0}));
    double q3 = r.hi / b.hi;
    return dd_add(quick_two_sum(q1, q2), {q3, 0.0});
}
dd dd_ldexp(dd a, int e) { return {std::ldexp(a.hi, e), std::ldexp(a.lo, e)}; }

// pi to about 107 bits
const dd DD_PI = {3.141592653589793116e+00, 1.224646799147353207e-16};

typedef unsigned __int128 u128;

// round(v * 2^128) mod 2^128 for |v| < 1.
u128 frac_to_q128(double v) {
    if (v == 0.0) return 0;
    int e;
    double m = std::frexp(std::fabs(v), &e);          // |v| = m 2^e, m in [1/2, 1)
    uint64_t M = (uint64_t)std::ldexp(m, 53);         // exact 53-bit integer
    int sh = e - 53 + 128;                            // |v| 2^128 = M 2^sh, sh <= 75
    u128 r;
    if (sh >= 0) r = (u128)M << sh;
    else if (sh > -64) r = (u128)((M + ((uint64_t)1 << (-sh - 1))) >> (-sh));
    else r = 0;
    return v < 0 ? (u128)0 - r : r;
}

// Fractional part of a double-double as a 128-bit turn fraction.
void dd_to_turns128(dd t, uint64_t* hi, uint64_t* lo) {
    // x - trunc(x) is exact for every double (x - floor(x) is not for small
    // negative x); the signed fractions wrap modulo one turn below.
    double fh = t.hi - std::trunc(t.hi);
    double fl = t.lo - std::trunc(t.lo);
    u128 q = frac_to_q128(fh) + frac_to_q128(fl);
    *hi = (uint64_t)(q >> 64);
    *lo = (uint64_t)q;
}

// Fractional part of a double (|v| moderate) as a 64-bit turn fraction.
uint64_t double_to_turns64(double v) {
    uint64_t hi, lo;
    dd_to_turns128({v, 0.0}, &hi, &lo);
    return hi + (lo >> 63);
}

typedef std::complex<double> cplx;

int ilog2_exact(int64_t N) {
    if (N < 2 || N > 65536) return -1;
    if ((N & (N - 1)) != 0) return -1;
    int p = 0;
    while ((int64_t(1) << p) < N) ++p;
    return p;
}

// Re(x/y) of complex FP64 numbers, in double-double.
dd dd_re_div(cplx x, cplx y) {
    dd num = dd_add(two_prod(x.real(), y.real()), two_prod(x.imag(), y.imag()));
    dd den = dd_add(two_prod(y.real(), y.real()), two_prod(y.imag(), y.imag()));
    return dd_div(num, den);
}
// Re(x*y) in double-double.
dd dd_re_mul(cplx x, cplx y) {
    return dd_sub(two_prod(x.real(), y.real()), two_prod(x.imag(), y.imag()));
}

bool symplectic(cplx a, cplx b, cplx c, cplx d) {
    cplx ad = a * d, bc = b * c;
    double tol = 1e-9 * std::fmax(1.0, std::fmax(std::abs(ad), std::abs(bc)));
    return std::abs(ad - bc - 1.0) <= tol;
}

// Build the descriptor of one signal.  Returns LCT_OK or a validation error.
lct_status make_desc(int64_t N, const double* p, int64_t offset, lct_desc* D) {
    int log2n = ilog2_exact(N);
    if (log2n < 0) return LCT_ERR_N;
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(p[i])) return LCT_ERR_ARG;
    cplx a(p[0], p[1]), b(p[2], p[3]), c(p[4], p[5]), d(p[6], p[7]);
    if (!symplectic(a, b, c, d)) return LCT_ERR_NOT_SYMPLECTIC;
    std::memset(D, 0, sizeof(*D));
    D->offset = offset;
    D->log2n = log2n;
    uint64_t hi, lo;
    if (b == cplx(0.0, 0.0)) {
        // b = 0: G_j = sqrt(d) e^{i c x_j^2 / (2d)} f_j on y_j = x_j / d;
        // c x^2/(2d) = Re(c/d) pi^2 m^2/(16N) -> turns Re(c/d) pi / (32N).
        D->kind = LCT_KIND_DIAG;
        dd t = dd_ldexp(dd_mul(dd_re_div(c, d), DD_PI), -(5 + log2n));
        dd_to_turns128(t, &hi, &lo);
        D->out_hi = hi;
        D->out_lo = lo;
        cplx sd = std::sqrt(d);                       // principal root
        D->scale = std::abs(sd);
        D->out_c = double_to_turns64(std::arg(sd) / (2.0 * M_PI));
        return LCT_OK;
    }
    D->kind = LCT_KIND_XFT;
    // pre-chirp a x_k^2/(2b) = (a/b) pi^2 m^2 / (16 N): turns (a/b) pi / (32 N)
    dd tin = dd_ldexp(dd_mul(dd_re_div(a, b), DD_PI), -(5 + log2n));
    dd_to_turns128(tin, &hi, &lo);
    D->in_hi = hi;
    D->in_lo = lo;
    cplx ab = a / b;
    double decay = ab.imag() * M_PI * M_PI / (16.0 * (double)N);
    D->decay = decay;
    if (decay != 0.0) D->flags |= LCT_FLAG_DECAY;
    // post-chirp d y_j^2/(2b) = b d m^2 / N: turns Re(b d) / (2 pi N)
    dd tout = dd_ldexp(dd_div(dd_re_mul(b, d), DD_PI), -(1 + log2n));
    dd_to_turns128(tout, &hi, &lo);
    D->out_hi = hi;
    D->out_lo = lo;
    // constant: -(N-1)^2/(4N) turns (exact) + arg(dx / sqrt(2 pi i b)) / (2 pi)
    uint64_t r = (uint64_t)(((N - 1) * (N - 1)) % (4 * N));
    uint64_t centre = (uint64_t)0 - (r << (62 - log2n));       // -r / (4N) as Q0.64
    double dx = M_PI / std::sqrt(2.0 * (double)N);
    cplx pre = dx / std::sqrt(cplx(0.0, 2.0 * M_PI) * b);
    D->scale = std::abs(pre);
    D->out_c = centre + double_to_turns64(std::arg(pre) / (2.0 * M_PI));
    return LCT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// twiddle tables of the Stockham engine (xft_engine.cuh)
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tw_mu;
std::map<std::tuple<int, int, int>, void*> g_tw;   // (device, dtype, log2n) -> table

// Table of the Stockham engine with radix E = 2^le passes (see xft_engine.cuh).
template <class T>
std::vector<T> build_twiddles(int log2n, int le = 4) {
    const int E = 1 << le;
    const int P = log2n >= le ? (log2n + le - 1) / le : 1;
    const int R0 = 1 << (log2n - le * (P - 1));
    std::vector<T> t;
    for (int p = 1; p < P; ++p) {
        const int64_t ns = (int64_t)R0 << (le * (p - 1));
        const int64_t M = E * ns;
        for (int j = 1; j < E; ++j)
            for (int64_t k = 0; k < ns; ++k) {
                const double ang = 2.0 * M_PI * (double)((j * k) % M) / (double)M;
                t.push_back((T)std::cos(ang));
                t.push_back((T)-std::sin(ang));
            }
    }
    return t;
}

// The cached device copy of the table `key`, built by make() on first use.
// Caller holds g_tw_mu.
template <class F>
const void* cached_table(const std::tuple<int, int, int>& key, F make) {
    auto it = g_tw.find(key);
    if (it != g_tw.end()) return it->second;
    const auto t = make();
    const size_t bytes = t.size() * sizeof(t[0]);
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, t.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    g_tw[key] = d;
    return d;
}
}  // namespace

const void* lct_twiddle_table(int dtype, int log2n) {
    if (log2n < 5) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    const auto key = std::make_tuple(dev, dtype, log2n);
    if (dtype == LCT_C64) return cached_table(key, [&] { return build_twiddles<float>(log2n); });
    return cached_table(key, [&] { return build_twiddles<double>(log2n); });
}

const void* lct_twiddle_table_r8(int log2n) {
    if (log2n < 4) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    return cached_table(std::make_tuple(dev, 30, log2n), [&] { return build_twiddles<float>(log2n, 3); });
}

const void* lct_twiddle_table_pair(int log2n, int le) {
    if (log2n <= le) return nullptr;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(g_tw_mu);
    return cached_table(std::make_tuple(dev, 10 + le, log2n), [&] {
        std::vector<float> t = build_twiddles<float>(log2n, le);
        std::vector<float> b(2 * t.size());
        for (size_t k = 0; k < t.size() / 2; ++k) {
            b[4 * k + 0] = t[2 * k];
            b[4 * k + 1] = t[2 * k];
            b[4 * k + 2] = t[2 * k + 1];
            b[4 * k + 3] = t[2 * k + 1];
        }
        return b;
    });
}

int lct_make_desc_host(int64_t N, const double* p, int64_t offset, lct_desc* D) {
    return (int)make_desc(N, p, offset, D);
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
struct lct_plan_s {
    lct_dtype dtype = LCT_C64;
    lct_precision prec = LCT_PREC_NATIVE;
    bool is_batch = false;
    int64_t count = 1;
    int64_t N0 = 0;                 // common N (uniform plans); 0 when ragged
    std::vector<int64_t> N;
    std::vector<double> abcd;       // count x 8
    std::vector<lct_desc> desc;     // count descriptors
    // device state
    std::mutex mu;
    int device = -1;
    lct_desc* d_desc = nullptr;
    int32_t* d_status = nullptr;
    void* d_work = nullptr;
    size_t work_bytes = 0;
    void* d_tp = nullptr;            // two-pass chunk workspace(s)
    size_t tp_bytes = 0;
    cufftHandle fft = 0;
    bool fft_valid = false;
    int64_t fft_n = 0, fft_batch = 0;
    int variant = -1;               // -1: not chosen (cache or default 0)
    // ragged execution (mixed N or kinds): groups of equal (N, kind), largest
    // N first, each an index list into desc; run as one CUDA graph
    // kind LCT_KIND_DIAG: one group for every diagonal signal (log2n = -1),
    // its idx list ordered by N, run through the chunk list chunks[chunk_off ..]
    struct group {
        int log2n, kind;
        int64_t count, idx_off;
        int64_t tp_off = -1;
        int64_t chunk_off = 0, nchunks = 0;
    };
    bool ragged = false;
    std::vector<group> groups;
    std::vector<int32_t> idx;       // concatenated index lists
    int32_t* d_idx = nullptr;
    std::vector<int32_t> chunks;    // diagonal-group chunks, 4 int32 each
    int32_t* d_chunks = nullptr;
    static constexpr int kBranches = 4;
    cudaStream_t cap = nullptr;
    cudaStream_t side[kBranches] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kBranches] = {};
    cudaGraphExec_t gexec = nullptr;
    // host-buffer execution: copy-in, compute and copy-out streams, two
    // staging buffer pairs of `hx_chunk` signals, and their events
    cudaStream_t hx_stream[3] = {};
    cudaEvent_t hx_start = nullptr;
    cudaEvent_t hx_in[2] = {}, hx_comp[2] = {}, hx_out[2] = {};
    void* hx_buf = nullptr;
    size_t hx_bytes = 0;
    const void* g_in = nullptr;
    void* g_out = nullptr;
    // backward: per-signal gradient coefficients and reduction workspace
    double* d_coef = nullptr;
    double* d_partial = nullptr;
    int64_t partial_count = 0;
    // offset properties, fixed at creation: every offset even (16-byte signal
    // starts when `in` is 16-byte aligned) and offset[s] == s N0
    bool even_offsets = true;
    bool contiguous = true;
};

// ---------------------------------------------------------------------------
// autotune cache: (gpu name, dtype, log2n) -> variant
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string gpu_name() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    std::string n = prop.name;
    for (char& ch : n)
        if (ch == '|' || ch == '\n') ch = '_';
    return n;
}

std::string tune_key(const std::string& gpu, int dtype, int log2n) {
    return gpu + "|" + std::to_string(dtype) + "|" + std::to_string(log2n);
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("LCT_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        std::string s(line);
        size_t p3 = s.rfind('|');
        if (p3 == std::string::npos) continue;
        int v = std::atoi(s.c_str() + p3 + 1);
        g_tune[s.substr(0, p3)] = v;
    }
    std::fclose(f);
}

int tune_lookup(int dtype, int log2n) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(tune_key(gpu_name(), dtype, log2n));
    return it == g_tune.end() ? -1 : it->second;
}

void tune_store(int dtype, int log2n, int variant) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    std::string key = tune_key(gpu_name(), dtype, log2n);
    g_tune[key] = variant;
    const char* path = std::getenv("LCT_AUTOTUNE_CACHE");
    if (path && *path) {
        FILE* f = std::fopen(path, "a");
        if (f) {
            std::fprintf(f, "%s|%d\n", key.c_str(), variant);
            std::fclose(f);
        }
    }
}
}  // namespace

namespace {

void release_device(lct_plan p) {
    if (p->device < 0) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    if (p->fft_valid) cufftDestroy(p->fft);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    for (int b = 0; b < lct_plan_s::kBranches; ++b) {
        if (p->side[b]) cudaStreamDestroy(p->side[b]);
        if (p->ev_join[b]) cudaEventDestroy(p->ev_join[b]);
        p->side[b] = nullptr;
        p->ev_join[b] = nullptr;
    }
    for (int k = 0; k < 3; ++k) {
        if (p->hx_stream[k]) cudaStreamDestroy(p->hx_stream[k]);
        p->hx_stream[k] = nullptr;
    }
    for (int b = 0; b < 2; ++b) {
        for (cudaEvent_t* e : {&p->hx_in[b], &p->hx_comp[b], &p->hx_out[b]}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
    }
    if (p->hx_start) cudaEventDestroy(p->hx_start);
    p->hx_start = nullptr;
    cudaFree(p->hx_buf);
    p->hx_buf = nullptr;
    p->hx_bytes = 0;
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    p->cap = nullptr;
    p->ev_fork = nullptr;
    p->gexec = nullptr;
    p->g_in = nullptr;
    p->g_out = nullptr;
    cudaFree(p->d_desc);
    cudaFree(p->d_status);
    cudaFree(p->d_work);
    cudaFree(p->d_tp);
    p->d_tp = nullptr;
    p->tp_bytes = 0;
    cudaFree(p->d_idx);
    p->d_idx = nullptr;
    cudaFree(p->d_chunks);
    p->d_chunks = nullptr;
    cudaFree(p->d_coef);
    cudaFree(p->d_partial);
    p->d_coef = nullptr;
    p->d_partial = nullptr;
    p->partial_count = 0;
    if (cur != p->device && cur >= 0) cudaSetDevice(cur);
    p->fft_valid = false;
    p->d_desc = nullptr;
    p->d_status = nullptr;
    p->d_work = nullptr;
    p->work_bytes = 0;
    p->device = -1;
}

// Upload descriptors to the current device (once per device).
lct_status ensure_device(lct_plan p) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return LCT_ERR_CUDA;
    if (p->device == dev) return LCT_OK;
    release_device(p);
    size_t bytes = sizeof(lct_desc) * p->desc.size();
    if (cudaMalloc(&p->d_desc, bytes) != cudaSuccess) return LCT_ERR_OOM;
    if (cudaMalloc(&p->d_status, sizeof(int32_t)) != cudaSuccess) {
        cudaFree(p->d_desc);
        p->d_desc = nullptr;
        return LCT_ERR_OOM;
    }
    if (cudaMemcpy(p->d_desc, p->desc.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaFree(p->d_desc);
        cudaFree(p->d_status);
        p->d_desc = nullptr;
        p->d_status = nullptr;
        return LCT_ERR_CUDA;
    }
    p->device = dev;
    if (p->ragged && !p->idx.empty()) {
        const size_t ib = sizeof(int32_t) * p->idx.size();
        if (cudaMalloc(&p->d_idx, ib) != cudaSuccess) {
            release_device(p);
            return LCT_ERR_OOM;
        }
        if (cudaMemcpy(p->d_idx, p->idx.data(), ib, cudaMemcpyHostToDevice) != cudaSuccess) {
            release_device(p);
            return LCT_ERR_CUDA;
        }
    }
    if (p->ragged && !p->chunks.empty()) {
        const size_t cb = sizeof(int32_t) * p->chunks.size();
        if (cudaMalloc(&p->d_chunks, cb) != cudaSuccess) {
            release_device(p);
            return LCT_ERR_OOM;
        }
        if (cudaMemcpy(p->d_chunks, p->chunks.data(), cb, cudaMemcpyHostToDevice) != cudaSuccess) {
            release_device(p);
            return LCT_ERR_CUDA;
        }
    }
    return LCT_OK;
}

// NVTX range over an entry point (visible in Nsight timelines; costs a
// call into the NVTX stub when no tool is attached).
struct trace_range {
    explicit trace_range(const char* name) { nvtxRangePushA(name); }
    ~trace_range() { nvtxRangePop(); }
    trace_range(const trace_range&) = delete;
    trace_range& operator=(const trace_range&) = delete;
};

// Debug mode (LCT_DEBUG=1 in the environment, or lct_set_debug): every
// lct_execute / lct_backward synchronises its stream, scans the outputs for
// non-finite samples and reports the device status word.
std::atomic<int> g_debug{-1};
bool debug_on() {
    int v = g_debug.load();
    if (v < 0) {
        const char* e = std::getenv("LCT_DEBUG");
        v = (e && e[0] && e[0] != '0') ? 1 : 0;
        int expect = -1;
        g_debug.compare_exchange_strong(expect, v);
        v = g_debug.load();
    }
    return v == 1;
}

lct_status check_ptr(const void* ptr, lct_dtype dt) {
    if (!ptr) return LCT_ERR_ARG;
    uintptr_t align = dt == LCT_C64 ? 8 : 16;
    if (((uintptr_t)ptr) % align) return LCT_ERR_ALIGN;
    return LCT_OK;
}

lct_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return LCT_OK;
    if (e == cudaErrorMemoryAllocation) return LCT_ERR_OOM;
    return LCT_ERR_CUDA;
}

lct_status new_plan(lct_plan* out, lct_dtype dtype, int64_t count, const int64_t* N,
                    const double* abcd, const int64_t* offsets, bool is_batch) {
    if (!out) return LCT_ERR_ARG;
    *out = nullptr;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    if (count < 1) return LCT_ERR_ARG;
    lct_plan p = new (std::nothrow) lct_plan_s();
    if (!p) return LCT_ERR_OOM;
    p->dtype = dtype;
    p->is_batch = is_batch;
    p->count = count;
    p->N.assign(N, N + count);
    p->abcd.assign(abcd, abcd + 8 * count);
    p->desc.resize(count);
    p->N0 = N[0];
    for (int64_t s = 0; s < count; ++s) {
        if (offsets && offsets[s] < 0) { delete p; return LCT_ERR_ARG; }
        lct_status st = make_desc(N[s], abcd + 8 * s, offsets ? offsets[s] : 0, &p->desc[s]);
        if (st != LCT_OK) { delete p; return st; }
        if (N[s] != p->N0) p->N0 = 0;
        if (p->desc[s].offset % 2) p->even_offsets = false;
        if (p->desc[s].offset != s * N[0]) p->contiguous = false;
    }
    bool mixed_kind = false;
    for (int64_t s = 1; s < count; ++s)
        if (p->desc[s].kind != p->desc[0].kind) mixed_kind = true;
    if (is_batch && (p->N0 == 0 || mixed_kind)) {
        // Group by (N, kind), largest N first.
        p->ragged = true;
        std::map<std::pair<int, int>, std::vector<int32_t>, std::greater<std::pair<int, int>>> by;
        for (int64_t s = 0; s < count; ++s) {
            const lct_desc& D = p->desc[s];
            by[{D.log2n, D.kind}].push_back((int32_t)s);
        }
        lct_plan_s::group diag;
        diag.log2n = -1;
        diag.kind = LCT_KIND_DIAG;
        diag.count = 0;
        std::vector<int32_t> diag_idx;
        for (auto& kv : by) {
            if (kv.first.second == LCT_KIND_DIAG) {
                // chunks of kDiagChunk elements, or whole small signals packed
                const int L = kv.first.first;
                const int64_t n = (int64_t)1 << L;
                const int64_t pos0 = (int64_t)diag_idx.size();
                const int64_t m = (int64_t)kv.second.size();
                if (n >= kDiagChunk) {
                    for (int64_t j = 0; j < m; ++j)
                        for (int64_t st = 0; st < n; st += kDiagChunk)
                            p->chunks.insert(p->chunks.end(),
                                             {(int32_t)(pos0 + j), (int32_t)st, L, 1});
                } else {
                    const int64_t per = kDiagChunk / n;
                    for (int64_t j = 0; j < m; j += per)
                        p->chunks.insert(p->chunks.end(),
                                         {(int32_t)(pos0 + j), 0, L,
                                          (int32_t)(m - j < per ? m - j : per)});
                }
                diag_idx.insert(diag_idx.end(), kv.second.begin(), kv.second.end());
                continue;
            }
            lct_plan_s::group g;
            g.log2n = kv.first.first;
            g.kind = kv.first.second;
            g.count = (int64_t)kv.second.size();
            g.idx_off = (int64_t)p->idx.size();
            p->idx.insert(p->idx.end(), kv.second.begin(), kv.second.end());
            p->groups.push_back(g);
        }
        if (!diag_idx.empty()) {
            diag.count = (int64_t)diag_idx.size();
            diag.idx_off = (int64_t)p->idx.size();
            diag.chunk_off = 0;
            diag.nchunks = (int64_t)(p->chunks.size() / 4);
            p->idx.insert(p->idx.end(), diag_idx.begin(), diag_idx.end());
            p->groups.push_back(diag);
        }
    }
    *out = p;
    return LCT_OK;
}

// Plain FP64 path: chirp kernel -> cuFFT Z2Z (forward) -> chirp+scale kernel.
lct_status run_plain(lct_plan p, const void* in, void* out, int64_t count, int desc_step,
                     cudaStream_t stream) {
    int64_t N = p->N0;
    int log2n = p->desc[0].log2n;
    size_t need = (size_t)count * (size_t)N * 16;
    if (need > p->work_bytes) {
        cudaFree(p->d_work);
        p->d_work = nullptr;
        p->work_bytes = 0;
        if (cudaMalloc(&p->d_work, need) != cudaSuccess) return LCT_ERR_OOM;
        p->work_bytes = need;
    }
    if (!p->fft_valid || p->fft_n != N || p->fft_batch != count) {
        if (p->fft_valid) cufftDestroy(p->fft);
        p->fft_valid = false;
        int n = (int)N;
        if (cufftPlanMany(&p->fft, 1, &n, nullptr, 1, n, nullptr, 1, n, CUFFT_Z2Z, (int)count) !=
            CUFFT_SUCCESS)
            return LCT_ERR_CUDA;
        p->fft_valid = true;
        p->fft_n = N;
        p->fft_batch = count;
    }
    if (cufftSetStream(p->fft, stream) != CUFFT_SUCCESS) return LCT_ERR_CUDA;
    lct_status st = from_cuda(lct_launch_plain_pre(p->dtype, log2n, in, p->d_work, p->d_desc,
                                                   desc_step, count, stream));
    if (st != LCT_OK) return st;
    cufftDoubleComplex* w = (cufftDoubleComplex*)p->d_work;
    if (cufftExecZ2Z(p->fft, w, w, CUFFT_FORWARD) != CUFFT_SUCCESS) return LCT_ERR_CUDA;
    return from_cuda(lct_launch_plain_post(p->dtype, log2n, p->d_work, out, p->d_desc, desc_step,
                                           count, stream));
}

// Can a bulk-async variant run this plan on `in` (16-byte aligned starts)?
// Smallest N that runs two-pass by default (measured on GB300: two passes
// beat the cluster kernel from here up).
constexpr int kTwoPassDefaultLog2 = 15;

bool tma_aligned(lct_plan p, const void* in) {
    return ((uintptr_t)in) % 16 == 0 && (!p->is_batch || p->even_offsets);
}

bool pair_tma_ok(lct_plan p, const void* in) {
    return lct_fused_pair_tma_supported(p->dtype, p->desc[0].log2n) && tma_aligned(p, in);
}

// Can variant 1 (persistent, bulk-async prefetch) run this plan on `in`?
bool tma_ok(lct_plan p, const void* in) {
    return lct_fused_tma_supported(p->dtype, p->desc[0].log2n) && tma_aligned(p, in);
}

// Variant used when neither the plan nor the tune cache chooses one.
int default_variant(lct_dtype dtype, int log2n) {
    return (lct_twopass_supported(dtype, log2n) && log2n >= kTwoPassDefaultLog2) ? 7 : 0;
}

int effective_variant(lct_plan p) {
    if (p->variant >= 0) return p->variant;
    int v = tune_lookup(p->dtype, p->desc[0].log2n);
    return v >= 0 ? v : default_variant(p->dtype, p->desc[0].log2n);
}

// Two-pass path ------------------------------------------------------------
size_t sample_bytes(lct_dtype dtype) { return dtype == LCT_C64 ? 8 : 16; }

// Workspace bytes of the two-pass path for `count` signals of N = 2^log2n:
// the ring slots, then the queue and counters.
lct_status twopass_work_bytes(lct_dtype dtype, int log2n, int64_t count, size_t* bytes) {
    int64_t slots = 0;
    if (lct_twopass_ring(dtype, log2n, count, &slots) != cudaSuccess) return LCT_ERR_CUDA;
    *bytes = (size_t)slots * (sample_bytes(dtype) << log2n) +
             (((size_t)(4 + 2 * slots) * 4 + 255) & ~(size_t)255);
    return LCT_OK;
}

lct_status ensure_tp_work(lct_plan p, size_t need) {
    if (need <= p->tp_bytes) return LCT_OK;
    cudaFree(p->d_tp);
    p->d_tp = nullptr;
    p->tp_bytes = 0;
    if (cudaMalloc(&p->d_tp, need) != cudaSuccess) return LCT_ERR_OOM;
    p->tp_bytes = need;
    return LCT_OK;
}

// The two-pass transform of `count` signals with the workspace `work` (of
// twopass_work_bytes bytes).
lct_status run_twopass(lct_plan p, int log2n, const void* in, void* out, int64_t count,
                       int desc_step, const int32_t* idx, void* work, cudaStream_t stream) {
    int l1, l2;
    lct_twopass_split(log2n, &l1, &l2);
    const void* tw1 = lct_twiddle_table(p->dtype, l1);
    const void* tw2 = lct_twiddle_table(p->dtype, l2);
    if (!tw1 || !tw2) return LCT_ERR_OOM;
    int64_t slots = 0;
    if (lct_twopass_ring(p->dtype, log2n, count, &slots) != cudaSuccess) return LCT_ERR_CUDA;
    int32_t* sync = (int32_t*)((char*)work + (size_t)slots * (sample_bytes(p->dtype) << log2n));
    return from_cuda(lct_launch_twopass(p->dtype, log2n, in, out, work, sync, p->d_desc,
                                        desc_step, count, idx, p->d_status, tw1, tw2, stream));
}

lct_status run_fused(lct_plan p, const void* in, void* out, int64_t batch, int desc_step,
                     int variant, cudaStream_t stream) {
    const int log2n = p->desc[0].log2n;
    if (variant == 7 && lct_twopass_supported(p->dtype, log2n)) {
        size_t need = 0;
        lct_status st = twopass_work_bytes(p->dtype, log2n, batch, &need);
        if (st == LCT_OK) st = ensure_tp_work(p, need);
        if (st != LCT_OK) return st;
        return run_twopass(p, log2n, in, out, batch, desc_step, nullptr, p->d_tp, stream);
    }
    const int lm = lct_cluster_local_log2(p->dtype, log2n);
    if (lm >= 0 && (variant == 5 || !lct_fused_supported(p->dtype, log2n))) {
        const void* twl = lct_twiddle_table(p->dtype, lm);
        if (!twl) return LCT_ERR_OOM;
        return from_cuda(lct_launch_cluster(p->dtype, log2n, in, out, p->d_desc, desc_step, batch,
                                            twl, nullptr, p->d_status, stream));
    }
    if (!lct_fused_supported(p->dtype, log2n)) return LCT_ERR_UNSUPPORTED;
    const void* tw = lct_twiddle_table(p->dtype, log2n);
    if (log2n >= 5 && !tw) return LCT_ERR_OOM;
    if (variant == 6 && lct_fused_pair8_supported(p->dtype, log2n)) {
        const void* tw8 = lct_twiddle_table_pair(log2n, 3);
        if (!tw8) return LCT_ERR_OOM;
        return from_cuda(lct_launch_fused_pair8(p->dtype, log2n, in, out, p->d_desc, desc_step,
                                                batch, tw8, stream));
    }
    if (variant == 4 && pair_tma_ok(p, in)) {
        const void* tw2 = lct_twiddle_table_pair(log2n);
        if (!tw2) return LCT_ERR_OOM;
        return from_cuda(lct_launch_fused_pair_tma(p->dtype, log2n, in, out, p->d_desc,
                                                   desc_step, batch, tw2, p->d_status, stream));
    }
    if ((variant == 3 || variant == 4) && lct_fused_pair_supported(p->dtype, log2n)) {
        const void* tw2 = lct_twiddle_table_pair(log2n);
        if (!tw2) return LCT_ERR_OOM;
        return from_cuda(lct_launch_fused_pair(p->dtype, log2n, in, out, p->d_desc, desc_step,
                                               batch, tw2, stream));
    }
    if ((variant == 1 || variant == 2) && tma_ok(p, in))
        return from_cuda(lct_launch_fused_tma(p->dtype, log2n, in, out, p->d_desc, desc_step,
                                              batch, tw, p->d_status, variant == 2, stream));
    return from_cuda(lct_launch_fused(p->dtype, log2n, in, out, p->d_desc, desc_step, batch, tw,
                                      nullptr, p->d_status, stream));
}

// Variant of a ragged group of N = 2^log2n: the tuned one, else the
// default (two passes for N >= 32768).
int group_variant(lct_dtype dtype, int log2n) {
    const int v = tune_lookup(dtype, log2n);
    if (v >= 0) return v;
    return default_variant(dtype, log2n);
}

// Launch one group of a ragged plan on `stream`.
lct_status launch_group(lct_plan p, const lct_plan_s::group& g, const void* in, void* out,
                        cudaStream_t stream) {
    const int32_t* idx = p->d_idx + g.idx_off;
    if (g.kind == LCT_KIND_DIAG)
        return from_cuda(lct_launch_diag_chunks(p->dtype, in, out, p->d_desc, idx,
                                                p->d_chunks + 4 * g.chunk_off, g.nchunks,
                                                p->d_status, stream));
    const int lm = lct_cluster_local_log2(p->dtype, g.log2n);
    const bool single = lct_fused_supported(p->dtype, g.log2n);
    const int v = tune_lookup(p->dtype, g.log2n);
    if (g.tp_off >= 0)
        return run_twopass(p, g.log2n, in, out, g.count, 1, idx, (char*)p->d_tp + g.tp_off, stream);
    if (lm >= 0 && (!single || v == 5))
        return from_cuda(lct_launch_cluster(p->dtype, g.log2n, in, out, p->d_desc, 1, g.count,
                                            lct_twiddle_table(p->dtype, lm), idx, p->d_status,
                                            stream));
    if (!single) return LCT_ERR_UNSUPPORTED;
    return from_cuda(lct_launch_fused(p->dtype, g.log2n, in, out, p->d_desc, 1, g.count,
                                      lct_twiddle_table(p->dtype, g.log2n), idx, p->d_status,
                                      stream));
}

// Capture every group into one graph: a fork to kBranches streams, groups
// dealt round-robin (largest N first), a join; instantiated once per
// (in, out) pair.
lct_status build_graph(lct_plan p, const void* in, void* out) {
    // tables and workspaces first: allocation is not allowed while capturing.
    // Every two-pass group gets its own chunk workspace (the branches run
    // concurrently).
    size_t tp_need = 0;
    for (auto& g : p->groups) {
        g.tp_off = -1;
        if (g.kind == LCT_KIND_DIAG || !lct_twopass_supported(p->dtype, g.log2n)) continue;
        if (group_variant(p->dtype, g.log2n) != 7) continue;
        int l1, l2;
        lct_twopass_split(g.log2n, &l1, &l2);
        if (!lct_twiddle_table(p->dtype, l1) || !lct_twiddle_table(p->dtype, l2)) return LCT_ERR_OOM;
        g.tp_off = (int64_t)tp_need;
        size_t bytes = 0;
        lct_status st = twopass_work_bytes(p->dtype, g.log2n, g.count, &bytes);
        if (st != LCT_OK) return st;
        tp_need += (bytes + 255) & ~(size_t)255;
    }
    if (tp_need) {
        lct_status st = ensure_tp_work(p, tp_need);
        if (st != LCT_OK) return st;
    }
    for (const auto& g : p->groups) {
        if (g.kind == LCT_KIND_DIAG) continue;
        const int lm = lct_cluster_local_log2(p->dtype, g.log2n);
        if (lm >= 0 && !lct_twiddle_table(p->dtype, lm)) return LCT_ERR_OOM;
        if (g.log2n >= 5 && lct_fused_supported(p->dtype, g.log2n) &&
            !lct_twiddle_table(p->dtype, g.log2n))
            return LCT_ERR_OOM;
    }
    if (!p->cap) {
        if (cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess)
            return LCT_ERR_CUDA;
        for (int b = 0; b < lct_plan_s::kBranches; ++b)
            if (cudaStreamCreateWithFlags(&p->side[b], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&p->ev_join[b], cudaEventDisableTiming) != cudaSuccess)
                return LCT_ERR_CUDA;
    }
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return LCT_ERR_CUDA;
    lct_status st = LCT_OK;
    if (cudaEventRecord(p->ev_fork, p->cap) != cudaSuccess) st = LCT_ERR_CUDA;
    for (int b = 0; b < lct_plan_s::kBranches && st == LCT_OK; ++b)
        if (cudaStreamWaitEvent(p->side[b], p->ev_fork, 0) != cudaSuccess) st = LCT_ERR_CUDA;
    for (size_t k = 0; k < p->groups.size() && st == LCT_OK; ++k)
        st = launch_group(p, p->groups[k], in, out, p->side[k % lct_plan_s::kBranches]);
    for (int b = 0; b < lct_plan_s::kBranches && st == LCT_OK; ++b) {
        if (cudaEventRecord(p->ev_join[b], p->side[b]) != cudaSuccess ||
            cudaStreamWaitEvent(p->cap, p->ev_join[b], 0) != cudaSuccess)
            st = LCT_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
    if (st != LCT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess || !graph) return LCT_ERR_CUDA;
    const cudaError_t ei = cudaGraphInstantiate(&p->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        p->gexec = nullptr;
        return LCT_ERR_CUDA;
    }
    p->g_in = in;
    p->g_out = out;
    return LCT_OK;
}

// Backward helpers ----------------------------------------------------------
// Coefficients of (SA, SR, SG) in (dl/da, dl/db, dl/dd), see k_general.cu.
void grad_coefs(const double* p, int64_t N, double* c) {
    const double a = p[0], b = p[2], d = p[6];
    const double pi2 = M_PI * M_PI, n = (double)N;
    c[0] = -pi2 / (16.0 * b * n);
    c[1] = a * pi2 / (16.0 * b * b * n);
    c[2] = -1.0 / (2.0 * b);
    c[3] = -d / n;
    c[4] = -b / n;
}

lct_status ensure_grad_state(lct_plan p, int64_t batch) {
    if (!p->d_coef) {
        std::vector<double> c(5 * p->count);
        for (int64_t s = 0; s < p->count; ++s) grad_coefs(&p->abcd[8 * s], p->N[s], &c[5 * s]);
        if (cudaMalloc(&p->d_coef, sizeof(double) * c.size()) != cudaSuccess) return LCT_ERR_OOM;
        if (cudaMemcpy(p->d_coef, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return LCT_ERR_CUDA;
    }
    if (batch > p->partial_count) {
        // per-signal sums, then the finalize scratch (zeroed once)
        cudaFree(p->d_partial);
        p->d_partial = nullptr;
        p->partial_count = 0;
        const size_t bytes = sizeof(double) * 3 * batch + lct_grad_finalize_scratch_bytes();
        if (cudaMalloc(&p->d_partial, bytes) != cudaSuccess) return LCT_ERR_OOM;
        if (cudaMemset(p->d_partial, 0, bytes) != cudaSuccess) return LCT_ERR_CUDA;
        p->partial_count = batch;
    }
    return LCT_OK;
}

bool real_params(const lct_plan p) {
    for (int64_t s = 0; s < p->count; ++s) {
        const double* q = &p->abcd[8 * s];
        if (q[1] != 0.0 || q[3] != 0.0 || q[5] != 0.0 || q[7] != 0.0) return false;
    }
    return true;
}

// Adjoint (and gradients) of one uniform plan: rows (cols = 0) or columns.
lct_status run_backward(lct_plan p, const void* g, const void* f, const void* G, void* h,
                        double* grad, int64_t batch, int cols, int64_t es, int64_t P, int64_t big,
                        cudaStream_t stream) {
    const int log2n = p->desc[0].log2n;
    if (!lct_gen_supported(p->dtype, log2n, cols)) return LCT_ERR_UNSUPPORTED;
    // complex64 columns run the radix-8 engine
    const bool r8 = cols && p->dtype == LCT_C64;
    const void* tw = r8 ? lct_twiddle_table_r8(log2n) : lct_twiddle_table(p->dtype, log2n);
    if (log2n >= 5 && !tw) return LCT_ERR_OOM;
    const int do_grad = grad != nullptr;
    if (do_grad) {
        lct_status st = ensure_grad_state(p, batch);
        if (st != LCT_OK) return st;
    }
    const int desc_step = p->is_batch ? 1 : 0;
    lct_status st = from_cuda(lct_launch_gen(p->dtype, log2n, cols, 1, do_grad, g, h, p->d_desc,
                                             desc_step, batch, tw, es, P, big, G, f,
                                             do_grad ? p->d_partial : nullptr,
                                             desc_step ? nullptr : p->desc.data(), stream));
    if (st != LCT_OK || !do_grad) return st;
    return from_cuda(lct_launch_grad_finalize(p->d_partial, p->d_coef, desc_step, batch,
                                              p->is_batch ? 0 : 1, grad,
                                              p->d_partial + 3 * p->partial_count, stream));
}

lct_status run_ragged(lct_plan p, const void* in, void* out, cudaStream_t stream) {
    if (p->prec != LCT_PREC_NATIVE) return LCT_ERR_UNSUPPORTED;
    if (!p->gexec || p->g_in != in || p->g_out != out) {
        lct_status st = build_graph(p, in, out);
        if (st != LCT_OK) return st;
    }
    return from_cuda(cudaGraphLaunch(p->gexec, stream));
}

// The transform on the current device with the plan's state set up (lock
// held).  desc: the descriptors of the launch's signals (the plan's, or a
// sub-range of them for chunked execution; batch plans address samples by
// each descriptor's offset into in/out).
lct_status execute_locked(lct_plan plan, const lct_desc* desc, const void* in, void* out,
                          int64_t batch, cudaStream_t stream) {
    if (plan->ragged) return run_ragged(plan, in, out, stream);
    // every path below reads the descriptors through plan->d_desc
    struct swap {
        lct_plan p;
        lct_desc* saved;
        ~swap() { p->d_desc = saved; }
    } restore{plan, plan->d_desc};
    plan->d_desc = const_cast<lct_desc*>(desc);
    const int desc_step = plan->is_batch ? 1 : 0;
    const lct_desc& D0 = plan->desc[0];
    const int log2n = D0.log2n;
    if (D0.kind == LCT_KIND_DIAG)
        return from_cuda(lct_launch_diag(plan->dtype, log2n, in, out, plan->d_desc, desc_step,
                                         batch, nullptr, plan->d_status, stream));
    if (plan->prec == LCT_PREC_PLAIN64) {
        // the plain path assumes contiguous rows
        if (plan->is_batch && !plan->contiguous) return LCT_ERR_UNSUPPORTED;
        return run_plain(plan, in, out, batch, desc_step, stream);
    }
    if (plan->prec == LCT_PREC_SPLIT_BF16 || plan->prec == LCT_PREC_SPLIT_FP16 ||
        plan->prec == LCT_PREC_FP16) {
        const void* tw = lct_twiddle_table(plan->dtype, log2n);
        if (log2n >= 5 && !tw) return LCT_ERR_OOM;
        return from_cuda(lct_launch_split((int)plan->prec, log2n, in, out, plan->d_desc,
                                          desc_step, batch, tw, tma_aligned(plan, in) ? 1 : 0,
                                          plan->contiguous ? 1 : 0, plan->d_status, stream));
    }
    return run_fused(plan, in, out, batch, desc_step, effective_variant(plan), stream);
}

// Debug mode: scan `count` output signals laid out as the plan's (batch plans:
// by descriptor; others: contiguous rows of N0), wait, report and clear the
// device status word.
lct_status debug_check(lct_plan plan, const void* out, int64_t count, cudaStream_t stream) {
    const int desc_step = plan->is_batch ? 1 : 0;
    const int log2n = plan->desc[0].log2n;
    if (lct_launch_scan(plan->dtype, out, plan->d_desc, desc_step, count, log2n, plan->d_status,
                        stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return LCT_ERR_CUDA;
    int32_t v = 0;
    if (cudaMemcpy(&v, plan->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LCT_ERR_CUDA;
    if (v == LCT_DEV_OK) return LCT_OK;
    cudaMemset(plan->d_status, 0, sizeof(int32_t));
    return v == LCT_DEV_TIMEOUT ? LCT_ERR_TIMEOUT : LCT_ERR_DEVICE;
}

// Host-buffer execution ----------------------------------------------------
// Signals per chunk: about 32 MiB of samples, at least one signal (measured
// on GB300 with 512 MiB each way: 16 MiB 3.62 ms, 32 MiB 3.46 ms, 64 MiB
// 3.52 ms, 128 MiB 5.66 ms -- fill and drain against too few chunks).
int64_t host_chunk(const lct_plan p) {
    const size_t per = (size_t)p->N0 * sample_bytes(p->dtype);
    int64_t c = (int64_t)(((size_t)32 << 20) / per);
    return c < 1 ? 1 : c;
}

lct_status ensure_host_state(lct_plan p, int64_t chunk) {
    if (!p->hx_stream[0]) {
        for (int k = 0; k < 3; ++k)
            if (cudaStreamCreateWithFlags(&p->hx_stream[k], cudaStreamNonBlocking) != cudaSuccess)
                return LCT_ERR_CUDA;
        if (cudaEventCreateWithFlags(&p->hx_start, cudaEventDisableTiming) != cudaSuccess)
            return LCT_ERR_CUDA;
        for (int b = 0; b < 2; ++b)
            for (cudaEvent_t* e : {&p->hx_in[b], &p->hx_comp[b], &p->hx_out[b]})
                if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
                    return LCT_ERR_CUDA;
    }
    const size_t need = 4 * (size_t)chunk * (size_t)p->N0 * sample_bytes(p->dtype);
    if (need > p->hx_bytes) {
        cudaFree(p->hx_buf);
        p->hx_buf = nullptr;
        p->hx_bytes = 0;
        if (cudaMalloc(&p->hx_buf, need) != cudaSuccess) return LCT_ERR_OOM;
        p->hx_bytes = need;
    }
    return LCT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

lct_status lct_plan_create(lct_plan* out, int64_t N, double a, double b, double c, double d,
                           lct_dtype dtype) {
    trace_range trace("lct_plan_create");
    double p[8] = {a, 0.0, b, 0.0, c, 0.0, d, 0.0};
    return new_plan(out, dtype, 1, &N, p, nullptr, false);
}

lct_status lct_plan_create_complex(lct_plan* out, int64_t N, const double abcd_reim[8],
                                   lct_dtype dtype) {
    if (!abcd_reim) return LCT_ERR_ARG;
    return new_plan(out, dtype, 1, &N, abcd_reim, nullptr, false);
}

lct_status lct_plan_create_batch(lct_plan* out, int64_t count, const int64_t* N,
                                 const double* abcd_reim, const int64_t* offsets,
                                 lct_dtype dtype) {
    trace_range trace("lct_plan_create_batch");
    if (!N || !abcd_reim || !offsets) return LCT_ERR_ARG;
    return new_plan(out, dtype, count, N, abcd_reim, offsets, true);
}

lct_status lct_plan_set_precision(lct_plan plan, lct_precision precision) {
    if (!plan) return LCT_ERR_ARG;
    switch (precision) {
        case LCT_PREC_NATIVE:
        case LCT_PREC_PLAIN64:
            plan->prec = precision;
            return LCT_OK;
        case LCT_PREC_SPLIT_BF16:
        case LCT_PREC_SPLIT_FP16:
        case LCT_PREC_FP16: {
            // tensor-core DFT: complex64, one N in [16, 4096] (b = 0 plans have
            // no DFT and run their diagonal kernel whatever the precision)
            if (plan->dtype != LCT_C64 || plan->ragged || plan->N0 == 0) return LCT_ERR_UNSUPPORTED;
            const int log2n = ilog2_exact(plan->N0);
            if (plan->desc[0].kind == LCT_KIND_XFT && !lct_split_supported(plan->dtype, log2n))
                return LCT_ERR_UNSUPPORTED;
            plan->prec = precision;
            return LCT_OK;
        }
        default:
            return LCT_ERR_ARG;
    }
}

lct_status lct_plan_set_variant(lct_plan plan, int variant) {
    if (!plan || variant < 0 || variant > 7) return LCT_ERR_ARG;
    plan->variant = variant;
    return LCT_OK;
}

lct_status lct_plan_get_variant(lct_plan plan, int* variant) {
    if (!plan || !variant) return LCT_ERR_ARG;
    *variant = plan->variant >= 0 ? plan->variant
                                  : default_variant(plan->dtype, plan->desc[0].log2n);
    return LCT_OK;
}

lct_status lct_plan_autotune(lct_plan plan, const void* in, void* out, int64_t batch,
                             lct_stream_t stream_) {
    trace_range trace("lct_plan_autotune");
    if (!plan) return LCT_ERR_ARG;
    if (plan->prec != LCT_PREC_NATIVE || plan->N0 == 0 || plan->desc[0].kind != LCT_KIND_XFT) {
        plan->variant = 0;
        return LCT_OK;
    }
    const int saved = plan->variant;
    int candidates[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int n_cand = 1;
    if (lct_fused_pair8_supported(plan->dtype, plan->desc[0].log2n)) candidates[n_cand++] = 6;
    if (lct_cluster_local_log2(plan->dtype, plan->desc[0].log2n) >= 0 &&
        lct_fused_supported(plan->dtype, plan->desc[0].log2n))
        candidates[n_cand++] = 5;
    if (lct_twopass_supported(plan->dtype, plan->desc[0].log2n)) candidates[n_cand++] = 7;
    if (lct_fused_pair_supported(plan->dtype, plan->desc[0].log2n)) candidates[n_cand++] = 3;
    if (pair_tma_ok(plan, in)) candidates[n_cand++] = 4;
    if (tma_ok(plan, in)) {
        candidates[n_cand++] = 1;
        candidates[n_cand++] = 2;
    }
    if (n_cand == 1) {
        plan->variant = 0;
        return LCT_OK;
    }
    cudaStream_t stream = (cudaStream_t)stream_;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LCT_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LCT_ERR_CUDA;
    }
    float best_ms = 1e30f;
    int best = 0;
    lct_status st = LCT_OK;
    for (int c = 0; c < n_cand && st == LCT_OK; ++c) {
        plan->variant = candidates[c];
        for (int w = 0; w < 2 && st == LCT_OK; ++w) st = lct_execute(plan, in, out, batch, stream_);
        if (st != LCT_OK) break;
        cudaEventRecord(e0, stream);
        for (int r = 0; r < 5 && st == LCT_OK; ++r) st = lct_execute(plan, in, out, batch, stream_);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = LCT_ERR_CUDA;
        float ms = 0.f;
        if (st == LCT_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = candidates[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LCT_OK) {
        plan->variant = saved;
        return st;
    }
    plan->variant = best;
    tune_store(plan->dtype, plan->desc[0].log2n, best);
    return LCT_OK;
}

lct_status lct_execute(lct_plan plan, const void* in, void* out, int64_t batch,
                       lct_stream_t stream_) {
    trace_range trace("lct_execute");
    if (!plan) return LCT_ERR_ARG;
    if (batch < 0) return LCT_ERR_ARG;
    if (plan->is_batch && batch != plan->count) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    lct_status st = check_ptr(in, plan->dtype);
    if (st != LCT_OK) return st;
    st = check_ptr(out, plan->dtype);
    if (st != LCT_OK) return st;
    std::lock_guard<std::mutex> g(plan->mu);
    st = ensure_device(plan);
    if (st != LCT_OK) return st;
    st = execute_locked(plan, plan->d_desc, in, out, batch, (cudaStream_t)stream_);
    if (st == LCT_OK && debug_on()) st = debug_check(plan, out, batch, (cudaStream_t)stream_);
    return st;
}

lct_status lct_execute_host(lct_plan plan, const void* h_in, void* h_out, int64_t batch,
                            lct_stream_t stream_) {
    trace_range trace("lct_execute_host");
    if (!plan || !h_in || !h_out || batch < 0) return LCT_ERR_ARG;
    if (plan->is_batch && batch != plan->count) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    if (plan->ragged || plan->N0 == 0 || (plan->is_batch && !plan->contiguous))
        return LCT_ERR_UNSUPPORTED;
    cudaStream_t stream = (cudaStream_t)stream_;
    std::lock_guard<std::mutex> g(plan->mu);
    lct_status st = ensure_device(plan);
    if (st != LCT_OK) return st;
    const int64_t chunk = host_chunk(plan) < batch ? host_chunk(plan) : batch;
    if ((st = ensure_host_state(plan, chunk)) != LCT_OK) return st;
    const int64_t N = plan->N0;
    const size_t es = sample_bytes(plan->dtype);
    const size_t cbytes = (size_t)chunk * (size_t)N * es;
    char* din[2] = {(char*)plan->hx_buf, (char*)plan->hx_buf + cbytes};
    char* dout[2] = {(char*)plan->hx_buf + 2 * cbytes, (char*)plan->hx_buf + 3 * cbytes};
    cudaStream_t s_in = plan->hx_stream[0], s_comp = plan->hx_stream[1], s_out = plan->hx_stream[2];
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // everything after the work already queued on `stream`
    if (!ok(cudaEventRecord(plan->hx_start, stream)) ||
        !ok(cudaStreamWaitEvent(s_in, plan->hx_start, 0)) ||
        !ok(cudaStreamWaitEvent(s_comp, plan->hx_start, 0)) ||
        !ok(cudaStreamWaitEvent(s_out, plan->hx_start, 0)))
        return LCT_ERR_CUDA;
    int64_t k = 0;
    for (int64_t c0 = 0; c0 < batch; c0 += chunk, ++k) {
        const int64_t cs = batch - c0 < chunk ? batch - c0 : chunk;
        const int b = (int)(k & 1);
        const size_t bytes = (size_t)cs * (size_t)N * es;
        const size_t hoff = (size_t)c0 * (size_t)N * es;
        // copy-in: after the compute of chunk k - 2 has read din[b]
        if (k >= 2 && !ok(cudaStreamWaitEvent(s_in, plan->hx_comp[b], 0))) return LCT_ERR_CUDA;
        if (!ok(cudaMemcpyAsync(din[b], (const char*)h_in + hoff, bytes, cudaMemcpyHostToDevice, s_in)) ||
            !ok(cudaEventRecord(plan->hx_in[b], s_in)))
            return LCT_ERR_CUDA;
        // compute: after its copy-in and after the copy-out of chunk k - 2
        if (!ok(cudaStreamWaitEvent(s_comp, plan->hx_in[b], 0))) return LCT_ERR_CUDA;
        if (k >= 2 && !ok(cudaStreamWaitEvent(s_comp, plan->hx_out[b], 0))) return LCT_ERR_CUDA;
        if (plan->is_batch) {
            // descriptors c0.. address samples at offset (c0 + j) N: shift the bases
            st = execute_locked(plan, plan->d_desc + c0, din[b] - hoff, dout[b] - hoff, cs, s_comp);
        } else {
            st = execute_locked(plan, plan->d_desc, din[b], dout[b], cs, s_comp);
        }
        if (st != LCT_OK) return st;
        if (!ok(cudaEventRecord(plan->hx_comp[b], s_comp))) return LCT_ERR_CUDA;
        // copy-out
        if (!ok(cudaStreamWaitEvent(s_out, plan->hx_comp[b], 0)) ||
            !ok(cudaMemcpyAsync((char*)h_out + hoff, dout[b], bytes, cudaMemcpyDeviceToHost, s_out)) ||
            !ok(cudaEventRecord(plan->hx_out[b], s_out)))
            return LCT_ERR_CUDA;
    }
    // `stream` continues after the last copy-out (s_out is in order)
    if (!ok(cudaEventRecord(plan->hx_out[0], s_out)) ||
        !ok(cudaStreamWaitEvent(stream, plan->hx_out[0], 0)))
        return LCT_ERR_CUDA;
    return LCT_OK;
}

lct_status frft_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                        int64_t batch, lct_dtype dtype, lct_stream_t stream) {
    trace_range trace("frft_execute");
    cplx z(z_re, z_im);
    double az = std::abs(z);
    if (!std::isfinite(az) || az == 0.0 || az > 1.0 + 1e-15) return LCT_ERR_ARG;
    if (ilog2_exact(N) < 0) return LCT_ERR_N;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    double p[8];
    double frft_scale_abs;
    double frft_scale_turns;
    cplx one_minus_z2 = 1.0 - z * z;
    if (one_minus_z2 == cplx(0.0, 0.0)) {
        // z = +-1: F_z = sqrt(2 pi) times the identity / the parity on y_j = x_j / z,
        // which is the b = 0 branch with d = z, scaled by sqrt(2 pi)/sqrt(d).
        cplx d = z;
        p[0] = d.real(); p[1] = 0.0; p[2] = 0.0; p[3] = 0.0;
        p[4] = 0.0; p[5] = 0.0; p[6] = d.real(); p[7] = 0.0;
        cplx s = std::sqrt(2.0 * M_PI) / std::sqrt(d);
        frft_scale_abs = std::abs(s);
        frft_scale_turns = std::arg(s) / (2.0 * M_PI);
    } else {
        cplx zi = 1.0 / z;
        cplx a = (z + zi) / 2.0;
        cplx b = (zi - z) / cplx(0.0, 2.0);
        cplx c = cplx(0.0, 1.0) * (zi - z) / 2.0;
        p[0] = a.real(); p[1] = a.imag(); p[2] = b.real(); p[3] = b.imag();
        p[4] = c.real(); p[5] = c.imag(); p[6] = a.real(); p[7] = a.imag();
        // F_z = sqrt(2/(1-z^2)) sqrt(2 pi i b) LCT: multiply the LCT prefactor.
        cplx s = std::sqrt(2.0 / one_minus_z2) * std::sqrt(cplx(0.0, 2.0 * M_PI) * b);
        frft_scale_abs = std::abs(s);
        frft_scale_turns = std::arg(s) / (2.0 * M_PI);
    }
    lct_plan plan = nullptr;
    // The mapped parameters satisfy ad - bc = 1 up to rounding.
    lct_status st = new_plan(&plan, dtype, 1, &N, p, nullptr, false);
    if (st != LCT_OK) return st;
    plan->desc[0].scale *= frft_scale_abs;
    plan->desc[0].out_c += double_to_turns64(frft_scale_turns);
    st = lct_execute(plan, in, out, batch, stream);
    // Free the plan's device state only after the stream has consumed it.
    if (st == LCT_OK && plan->device >= 0) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = LCT_ERR_CUDA;
    }
    lct_plan_destroy(plan);
    return st;
}

lct_status lct_output_grid(lct_plan plan, int64_t index, double* y_reim, double* rho) {
    if (!plan || !y_reim || index < 0 || index >= plan->count) return LCT_ERR_ARG;
    int64_t N = plan->N[index];
    const double* p = plan->abcd.data() + 8 * index;
    cplx b(p[2], p[3]), c(p[4], p[5]), d(p[6], p[7]);
    for (int64_t j = 0; j < N; ++j) {
        double m = (double)(2 * j - N + 1);
        double x = M_PI * m / (2.0 * std::sqrt(2.0 * (double)N));
        cplx y;
        double r;
        if (b == cplx(0.0, 0.0)) {
            y = x / d;
            r = -(c / d).imag() * M_PI * M_PI * m * m / (16.0 * (double)N);
        } else {
            y = 4.0 * b * x / M_PI;
            r = -(b * d).imag() * m * m / (double)N;
        }
        y_reim[2 * j] = y.real();
        y_reim[2 * j + 1] = y.imag();
        if (rho) rho[j] = r;
    }
    return LCT_OK;
}

lct_status lct_input_grid(int64_t N, double* x) {
    if (!x) return LCT_ERR_ARG;
    if (ilog2_exact(N) < 0) return LCT_ERR_N;
    for (int64_t k = 0; k < N; ++k)
        x[k] = M_PI * (double)(2 * k - N + 1) / (2.0 * std::sqrt(2.0 * (double)N));
    return LCT_OK;
}

lct_status lct_plan_phase_turns(lct_plan plan, int64_t index, uint64_t out[5]) {
    if (!plan || !out || index < 0 || index >= plan->count) return LCT_ERR_ARG;
    const lct_desc& D = plan->desc[index];
    out[0] = D.in_hi;
    out[1] = D.in_lo;
    out[2] = D.out_hi;
    out[3] = D.out_lo;
    out[4] = D.out_c;
    return LCT_OK;
}

lct_status lct_device_status(lct_plan plan, lct_stream_t stream) {
    if (!plan) return LCT_ERR_ARG;
    std::lock_guard<std::mutex> g(plan->mu);
    if (plan->device < 0) return LCT_OK;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LCT_ERR_CUDA;
    int32_t v = 0;
    if (cudaMemcpy(&v, plan->d_status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LCT_ERR_CUDA;
    if (v != LCT_DEV_OK) {
        cudaMemset(plan->d_status, 0, sizeof(int32_t));
        return v == LCT_DEV_TIMEOUT ? LCT_ERR_TIMEOUT : LCT_ERR_DEVICE;
    }
    return LCT_OK;
}

lct_status lct_plan_destroy(lct_plan plan) {
    if (!plan) return LCT_ERR_ARG;
    release_device(plan);
    delete plan;
    return LCT_OK;
}

lct_status lct_backward(lct_plan plan, const void* grad_out, const void* in, const void* out,
                        void* grad_in, double* grad_abd, int64_t batch, lct_stream_t stream_) {
    trace_range trace("lct_backward");
    if (!plan || batch < 0) return LCT_ERR_ARG;
    if (plan->is_batch && batch != plan->count) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    lct_status st = check_ptr(grad_out, plan->dtype);
    if (st == LCT_OK) st = check_ptr(grad_in, plan->dtype);
    if (st != LCT_OK) return st;
    if (grad_abd) {
        if ((st = check_ptr(in, plan->dtype)) != LCT_OK) return st;
        if ((st = check_ptr(out, plan->dtype)) != LCT_OK) return st;
        if (!real_params(plan)) return LCT_ERR_UNSUPPORTED;
    }
    if (plan->ragged || plan->N0 == 0 || plan->prec != LCT_PREC_NATIVE) return LCT_ERR_UNSUPPORTED;
    for (const lct_desc& D : plan->desc)
        if (D.kind != LCT_KIND_XFT) return LCT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(plan->mu);
    st = ensure_device(plan);
    if (st != LCT_OK) return st;
    return run_backward(plan, grad_out, in, out, grad_in, grad_abd, batch, 0, 1, 1, plan->N0,
                        (cudaStream_t)stream_);
}

// ---------------------------------------------------------------------------
// separable 2-D transform
// ---------------------------------------------------------------------------
struct lct2d_plan_s {
    lct_plan px = nullptr;   // rows: length nx
    lct_plan py = nullptr;   // columns: length ny
    int64_t nx = 0, ny = 0;
    lct_dtype dtype = LCT_C64;
};

lct_status lct2d_plan_create(lct2d_plan* out, int64_t ny, int64_t nx, const double abcd_y[4],
                             const double abcd_x[4], lct_dtype dtype) {
    if (!out || !abcd_y || !abcd_x) return LCT_ERR_ARG;
    *out = nullptr;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    const int lx = ilog2_exact(nx), ly = ilog2_exact(ny);
    if (lx < 0 || ly < 0) return LCT_ERR_N;
    if (!lct_gen_supported(dtype, ly, 1) || !lct_gen_supported(dtype, lx, 0) || !lct_fused_supported(dtype, lx))
        return LCT_ERR_UNSUPPORTED;
    if (abcd_x[1] == 0.0 || abcd_y[1] == 0.0) return LCT_ERR_UNSUPPORTED;
    lct2d_plan p = new (std::nothrow) lct2d_plan_s();
    if (!p) return LCT_ERR_OOM;
    p->nx = nx;
    p->ny = ny;
    p->dtype = dtype;
    lct_status st = lct_plan_create(&p->px, nx, abcd_x[0], abcd_x[1], abcd_x[2], abcd_x[3], dtype);
    if (st == LCT_OK)
        st = lct_plan_create(&p->py, ny, abcd_y[0], abcd_y[1], abcd_y[2], abcd_y[3], dtype);
    if (st != LCT_OK) {
        lct2d_plan_destroy(p);
        return st;
    }
    *out = p;
    return LCT_OK;
}

lct_status lct2d_execute(lct2d_plan plan, const void* in, void* mid, void* out, int64_t batch,
                         lct_stream_t stream_) {
    trace_range trace("lct2d_execute");
    if (!plan || batch < 0) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    lct_status st = check_ptr(mid, plan->dtype);
    if (st == LCT_OK) st = check_ptr(out, plan->dtype);
    if (st != LCT_OK) return st;
    // rows: batch * ny contiguous signals of length nx
    st = lct_execute(plan->px, in, mid, batch * plan->ny, stream_);
    if (st != LCT_OK) return st;
    lct_plan py = plan->py;
    std::lock_guard<std::mutex> g(py->mu);
    st = ensure_device(py);
    if (st != LCT_OK) return st;
    const int ly = py->desc[0].log2n;
    const void* tw = py->dtype == LCT_C64 ? lct_twiddle_table_r8(ly) : lct_twiddle_table(py->dtype, ly);
    if (ly >= 5 && !tw) return LCT_ERR_OOM;
    // columns: batch * nx signals of length ny, element stride nx
    return from_cuda(lct_launch_gen(py->dtype, ly, 1, 0, 0, mid, out, py->d_desc, 0,
                                    batch * plan->nx, tw, plan->nx, plan->nx,
                                    plan->nx * plan->ny, nullptr, nullptr, nullptr,
                                    py->desc.data(), (cudaStream_t)stream_));
}

lct_status lct2d_backward(lct2d_plan plan, const void* grad_out, const void* in, const void* mid,
                          const void* out, void* grad_mid, void* grad_in, double* grad_abd,
                          int64_t batch, lct_stream_t stream_) {
    trace_range trace("lct2d_backward");
    if (!plan || batch < 0) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    const void* ptrs[4] = {grad_out, grad_mid, grad_in, grad_abd ? mid : grad_out};
    for (const void* q : ptrs) {
        lct_status st = check_ptr(q, plan->dtype);
        if (st != LCT_OK) return st;
    }
    if (grad_abd && (check_ptr(in, plan->dtype) != LCT_OK || check_ptr(out, plan->dtype) != LCT_OK))
        return LCT_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    lct_status st;
    {
        lct_plan py = plan->py;
        std::lock_guard<std::mutex> g(py->mu);
        if ((st = ensure_device(py)) != LCT_OK) return st;
        st = run_backward(py, grad_out, mid, out, grad_mid, grad_abd ? grad_abd + 3 : nullptr,
                          batch * plan->nx, 1, plan->nx, plan->nx, plan->nx * plan->ny, stream);
        if (st != LCT_OK) return st;
    }
    lct_plan px = plan->px;
    std::lock_guard<std::mutex> g(px->mu);
    if ((st = ensure_device(px)) != LCT_OK) return st;
    return run_backward(px, grad_mid, in, mid, grad_in, grad_abd, batch * plan->ny, 0, 1, 1,
                        plan->nx, stream);
}

lct_status lct2d_plan_destroy(lct2d_plan plan) {
    if (!plan) return LCT_ERR_ARG;
    if (plan->px) lct_plan_destroy(plan->px);
    if (plan->py) lct_plan_destroy(plan->py);
    delete plan;
    return LCT_OK;
}

lct_status lct_set_debug(int on) {
    g_debug.store(on ? 1 : 0);
    return LCT_OK;
}

lct_status lct_selftest_timeout(int which, double limit_ms, lct_stream_t stream_) {
    if ((which != 0 && which != 1) || !(limit_ms > 0.0) || limit_ms > 1000.0) return LCT_ERR_ARG;
    cudaStream_t stream = (cudaStream_t)stream_;
    int32_t* word = nullptr;
    if (cudaMalloc(&word, 4 * sizeof(int32_t)) != cudaSuccess) return LCT_ERR_OOM;
    lct_status st = LCT_OK;
    int32_t result = -1;
    if (cudaMemsetAsync(word, 0, 4 * sizeof(int32_t), stream) != cudaSuccess ||
        lct_launch_selftest_wait(which, (uint64_t)(limit_ms * 1e6), word, stream) != cudaSuccess ||
        cudaMemcpyAsync(&result, word, sizeof(int32_t), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        st = LCT_ERR_CUDA;
    cudaFree(word);
    if (st != LCT_OK) return st;
    return result == LCT_DEV_TIMEOUT ? LCT_ERR_TIMEOUT : (result == LCT_DEV_OK ? LCT_OK : LCT_ERR_CUDA);
}

lct_status lct_partition(int64_t count, const int64_t* N, const double* abcd_reim, int32_t world,
                         int32_t* owner, double* load) {
    if (count < 0 || world < 1 || (count > 0 && (!N || !owner))) return LCT_ERR_ARG;
    std::vector<double> cost((size_t)count);
    for (int64_t s = 0; s < count; ++s) {
        if (ilog2_exact(N[s]) < 0) return LCT_ERR_N;
        const bool diag = abcd_reim && abcd_reim[8 * s + 2] == 0.0 && abcd_reim[8 * s + 3] == 0.0;
        cost[(size_t)s] = diag ? (double)N[s] : (double)N[s] * ilog2_exact(N[s]);
    }
    std::vector<int64_t> order((size_t)count);
    std::iota(order.begin(), order.end(), (int64_t)0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return cost[(size_t)x] > cost[(size_t)y]; });
    // least-loaded rank first, then the lowest rank
    using slot = std::pair<double, int32_t>;
    std::priority_queue<slot, std::vector<slot>, std::greater<slot>> ranks;
    for (int32_t r = 0; r < world; ++r) ranks.push({0.0, r});
    std::vector<double> total((size_t)world, 0.0);
    for (int64_t s : order) {
        slot r = ranks.top();
        ranks.pop();
        owner[s] = r.second;
        r.first += cost[(size_t)s];
        total[(size_t)r.second] = r.first;
        ranks.push(r);
    }
    if (load)
        for (int32_t r = 0; r < world; ++r) load[r] = total[(size_t)r];
    return LCT_OK;
}

const char* lct_status_string(lct_status s) {
    switch (s) {
        case LCT_OK: return "ok";
        case LCT_ERR_ARG: return "invalid argument";
        case LCT_ERR_N: return "N must be a power of two in [2, 65536]";
        case LCT_ERR_NOT_SYMPLECTIC: return "parameters do not satisfy ad - bc = 1";
        case LCT_ERR_DTYPE: return "unknown dtype";
        case LCT_ERR_ALIGN: return "pointer not aligned to the sample size";
        case LCT_ERR_OOM: return "out of device memory";
        case LCT_ERR_CUDA: return "CUDA runtime or cuFFT error";
        case LCT_ERR_DEVICE: return "a kernel recorded a per-item error";
        case LCT_ERR_TIMEOUT: return "a bounded device wait timed out";
        case LCT_ERR_UNSUPPORTED: return "combination not supported";
    }
    return "unknown status";
}

}  // extern "C"
