// Plans and their device state, the autotune cache, debug mode, sharding
// over ranks and the status strings (include/lct.h).
#include "lct_plan.h"

#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <queue>
#include <string>
#include <tuple>
#include <vector>

// ---------------------------------------------------------------------------
// autotune cache: (gpu name, dtype, log2n) -> variant
// ---------------------------------------------------------------------------
namespace lcth {
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

}  // namespace
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
}  // namespace lcth

namespace lcth {


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
    cudaFree(p->d_rg_items);
    cudaFree(p->d_rg_groups);
    cudaFree(p->d_rg_work);
    cudaFree(p->d_rg_sync);
    p->d_rg_items = nullptr;
    p->d_rg_groups = nullptr;
    p->d_rg_work = nullptr;
    p->d_rg_sync = nullptr;
    p->rg_items = 0;
    p->rg_sync_bytes = 0;
    cudaFree(p->d_coef);
    cudaFree(p->d_partial);
    cudaFree(p->d_desc_adj);
    p->d_coef = nullptr;
    p->d_partial = nullptr;
    p->d_desc_adj = nullptr;
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

std::recursive_mutex& launch_mutex() {
    static std::recursive_mutex m;
    return m;
}

// Debug mode (LCT_DEBUG=1 in the environment, or lct_set_debug): every
// lct_execute / lct_backward synchronises its stream, scans the outputs for
// non-finite samples and reports the device status word.
namespace {
std::atomic<int> g_debug{-1};
}  // namespace

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
        // N: a power of two in [2, 65536], or another N the chirp-convolution
        // kernel takes in this dtype
        if (ilog2_exact(N[s]) < 0 && !lct_blue_supported(dtype, N[s])) { delete p; return LCT_ERR_N; }
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
        // Group by (N, kind), largest N first (tile size log2n, then N).
        p->ragged = true;
        typedef std::tuple<int, int, int> gkey;                   // (log2n, n, kind)
        std::map<gkey, std::vector<int32_t>, std::greater<gkey>> by;
        for (int64_t s = 0; s < count; ++s) {
            const lct_desc& D = p->desc[s];
            by[gkey{D.log2n, D.n, D.kind}].push_back((int32_t)s);
        }
        lct_plan_s::group diag;
        diag.log2n = -1;
        diag.kind = LCT_KIND_DIAG;
        diag.count = 0;
        std::vector<int32_t> diag_idx;
        for (auto& kv : by) {
            if (std::get<2>(kv.first) == LCT_KIND_DIAG) {
                // chunks of kDiagChunk elements, or whole small signals packed
                const int L = std::get<0>(kv.first);
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
            g.log2n = std::get<0>(kv.first);
            g.n = std::get<1>(kv.first);
            g.kind = std::get<2>(kv.first);
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


}  // namespace lcth

using namespace lcth;

// ---------------------------------------------------------------------------
// C ABI: plans
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
            plan->prec = precision;
            return LCT_OK;
        case LCT_PREC_PLAIN64:
            // the unfused paths take powers of two only
            if (blue_kind(plan->desc[0].kind)) return LCT_ERR_UNSUPPORTED;
            plan->prec = precision;
            return LCT_OK;
        case LCT_PREC_PLAIN32:
            if (blue_kind(plan->desc[0].kind)) return LCT_ERR_UNSUPPORTED;
            // FP32 chirps around cuFFT C2C: complex64 plans of one N
            if (plan->dtype != LCT_C64 || plan->ragged || plan->N0 == 0) return LCT_ERR_UNSUPPORTED;
            plan->prec = precision;
            return LCT_OK;
        case LCT_PREC_SPLIT_BF16:
        case LCT_PREC_SPLIT_FP16:
        case LCT_PREC_FP16: {
            // tensor-core DFT: complex64, one N in [16, 4096] (b = 0 plans have
            // no DFT and run their diagonal kernel whatever the precision)
            if (plan->dtype != LCT_C64 || plan->ragged || plan->N0 == 0) return LCT_ERR_UNSUPPORTED;
            const int log2n = ilog2_exact(plan->N0);
            if (log2n < 0) return LCT_ERR_UNSUPPORTED;
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
    if (!plan || variant < 0 || variant > 11) return LCT_ERR_ARG;
    plan->variant = variant;
    return LCT_OK;
}

lct_status lct_plan_get_variant(lct_plan plan, int* variant) {
    if (!plan || !variant) return LCT_ERR_ARG;
    *variant = plan->variant >= 0 ? plan->variant
                                  : default_variant(plan->dtype, plan->desc[0].log2n);
    return LCT_OK;
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
    if (N < 2 || N > 65536) return LCT_ERR_N;
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
        if (N[s] < 2 || N[s] > 65536) return LCT_ERR_N;
        const bool diag = abcd_reim && abcd_reim[8 * s + 2] == 0.0 && abcd_reim[8 * s + 3] == 0.0;
        const int l = ilog2_exact(N[s]);
        // a DFT of N (power of two or 7-smooth, mixed radix), or two DFTs of
        // M >= 2N - 1 (other N)
        const double dft = l >= 0 ? (double)N[s] * l
                         : lct_mixed_ok(N[s]) ? (double)N[s] * std::ceil(std::log2((double)N[s]))
                                  : 2.0 * (double)((int64_t)1 << lct_blue_log2m(N[s])) * lct_blue_log2m(N[s]);
        cost[(size_t)s] = diag ? (double)N[s] : dft;
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
        case LCT_ERR_N:
            return "N must be a power of two in [2, 65536] or another N in [3, 8192] (complex64) / "
                   "[3, 4096] (complex128)";
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
