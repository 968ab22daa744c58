// Host-side internals of the library, shared by lct_phase.cpp (exact phase
// constants, descriptors, twiddle tables), lct_plan.cpp (plans, device
// state, tune cache, sharding), lct_exec.cpp (forward execution) and
// lct_grad.cpp (backward and the separable 2-D transform): the plan object
// and the helpers the entry points share.  Not installed; include/lct.h is
// the public interface.
#pragma once
#include "lct_internal.h"
#include "../../include/lct.h"

#include <cuda_runtime.h>
#include <cufft.h>
#include <nvtx3/nvToolsExt.h>

#include <complex>
#include <cstdint>
#include <mutex>
#include <vector>

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
    int fft_type = 0;
    int variant = -1;               // -1: not chosen (cache or default 0)
    // ragged execution (mixed N or kinds): groups of equal (N, kind), largest
    // N first, each an index list into desc; run as one CUDA graph
    // kind LCT_KIND_DIAG: one group for every diagonal signal (log2n = -1),
    // its idx list ordered by N, run through the chunk list chunks[chunk_off ..]
    struct group {
        int log2n, kind;
        int n = 0;                  // N of the group's signals
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
    // persistent ragged launch (variant 9): its work queue, two-pass group
    // table, ring workspace and counters, built on first use
    int4* d_rg_items = nullptr;
    lct_rg_group* d_rg_groups = nullptr;
    int64_t rg_items = 0;
    void* d_rg_work = nullptr;
    int32_t* d_rg_sync = nullptr;
    size_t rg_sync_bytes = 0;
    const void* rg_tw[17] = {};
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
    // backward through the forward kernels: descriptors with the two chirps exchanged
    lct_desc* d_desc_adj = nullptr;
    int64_t partial_count = 0;
    // offset properties, fixed at creation: every offset even (16-byte signal
    // starts when `in` is 16-byte aligned) and offset[s] == s N0
    bool even_offsets = true;
    bool contiguous = true;
    // set by execute_locked: the launch reads the plan's own descriptor array
    // (not a shifted sub-range of it, as chunked host-buffer execution passes)
    bool own_desc = true;
};

namespace lcth {

typedef std::complex<double> cplx;

// ---- lct_phase.cpp --------------------------------------------------------
// log2 N for N a power of two in [2, 65536], else -1.
int ilog2_exact(int64_t N);
// Is this a plan of N that is not a power of two (mixed-radix or chirp-convolution kernel)?
inline bool blue_kind(int kind) {
    return kind == LCT_KIND_BLUE || kind == LCT_KIND_DIAGN || kind == LCT_KIND_MIXED;
}
// round(v 2^64) mod 2^64 for a turn fraction v (|v| < 1).
uint64_t double_to_turns64(double v);
// Validates p = {a, b, c, d} (re, im pairs; ad - bc = 1) and fills the
// descriptor of one N-point signal at element `offset`.
lct_status make_desc(int64_t N, const double* p, int64_t offset, lct_desc* D);
// Complex-z fractional transform on the nodes (kind LCT_KIND_MEHLER): the
// descriptor and the lag-kernel constants h_l = c e^{-a_h l^2} e^{2 pi i phi_h l^2}.
struct mehler_consts {
    double a_h, c_re, c_im;
    uint64_t phi_hi, phi_lo;
};
// |z| <= 1 (+1e-15), z != +-1, finite; else LCT_ERR_ARG.  N is not checked.
lct_status mehler_setup(int64_t N, double z_re, double z_im, lct_desc* D, mehler_consts* K);

// ---- lct_plan.cpp ---------------------------------------------------------
int tune_lookup(int dtype, int log2n);               // -1: no cached choice
void tune_store(int dtype, int log2n, int variant);
void release_device(lct_plan p);
lct_status ensure_device(lct_plan p);                // descriptors on the current device
bool debug_on();
lct_status check_ptr(const void* ptr, lct_dtype dt);
lct_status from_cuda(cudaError_t e);
lct_status new_plan(lct_plan* out, lct_dtype dtype, int64_t count, const int64_t* N,
                    const double* abcd, const int64_t* offsets, bool is_batch);

// ---- lct_exec.cpp ---------------------------------------------------------
int default_variant(lct_dtype dtype, int log2n);
int effective_variant(lct_plan p);
bool tma_aligned(lct_plan p, const void* in);
bool pair_tma_ok(lct_plan p, const void* in);
bool tma_ok(lct_plan p, const void* in);
bool tmat_ok(lct_plan p, const void* in, int64_t batch);
lct_status execute_locked(lct_plan plan, const lct_desc* desc, const void* in, void* out,
                          int64_t batch, cudaStream_t stream);
lct_status debug_check(lct_plan plan, const void* out, int64_t count, cudaStream_t stream);

// ---- lct_grad.cpp ---------------------------------------------------------
bool real_params(const lct_plan p);
lct_status run_backward(lct_plan p, const void* g, const void* f, const void* G, void* h,
                        double* grad, int64_t batch, int cols, int64_t es, int64_t P, int64_t big,
                        cudaStream_t stream);

inline size_t sample_bytes(lct_dtype dtype) { return dtype == LCT_C64 ? 8 : 16; }

// Launch lock of the entry points that run kernels, taken before any plan's
// own lock.  The kernel launchers keep per-device launch configurations
// (resident CTAs per multiprocessor, shared-memory opt-ins) in plain statics
// filled by their first launch on a device; one process-wide lock around
// the host-side submission makes those first writes happen before every
// later read, from any thread.  Recursive: an entry point may call another
// (frft_execute runs lct_execute, lct2d_execute runs lct_execute).  It is
// held only while launches are enqueued (and the waits of lct_execute_host
// and lct_plan_autotune), not while kernels run.
std::recursive_mutex& launch_mutex();
struct launch_lock {
    launch_lock() : g(launch_mutex()) {}
    std::lock_guard<std::recursive_mutex> g;
};

// NVTX range over an entry point (visible in Nsight timelines; costs a
// call into the NVTX stub when no tool is attached).
struct trace_range {
    explicit trace_range(const char* name) { nvtxRangePushA(name); }
    ~trace_range() { nvtxRangePop(); }
    trace_range(const trace_range&) = delete;
    trace_range& operator=(const trace_range&) = delete;
};

}  // namespace lcth
