// Forward execution: the plain FP64 path, the fused / persistent / paired /
// cluster / two-pass kernels and their variant choice, ragged batches as
// one CUDA graph, the split-precision path, host-buffer execution with
// overlapped copies, the autotuner and the FrFT entry (include/lct.h).
#include "lct_plan.h"

#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <complex>
#include <mutex>
#include <vector>

namespace lcth {

namespace {
// Plain paths: chirp kernel -> cuFFT (forward) -> chirp+scale kernel, on an
// FP64 workspace with Z2Z (PLAIN64) or an FP32 one with C2C (PLAIN32).
lct_status run_plain(lct_plan p, const void* in, void* out, int64_t count, int desc_step,
                     cudaStream_t stream) {
    const bool fp32 = p->prec == LCT_PREC_PLAIN32;
    int64_t N = p->N0;
    int log2n = p->desc[0].log2n;
    size_t need = (size_t)count * (size_t)N * (fp32 ? 8 : 16);
    if (need > p->work_bytes) {
        cudaFree(p->d_work);
        p->d_work = nullptr;
        p->work_bytes = 0;
        if (cudaMalloc(&p->d_work, need) != cudaSuccess) return LCT_ERR_OOM;
        p->work_bytes = need;
    }
    const cufftType type = fp32 ? CUFFT_C2C : CUFFT_Z2Z;
    if (!p->fft_valid || p->fft_n != N || p->fft_batch != count || p->fft_type != (int)type) {
        if (p->fft_valid) cufftDestroy(p->fft);
        p->fft_valid = false;
        int n = (int)N;
        if (cufftPlanMany(&p->fft, 1, &n, nullptr, 1, n, nullptr, 1, n, type, (int)count) !=
            CUFFT_SUCCESS)
            return LCT_ERR_CUDA;
        p->fft_valid = true;
        p->fft_n = N;
        p->fft_batch = count;
        p->fft_type = (int)type;
    }
    if (cufftSetStream(p->fft, stream) != CUFFT_SUCCESS) return LCT_ERR_CUDA;
    if (fp32) {
        lct_status st = from_cuda(lct_launch_plain32_pre(in, p->d_work, p->d_desc, log2n,
                                                         desc_step, count, stream));
        if (st != LCT_OK) return st;
        cufftComplex* w = (cufftComplex*)p->d_work;
        if (cufftExecC2C(p->fft, w, w, CUFFT_FORWARD) != CUFFT_SUCCESS) return LCT_ERR_CUDA;
        return from_cuda(lct_launch_plain32_post(p->d_work, out, p->d_desc, log2n, desc_step,
                                                 count, stream));
    }
    lct_status st = from_cuda(lct_launch_plain_pre(p->dtype, log2n, in, p->d_work, p->d_desc,
                                                   desc_step, count, stream));
    if (st != LCT_OK) return st;
    cufftDoubleComplex* w = (cufftDoubleComplex*)p->d_work;
    if (cufftExecZ2Z(p->fft, w, w, CUFFT_FORWARD) != CUFFT_SUCCESS) return LCT_ERR_CUDA;
    return from_cuda(lct_launch_plain_post(p->dtype, log2n, p->d_work, out, p->d_desc, desc_step,
                                           count, stream));
}
}  // namespace

// The split modes at N = 4096 run on tcgen05 unless LCT_SPLIT_KERNEL=mma
// selects the mma.sync kernel (a diagnostic, read once).
bool split_on_tcgen05() {
    static const bool on = [] {
        const char* e = std::getenv("LCT_SPLIT_KERNEL");
        return !(e && std::strcmp(e, "mma") == 0);
    }();
    return on;
}

// Smallest N that runs two-pass by default (measured on GB300: two passes
// beat the cluster kernel from here up).
constexpr int kTwoPassDefaultLog2 = 15;

// Can a bulk-async variant run this plan on `in` (16-byte aligned starts)?
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

// Can variant 8 (tensor-map staged loads) run this launch: contiguous
// signals addressed from `in` itself (the plan's own descriptors), 16-byte
// aligned, whole 256-sample rows?
bool tmat_ok(lct_plan p, const void* in, int64_t batch) {
    const int log2n = p->desc[0].log2n;
    return lct_fused_tmat_supported(p->dtype, log2n) && ((uintptr_t)in) % 16 == 0 &&
           p->own_desc && (!p->is_batch || p->contiguous) &&
           ((batch << log2n) % 256) == 0;
}

// Variant used when neither the plan nor the tune cache chooses one: two
// passes from N = 32768, else the fused kernel's schedule that measured
// fastest on GB300 for complex64 batches (64 Mi points, per-signal
// parameters; the schedule sweep is in the design notes).
int default_variant(lct_dtype dtype, int log2n) {
    if (lct_twopass_supported(dtype, log2n) && log2n >= kTwoPassDefaultLog2) return 7;
    if (dtype == LCT_C64) {
        if (log2n >= 5 && log2n <= 8) return 10;       // N = 32..256: radix-8 passes
        if (log2n >= 9 && log2n <= 11) return 11;      // N = 512..2048: one signal per CTA
    }
    return 0;
}

// Does schedule variant 10 (radix-8 passes) or 11 (one signal per CTA)
// apply to this N and dtype?
bool sched_applies(lct_dtype dtype, int log2n, int variant) {
    if (variant == 10) return lct_fused_sched_supported(dtype, log2n, 3, 0);
    if (variant == 11)
        return lct_fused_sched_supported(dtype, log2n, 2, 1) || lct_fused_sched_supported(dtype, log2n, 4, 1);
    return false;
}

// Twiddle table of a schedule variant (radix-4 passes for complex128 one
// signal per CTA up to N = 2048), or nullptr when the variant does not apply
// to this N and dtype (or the table cannot be made).
const void* sched_table(lct_dtype dtype, int log2n, int variant) {
    if (variant == 10 && lct_fused_sched_supported(dtype, log2n, 3, 0))
        return lct_twiddle_table_le(dtype, log2n, 3);
    if (variant == 11 && lct_fused_sched_supported(dtype, log2n, 2, 1))
        return lct_twiddle_table_le(dtype, log2n, 2);
    if (variant == 11 && lct_fused_sched_supported(dtype, log2n, 4, 1))
        return lct_twiddle_table(dtype, log2n);
    return nullptr;
}

// Launch a schedule variant (10 or 11) of the fused kernel; false if it does
// not apply (the caller then takes variant 0).
bool launch_sched(lct_plan p, int log2n, int variant, const void* in, void* out, int desc_step,
                  int64_t count, const int32_t* idx, cudaStream_t stream, lct_status* st) {
    const void* tw = sched_table(p->dtype, log2n, variant);
    if (!tw) return false;
    const bool r4 = variant == 11 && lct_fused_sched_supported(p->dtype, log2n, 2, 1);
    const int le = variant == 10 ? 3 : (r4 ? 2 : 4);
    *st = from_cuda(lct_launch_fused_sched(p->dtype, log2n, le, variant == 11 ? 1 : 0, in, out, p->d_desc,
                                           desc_step, count, tw, idx, p->d_status, stream));
    return true;
}

int effective_variant(lct_plan p) {
    if (p->variant >= 0) return p->variant;
    int v = tune_lookup(p->dtype, p->desc[0].log2n);
    return v >= 0 ? v : default_variant(p->dtype, p->desc[0].log2n);
}

namespace {
// Two-pass path ------------------------------------------------------------
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
    if (variant == 10 || variant == 11) {
        lct_status st = LCT_OK;
        if (launch_sched(p, log2n, variant, in, out, desc_step, batch, nullptr, stream, &st)) return st;
    }
    if (variant == 8 && tmat_ok(p, in, batch))
        return from_cuda(lct_launch_fused_tmat(log2n, in, out, p->d_desc, desc_step, batch, tw,
                                               p->d_status, stream));
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

// N that is not a power of two: the chirp-convolution kernel (b != 0) or the
// diagonal (b == 0) for `count` signals of one N.
lct_status run_blue(lct_plan p, int kind, int64_t n, const void* in, void* out, int64_t count,
                    int desc_step, const int32_t* idx, cudaStream_t stream) {
    if (kind == LCT_KIND_DIAGN)
        return from_cuda(lct_launch_diag_any(p->dtype, n, in, out, p->d_desc, desc_step, count, idx,
                                             p->d_status, stream));
    if (kind == LCT_KIND_MIXED) {
        lct_mixed_plan pl;
        if (!lct_mixed_make_plan(n, p->dtype, &pl)) return LCT_ERR_N;
        const void* tw = lct_mixed_twiddles(p->dtype, n);
        if (!tw) return LCT_ERR_OOM;
        return from_cuda(lct_launch_mixed(p->dtype, pl, in, out, p->d_desc, desc_step, count, tw, idx,
                                          p->d_status, stream));
    }
    const int lm = lct_blue_log2m(n);
    const void* tw = lct_twiddle_table(p->dtype, lm);
    const void* spec = lct_blue_spectrum(p->dtype, n);
    if ((lm >= 5 && !tw) || !spec) return LCT_ERR_OOM;
    return from_cuda(lct_launch_blue(p->dtype, n, in, out, p->d_desc, desc_step, count, tw, spec,
                                     idx, p->d_status, stream));
}

// Launch one group of a ragged plan on `stream`.
lct_status launch_group(lct_plan p, const lct_plan_s::group& g, const void* in, void* out,
                        cudaStream_t stream) {
    const int32_t* idx = p->d_idx + g.idx_off;
    if (blue_kind(g.kind)) return run_blue(p, g.kind, g.n, in, out, g.count, 1, idx, stream);
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
    const int gv = group_variant(p->dtype, g.log2n);
    if (gv == 10 || gv == 11) {
        lct_status st = LCT_OK;
        if (launch_sched(p, g.log2n, gv, in, out, 1, g.count, idx, stream, &st)) return st;
    }
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
        if (g.kind != LCT_KIND_XFT || !lct_twopass_supported(p->dtype, g.log2n)) continue;
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
        if (g.kind == LCT_KIND_DIAG || g.kind == LCT_KIND_DIAGN) continue;
        if (g.kind == LCT_KIND_MIXED) {
            if (!lct_mixed_twiddles(p->dtype, g.n)) return LCT_ERR_OOM;
            continue;
        }
        if (g.kind == LCT_KIND_BLUE) {
            if ((g.log2n >= 5 && !lct_twiddle_table(p->dtype, g.log2n)) ||
                !lct_blue_spectrum(p->dtype, g.n))
                return LCT_ERR_OOM;
            continue;
        }
        const int lm = lct_cluster_local_log2(p->dtype, g.log2n);
        if (lm >= 0 && !lct_twiddle_table(p->dtype, lm)) return LCT_ERR_OOM;
        if (g.log2n >= 5 && lct_fused_supported(p->dtype, g.log2n) &&
            !lct_twiddle_table(p->dtype, g.log2n))
            return LCT_ERR_OOM;
        const int gv = group_variant(p->dtype, g.log2n);       // schedule tables before capture
        if (sched_applies(p->dtype, g.log2n, gv) && !sched_table(p->dtype, g.log2n, gv)) return LCT_ERR_OOM;
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

// Persistent ragged launch (variant 9, complex64 plans of power-of-two N):
// the work queue, largest N first -- the two-pass tiles of each group of
// N >= 8192, then the fused items of N <= 4096, then the b = 0 chunks.
bool ragged_persistent_ok(lct_plan p) {
    if (p->dtype != LCT_C64) return false;
    for (const auto& g : p->groups)
        if (g.kind != LCT_KIND_DIAG && !(g.kind == LCT_KIND_XFT && g.log2n >= 1 && g.log2n <= 16))
            return false;
    return true;
}

lct_status build_ragged_persistent(lct_plan p) {
    std::vector<int4> items;
    std::vector<lct_rg_group> tg;
    int64_t work = 0, sync = 0;
    for (const auto& g : p->groups) {
        if (g.kind == LCT_KIND_DIAG) {
            for (int64_t c = 0; c < g.nchunks; ++c)
                items.push_back(make_int4(LCT_RG_DIAG, (int)(g.chunk_off + c), (int)g.idx_off, 0));
            continue;
        }
        if (g.log2n >= 13) {
            int64_t slots = 0;
            if (lct_twopass_ring(0, g.log2n, g.count, &slots) != cudaSuccess || slots < 3)
                return LCT_ERR_CUDA;
            int cb = 0, rb = 0;
            lct_twopass_tiles(g.log2n, &cb, &rb);
            lct_rg_group r;
            r.count = g.count;
            r.slots = slots;
            r.lag = slots - 2;
            r.idx_off = g.idx_off;
            r.work_off = work;
            r.sync_off = sync;
            r.log2n = g.log2n;
            r.pad = 0;
            work += slots << g.log2n;
            sync += 4 + 2 * slots;
            const int gi = (int)tg.size();
            tg.push_back(r);
            const int64_t total = g.count * (cb + rb);
            for (int64_t q = 0; q < total; ++q)
                items.push_back(make_int4(LCT_RG_TP, gi, (int)(uint32_t)(q >> 32), (int)(uint32_t)q));
            continue;
        }
        const int spc = lct_ragged_fused_spc(g.log2n);
        for (int64_t j = 0; j < g.count; j += spc)
            items.push_back(make_int4(LCT_RG_FUSED, g.log2n, (int)(g.idx_off + j),
                                      (int)(g.count - j < spc ? g.count - j : spc)));
    }
    for (int l = 5; l <= 12; ++l) {
        p->rg_tw[l] = lct_twiddle_table(LCT_C64, l);
        if (!p->rg_tw[l]) return LCT_ERR_OOM;
    }
    const size_t ib = items.size() * sizeof(int4), gb = (tg.empty() ? 1 : tg.size()) * sizeof(lct_rg_group);
    p->rg_sync_bytes = (size_t)(2 + sync) * sizeof(int32_t);
    if (cudaMalloc(&p->d_rg_items, ib ? ib : sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&p->d_rg_groups, gb) != cudaSuccess ||
        cudaMalloc(&p->d_rg_work, (size_t)(work ? work : 1) * sample_bytes(p->dtype)) != cudaSuccess ||
        cudaMalloc(&p->d_rg_sync, p->rg_sync_bytes) != cudaSuccess)
        return LCT_ERR_OOM;
    if ((ib && cudaMemcpy(p->d_rg_items, items.data(), ib, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (!tg.empty() && cudaMemcpy(p->d_rg_groups, tg.data(), tg.size() * sizeof(lct_rg_group),
                                   cudaMemcpyHostToDevice) != cudaSuccess))
        return LCT_ERR_CUDA;
    p->rg_items = (int64_t)items.size();
    return LCT_OK;
}

lct_status run_ragged(lct_plan p, const void* in, void* out, cudaStream_t stream) {
    if (p->prec != LCT_PREC_NATIVE) return LCT_ERR_UNSUPPORTED;
    if (p->variant == 9 && ragged_persistent_ok(p)) {
        if (!p->d_rg_items) {
            lct_status st = build_ragged_persistent(p);
            if (st != LCT_OK) return st;
        }
        return from_cuda(lct_launch_ragged(in, out, p->d_desc, p->d_idx, p->d_rg_items, p->rg_items,
                                           p->d_rg_groups, (const int4*)p->d_chunks, p->d_rg_work,
                                           p->d_rg_sync, p->rg_sync_bytes, p->rg_tw, p->d_status,
                                           stream));
    }
    if (!p->gexec || p->g_in != in || p->g_out != out) {
        lct_status st = build_graph(p, in, out);
        if (st != LCT_OK) return st;
    }
    return from_cuda(cudaGraphLaunch(p->gexec, stream));
}
}  // namespace

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
    plan->own_desc = desc == plan->d_desc;
    plan->d_desc = const_cast<lct_desc*>(desc);
    const int desc_step = plan->is_batch ? 1 : 0;
    const lct_desc& D0 = plan->desc[0];
    const int log2n = D0.log2n;
    if (blue_kind(D0.kind)) {
        if (plan->prec != LCT_PREC_NATIVE) return LCT_ERR_UNSUPPORTED;
        return run_blue(plan, D0.kind, D0.n, in, out, batch, desc_step, nullptr, stream);
    }
    if (D0.kind == LCT_KIND_DIAG)
        return from_cuda(lct_launch_diag(plan->dtype, log2n, in, out, plan->d_desc, desc_step,
                                         batch, nullptr, plan->d_status, stream));
    if (plan->prec == LCT_PREC_PLAIN64 || plan->prec == LCT_PREC_PLAIN32) {
        // the plain path assumes contiguous rows
        if (plan->is_batch && !plan->contiguous) return LCT_ERR_UNSUPPORTED;
        return run_plain(plan, in, out, batch, desc_step, stream);
    }
    if (plan->prec == LCT_PREC_SPLIT_BF16 || plan->prec == LCT_PREC_SPLIT_FP16 ||
        plan->prec == LCT_PREC_FP16) {
        const void* tw = lct_twiddle_table(plan->dtype, log2n);
        if (log2n >= 5 && !tw) return LCT_ERR_OOM;
        if (lct_split_umma_supported(plan->dtype, log2n) && split_on_tcgen05())
            return from_cuda(lct_launch_split_umma((int)plan->prec, log2n, in, out, plan->d_desc,
                                                   desc_step, batch, tw, plan->d_status, stream));
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
    if (lct_launch_scan(plan->dtype, out, plan->d_desc, desc_step, count, plan->desc[0].n, plan->d_status,
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

namespace {
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

}  // namespace lcth

using namespace lcth;

// ---------------------------------------------------------------------------
// C ABI: execution
// ---------------------------------------------------------------------------
extern "C" {

lct_status lct_plan_autotune(lct_plan plan, const void* in, void* out, int64_t batch,
                             lct_stream_t stream_) {
    trace_range trace("lct_plan_autotune");
    launch_lock launch;
    if (!plan) return LCT_ERR_ARG;
    if (plan->prec != LCT_PREC_NATIVE || plan->N0 == 0 || plan->desc[0].kind != LCT_KIND_XFT) {
        plan->variant = 0;
        return LCT_OK;
    }
    const int saved = plan->variant;
    int candidates[16] = {0};
    int n_cand = 1;
    // schedules of the fused kernel: radix-8 passes, one signal per CTA
    if (sched_applies(plan->dtype, plan->desc[0].log2n, 10)) candidates[n_cand++] = 10;
    if (sched_applies(plan->dtype, plan->desc[0].log2n, 11)) candidates[n_cand++] = 11;
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
    plan->own_desc = true;
    if (tmat_ok(plan, in, batch)) candidates[n_cand++] = 8;
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
    launch_lock launch;
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

// Is p page-locked host memory mapped into the device's address space?
// Then *dp is its device address.
static bool host_mapped(const void* p, void** dp) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();                  // not a CUDA pointer: clear the query's error
        return false;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
    *dp = a.devicePointer;
    return true;
}

lct_status lct_execute_host(lct_plan plan, const void* h_in, void* h_out, int64_t batch,
                            lct_stream_t stream_) {
    trace_range trace("lct_execute_host");
    launch_lock launch;
    if (!plan || !h_in || !h_out || batch < 0) return LCT_ERR_ARG;
    if (plan->is_batch && batch != plan->count) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    if (plan->ragged || plan->N0 == 0 || (plan->is_batch && !plan->contiguous))
        return LCT_ERR_UNSUPPORTED;
    cudaStream_t stream = (cudaStream_t)stream_;
    std::lock_guard<std::mutex> g(plan->mu);
    lct_status st = ensure_device(plan);
    if (st != LCT_OK) return st;
    // Page-locked buffers the device can address: the kernels read and write
    // them in place over the host link, with no staging copies (measured on
    // GB300: 3.28 against 3.46 ms per GiB in each direction).  Kept to the
    // kernels that load with plain instructions: not the bulk-copy and
    // tensor-map variants (1, 2, 4, 8) nor the split precisions.
    {
        void* din = nullptr;
        void* dout = nullptr;
        const int v = effective_variant(plan);
        if (plan->prec == LCT_PREC_NATIVE && v != 1 && v != 2 && v != 4 && v != 8 &&
            host_mapped(h_in, &din) && host_mapped(h_out, &dout))
            return execute_locked(plan, plan->d_desc, din, dout, batch, stream);
    }
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
    launch_lock launch;
    cplx z(z_re, z_im);
    double az = std::abs(z);
    if (!std::isfinite(az) || az == 0.0 || az > 1.0 + 1e-15) return LCT_ERR_ARG;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    if (ilog2_exact(N) < 0 && !lct_blue_supported(dtype, N)) return LCT_ERR_N;
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

// Complex-z fractional transform on the nodes (Sec. 2, eqs. (fasy),
// (primcuad)) as one convolution of length M = 2^ceil(log2(2N - 1)): a
// one-CTA launch forms the lag kernel's spectrum and the descriptor in a
// stream-ordered workspace, then the chirp-convolution kernel transforms the
// batch (lct_internal.h derives the form).
lct_status frft_mehler_execute(int64_t N, double z_re, double z_im, const void* in, void* out,
                               int64_t batch, lct_dtype dtype, lct_stream_t stream_) {
    trace_range trace("frft_mehler_execute");
    launch_lock launch;
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    if (N < 2 || N > (dtype == LCT_C64 ? kBlueMaxN64 : kBlueMaxN128)) return LCT_ERR_N;
    lct_desc D;
    mehler_consts K;
    lct_status st = mehler_setup(N, z_re, z_im, &D, &K);
    if (st != LCT_OK) return st;
    if (batch < 0 || batch > (int64_t)0x7fffffff) return LCT_ERR_ARG;
    if (batch == 0) return LCT_OK;
    st = check_ptr(in, dtype);
    if (st == LCT_OK) st = check_ptr(out, dtype);
    if (st != LCT_OK) return st;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int lm = D.log2n;
    const void* tw = lct_twiddle_table(dtype, lm);
    if (lm >= 5 && !tw) return LCT_ERR_OOM;
    // workspace: descriptor (80 B), status word, spectrum (M samples) at 256 B
    const size_t spec_bytes = ((size_t)1 << lm) * sample_bytes(dtype);
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, 256 + spec_bytes, stream) != cudaSuccess) return LCT_ERR_OOM;
    lct_desc* d_desc = (lct_desc*)ws;
    int32_t* d_status = (int32_t*)((char*)ws + 128);
    void* spec = (char*)ws + 256;
    cudaError_t e = lct_launch_mehler_spectrum(dtype, N, K.a_h, K.phi_hi, K.phi_lo, K.c_re, K.c_im,
                                               D, d_desc, spec, d_status, tw, stream);
    if (e == cudaSuccess)
        e = lct_launch_mehler(dtype, N, in, out, d_desc, batch, tw, spec, d_status, stream);
    const cudaError_t ef = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return from_cuda(e);
    return from_cuda(ef);
}

}  // extern "C"
