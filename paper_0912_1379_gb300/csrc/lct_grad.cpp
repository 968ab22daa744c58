// Backward (adjoint transform and parameter gradients) and the separable
// 2-D transform (include/lct.h).
#include "lct_plan.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

namespace lcth {

namespace {
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

}  // namespace

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

// Adjoint of a plan the backward kernel does not take (N >= 8192, N that is
// not a power of two, b = 0), real parameters: the discrete operator is
// L = S_out K S_in with diagonal chirps S and a symmetric K (the kernel
// e^{-i pi m_j m_k/(2N)} of Sec. 3, or the identity for b = 0), so
//   L^H g = conj(L' conj(g)),  L' = S_in K S_out,
// the forward transform with the two chirps exchanged (for b = 0 the plan's
// own diagonal).  Two conjugation passes around one forward launch, in place
// in h; signals contiguous (offset s N).
lct_status run_adjoint_forward(lct_plan p, const void* g, void* h, int64_t batch, cudaStream_t stream) {
    if (!p->d_desc_adj) {
        std::vector<lct_desc> a(p->desc);
        for (lct_desc& D : a)
            if (D.kind == LCT_KIND_XFT || D.kind == LCT_KIND_MIXED || D.kind == LCT_KIND_BLUE) {
                std::swap(D.in_hi, D.out_hi);
                std::swap(D.in_lo, D.out_lo);
            }
        const size_t bytes = sizeof(lct_desc) * a.size();
        if (cudaMalloc(&p->d_desc_adj, bytes) != cudaSuccess) return LCT_ERR_OOM;
        if (cudaMemcpy(p->d_desc_adj, a.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
            return LCT_ERR_CUDA;
    }
    const int64_t n = batch * p->N0;
    lct_status st = from_cuda(lct_launch_conj(p->dtype, g, h, n, stream));
    if (st == LCT_OK) st = execute_locked(p, p->d_desc_adj, h, h, batch, stream);
    if (st == LCT_OK) st = from_cuda(lct_launch_conj(p->dtype, h, h, n, stream));
    return st;
}

}  // namespace lcth

using namespace lcth;

extern "C" {

lct_status lct_backward(lct_plan plan, const void* grad_out, const void* in, const void* out,
                        void* grad_in, double* grad_abd, int64_t batch, lct_stream_t stream_) {
    trace_range trace("lct_backward");
    launch_lock launch;
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
    bool gen = lct_gen_supported(plan->dtype, plan->desc[0].log2n, 0);
    for (const lct_desc& D : plan->desc)
        if (D.kind != LCT_KIND_XFT) gen = false;
    std::lock_guard<std::mutex> g(plan->mu);
    st = ensure_device(plan);
    if (st != LCT_OK) return st;
    if (!gen) {
        // input gradient only: through the forward kernels
        if (grad_abd || !real_params(plan) || (plan->is_batch && !plan->contiguous))
            return LCT_ERR_UNSUPPORTED;
        st = run_adjoint_forward(plan, grad_out, grad_in, batch, (cudaStream_t)stream_);
        if (st == LCT_OK && debug_on()) st = debug_check(plan, grad_in, batch, (cudaStream_t)stream_);
        return st;
    }
    st = run_backward(plan, grad_out, in, out, grad_in, grad_abd, batch, 0, 1, 1, plan->N0,
                      (cudaStream_t)stream_);
    if (st == LCT_OK && debug_on()) st = debug_check(plan, grad_in, batch, (cudaStream_t)stream_);
    return st;
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
    launch_lock launch;
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
    launch_lock launch;
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

}  // extern "C"

// ---------------------------------------------------------------------------
// transposes for the multi-GPU separable 2-D transform
// ---------------------------------------------------------------------------
extern "C" lct_status lct_transpose(lct_dtype dtype, const void* in, void* out, int64_t rows,
                                    int64_t cols, int64_t vec, int64_t batch, lct_stream_t stream) {
    if (dtype != LCT_C64 && dtype != LCT_C128) return LCT_ERR_DTYPE;
    if (rows < 0 || cols < 0 || vec < 1 || batch < 0) return LCT_ERR_ARG;
    if (rows == 0 || cols == 0 || batch == 0) return LCT_OK;
    if (in == out) return LCT_ERR_ARG;
    lct_status st = check_ptr(in, dtype);
    if (st == LCT_OK) st = check_ptr(out, dtype);
    if (st != LCT_OK) return st;
    launch_lock launch;
    return from_cuda(lct_launch_transpose((int)dtype, in, out, rows, cols, vec, batch,
                                          (cudaStream_t)stream));
}
