// C ABI entry points: one pass of the objective, one optimiser step, the FP64
// certificate.  Every device call is stream-ordered on the caller's stream;
// nothing here synchronises except sos_read_status and sos_certify.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

using namespace sos;

namespace {

template <typename T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

bool bad_prec(int prec) { return prec < SOS_BF16 || prec > SOS_FP64_TC; }

int check_ptr(const void* p, const char* what) {
    if (!p) return fail(SOS_E_INVALID, std::string(what) + " is NULL");
    return SOS_OK;
}

// SOS_FP64_TC: forward on tensor cores by slices, FP64 residual and loss, and
// (when g32 is not NULL) the adjoint 2 H(r) A on tensor cores from bf16 H and
// bf16 A into the float buffer g32.
int pass_tc64(sos_plan_s* p, const double* A, const double* pv, float* g32, void* loss, void* ws, cudaStream_t st,
              int slices) {
    const Workspace w = workspace_layout(p, SOS_FP64_TC);
    double* c = at<double>(ws, w.c);
    SOS_CHECK(forward_tc64(p, A, ws, c, slices, st));
    double* L = loss ? static_cast<double*>(loss) : at<double>(ws, w.loss);
    int32_t* status = at<int32_t>(ws, w.status);
    double* resid = at<double>(ws, w.resid);
    SOS_CHECK(launch_residual<double>(p, c, pv, resid, L, at<double>(ws, w.partials), status, 1, st));
    if (!g32) return SOS_OK;
    float* r32 = at<float>(ws, w.resid32);
    SOS_CHECK(launch_convert<double, float>(resid, r32, p->M, st));
    SOS_CHECK(launch_build_h16(p, r32, at<char>(ws, w.h16), status, st));
    return launch_tc_adjoint_pair(p, at<char>(ws, w.h16), at<char>(ws, w.a16), g32, status, st);
}

// Forward into ws.c (zeroed here).  For BF16 also writes the bf16 copy of A.
int forward(sos_plan_s* p, int prec, const void* A, void* ws, cudaStream_t st, void* c_out) {
    const Workspace w = workspace_layout(p, prec);
    if (prec == SOS_FP64_TC) {
        double* c = c_out ? static_cast<double*>(c_out) : at<double>(ws, w.c);
        return forward_tc64(p, static_cast<const double*>(A), ws, c, kMaxSlices, st);
    }
    if (prec == SOS_FP64) {
        double* c = c_out ? static_cast<double*>(c_out) : at<double>(ws, w.c);
        SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(double), st));
        return launch_simt_forward<double, double>(p, static_cast<const double*>(A), c, 1, st);
    }
    float* c = c_out ? static_cast<float*>(c_out) : at<float>(ws, w.c);
    SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(float), st));
    if (prec == SOS_FP32) return launch_simt_forward<float, float>(p, static_cast<const float*>(A), c, 1, st);
    void* a16 = at<char>(ws, w.a16);
    SOS_CHECK(launch_cast_bf16(static_cast<const float*>(A), p->N, p->r, a16, p->ld16, st));
    if (!use_cta_pairs()) return launch_tc_forward(p, a16, c, at<int32_t>(ws, w.status), st);
    float* diag = nullptr;
    if (use_exact_diag()) {
        diag = at<float>(ws, w.diag);
        SOS_CHECK(launch_diag_sumsq(a16, p->ld16, p->N, p->r, diag, st));
    }
    return launch_tc_forward_pair(p, a16, c, at<int32_t>(ws, w.status), st, diag);
}

int loss_grad(sos_plan_s* p, int prec, const void* A, const void* pv, void* grad, void* loss, void* ws,
              cudaStream_t st, bool fp32_contraction = false) {
    const Workspace w = workspace_layout(p, prec);
    if (prec == SOS_FP64_TC) {
        float* g32 = grad ? at<float>(ws, w.grad) : nullptr;
        SOS_CHECK(pass_tc64(p, static_cast<const double*>(A), static_cast<const double*>(pv), g32, loss, ws, st,
                            kMaxSlices));
        if (grad) SOS_CHECK(launch_convert<float, double>(g32, static_cast<double*>(grad), p->N * p->r, st));
        return SOS_OK;
    }
    SOS_CHECK(forward(p, prec, A, ws, st, nullptr));
    double* L = loss ? static_cast<double*>(loss) : at<double>(ws, w.loss);
    int32_t* status = at<int32_t>(ws, w.status);
    double* partials = at<double>(ws, w.partials);
    if (prec == SOS_FP64) {
        double* resid = at<double>(ws, w.resid);
        SOS_CHECK(launch_residual<double>(p, at<double>(ws, w.c), static_cast<const double*>(pv), resid, L,
                                          partials, status, 1, st));
        if (grad)
            SOS_CHECK(launch_simt_adjoint<double>(p, static_cast<const double*>(A), resid,
                                                  static_cast<double*>(grad), 1, st, fp32_contraction));
        return SOS_OK;
    }
    float* resid = at<float>(ws, w.resid);
    SOS_CHECK(launch_residual<float>(p, at<float>(ws, w.c), static_cast<const float*>(pv), resid, L, partials,
                                     status, 1, st));
    if (!grad) return SOS_OK;
    if (prec == SOS_FP32)
        return launch_simt_adjoint<float>(p, static_cast<const float*>(A), resid, static_cast<float*>(grad), 1,
                                          st);
    if (use_h_ring())
        return launch_tc_adjoint_ring_pair(p, resid, at<char>(ws, w.ring), at<uint32_t>(ws, w.ring_flags),
                                           at<char>(ws, w.a16), static_cast<float*>(grad), status, st);
    void* h16 = at<char>(ws, w.h16);
    SOS_CHECK(launch_build_h16(p, resid, h16, status, st));
    return use_cta_pairs()
               ? launch_tc_adjoint_pair(p, h16, at<char>(ws, w.a16), static_cast<float*>(grad), status, st)
               : launch_tc_adjoint(p, h16, at<char>(ws, w.a16), static_cast<float*>(grad), status, st);
}

Workspace batched_layout(const sos_plan_s* p, int prec, int64_t batch) {
    Workspace w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t a = off;
        off += (bytes + 255) / 256 * 256;
        return a;
    };
    const size_t elt = prec == SOS_FP64 ? 8 : 4;
    w.status = take(64 * sizeof(int32_t));
    w.partials = take((size_t)std::max<int64_t>(2 * kResidBlocks, 2 * batch) * sizeof(double));
    w.loss = take((size_t)batch * 2 * sizeof(double));
    w.c = take((size_t)batch * p->M * elt);
    w.resid = take((size_t)batch * p->M * elt);
    w.total = off;
    return w;
}

}  // namespace

int sos::core_loss_grad(sos_plan_s* p, int prec, const void* A, const void* pv, void* grad, void* loss, void* ws,
                        cudaStream_t st, bool fp32_contraction) {
    return loss_grad(p, prec, A, pv, grad, loss, ws, st, fp32_contraction);
}

extern "C" {

int sos_workspace_init(sos_plan_t p, int prec, void* ws, void* stream) {
    if (!p || bad_prec(prec) || !ws) return fail(SOS_E_INVALID, "sos_workspace_init: bad argument");
    SOS_CUDA(cudaMemsetAsync(ws, 0, 64 * sizeof(int32_t), (cudaStream_t)stream));
    return SOS_OK;
}

int sos_coeffs(sos_plan_t p, int prec, const void* A, void* c, void* ws, void* stream) {
    TraceRange trace_("sos_coeffs");
    if (!p || bad_prec(prec)) return fail(SOS_E_INVALID, "sos_coeffs: bad plan or precision");
    SOS_CHECK(check_ptr(A, "sos_coeffs: A"));
    SOS_CHECK(check_ptr(c, "sos_coeffs: c"));
    SOS_CHECK(check_ptr(ws, "sos_coeffs: workspace"));
    SOS_CHECK(ensure_device(p));
    return forward(p, prec, A, ws, (cudaStream_t)stream, c);
}

int sos_loss_grad(sos_plan_t p, int prec, const void* A, const void* pv, void* grad, void* loss, void* ws,
                  void* stream) {
    TraceRange trace_("sos_loss_grad");
    if (!p || bad_prec(prec)) return fail(SOS_E_INVALID, "sos_loss_grad: bad plan or precision");
    SOS_CHECK(check_ptr(A, "sos_loss_grad: A"));
    SOS_CHECK(check_ptr(pv, "sos_loss_grad: p"));
    SOS_CHECK(check_ptr(ws, "sos_loss_grad: workspace"));
    SOS_CHECK(ensure_device(p));
    return loss_grad(p, prec, A, pv, grad, loss, ws, (cudaStream_t)stream);
}

int sos_workspace_size_batched(sos_plan_t p, int prec, int64_t batch, size_t* bytes) {
    if (!p || !bytes || batch < 1 || (prec != SOS_FP32 && prec != SOS_FP64))
        return fail(SOS_E_INVALID, "sos_workspace_size_batched: bad argument");
    *bytes = batched_layout(p, prec, batch).total;
    return SOS_OK;
}

int sos_loss_grad_batched(sos_plan_t p, int prec, int64_t batch, const void* A, const void* pv, void* grad,
                          void* loss, void* ws, void* stream) {
    TraceRange trace_("sos_loss_grad_batched");
    if (!p || batch < 1 || (prec != SOS_FP32 && prec != SOS_FP64))
        return fail(SOS_E_INVALID, "sos_loss_grad_batched: FP32 or FP64 and batch >= 1");
    SOS_CHECK(check_ptr(A, "sos_loss_grad_batched: A"));
    SOS_CHECK(check_ptr(pv, "sos_loss_grad_batched: p"));
    SOS_CHECK(check_ptr(loss, "sos_loss_grad_batched: loss"));
    SOS_CHECK(check_ptr(ws, "sos_loss_grad_batched: workspace"));
    SOS_CHECK(ensure_device(p));
    cudaStream_t st = (cudaStream_t)stream;
    const Workspace w = batched_layout(p, prec, batch);
    int32_t* status = at<int32_t>(ws, w.status);
    double* partials = at<double>(ws, w.partials);
    double* L = static_cast<double*>(loss);
    if (prec == SOS_FP64) {
        double* c = at<double>(ws, w.c);
        double* resid = at<double>(ws, w.resid);
        SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)batch * p->M * sizeof(double), st));
        SOS_CHECK(launch_simt_forward<double, double>(p, static_cast<const double*>(A), c, batch, st));
        SOS_CHECK(launch_residual<double>(p, c, static_cast<const double*>(pv), resid, L, partials, status, batch,
                                          st));
        if (grad)
            SOS_CHECK(launch_simt_adjoint<double>(p, static_cast<const double*>(A), resid,
                                                  static_cast<double*>(grad), batch, st));
        return SOS_OK;
    }
    float* c = at<float>(ws, w.c);
    float* resid = at<float>(ws, w.resid);
    SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)batch * p->M * sizeof(float), st));
    SOS_CHECK(launch_simt_forward<float, float>(p, static_cast<const float*>(A), c, batch, st));
    SOS_CHECK(launch_residual<float>(p, c, static_cast<const float*>(pv), resid, L, partials, status, batch, st));
    if (grad)
        SOS_CHECK(launch_simt_adjoint<float>(p, static_cast<const float*>(A), resid, static_cast<float*>(grad),
                                             batch, st));
    return SOS_OK;
}

int sos_step(sos_plan_t p, int prec, sos_state* s, const void* pv, const sos_step_opts* o, void* loss, void* ws,
             void* stream) {
    TraceRange trace_("sos_step");
    if (!p || bad_prec(prec) || !s || !o) return fail(SOS_E_INVALID, "sos_step: bad argument");
    SOS_CHECK(check_ptr(s->A, "sos_step: state A"));
    SOS_CHECK(check_ptr(pv, "sos_step: p"));
    SOS_CHECK(check_ptr(ws, "sos_step: workspace"));
    if (o->optimizer == SOS_ADAM && (!s->m || !s->v)) return fail(SOS_E_INVALID, "sos_step: Adam needs m and v");
    if (o->optimizer != SOS_ADAM && o->optimizer != SOS_GD) return fail(SOS_E_INVALID, "sos_step: bad optimizer");
    if (o->flags & ~SOS_STEP_FP32_ADJOINT) return fail(SOS_E_INVALID, "sos_step: unknown flags");
    if (o->slices != 0 && (o->slices < 2 || o->slices > kMaxSlices))
        return fail(SOS_E_INVALID, "sos_step: slices must be 0 or 2..8");
    SOS_CHECK(ensure_device(p));
    cudaStream_t st = (cudaStream_t)stream;
    const Workspace w = workspace_layout(p, prec);
    const int64_t t = s->t + 1;
    if (prec == SOS_BF16) {
        // forward on the current bf16 copy, adjoint with the update fused into
        // its epilogue, which writes the next bf16 copy
        const size_t half = (size_t)p->N * (size_t)p->ld16 * 2;
        const int cur = (s->flags & SOS_STATE_BF16_INDEX) ? 1 : 0;
        char* a16_cur = at<char>(ws, w.a16) + cur * half;
        char* a16_next = at<char>(ws, w.a16) + (1 - cur) * half;
        int32_t* status = at<int32_t>(ws, w.status);
        float* c = at<float>(ws, w.c);
        float* resid = at<float>(ws, w.resid);
        if (!(s->flags & SOS_STATE_BF16_CURRENT))
            SOS_CHECK(launch_cast_bf16(static_cast<const float*>(s->A), p->N, p->r, a16_cur, p->ld16, st));
        SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(float), st));
        if (use_cta_pairs()) {
            float* diag = nullptr;
            if (use_exact_diag()) {
                diag = at<float>(ws, w.diag);
                SOS_CHECK(launch_diag_sumsq(a16_cur, p->ld16, p->N, p->r, diag, st));
            }
            SOS_CHECK(launch_tc_forward_pair(p, a16_cur, c, status, st, diag));
        } else {
            SOS_CHECK(launch_tc_forward(p, a16_cur, c, status, st));
        }
        double* L = loss ? static_cast<double*>(loss) : at<double>(ws, w.loss);
        SOS_CHECK(launch_residual<float>(p, c, static_cast<const float*>(pv), resid, L, at<double>(ws, w.partials),
                                         status, 1, st));
        if (use_h_ring()) {
            SOS_CHECK(launch_tc_adjoint_update_ring_pair(
                p, resid, at<char>(ws, w.ring), at<uint32_t>(ws, w.ring_flags), a16_cur, a16_next,
                static_cast<float*>(s->A), static_cast<float*>(s->m), static_cast<float*>(s->v), o->optimizer, t,
                o->lr, o->beta1, o->beta2, o->eps, status, st));
        } else {
            void* h16 = at<char>(ws, w.h16);
            SOS_CHECK(launch_build_h16(p, resid, h16, status, st));
            auto adj = use_cta_pairs() ? launch_tc_adjoint_update_pair : launch_tc_adjoint_update;
            SOS_CHECK(adj(p, h16, a16_cur, a16_next, static_cast<float*>(s->A), static_cast<float*>(s->m),
                          static_cast<float*>(s->v), o->optimizer, t, o->lr, o->beta1, o->beta2, o->eps, status,
                          st));
        }
        s->flags = SOS_STATE_BF16_CURRENT | (cur ? 0 : SOS_STATE_BF16_INDEX);
        s->t = t;
        return SOS_OK;
    }
    if (prec == SOS_FP64_TC) {
        const int slices = o->slices == 0 ? kMaxSlices : o->slices;
        float* g32 = at<float>(ws, w.grad);
        SOS_CHECK(pass_tc64(p, static_cast<const double*>(s->A), static_cast<const double*>(pv), g32, loss, ws, st,
                            slices));
        SOS_CHECK(launch_update_mixed(p->N, p->r, static_cast<double*>(s->A), static_cast<float*>(s->m),
                                      static_cast<float*>(s->v), g32, o->optimizer, t, o->lr, o->beta1, o->beta2,
                                      o->eps, st));
        s->flags = 0;
        s->t = t;
        return SOS_OK;
    }
    void* grad = at<char>(ws, w.grad);
    SOS_CHECK(loss_grad(p, prec, s->A, pv, grad, loss, ws, st,
                        prec == SOS_FP64 && (o->flags & SOS_STEP_FP32_ADJOINT)));
    if (prec == SOS_FP64)
        SOS_CHECK(launch_update<double>(p->N, p->r, static_cast<double*>(s->A), static_cast<double*>(s->m),
                                        static_cast<double*>(s->v), static_cast<const double*>(grad), o->optimizer,
                                        t, o->lr, o->beta1, o->beta2, o->eps, nullptr, 0, st));
    else
        SOS_CHECK(launch_update<float>(p->N, p->r, static_cast<float*>(s->A), static_cast<float*>(s->m),
                                       static_cast<float*>(s->v), static_cast<const float*>(grad), o->optimizer, t,
                                       o->lr, o->beta1, o->beta2, o->eps, nullptr, 0, st));
    s->flags = 0;
    s->t = t;
    return SOS_OK;
}

int sos_convert(const void* x, int x_prec, void* y, int y_prec, int64_t count, void* stream) {
    if (!x || !y || count < 0 || (x_prec != SOS_FP32 && x_prec != SOS_FP64) ||
        (y_prec != SOS_FP32 && y_prec != SOS_FP64))
        return fail(SOS_E_INVALID, "sos_convert: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (count == 0) return SOS_OK;
    if (x_prec == y_prec) {
        SOS_CUDA(cudaMemcpyAsync(y, x, (size_t)count * (x_prec == SOS_FP64 ? 8 : 4), cudaMemcpyDeviceToDevice, st));
        return SOS_OK;
    }
    if (x_prec == SOS_FP64) return launch_convert<double, float>(static_cast<const double*>(x), static_cast<float*>(y), count, st);
    return launch_convert<float, double>(static_cast<const float*>(x), static_cast<double*>(y), count, st);
}

int sos_read_status(sos_plan_t p, int prec, void* ws, void* stream) {
    if (!p || bad_prec(prec) || !ws) return fail(SOS_E_INVALID, "sos_read_status: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t word = 0;
    SOS_CUDA(cudaMemcpyAsync(&word, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SOS_CUDA(cudaStreamSynchronize(st));
    if (word != 0) {
        SOS_CUDA(cudaMemsetAsync(ws, 0, sizeof(int32_t), st));
        return fail(word, word == SOS_E_NONFINITE ? "non-finite value in c, p or the residual"
                                                  : "a bounded device wait timed out");
    }
    return SOS_OK;
}

int sos_certify(sos_plan_t p, const void* A, int a_is_double, const double* pv, double tol_rel, double* rel_out,
                int* verdict_out, void* ws_unused, void* stream) {
    TraceRange trace_("sos_certify");
    (void)ws_unused;
    if (!p || !A || !pv || !rel_out || !verdict_out) return fail(SOS_E_INVALID, "sos_certify: bad argument");
    SOS_CHECK(ensure_device(p));
    cudaStream_t st = (cudaStream_t)stream;
    // private FP64 scratch: c (M), partials, loss, status
    const size_t c_bytes = ((size_t)p->M * sizeof(double) + 255) / 256 * 256;
    const size_t extra = 2 * kResidBlocks * sizeof(double) + 2 * sizeof(double) + 64 * sizeof(int32_t);
    char* scratch = nullptr;
    SOS_CUDA(cudaMalloc(&scratch, c_bytes + extra));
    double* c = reinterpret_cast<double*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + c_bytes);
    double* loss = partials + 2 * kResidBlocks;
    int32_t* status = reinterpret_cast<int32_t*>(loss + 2);
    int rc = SOS_OK;
    cudaError_t e = cudaMemsetAsync(scratch, 0, c_bytes + extra, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "sos_certify: memset");
    if (rc == SOS_OK)
        rc = a_is_double ? launch_simt_forward<double, double>(p, static_cast<const double*>(A), c, 1, st)
                         : launch_simt_forward<float, double>(p, static_cast<const float*>(A), c, 1, st);
    if (rc == SOS_OK) rc = launch_residual<double>(p, c, pv, nullptr, loss, partials, status, 1, st);
    double host[2] = {0, 0};
    int32_t word = 0;
    if (rc == SOS_OK) {
        e = cudaMemcpyAsync(host, loss, sizeof(host), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&word, status, sizeof(word), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "sos_certify: read back");
    }
    cudaFree(scratch);
    if (rc != SOS_OK) return rc;
    if (word != 0) {
        *verdict_out = SOS_VERDICT_ERROR;
        *rel_out = NAN;
        return fail(word, "sos_certify: non-finite value");
    }
    const double pn = std::sqrt(host[1]);
    *rel_out = pn > 0 ? std::sqrt(2.0 * host[0]) / pn : std::sqrt(2.0 * host[0]);
    *verdict_out = (*rel_out <= tol_rel) ? SOS_VERDICT_SOS : SOS_VERDICT_NOT_CONVERGED;
    return SOS_OK;
}

}  // extern "C"
