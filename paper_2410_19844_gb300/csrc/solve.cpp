// sos_solve: the precision ladder around sos_step, and the certificate.
//
// Stages (Sec. 3's optimiser is Adam; its success measure is the minimum
// error over all iterations, which is what is tracked here):
//   1. BF16 contractions (tensor cores, FP32 accumulation) until the relative
//      residual ||c - p|| / ||p|| drops below switch_rel or stops improving;
//   2. FP32 on CUDA cores until it stops improving;
//   3. FP64 on CUDA cores, on an FP64 copy of A, for at most fp64_steps;
// then the FP64 certificate (||c - p|| <= cert_tol ||p||, Sec. 3) of the best
// checked A.  The optimiser state (m, v, t) carries over between stages: a
// fresh Adam state would move every entry by about lr on its first step.
#include <cmath>
#include <vector>

#include "internal.h"

using namespace sos;

namespace {

struct DeviceBuffers {
    std::vector<void*> ptrs;
    ~DeviceBuffers() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename T>
    int alloc(T** out, size_t count) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T) + 256);
        if (e != cudaSuccess) return cuda_fail(e, "sos_solve: allocation");
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return SOS_OK;
    }
};

int read_loss(const double* dev, double* host, cudaStream_t st) {
    SOS_CUDA(cudaMemcpyAsync(host, dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    SOS_CUDA(cudaStreamSynchronize(st));
    return SOS_OK;
}

}  // namespace

extern "C" {

int sos_solve_opts_default(sos_solve_opts* o) {
    if (!o) return fail(SOS_E_INVALID, "sos_solve_opts_default: NULL");
    o->optimizer = SOS_ADAM;
    o->lr_bf16 = 1e-2;
    o->lr_fp32 = 1e-2;
    o->lr_fp64 = 1e-2;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->max_steps = 20000;
    o->check_every = 50;
    o->switch_rel = 1e-3;
    o->stall_checks = 4;
    o->fp64_steps = 2000;
    o->fp64_fp32_adjoint = 1;
    o->cert_tol = 1e-8;
    o->start_prec = SOS_BF16;
    o->tc_fp64 = 1;
    return SOS_OK;
}

int sos_solve(sos_plan_t p, const double* p64, double* A, const sos_solve_opts* o, sos_result* out, void* stream) {
    TraceRange trace_("sos_solve");
    if (!p || !p64 || !A || !o || !out) return fail(SOS_E_INVALID, "sos_solve: NULL argument");
    if (o->start_prec != SOS_BF16 && o->start_prec != SOS_FP32 && o->start_prec != SOS_FP64)
        return fail(SOS_E_INVALID, "sos_solve: bad start_prec");
    if (o->check_every < 1 || o->max_steps < 0 || o->fp64_steps < 0)
        return fail(SOS_E_INVALID, "sos_solve: bad step counts");
    SOS_CHECK(ensure_device(p));
    cudaStream_t st = (cudaStream_t)stream;
    *out = sos_result{};
    out->verdict = SOS_VERDICT_ERROR;
    out->min_rel = INFINITY;
    const size_t NR = (size_t)p->N * (size_t)p->r;
    const size_t M = (size_t)p->M;

    DeviceBuffers mem;
    float *p32 = nullptr, *A32 = nullptr, *m32 = nullptr, *v32 = nullptr, *best32 = nullptr;
    double *loss = nullptr, *A64 = nullptr, *m64 = nullptr, *v64 = nullptr, *best64 = nullptr;
    SOS_CHECK(mem.alloc(&p32, M));
    SOS_CHECK(mem.alloc(&A32, NR));
    SOS_CHECK(mem.alloc(&m32, NR));
    SOS_CHECK(mem.alloc(&v32, NR));
    SOS_CHECK(mem.alloc(&best32, NR));
    SOS_CHECK(mem.alloc(&loss, 2));
    void *ws16 = nullptr, *ws32 = nullptr, *ws64 = nullptr;
    size_t b16 = workspace_layout(p, SOS_BF16).total, b32 = workspace_layout(p, SOS_FP32).total;
    size_t b64 = workspace_layout(p, SOS_FP64).total;
    SOS_CHECK(mem.alloc(reinterpret_cast<char**>(&ws16), b16));
    SOS_CHECK(mem.alloc(reinterpret_cast<char**>(&ws32), b32));
    SOS_CHECK(mem.alloc(reinterpret_cast<char**>(&ws64), b64));
    SOS_CHECK(sos_workspace_init(p, SOS_BF16, ws16, stream));
    SOS_CHECK(sos_workspace_init(p, SOS_FP32, ws32, stream));
    SOS_CHECK(sos_workspace_init(p, SOS_FP64, ws64, stream));
    SOS_CHECK(launch_convert<double, float>(p64, p32, (int64_t)M, st));
    SOS_CHECK(launch_convert<double, float>(A, A32, (int64_t)NR, st));
    SOS_CUDA(cudaMemsetAsync(m32, 0, NR * sizeof(float), st));
    SOS_CUDA(cudaMemsetAsync(v32, 0, NR * sizeof(float), st));
    SOS_CUDA(cudaMemcpyAsync(best32, A32, NR * sizeof(float), cudaMemcpyDeviceToDevice, st));

    // ||p||^2 from an FP64 pass at the start point, which also fills the
    // start point's FP64 relative residual
    double host[2];
    SOS_CHECK(sos_loss_grad(p, SOS_FP64, A, p64, nullptr, loss, ws64, stream));
    SOS_CHECK(read_loss(loss, host, st));
    const double pp = host[1] > 0 ? host[1] : 1.0;
    auto rel_of = [&](double l) { return std::sqrt(2.0 * std::max(l, 0.0) / pp); };
    out->rel_start_fp64 = rel_of(host[0]);

    // the SOS_FP64_TC stage needs exact slice products (r dmax^2 < 2^24) and the
    // CTA-pair kernels; without them the CUDA-core stages run instead
    const bool tc = o->tc_fp64 && slice_format(p).exact_for(p->r) && use_cta_pairs();
    int prec = o->start_prec == SOS_FP64 ? SOS_FP32 : o->start_prec;
    sos_state s{A32, m32, v32, 0, 0, 0};
    double best = INFINITY, last_gain = INFINITY;
    int stall = 0;
    bool have_best64 = false;
    int64_t step = 0;
    const bool run32 = o->start_prec != SOS_FP64;

    // ---- BF16 and FP32 stages on the FP32 master ----
    while (run32 && step < o->max_steps) {
        if (step % o->check_every == 0) {
            void* ws = prec == SOS_BF16 ? ws16 : ws32;
            SOS_CHECK(sos_loss_grad(p, prec, A32, p32, nullptr, loss, ws, stream));
            SOS_CHECK(read_loss(loss, host, st));
            if (!std::isfinite(host[0])) return fail(SOS_E_NONFINITE, "sos_solve: non-finite loss");
            const double rel = rel_of(host[0]);
            if (rel < best) {
                best = rel;
                SOS_CUDA(cudaMemcpyAsync(best32, A32, NR * sizeof(float), cudaMemcpyDeviceToDevice, st));
            }
            if (rel < 0.99 * last_gain) {
                last_gain = rel;
                stall = 0;
            } else {
                ++stall;
            }
            if (prec == SOS_BF16 && (rel < o->switch_rel || stall >= o->stall_checks)) {
                if (tc) {                             // the FP64_TC stage follows instead
                    out->rel_at_switch = rel;
                    out->steps_bf16 = step;
                    prec = SOS_FP64_TC;
                    break;
                }
                nvtxMarkA("sos_solve: BF16 -> FP32");
                out->rel_at_switch = rel;
                out->steps_bf16 = step;
                prec = SOS_FP32;
                s.flags = 0;
                stall = 0;
                last_gain = rel;
                best = INFINITY;          // FP32 losses are not comparable with BF16 ones
                continue;
            }
            if (prec == SOS_FP32 && (stall >= o->stall_checks || rel <= 0.25 * o->cert_tol)) break;
        }
        sos_step_opts so{o->optimizer, prec == SOS_BF16 ? o->lr_bf16 : o->lr_fp32, o->beta1, o->beta2, o->eps, 0};
        SOS_CHECK(sos_step(p, prec, &s, p32, &so, nullptr, prec == SOS_BF16 ? ws16 : ws32, stream));
        ++step;
    }
    if (prec == SOS_BF16) out->steps_bf16 = step;
    out->steps_fp32 = prec == SOS_FP64_TC ? 0 : step - out->steps_bf16;
    out->min_rel = best;
    if (prec == SOS_FP64_TC || (tc && prec == SOS_BF16)) {
        // ---- SOS_FP64_TC stage on an FP64 copy of the best BF16 point ----
        nvtxMarkA("sos_solve: FP64_TC stage");
        // the FP32 moments carry over as they are (SOS_FP64_TC keeps m, v in FP32)
        double *A64t = nullptr, *best64t = nullptr;
        SOS_CHECK(mem.alloc(&A64t, NR));
        SOS_CHECK(mem.alloc(&best64t, NR));
        void* wst = nullptr;
        SOS_CHECK(mem.alloc(reinterpret_cast<char**>(&wst), workspace_layout(p, SOS_FP64_TC).total));
        SOS_CHECK(sos_workspace_init(p, SOS_FP64_TC, wst, stream));
        SOS_CHECK(launch_convert<float, double>(best32, A64t, (int64_t)NR, st));
        sos_state st64{A64t, m32, v32, s.t, 0, 0};
        double best_t = INFINITY, gain = INFINITY;
        int stall_t = 0, slices = kMaxSlices;
        bool have = false;
        for (int64_t k = 0; k <= o->fp64_steps; ++k) {
            if (k % o->check_every == 0 || k == o->fp64_steps) {
                // the loss of the previous step is at most check_every steps old; the
                // check evaluates the current point at full slice accuracy
                SOS_CHECK(sos_loss_grad(p, SOS_FP64_TC, A64t, p64, nullptr, loss, wst, stream));
                SOS_CHECK(read_loss(loss, host, st));
                if (!std::isfinite(host[0])) return fail(SOS_E_NONFINITE, "sos_solve: non-finite FP64_TC loss");
                const double rel = rel_of(host[0]);
                if (rel < best_t) {
                    best_t = rel;
                    have = true;
                    SOS_CUDA(cudaMemcpyAsync(best64t, A64t, NR * sizeof(double), cudaMemcpyDeviceToDevice, st));
                }
                if (rel < 0.99 * gain) {
                    gain = rel;
                    stall_t = 0;
                } else {
                    ++stall_t;
                }
                if (rel <= 0.5 * o->cert_tol || stall_t >= o->stall_checks || k == o->fp64_steps) break;
                // slices for a forward about 2^-10 of the residual
                const double bits = -std::log2(std::max(rel, 1e-300)) + 10.0;
                slices = std::min(kMaxSlices, std::max(3, (int)std::ceil(bits / kSliceBits)));
            }
            sos_step_opts so{o->optimizer, o->lr_fp64, o->beta1, o->beta2, o->eps, 0, slices};
            SOS_CHECK(sos_step(p, SOS_FP64_TC, &st64, p64, &so, nullptr, wst, stream));
            ++out->steps_fp64;
        }
        out->min_rel_fp64 = best_t;
        const double* final_A = have ? best64t : A64t;
        double rel = 0.0;
        int verdict = SOS_VERDICT_ERROR;
        SOS_CHECK(sos_certify(p, final_A, 1, p64, o->cert_tol, &rel, &verdict, nullptr, stream));
        SOS_CUDA(cudaMemcpyAsync(A, final_A, NR * sizeof(double), cudaMemcpyDeviceToDevice, st));
        SOS_CUDA(cudaStreamSynchronize(st));
        out->steps = out->steps_bf16 + out->steps_fp32 + out->steps_fp64;
        out->rel_resid_fp64 = rel;
        out->verdict = verdict;
        return SOS_OK;
    }

    // ---- FP64 stage on an FP64 copy of the best FP32 point ----
    nvtxMarkA("sos_solve: FP64 stage");
    SOS_CHECK(mem.alloc(&A64, NR));
    SOS_CHECK(mem.alloc(&best64, NR));
    if (run32)
        SOS_CHECK(launch_convert<float, double>(best32, A64, (int64_t)NR, st));
    else
        SOS_CUDA(cudaMemcpyAsync(A64, A, NR * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (o->fp64_steps > 0) {
        SOS_CHECK(mem.alloc(&m64, NR));
        SOS_CHECK(mem.alloc(&v64, NR));
        SOS_CHECK(launch_convert<float, double>(m32, m64, (int64_t)NR, st));
        SOS_CHECK(launch_convert<float, double>(v32, v64, (int64_t)NR, st));
        sos_state s64{A64, m64, v64, s.t, 0, 0};
        double best64_rel = INFINITY;
        for (int64_t k = 0; k <= o->fp64_steps; ++k) {
            if (k % o->check_every == 0 || k == o->fp64_steps) {
                SOS_CHECK(sos_loss_grad(p, SOS_FP64, A64, p64, nullptr, loss, ws64, stream));
                SOS_CHECK(read_loss(loss, host, st));
                if (!std::isfinite(host[0])) return fail(SOS_E_NONFINITE, "sos_solve: non-finite FP64 loss");
                const double rel = rel_of(host[0]);
                if (rel < best64_rel) {
                    best64_rel = rel;
                    have_best64 = true;
                    SOS_CUDA(cudaMemcpyAsync(best64, A64, NR * sizeof(double), cudaMemcpyDeviceToDevice, st));
                }
                if (rel <= 0.5 * o->cert_tol || k == o->fp64_steps) break;
            }
            sos_step_opts so{o->optimizer, o->lr_fp64, o->beta1, o->beta2, o->eps,
                             o->fp64_fp32_adjoint ? SOS_STEP_FP32_ADJOINT : 0};
            SOS_CHECK(sos_step(p, SOS_FP64, &s64, p64, &so, nullptr, ws64, stream));
            ++out->steps_fp64;
        }
        out->min_rel_fp64 = best64_rel;
    }
    const double* final_A = have_best64 ? best64 : A64;
    double rel = 0.0;
    int verdict = SOS_VERDICT_ERROR;
    SOS_CHECK(sos_certify(p, final_A, 1, p64, o->cert_tol, &rel, &verdict, nullptr, stream));
    SOS_CUDA(cudaMemcpyAsync(A, final_A, NR * sizeof(double), cudaMemcpyDeviceToDevice, st));
    SOS_CUDA(cudaStreamSynchronize(st));
    out->steps = out->steps_bf16 + out->steps_fp32 + out->steps_fp64;
    out->rel_resid_fp64 = rel;
    out->verdict = verdict;
    return SOS_OK;
}

}  // extern "C"
