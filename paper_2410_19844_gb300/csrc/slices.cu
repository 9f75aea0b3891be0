// SOS_FP64_TC: the forward c(A) to FP64 accuracy on tensor cores, by error-free
// slicing of the matrix product (Ozaki, Ogita, Oishi, Rump: "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Row a of A is scaled by 2^-e_a with e_a the exponent of its largest entry
// (|A[a][k]| 2^-e_a < 1) and cut into 5-bit digits:
//     A[a][k] = 2^e_a sum_{i >= 0} d_i[a][k] 2^(-5 (i + 1)),   |d_i| <= 31,
// each digit an integer held exactly in bf16.  Then
//     G[a][b] = sum_k A[a][k] A[b][k]
//             = sum_{i, j} 2^(e_a + e_b - 5 (i + j + 2)) sum_k d_i[a][k] d_j[b][k],
// and the inner sums are integers below r 31^2 < 2^24, so the tensor core's
// FP32 accumulator holds them exactly whatever its rounding.  Keeping the
// terms with i + j < s (s slices) leaves, per term A[a][k] A[b][k], at most
// s 2^(-5 s) 2^(e_a + e_b) from the dropped products and 2 2^(-5 s) 2^(e_a + e_b)
// from the truncated tails of the two rows.  Unit (i, i) is a symmetric product: the upper-triangle
// tiles with weights 1 / 2, as in the BF16 forward.  Units (i, j) and (j, i),
// i < j, add up to twice the full product over every ordered (a, b).  Each
// unit's epilogue scales its exact integers by powers of two and adds them to
// the FP64 coefficients.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace sos {
namespace {

constexpr int kThreads = 256;

// One block per row: the row's largest magnitude, then its digits.
__global__ void __launch_bounds__(kThreads) split_rows_kernel(const double* __restrict__ A, int64_t N, int64_t r,
                                                              int slices, __nv_bfloat16* __restrict__ S,
                                                              int64_t slice_stride, int64_t ld16,
                                                              int32_t* __restrict__ ex) {
    __shared__ double red[kThreads / 32];
    const int64_t a = blockIdx.x;
    if (a >= N) return;
    const double* row = A + a * r;
    double mx = 0.0;
    for (int64_t k = threadIdx.x; k < r; k += kThreads) mx = fmax(mx, fabs(row[k]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) red[0] = mx;
    }
    __syncthreads();
    mx = red[0];
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);      // mx = f 2^e, f in [0.5, 1)
    if (threadIdx.x == 0) ex[a] = e;
    const double scale = ldexp(1.0, -e);
    for (int64_t k = threadIdx.x; k < r; k += kThreads) {
        double x = row[k] * scale;                        // |x| < 1, exact
        for (int i = 0; i < slices; ++i) {
            x *= 32.0;                                    // exact
            const double d = trunc(x);
            x -= d;                                       // exact
            S[i * slice_stride + a * ld16 + k] = __double2bfloat16(d);   // |d| <= 31: exact
        }
    }
}

__global__ void cast_bf16_from_double_kernel(const double* __restrict__ A, int64_t N, int64_t r,
                                             __nv_bfloat16* __restrict__ a16, int64_t ld16) {
    const int64_t total = N * r;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / r, col = i - row * r;
        a16[row * ld16 + col] = __float2bfloat16_rn((float)A[i]);
    }
}

__global__ void update_mixed_kernel(int64_t count, double* __restrict__ A, double* __restrict__ m,
                                    double* __restrict__ v, const float* __restrict__ g, int optimizer, double lr,
                                    double b1, double b2, double eps, double c1, double c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double gi = (double)g[i];
        double a = A[i];
        if (optimizer == SOS_GD) {
            a -= lr * gi;
        } else {
            const double mi = b1 * m[i] + (1.0 - b1) * gi;
            const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            a -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
        }
        A[i] = a;
    }
}

int grid_for(int64_t count) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((count + kThreads - 1) / kThreads, 152 * 16));
}

// Every 256 x 256 tile of N x N, in bands of 8 row blocks (rows fastest in a band).
int ensure_full_tiles(sos_plan_s* p) {
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->dev.full_tiles2) return SOS_OK;
    const int TP = (int)ceil_div(p->N, 256), band = 8;
    std::vector<int2> t;
    for (int i0 = 0; i0 < TP; i0 += band) {
        const int i1 = std::min(TP, i0 + band);
        for (int J = 0; J < TP; ++J)
            for (int I = i0; I < i1; ++I) t.push_back(make_int2(I, J));
    }
    int2* d = nullptr;
    cudaError_t e = cudaMalloc(&d, t.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(d, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "SOS_FP64_TC: tile list");
    }
    p->dev.full_tiles2 = d;
    p->dev.num_full_tiles2 = (int)t.size();
    return SOS_OK;
}

}  // namespace

int launch_cast_bf16_from_double(const double* A, int64_t N, int64_t r, void* a16, int64_t ld16, cudaStream_t st) {
    {
        KernelScope ks_("cast_bf16", st);
        cast_bf16_from_double_kernel<<<grid_for(N * r), kThreads, 0, st>>>(A, N, r, (__nv_bfloat16*)a16, ld16);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

int launch_update_mixed(int64_t N, int64_t r, double* A, double* m, double* v, const float* grad, int optimizer,
                        int64_t t, double lr, double b1, double b2, double eps, cudaStream_t st) {
    const double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
    {
        KernelScope ks_("update", st);
        update_mixed_kernel<<<grid_for(N * r), kThreads, 0, st>>>(N * r, A, m, v, grad, optimizer, lr, b1, b2, eps,
                                                                  c1, c2);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

int forward_tc64(sos_plan_s* p, const double* A, void* ws, double* c, int slices, cudaStream_t st) {
    if (!use_cta_pairs()) return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC needs the CTA-pair kernels (SOS_CTA_PAIRS=1)");
    if (slices < 2 || slices > kMaxSlices) return fail(SOS_E_INVALID, "SOS_FP64_TC: slices must be 2..8");
    if (p->r * 31 * 31 >= (int64_t)1 << 24)
        return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC: r too large for exact slice products (r <= 17458)");
    if (p->N > INT32_MAX / 2) return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC: N too large");
    SOS_CHECK(ensure_full_tiles(p));
    const Workspace w = workspace_layout(p, SOS_FP64_TC);
    char* base = static_cast<char*>(ws);
    __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(base + w.slices);
    int32_t* ex = reinterpret_cast<int32_t*>(base + w.ex);
    int32_t* status = reinterpret_cast<int32_t*>(base + w.status);
    const int64_t stride = p->N * p->ld16;
    SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(double), st));
    {
        KernelScope ks_("split_rows", st);
        split_rows_kernel<<<(unsigned)p->N, kThreads, 0, st>>>(A, p->N, p->r, slices, S, stride, p->ld16, ex);
    }
    SOS_CUDA(cudaGetLastError());
    // smallest terms first, so the FP64 sums add the large contributions last
    for (int o = slices - 1; o >= 0; --o)          // o = i + j
        for (int i = 0; 2 * i <= o; ++i) {
            const int j = o - i;
            const bool cross = i != j;
            SOS_CHECK(launch_tc_slices_pair(p, S + i * stride, S + j * stride, cross,
                                            cross ? p->dev.full_tiles2 : p->dev.fwd_tiles2,
                                            cross ? p->dev.num_full_tiles2 : p->dev.num_fwd_tiles2, ex,
                                            -kSliceBits * (o + 2), c, status, st));
        }
    return SOS_OK;
}

}  // namespace sos
