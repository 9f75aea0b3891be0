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

// One block per row: the row's largest magnitude, then its digits, computed on
// the integer pipes from the bits of each double (FP64 arithmetic is slow on
// this GPU): |x| = m 2^q with m the 53-bit significand, X = floor(|x| 2^(52 - e))
// by a right shift of m, and digit i = bits 52 - 5 (i + 1) .. 52 - 5 i - 1 of X,
// with the sign of x.  Also writes the bf16 copy of A that the adjoint reads.
__global__ void __launch_bounds__(kThreads) split_rows_kernel(const double* __restrict__ A, int64_t N, int64_t r,
                                                              int slices, __nv_bfloat16* __restrict__ S,
                                                              int64_t slice_stride, int64_t ld16,
                                                              int32_t* __restrict__ ex,
                                                              __nv_bfloat16* __restrict__ a16) {
    __shared__ unsigned long long red[kThreads / 32];
    const int64_t a = blockIdx.x;
    if (a >= N) return;
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(A + a * r);
    const unsigned long long kAbs = 0x7fffffffffffffffull;
    unsigned long long mx = 0;      // largest |x| by its bits (monotone for non-negative doubles)
    for (int64_t k = threadIdx.x; k < r; k += kThreads) mx = max(mx, row[k] & kAbs);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        mx = threadIdx.x < kThreads / 32 ? red[threadIdx.x] : 0ull;
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (threadIdx.x == 0) red[0] = mx;
    }
    __syncthreads();
    const double mxd = __longlong_as_double((long long)red[0]);
    int e = 0;
    if (mxd > 0.0 && isfinite(mxd)) frexp(mxd, &e);     // mxd = f 2^e, f in [0.5, 1)
    if (threadIdx.x == 0) ex[a] = e;
    for (int64_t k = threadIdx.x; k < r; k += kThreads) {
        const unsigned long long bits = row[k];
        const int biased = (int)((bits >> 52) & 0x7ff);
        const unsigned long long frac = bits & 0xfffffffffffffull;
        // |x| = sig 2^(q), q = biased - 1075 (normal) or -1074 (subnormal)
        const unsigned long long sig = biased ? (frac | (1ull << 52)) : frac;
        const int q = biased ? biased - 1075 : -1074;
        // X = sig 2^(q + 52 - e) < 2^52; for normal x, |x| < 2^e gives a right shift of at least 1
        const int rshift = e - 52 - q;
        const unsigned long long X = rshift >= 64 ? 0ull : rshift >= 0 ? (sig >> rshift) : (sig << (-rshift));
        const bool neg = (bits >> 63) != 0;
        const bool nonfinite = biased == 0x7ff;            // carried into the products as NaN
        for (int i = 0; i < slices; ++i) {
            const int d = (int)((X >> (52 - kSliceBits * (i + 1))) & 31ull);
            const float f = nonfinite ? __int_as_float(0x7fc00000) : (float)(neg ? -d : d);
            S[i * slice_stride + a * ld16 + k] = __float2bfloat16_rn(f);   // exact for |d| <= 31
        }
        a16[a * ld16 + k] = __float2bfloat16_rn((float)__longlong_as_double((long long)bits));
    }
}

// FP64 iterate, FP32 gradient and FP32 moments: only the final subtraction (and
// its conversion) runs on the FP64 pipe.
__global__ void update_mixed_kernel(int64_t count, double* __restrict__ A, float* __restrict__ m,
                                    float* __restrict__ v, const float* __restrict__ g, int optimizer, float lr,
                                    float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        float step;
        if (optimizer == SOS_GD) {
            step = lr * gi;
        } else {
            const float mi = b1 * m[i] + (1.0f - b1) * gi;
            const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        }
        A[i] -= (double)step;
    }
}

int grid_for(int64_t count) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((count + kThreads - 1) / kThreads, 152 * 16));
}

// Tile lists of the slice products, in one of two forms.
//  * Grouped (k = floor((2^24 - 1) / (31^2 r)) >= 2): for each order o the
//    products (i, o - i) are packed into symmetric groups of at most
//    min(k, kMaxGroupSeg) segments -- the diagonal (o/2, o/2) as one segment,
//    each cross pair as two -- and every group covers the upper triangle: tiles
//    (g * TP + I, J), J >= I.
//  * Per pair (k = 1, r > 8729): the diagonal pairs cover the upper triangle
//    and the cross pairs every tile, in stacked coordinates (i * TP + I,
//    j * TP + J).
// Either way the entries are ordered by o, so the products with o < s are the
// first slice_tile_count[s] entries; rows are walked in bands of 8 row blocks.
int ensure_slice_tiles(sos_plan_s* p) {
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->dev.slice_tiles2) return SOS_OK;
    const int TP = (int)ceil_div(p->N, 256), band = 8;
    const int64_t kexact = (((int64_t)1 << 24) - 1) / (31 * 31 * p->r);
    const bool grouped = kexact >= 2;
    const int kseg = (int)std::min<int64_t>(kexact, kMaxGroupSeg);
    std::vector<int2> t;
    std::vector<SliceGroup> groups;
    int count[kMaxSlices + 1] = {0};
    int u = 0;
    auto upper = [&](int xoff, int yoff) {
        for (int i0 = 0; i0 < TP; i0 += band) {
            const int i1 = std::min(TP, i0 + band);
            for (int J = i0; J < TP; ++J)
                for (int I = i0; I < i1; ++I)
                    if (J >= I) t.push_back(make_int2(xoff + I, yoff + J));
        }
    };
    for (int o = 0; o < kMaxSlices; ++o) {
        if (grouped) {
            SliceGroup g{};
            g.order = o;
            auto flush = [&]() {
                if (g.nseg == 0) return;
                upper((int)groups.size() * TP, 0);
                groups.push_back(g);
                g = SliceGroup{};
                g.order = o;
            };
            for (int i = o / 2; i >= 0; --i) {            // the diagonal first, when o is even
                const int j = o - i;
                const int need = i == j ? 1 : 2;
                if (g.nseg + need > kseg) flush();
                g.sa[g.nseg] = i;
                g.sb[g.nseg] = j;
                ++g.nseg;
                if (i != j) {
                    g.sa[g.nseg] = j;
                    g.sb[g.nseg] = i;
                    ++g.nseg;
                }
            }
            flush();
        } else {
            for (int i = 0; 2 * i <= o; ++i) {
                const int j = o - i;
                p->dev.slice_pair_offset[u++] = (int)t.size();
                for (int i0 = 0; i0 < TP; i0 += band) {
                    const int i1 = std::min(TP, i0 + band);
                    for (int J = (i == j ? i0 : 0); J < TP; ++J)
                        for (int I = i0; I < i1; ++I)
                            if (i != j || J >= I) t.push_back(make_int2(i * TP + I, j * TP + J));
                }
            }
        }
        count[o + 1] = (int)t.size();
    }
    p->dev.slice_pair_offset[u] = (int)t.size();
    p->dev.slice_pairs = u;
    int2* d = nullptr;
    SliceGroup* dg = nullptr;
    cudaError_t e = cudaMalloc(&d, t.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(d, t.data(), t.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && grouped) e = cudaMalloc(&dg, groups.size() * sizeof(SliceGroup));
    if (e == cudaSuccess && grouped)
        e = cudaMemcpy(dg, groups.data(), groups.size() * sizeof(SliceGroup), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        cudaFree(dg);
        return cuda_fail(e, "SOS_FP64_TC: tile list");
    }
    p->dev.slice_tiles2 = d;
    p->dev.slice_groups = dg;
    p->dev.slice_grouped = grouped;
    for (int s = 0; s <= kMaxSlices; ++s) p->dev.slice_tile_count[s] = count[s];
    return SOS_OK;
}

}  // namespace

int launch_update_mixed(int64_t N, int64_t r, double* A, float* m, float* v, const float* grad, int optimizer,
                        int64_t t, double lr, double b1, double b2, double eps, cudaStream_t st) {
    const double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
    {
        KernelScope ks_("update", st);
        update_mixed_kernel<<<grid_for(N * r), kThreads, 0, st>>>(N * r, A, m, v, grad, optimizer, (float)lr,
                                                                  (float)b1, (float)b2, (float)eps, (float)c1,
                                                                  (float)c2);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

int forward_tc64(sos_plan_s* p, const double* A, void* ws, double* c, int slices, cudaStream_t st) {
    // the slices, the row exponents and the bf16 copy of A all come from one pass over A
    if (!use_cta_pairs()) return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC needs the CTA-pair kernels (SOS_CTA_PAIRS=1)");
    if (slices < 2 || slices > kMaxSlices) return fail(SOS_E_INVALID, "SOS_FP64_TC: slices must be 2..8");
    if (p->r * 31 * 31 >= (int64_t)1 << 24)
        return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC: r too large for exact slice products (r <= 17458)");
    const int64_t NP = round_up(p->N, 256);
    if ((int64_t)kMaxSlices * NP > INT32_MAX / 2) return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC: N too large");
    SOS_CHECK(ensure_slice_tiles(p));
    const Workspace w = workspace_layout(p, SOS_FP64_TC);
    char* base = static_cast<char*>(ws);
    __nv_bfloat16* S = reinterpret_cast<__nv_bfloat16*>(base + w.slices);
    int32_t* ex = reinterpret_cast<int32_t*>(base + w.ex);
    int32_t* status = reinterpret_cast<int32_t*>(base + w.status);
    SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(double), st));
    {
        KernelScope ks_("split_rows", st);
        split_rows_kernel<<<(unsigned)p->N, kThreads, 0, st>>>(A, p->N, p->r, slices, S, NP * p->ld16, p->ld16, ex,
                                                               reinterpret_cast<__nv_bfloat16*>(base + w.a16));
    }
    SOS_CUDA(cudaGetLastError());
    if (p->dev.slice_grouped)
        return launch_tc_slice_groups_pair(p, S, NP, p->dev.slice_tiles2, p->dev.slice_tile_count[slices],
                                           p->dev.slice_groups, ex, c, status, st);
    // Every pair with i + j < slices.  Small plans run them all in one
    // persistent launch (a pair alone would leave most of its last wave of
    // CTA pairs idle); when one pair alone fills at least 8 waves, one launch
    // per pair runs faster (measured at N = 10,626: 0.93 against 0.84 of the
    // tensor peak).
    const int64_t TP = ceil_div(p->N, 256);
    const int64_t waves = TP * TP / std::max(1, p->dev.num_sms / 2);
    const int total = p->dev.slice_tile_count[slices];
    if (waves < 8)
        return launch_tc_slices_pair(p, S, NP, p->dev.slice_tiles2, total, ex, c, status, st);
    for (int u = 0; u < p->dev.slice_pairs && p->dev.slice_pair_offset[u] < total; ++u) {
        const int off = p->dev.slice_pair_offset[u];
        SOS_CHECK(launch_tc_slices_pair(p, S, NP, p->dev.slice_tiles2 + off, p->dev.slice_pair_offset[u + 1] - off,
                                        ex, c, status, st));
    }
    return SOS_OK;
}

}  // namespace sos
