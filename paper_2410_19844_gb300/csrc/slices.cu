// SOS_FP64_TC: the forward c(A) to FP64 accuracy on tensor cores, by error-free
// slicing of the matrix product (Ozaki, Ogita, Oishi, Rump: "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Row a of A is scaled by 2^-e_a with e_a the exponent of its largest entry
// (|A[a][k]| 2^-e_a < 1) and cut into b-bit digits:
//     A[a][k] = 2^e_a sum_{i >= 0} d_i[a][k] 2^(-b (i + 1)),   |d_i| <= 2^b - 1,
// each digit an integer held exactly in the slice type: b = 5 in bf16, or
// b = 4 in E4M3 bytes (SOS_SLICE_FP8 = 1), whose products the tensor core runs
// at twice the K per byte of operand.  Then
//     G[a][b] = sum_k A[a][k] A[b][k]
//             = sum_{i, j} 2^(e_a + e_b - b (i + j + 2)) sum_k d_i[a][k] d_j[b][k],
// and the inner sums are integers below r (2^b - 1)^2 < 2^24, so the tensor
// core's FP32 accumulator holds them exactly whatever its rounding.  Keeping
// the terms with i + j < s (s slices) leaves, per term A[a][k] A[b][k], at most
// s 2^(-b s) 2^(e_a + e_b) from the dropped products and 2 2^(-b s) 2^(e_a + e_b)
// from the truncated tails of the two rows.  The API counts slices in 5-bit
// units; E4M3 slicing takes ceil(5 s / 4) of its own, at least as many bits.
// Unit (i, i) is a symmetric product: the upper-triangle tiles with weights
// 1 / 2, as in the BF16 forward.  Units (i, j) and (j, i), i < j, add up to
// twice the full product over every ordered (a, b).  Each unit's epilogue
// scales its exact integers by powers of two and adds them to the FP64
// coefficients.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace sos {
namespace {

constexpr int kThreads = 256;

// Digit codes without conversion instructions (which run at a quarter of the
// integer rate): the float 2^23 + m, 0 <= m < 2^23, holds m in its low
// significand bits, so subtracting 2^23 gives float(m) exactly.  From its bits:
//   * bf16(m) is the upper half (m <= 31 has at most five significant bits);
//   * E4M3(m), m = 2^E (1 + f / 8) with E <= 3 and f three bits (m <= 15 has
//     at most four significant bits), is (E + 7) << 3 | f: the float's
//     exponent field and top three fraction bits, bits 20..30, less
//     (127 - 7) << 3; and 0 for m = 0.
// Signs are or-ed in afterwards; NaN (a non-finite entry) replaces the code.
__device__ __forceinline__ uint32_t float_bits_of_small(uint32_t m) {
    return __float_as_uint(__uint_as_float(0x4b000000u | m) - 8388608.0f);
}

// Slice i of four entries (their 52-bit scaled significands X) as four codes:
// 8 bytes of bf16 or 4 of E4M3, with sign and NaN masks of the same layout.
template <int BITS>
struct DigitCodes;
template <>
struct DigitCodes<5> {
    using Word = uint2;
    static __device__ __forceinline__ Word masks(const bool* flag, uint32_t bit) {
        return make_uint2((flag[0] ? bit : 0u) | (flag[1] ? bit << 16 : 0u),
                          (flag[2] ? bit : 0u) | (flag[3] ? bit << 16 : 0u));
    }
    static __device__ __forceinline__ Word sign_masks(const bool* neg) { return masks(neg, 0x8000u); }
    static __device__ __forceinline__ Word nan_masks(const bool* nf) { return masks(nf, 0xffffu); }
    static __device__ __forceinline__ Word code(const uint32_t* m, Word sign, Word nan) {
        const uint32_t f0 = float_bits_of_small(m[0]), f1 = float_bits_of_small(m[1]);
        const uint32_t f2 = float_bits_of_small(m[2]), f3 = float_bits_of_small(m[3]);
        const uint32_t lo = __byte_perm(f0, f1, 0x7632) | sign.x;   // upper halves of f0, f1
        const uint32_t hi = __byte_perm(f2, f3, 0x7632) | sign.y;
        return make_uint2((lo & ~nan.x) | (0x7fc07fc0u & nan.x), (hi & ~nan.y) | (0x7fc07fc0u & nan.y));
    }
    static __device__ __forceinline__ void put(__nv_bfloat16* dst, Word w, int j) {
        const uint32_t h = ((j < 2 ? w.x : w.y) >> (16 * (j & 1))) & 0xffffu;
        *dst = __ushort_as_bfloat16((unsigned short)h);
    }
};
template <>
struct DigitCodes<4> {
    using Word = uint32_t;
    static __device__ __forceinline__ Word masks(const bool* flag, uint32_t byte) {
        return (flag[0] ? byte : 0u) | (flag[1] ? byte << 8 : 0u) | (flag[2] ? byte << 16 : 0u) |
               (flag[3] ? byte << 24 : 0u);
    }
    static __device__ __forceinline__ Word sign_masks(const bool* neg) { return masks(neg, 0x80u); }
    static __device__ __forceinline__ Word nan_masks(const bool* nf) { return masks(nf, 0xffu); }
    static __device__ __forceinline__ uint32_t one(uint32_t m) {
        return m ? (float_bits_of_small(m) >> 20) - ((127u - 7u) << 3) : 0u;
    }
    static __device__ __forceinline__ Word code(const uint32_t* m, Word sign, Word nan) {
        const uint32_t c = one(m[0]) | (one(m[1]) << 8) | (one(m[2]) << 16) | (one(m[3]) << 24) | sign;
        return (c & ~nan) | (0x7f7f7f7fu & nan);                    // 0x7f: E4M3 NaN
    }
    static __device__ __forceinline__ void put(uint8_t* dst, Word w, int j) { *dst = (uint8_t)(w >> (8 * j)); }
};

// One block per row: the row's largest magnitude, then its digits (BITS bits
// each: 5 in bf16 slices, 4 in E4M3 slices), computed on the integer pipes
// from the bits of each double (FP64 arithmetic is slow on this GPU): |x| =
// m 2^q with m the 53-bit significand, X = floor(|x| 2^(52 - e)) by a right
// shift of m, and digit i = bits 52 - BITS (i + 1) .. 52 - BITS i - 1 of X,
// with the sign of x.  Also writes the bf16 copy of A that the adjoint reads.
// Each thread takes four consecutive entries, so every slice row is written
// in 8- or 4-byte stores (lds and ld16 are multiples of 4 elements).
template <int BITS, int MAXS, class T>
__global__ void __launch_bounds__(kThreads) split_rows_kernel(const double* __restrict__ A, int64_t N, int64_t r,
                                                              int slices, T* __restrict__ S, int64_t slice_stride,
                                                              int64_t lds, int64_t ld16, int32_t* __restrict__ ex,
                                                              __nv_bfloat16* __restrict__ a16) {
    using Codes = DigitCodes<BITS>;
    using Word = typename Codes::Word;
    static_assert(sizeof(Word) == 4 * sizeof(T), "four codes per store");
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
    constexpr unsigned long long kDigit = (1ull << BITS) - 1;
    for (int64_t k0 = 4 * (int64_t)threadIdx.x; k0 < r; k0 += 4 * kThreads) {
        const int cnt = (int)min((int64_t)4, r - k0);
        unsigned long long X[4];
        bool neg[4], nonfinite[4];
        __nv_bfloat16 copy[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned long long bits = j < cnt ? row[k0 + j] : 0ull;
            const int biased = (int)((bits >> 52) & 0x7ff);
            const unsigned long long frac = bits & 0xfffffffffffffull;
            // |x| = sig 2^(q), q = biased - 1075 (normal) or -1074 (subnormal)
            const unsigned long long sig = biased ? (frac | (1ull << 52)) : frac;
            const int q = biased ? biased - 1075 : -1074;
            // X = sig 2^(q + 52 - e) < 2^52; for normal x, |x| < 2^e gives a right shift of at least 1
            const int rshift = e - 52 - q;
            X[j] = rshift >= 64 ? 0ull : rshift >= 0 ? (sig >> rshift) : (sig << (-rshift));
            neg[j] = (bits >> 63) != 0;
            nonfinite[j] = biased == 0x7ff;                // carried into the products as NaN
            copy[j] = __float2bfloat16_rn((float)__longlong_as_double((long long)bits));
        }
        const Word sign = Codes::sign_masks(neg), nan = Codes::nan_masks(nonfinite);
#pragma unroll
        for (int i = 0; i < MAXS; ++i) {
            if (i >= slices) break;
            uint32_t m[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) m[j] = (uint32_t)((X[j] >> (52 - BITS * (i + 1))) & kDigit);
            const Word w = Codes::code(m, sign, nan);
            T* dst = S + i * slice_stride + a * lds + k0;
            if (cnt == 4) {
                *reinterpret_cast<Word*>(dst) = w;
            } else {
                for (int j = 0; j < cnt; ++j) Codes::put(dst + j, w, j);
            }
        }
        __nv_bfloat16* dst16 = a16 + a * ld16 + k0;
        auto u16 = [&](int j) { return (uint32_t)__bfloat16_as_ushort(copy[j]); };
        const uint2 cw = make_uint2(u16(0) | (u16(1) << 16), u16(2) | (u16(3) << 16));
        if (cnt == 4) {
            *reinterpret_cast<uint2*>(dst16) = cw;
        } else {
            for (int j = 0; j < cnt; ++j) DigitCodes<5>::put(dst16 + j, cw, j);
        }
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

// Tile lists of the slice products of format f, in one of two forms.
//  * Grouped (k = floor((2^24 - 1) / (dmax^2 r)) >= 2): for each order o the
//    products (i, o - i) are packed into symmetric groups of at most
//    min(k, kMaxGroupSeg) segments -- the diagonal (o/2, o/2) as one segment,
//    each cross pair as two -- and every group covers the upper triangle: tiles
//    (g * TP + I, J), J >= I.
//  * Per pair (k = 1: r > 8729 for bf16 slices, r > 37282 for E4M3): the
//    diagonal pairs cover the upper triangle
//    and the cross pairs every tile, in stacked coordinates (i * TP + I,
//    j * TP + J).
// Either way the entries are ordered by o, so the products with o < s are the
// first slice_tile_count[s] entries; rows are walked in bands of 8 row blocks.
int ensure_slice_tiles(sos_plan_s* p, const SliceFormat& f) {
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->dev.slice_tiles2) return SOS_OK;
    const int TP = (int)ceil_div(p->N, 256), band = 8;
    const int64_t kexact = (((int64_t)1 << 24) - 1) / ((int64_t)f.dmax * f.dmax * p->r);
    const bool grouped = kexact >= 2;
    const int kseg = (int)std::min<int64_t>(kexact, kMaxGroupSeg);
    std::vector<int2> t;
    std::vector<SliceGroup> groups;
    int count[kMaxSlices8 + 1] = {0};
    int u = 0;
    auto upper = [&](int xoff, int yoff) {
        for (int i0 = 0; i0 < TP; i0 += band) {
            const int i1 = std::min(TP, i0 + band);
            for (int J = i0; J < TP; ++J)
                for (int I = i0; I < i1; ++I)
                    if (J >= I) t.push_back(make_int2(xoff + I, yoff + J));
        }
    };
    for (int o = 0; o < f.max_slices; ++o) {
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
                if (u >= kMaxSlicePairs) return fail(SOS_E_INVALID, "SOS_FP64_TC: too many slice pairs");
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
    for (int s = 0; s <= f.max_slices; ++s) p->dev.slice_tile_count[s] = count[s];
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
    const SliceFormat f = slice_format(p);
    if (!f.exact_for(p->r))
        return fail(SOS_E_UNSUPPORTED, f.fp8 ? "SOS_FP64_TC: r too large for exact E4M3 slice products (r <= 74565)"
                                             : "SOS_FP64_TC: r too large for exact bf16 slice products (r <= 17458; "
                                               "SOS_SLICE_FP8=0 forbids the E4M3 slices that reach 74565)");
    const int sf = f.slices_for(slices);     // slices of this format with the bits of `slices` 5-bit ones
    const int64_t NP = round_up(p->N, 256);
    if ((int64_t)f.max_slices * NP > INT32_MAX / 2) return fail(SOS_E_UNSUPPORTED, "SOS_FP64_TC: N too large");
    SOS_CHECK(ensure_slice_tiles(p, f));
    const Workspace w = workspace_layout(p, SOS_FP64_TC);
    char* base = static_cast<char*>(ws);
    void* S = base + w.slices;
    int32_t* ex = reinterpret_cast<int32_t*>(base + w.ex);
    int32_t* status = reinterpret_cast<int32_t*>(base + w.status);
    __nv_bfloat16* a16 = reinterpret_cast<__nv_bfloat16*>(base + w.a16);
    SOS_CUDA(cudaMemsetAsync(c, 0, (size_t)p->M * sizeof(double), st));
    {
        KernelScope ks_("split_rows", st);
        if (f.fp8)
            split_rows_kernel<4, kMaxSlices8><<<(unsigned)p->N, kThreads, 0, st>>>(
                A, p->N, p->r, sf, static_cast<uint8_t*>(S), NP * f.ld, f.ld, p->ld16, ex, a16);
        else
            split_rows_kernel<kSliceBits, kMaxSlices><<<(unsigned)p->N, kThreads, 0, st>>>(
                A, p->N, p->r, sf, static_cast<__nv_bfloat16*>(S), NP * f.ld, f.ld, p->ld16, ex, a16);
    }
    SOS_CUDA(cudaGetLastError());
    if (p->dev.slice_grouped)
        return launch_tc_slice_groups_pair(p, f, S, NP, p->dev.slice_tiles2, p->dev.slice_tile_count[sf],
                                           p->dev.slice_groups, ex, c, status, st);
    // Every pair with i + j < sf.  Small plans run them all in one persistent
    // launch (a pair alone would leave most of its last wave of CTA pairs
    // idle); when one pair alone fills at least 8 waves, one launch per pair
    // runs faster (measured at N = 10,626 with bf16 slices: 0.93 against 0.84
    // of the tensor peak).
    const int64_t TP = ceil_div(p->N, 256);
    const int64_t waves = TP * TP / std::max(1, p->dev.num_sms / 2);
    const int total = p->dev.slice_tile_count[sf];
    if (waves < 8)
        return launch_tc_slices_pair(p, f, S, NP, p->dev.slice_tiles2, total, ex, c, status, st);
    for (int u = 0; u < p->dev.slice_pairs && p->dev.slice_pair_offset[u] < total; ++u) {
        const int off = p->dev.slice_pair_offset[u];
        SOS_CHECK(launch_tc_slices_pair(p, f, S, NP, p->dev.slice_tiles2 + off,
                                        p->dev.slice_pair_offset[u + 1] - off, ex, c, status, st));
    }
    return SOS_OK;
}

}  // namespace sos
