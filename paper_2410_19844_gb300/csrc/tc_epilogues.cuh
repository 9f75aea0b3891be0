// Epilogues of the tcgen05 GEMM cores (kernels_tc.cu, kernels_tc2.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"

namespace sos {

// Tensor map of a bf16 matrix (kernels_tc.cu).
int make_bf16_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                  uint32_t box_inner, uint32_t box_outer);
// Tensor map of a uint8 matrix (kernels_tc.cu): inner and ld in bytes.
int make_u8_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_inner,
                uint32_t box_outer);
int diag_gemm_pair(int b_mn_major, const void* X, const void* Y, float* D, int64_t m, int64_t n, int64_t k,
                   int64_t ldx, int64_t ldy, const int2* tiles, int num_tiles, int32_t* status, cudaStream_t st);

namespace tc {

// ---- epilogues ---------------------------------------------------------------
//
// The epilogue warps read the accumulator 32 x 32 at a time: warp q (= warp % 4)
// owns rows 32q .. 32q+31 of the 128-row tile, and each tcgen05.ld gives lane i
// row 32q+i, 32 consecutive columns.  The block is transposed through shared
// memory so that an epilogue works with lane j = column j and walks the 32
// rows: every global load and store of a row segment is then one coalesced
// 128-byte access.
//
// The 32 x 32 float block is stored unpadded, row i, column j at
// stage_idx(i, j) = 32 i + (j XOR stage_swz(i)), where stage_swz moves the two
// low bits of i to bits 3-4 and its three high bits to bits 0-2 (a permutation
// of 0..31).  Each of the three access patterns then reaches 32 distinct banks:
//   * the row write after tcgen05.ld (lane = row i, fixed column j): bank
//     j ^ swz(i), distinct because swz is a permutation;
//   * a row read (fixed row i, lane = column j): bank j ^ swz(i);
//   * the forward's 4 x 8 patch read (lane = 8 dr + dc at row 4u + dr, column
//     8v + dc): bits 0-2 of the bank are dc ^ u and bits 3-4 are v ^ dr.

constexpr int STAGE_FLOATS = 32 * 32;

__device__ __forceinline__ int stage_swz(int i) { return ((i & 3) << 3) | ((i >> 2) & 7); }
__device__ __forceinline__ int stage_idx(int i, int j) { return i * 32 + (j ^ stage_swz(i)); }

// Forward: c[idx(a, b)] += w G_ab for b >= a (w = 1 on the diagonal, 2 above).
// With diag given, G_aa comes from diag[a] (a CUDA-core sum of the bf16
// squares, rounded to nearest) instead of the accumulator.
// The warp walks the 32 x 32 block in 4 x 8 patches (lane = 8 dr + dc: row
// 4 (t / 4) + dr, column 8 (t % 4) + dc at step t): entries (a, b) and
// (a + 1, b - 1) often share the monomial a + b, so a compact patch's 32
// atomics touch about half the 32-byte sectors of c that one row's do.  All
// 32 index loads are issued before the first atomic, so they overlap.
struct SegmentSumEpilogue {
    static constexpr const char* kName = "tc_forward";
    static constexpr bool kSegmented = false;
    int N;
    const int32_t* idx;
    int64_t ld_idx;
    float* c;
    const float* diag = nullptr;

    __device__ __forceinline__ void operator()(int a0, int b0, const float* stage, int lane) const {
        if (a0 >= N || b0 >= N || b0 + 31 < a0) return;
        const int dr = lane >> 3, dc = lane & 7;
        int32_t g[32];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int a = a0 + 4 * (t >> 2) + dr, b = b0 + 8 * (t & 3) + dc;
            g[t] = (a < N && b < N && a <= b) ? __ldg(idx + (int64_t)a * ld_idx + b) : -1;
        }
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            if (g[t] >= 0) {
                const int i = 4 * (t >> 2) + dr, j = 8 * (t & 3) + dc;
                const bool on_diag = a0 + i == b0 + j;
                const float v = (diag != nullptr && on_diag) ? __ldg(diag + a0 + i) : stage[stage_idx(i, j)];
                atomicAdd(c + g[t], on_diag ? v : 2.0f * v);
            }
        }
    }
};

// 2^e as a double (e in the normal range; outside it falls back to ldexp).
__device__ __forceinline__ double pow2_int(int e) {
    if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(1023 + e) << 52);
    return ldexp(1.0, e);
}

// Forward of SOS_FP64_TC.  The slices of A are stacked (slice i in rows
// i * NP .. i * NP + N - 1, NP a multiple of 256), so one launch runs every
// slice pair: a tile at stacked rows (i * NP + a, j * NP + b) is the product of
// slices i and j.  acc is that product, exact in FP32 (every partial sum is an
// integer below 2^24); scaled by 2^(ex[a] + ex[b] - bits (i + j + 2)) it is an
// exact FP64 value, summed into the FP64 coefficients.  Diagonal pairs (i = j)
// cover the upper triangle with weights 1 (a = b) and 2 (a < b); cross pairs
// (i < j) cover every ordered (a, b) with weight 2, which also counts (j, i).
struct SliceSumEpilogue {
    static constexpr const char* kName = "tc_slices";
    static constexpr const char* kF8Name = "tc_slices_e4m3";
    static constexpr bool kSegmented = false;
    int N, NP;
    const int32_t* idx;
    int64_t ld_idx;
    double* c;
    const int32_t* ex;
    int bits = 5;         // bits per slice: 5 (bf16 slices) or 4 (E4M3 slices)

    __device__ __forceinline__ void operator()(int a0, int b0, const float* stage, int lane) const {
        const int si = a0 / NP, sj = b0 / NP;
        const int al = a0 - si * NP, bl = b0 - sj * NP;
        if (al >= N || bl >= N) return;
        const bool full = si != sj;
        if (!full && bl + 31 < al) return;
        const int b = bl + lane;
        if (b >= N) return;
        const int eb = ex[b] - bits * (si + sj + 2);
        const int32_t* col = idx + (int64_t)al * ld_idx + b;
        int32_t g[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int a = al + i;
            g[i] = (a < N && (full || a <= b)) ? __ldg(col + (int64_t)i * ld_idx) : -1;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (g[i] >= 0) {
                const double v = (double)stage[stage_idx(i, lane)] * pow2_int(ex[al + i] + eb);
                atomicAdd(c + g[i], (full || al + i != b) ? 2.0 * v : v);
            }
        }
    }
};

// SOS_FP64_TC for plans with r 31^2 k < 2^24, k >= 2: a group sums k slice
// products of one order o = i + j in a single accumulator (the sum of k exact
// integers below 2^24 / k is still exact).  The tile's K runs over the group's
// segments one after another -- segment s multiplies slice sa[s] (rows) with
// slice sb[s] (columns), both from the stacked slices -- and every group is
// symmetric: a diagonal product (i, i), or a cross product as the two segments
// (i, j) and (j, i).  So each group needs only the upper triangle, with weights
// 1 (a = b) and 2 (a < b), and one FP64 atomic per output element for all its
// products.  Tiles are (g * TP + I, J), g the group.
struct SliceGroupEpilogue {
    static constexpr const char* kName = "tc_slices";
    static constexpr const char* kF8Name = "tc_slices_e4m3";
    static constexpr bool kSegmented = true;
    int N, NP, TP;
    const int32_t* idx;
    int64_t ld_idx;
    double* c;
    const int32_t* ex;
    const SliceGroup* groups;
    int bits = 5;         // bits per slice: 5 (bf16 slices) or 4 (E4M3 slices)

    __device__ __forceinline__ int segments(int2 tile) const { return groups[tile.x / TP].nseg; }
    // first stacked row of the pair tile in the segment's A and B operands
    __device__ __forceinline__ int seg_arow(int2 tile, int seg) const {
        const int g = tile.x / TP;
        return groups[g].sa[seg] * NP + (tile.x - g * TP) * 256;
    }
    __device__ __forceinline__ int seg_brow(int2 tile, int seg) const {
        return groups[tile.x / TP].sb[seg] * NP + tile.y * 256;
    }

    __device__ __forceinline__ void operator()(int a0, int b0, const float* stage, int lane) const {
        const int g = a0 / NP;
        const int al = a0 - g * NP;
        if (al >= N || b0 >= N || b0 + 31 < al) return;
        const int b = b0 + lane;
        if (b >= N) return;
        const int eb = ex[b] - bits * (groups[g].order + 2);
        const int32_t* col = idx + (int64_t)al * ld_idx + b;
        int32_t gi[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int a = al + i;
            gi[i] = (a < N && a <= b) ? __ldg(col + (int64_t)i * ld_idx) : -1;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            if (gi[i] >= 0) {
                const double v = (double)stage[stage_idx(i, lane)] * pow2_int(ex[al + i] + eb);
                atomicAdd(c + gi[i], al + i != b ? 2.0 * v : v);
            }
        }
    }
};

// Adjoint / diagnostic GEMM: out[row][col] = scale * acc.
struct StoreEpilogue {
    static constexpr const char* kName = "tc_adjoint";
    static constexpr const char* kRingName = "tc_adjoint_ring";
    static constexpr bool kSegmented = false;
    int rows, cols;
    int64_t ld;
    float scale;
    float* out;

    __device__ __forceinline__ void operator()(int a0, int k0, const float* stage, int lane) const {
        const int k = k0 + lane;
        if (a0 >= rows || k >= cols) return;
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const int a = a0 + i;
            if (a >= rows) break;
            out[(int64_t)a * ld + k] = scale * stage[stage_idx(i, lane)];
        }
    }
};

struct DiagEpilogue : StoreEpilogue {
    static constexpr const char* kName = "tc_gemm_diag";
};

// Adjoint with the optimiser step fused in: grad = 2 acc, then gradient
// descent or Adam on the FP32 master A (and m, v), and the bf16 copy of the
// updated A written to the other buffer of the ping-pong pair (the current one
// is still being read as an operand by other tiles).
struct UpdateEpilogue {
    static constexpr const char* kName = "tc_adjoint_update";
    static constexpr const char* kRingName = "tc_adjoint_update_ring";
    static constexpr bool kSegmented = false;
    int rows, cols, optimizer;
    float lr, b1, b2, eps, c1, c2;
    float* A;
    float* m;
    float* v;
    __nv_bfloat16* a16_next;
    int64_t ld16;

    // Processes the 32 rows in two halves; each half issues all its global
    // loads before using any of them.
    __device__ __forceinline__ void operator()(int a0, int k0, const float* stage, int lane) const {
        const int k = k0 + lane;
        if (a0 >= rows || k >= cols) return;
        const float one = 1.0f;
        const int nrows = rows - a0 < 32 ? rows - a0 : 32;
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            float x[16], mm[16], vv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int64_t e = (int64_t)(a0 + h + i) * cols + k;
                const bool ok = h + i < nrows;
                x[i] = ok ? A[e] : 0.0f;
                if (optimizer != SOS_GD) {
                    mm[i] = ok ? m[e] : 0.0f;
                    vv[i] = ok ? v[e] : 0.0f;
                }
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (h + i >= nrows) break;
                const int64_t e = (int64_t)(a0 + h + i) * cols + k;
                const float g = 2.0f * stage[stage_idx(h + i, lane)];
                float xi = x[i];
                if (optimizer == SOS_GD) {
                    xi -= lr * g;
                } else {
                    const float mi = b1 * mm[i] + (one - b1) * g;
                    const float vi = b2 * vv[i] + (one - b2) * g * g;
                    m[e] = mi;
                    v[e] = vi;
                    const float mhat = mi / c1;
                    const float vhat = vi / c2;
                    xi -= lr * mhat / (sqrtf(vhat) + eps);
                }
                A[e] = xi;
                a16_next[(int64_t)(a0 + h + i) * ld16 + k] = __float2bfloat16_rn(xi);
            }
        }
    }
};

}  // namespace tc
}  // namespace sos
