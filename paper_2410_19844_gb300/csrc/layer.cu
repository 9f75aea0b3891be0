// The paper's network with its first layer (Sec. 2, Sec. 2.1): the quartic form
// ||B Z A1 x||^2 in nf = n + 1 variables.
//
// A1 (m x nf) is the linear first layer, v = A1 x; Z multiplies v by every x_i,
// giving the nf*m entries x_i v_j (index i*m + j); B (k x nf*m) forms k outputs.
// Output k is therefore the quadratic form x^T M_k A1 x with M_k[i][j] =
// B[k][i*m + j], i.e. B read as a stack of nf x m blocks.  Writing P_k = M_k A1
// (nf x nf), the form is sum_k (x^T P_k x)^2, whose coefficient matrix over the
// degree-2 monomials x_i x_j (i <= j) has entries
//     A_hat[(i, j)][k] = P_k[i][j] + P_k[j][i]  (i < j),   P_k[i][i]  (i = j).
// The plan's degree-<=4 basis in n = nf - 1 variables is the form dehomogenised
// (x_nf = 1), so A_hat is the plan's N x k coefficient matrix and the loss and
// its gradient with respect to A_hat are the core pass.  The gradient comes
// back through the expansion by the chain rule:
//     dL/dP_k[i][j] = dL/dA_hat[(min, max)(i, j)][k]      (the symmetric S_k)
//     dL/dB (as the stack of M_k) = S A1^T,   dL/dA1 = sum_k M_k^T S_k,
// three plain GEMMs with B viewed as a (k nf) x m matrix.  They are small next
// to the core pass (k nf^2 m against k N^2 multiply-adds).  In FP32 and FP64
// they run on CUDA cores.  In BF16 steps with nf and m of 64 or more, the two
// with k nf output rows -- P = B A1 and dL/dB = S A1^T -- run on the tensor
// cores from bf16 copies of B, A1 and S (CTA pairs, FP32 accumulation), like
// the core contractions; the long reduction dL/dA1 stays on CUDA cores (split
// over K).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "tc_epilogues.cuh"

namespace sos {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 8;

// C = A B with A(i, l) = A[i * as0 + l * as1] and B(l, j) = B[l * bs0 + j * bs1];
// grid (ceil(Ncol / 128), ceil(M / 128), splits).  Split z covers l in
// [z * kchunk, (z + 1) * kchunk) and writes its own M x Ncol block of C (at
// C + z * split_stride), summed afterwards by split_sum_kernel in a fixed order.
// 256 threads, 8 x 8 outputs each (rows ty + 16 u, columns tx + 16 v): 64
// multiply-adds per 16 shared-memory loads.  The next K-slice is read from
// global memory into registers while the current one is multiplied.
template <typename T>
__global__ void __launch_bounds__(256) strided_gemm_kernel(int64_t M, int64_t Ncol, int64_t K, int64_t kchunk,
                                                           const T* __restrict__ A, int64_t as0, int64_t as1,
                                                           const T* __restrict__ B, int64_t bs0, int64_t bs1,
                                                           T* __restrict__ C, int64_t ldc, int64_t split_stride) {
    __shared__ T As[kBK][kBM + 1];
    __shared__ T Bs[kBK][kBN + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t i0 = (int64_t)blockIdx.y * kBM, j0 = (int64_t)blockIdx.x * kBN;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    // staging map: element q = threadIdx.x + 256 e (e < 4) of each 128 x 8 slice,
    // walking the operand's contiguous dimension fastest
    T ra[4], rb[4];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = threadIdx.x + 256 * e;
            int ii, kk;
            if (as1 == 1) {
                ii = q / kBK;
                kk = q % kBK;
            } else {
                kk = q / kBM;
                ii = q % kBM;
            }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            ra[e] = (gi < M && gk < kend) ? A[gi * as0 + gk * as1] : T(0);
            int jj;
            if (bs1 == 1) {
                kk = q / kBN;
                jj = q % kBN;
            } else {
                jj = q / kBK;
                kk = q % kBK;
            }
            const int64_t gj = j0 + jj, gk2 = k0 + kk;
            rb[e] = (gj < Ncol && gk2 < kend) ? B[gk2 * bs0 + gj * bs1] : T(0);
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = threadIdx.x + 256 * e;
            if (as1 == 1)
                As[q % kBK][q / kBK] = ra[e];
            else
                As[q / kBM][q % kBM] = ra[e];
            if (bs1 == 1)
                Bs[q / kBN][q % kBN] = rb[e];
            else
                Bs[q % kBK][q / kBK] = rb[e];
        }
    };
    T acc[8][8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = T(0);
    if (kbeg < kend) fetch(kbeg);
    for (int64_t k0 = kbeg; k0 < kend; k0 += kBK) {
        stash();
        __syncthreads();
        if (k0 + kBK < kend) fetch(k0 + kBK);     // in flight during the products below
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            T a[8], b[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < 8; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
    T* Cz = C + (int64_t)blockIdx.z * split_stride;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + ty + 16 * u;
        if (i >= M) continue;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int64_t j = j0 + tx + 16 * v;
            if (j < Ncol) Cz[i * ldc + j] = acc[u][v];
        }
    }
}

// C[i][j] = sum over z = 0, 1, ... of part[z][i][j], in that order.
template <typename T>
__global__ void split_sum_kernel(const T* __restrict__ part, int splits, int64_t M, int64_t Ncol,
                                 T* __restrict__ C, int64_t ldc) {
    const int64_t count = M * Ncol;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int z = 0; z < splits; ++z) s += part[(int64_t)z * count + e];
        C[(e / Ncol) * ldc + e % Ncol] = s;
    }
}

constexpr int kTT = 32;   // tile edge of the expand and scatter transposes (blocks of 32 x 8 threads)

// A_hat[a][kk] = P_kk[i][j] + P_kk[j][i] (i < j) or P_kk[i][i], (i, j) = pairs[a].
// A block takes 32 monomials a by 32 outputs kk through shared memory, so that
// the reads walk a (consecutive pairs are mostly consecutive j in one row of
// P_kk) and the writes walk kk along a row of A_hat.  Grid (ceil(N / 32),
// ceil(k / 32)).
template <typename T>
__global__ void __launch_bounds__(256) form_expand_kernel(const T* __restrict__ P, const int2* __restrict__ pairs,
                                                          int64_t N, int64_t k, int nf, T* __restrict__ Ahat) {
    __shared__ T tile[kTT][kTT + 1];
    const int64_t a0 = (int64_t)blockIdx.x * kTT, kk0 = (int64_t)blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t nf2 = (int64_t)nf * nf, a = a0 + tx;
    const int2 ij = a < N ? pairs[a] : make_int2(0, 0);
#pragma unroll
    for (int r = 0; r < kTT; r += 8) {
        const int64_t kk = kk0 + ty + r;
        T v = T(0);
        if (a < N && kk < k) {
            const T* Pk = P + kk * nf2;
            v = Pk[ij.x * nf + ij.y];
            if (ij.x != ij.y) v += Pk[ij.y * nf + ij.x];
        }
        tile[ty + r][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kTT; r += 8) {
        const int64_t row = a0 + ty + r, kk = kk0 + tx;
        if (row < N && kk < k) Ahat[row * k + kk] = tile[tx][ty + r];
    }
}

// S_kk[i][j] = G[rows[i][j]][kk] for every (i, j): the gradient with respect to
// P_kk, symmetric because x_i x_j and x_j x_i are one monomial.  When S16 is
// not NULL the same values also go to S16 in bf16, row kk * nf + i of stride
// ld (the tensor-core operand).  A block takes 32 entries ij by 32 outputs kk
// through shared memory: the reads walk kk along a row of G, the writes walk
// ij.  Grid (ceil(nf^2 / 32), ceil(k / 32)).
template <typename T>
__global__ void __launch_bounds__(256) form_scatter_kernel(const T* __restrict__ G, const int32_t* __restrict__ rows,
                                                           int64_t k, int nf, T* __restrict__ S,
                                                           __nv_bfloat16* __restrict__ S16, int64_t ld) {
    __shared__ T tile[kTT][kTT + 1];
    const int64_t nf2 = (int64_t)nf * nf;
    const int64_t ij0 = (int64_t)blockIdx.x * kTT, kk0 = (int64_t)blockIdx.y * kTT;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < kTT; r += 8) {
        const int64_t ij = ij0 + ty + r, kk = kk0 + tx;
        tile[ty + r][tx] = (ij < nf2 && kk < k) ? G[(int64_t)rows[ij] * k + kk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kTT; r += 8) {
        const int64_t kk = kk0 + ty + r, ij = ij0 + tx;
        if (ij < nf2 && kk < k) {
            const T v = tile[tx][ty + r];
            S[kk * nf2 + ij] = v;
            if (S16) {
                const int64_t i = ij / nf, j = ij - i * nf;
                S16[(kk * nf + i) * ld + j] = __float2bfloat16_rn((float)v);
            }
        }
    }
}

// bf16 copy of a rows x cols float matrix into rows of ld (ld >= cols).
__global__ void cast_rows_bf16_kernel(const float* __restrict__ x, int64_t rows, int64_t cols,
                                      __nv_bfloat16* __restrict__ y, int64_t ld) {
    const int64_t count = rows * cols;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, j = e - i * cols;
        y[i * ld + j] = __float2bfloat16_rn(x[e]);
    }
}

// The 256 x 256 output tiles (i, j) of a TI x TJ grid, row by row.
__global__ void tile_grid_kernel(int TI, int TJ, int2* __restrict__ tiles) {
    const int count = TI * TJ;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
        tiles[e] = make_int2(e / TJ, e % TJ);
}

int grid_for(int64_t count) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 16));
}

// Split count for a GEMM whose output has `tiles` tiles and depth K: enough
// blocks for two waves on 152 SMs, each split at least a few K-slices deep.
int split_count(int64_t tiles, int64_t K) {
    const int64_t want = std::max<int64_t>(1, 304 / std::max<int64_t>(1, tiles));
    const int64_t most = std::max<int64_t>(1, K / (4 * kBK));
    return (int)std::min<int64_t>(std::min<int64_t>(want, most), 1024);
}

struct LayerLayout {
    size_t core = 0;    // the plan's workspace for prec, at offset 0
    size_t P = 0;       // k x nf x nf: P_k, then S_k
    size_t Ahat = 0;    // N x k
    size_t gAhat = 0;   // N x k
    size_t gB = 0;      // k x nf*m
    size_t gA1 = 0;     // m x nf
    size_t part = 0;    // split partial sums of dL/dA1
    // BF16 steps on CTA pairs: bf16 operands of the two tensor-core GEMMs and their tile lists
    size_t B16 = 0, A116 = 0, S16 = 0, tilesP = 0, tilesG = 0;
    int64_t ldm = 0, ldnf = 0;
    int ntP = 0, ntG = 0;
    bool tc = false;
    size_t total = 0;
    int splits = 1;
    int64_t kchunk = 0;
};

LayerLayout layer_layout(const sos_plan_s* p, int prec, int m) {
    LayerLayout w;
    const size_t elt = prec == SOS_FP64 ? 8 : 4;
    const int64_t nf = p->n + 1, k = p->r;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t a = off;
        off += (bytes + 255) / 256 * 256;
        return a;
    };
    w.core = take(workspace_layout(p, prec).total);
    w.P = take((size_t)k * nf * nf * elt);
    w.Ahat = take((size_t)p->N * k * elt);
    w.gAhat = take((size_t)p->N * k * elt);
    w.gB = take((size_t)k * nf * m * elt);
    w.gA1 = take((size_t)m * nf * elt);
    const int64_t K = k * nf;
    const int64_t tiles = ((m + kBM - 1) / kBM) * ((nf + kBN - 1) / kBN);
    w.splits = split_count(tiles, K);
    w.kchunk = ((K + w.splits - 1) / w.splits + kBK - 1) / kBK * kBK;
    w.splits = (int)((K + w.kchunk - 1) / w.kchunk);
    w.part = take((size_t)w.splits * m * nf * elt);
    // below 64 form variables or first-layer outputs the 256 x 256 tensor-core
    // tiles are mostly padding and the extra casts cost more than they save
    // (measured: nf = 31 slower by 13%, nf = 101 faster by 8%)
    w.tc = prec == SOS_BF16 && use_cta_pairs() && nf >= 64 && m >= 64;
    if (w.tc) {
        w.ldm = round_up(m, 64);
        w.ldnf = round_up(nf, 64);
        w.B16 = take((size_t)K * w.ldm * 2);
        w.A116 = take((size_t)m * w.ldnf * 2);
        w.S16 = take((size_t)K * w.ldnf * 2);
        const int64_t TI = ceil_div(K, 256);
        w.ntP = (int)(TI * ceil_div(nf, 256));
        w.ntG = (int)(TI * ceil_div(m, 256));
        w.tilesP = take((size_t)w.ntP * sizeof(int2));
        w.tilesG = take((size_t)w.ntG * sizeof(int2));
    }
    w.total = off;
    return w;
}

template <typename T>
T* at(void* ws, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int check_layer(sos_plan_s* p, int prec, int m, const char* who) {
    if (!p || prec < SOS_BF16 || prec > SOS_FP64) return fail(SOS_E_INVALID, std::string(who) + ": bad plan or precision");
    if (p->two_d != 4)
        return fail(SOS_E_INVALID, std::string(who) + ": the first layer produces quartics; the plan needs two_d = 4");
    if (m < 1 || m > 65536) return fail(SOS_E_INVALID, std::string(who) + ": need 1 <= m <= 65536");
    return SOS_OK;
}

// Row of x_i x_j (0 <= i, j < nf) in the plan's degree-<=2 table.
int ensure_form_tables(sos_plan_s* p) {
    SOS_CHECK(ensure_device(p));
    std::lock_guard<std::mutex> lock(p->mu);
    if (p->dev.form_rows) return SOS_OK;
    const int n = p->n, nf = n + 1;
    std::vector<int32_t> rows((size_t)nf * nf, -1);
    std::vector<int2> pairs((size_t)p->N);
    for (int64_t a = 0; a < p->N; ++a) {
        const uint8_t* e = &p->Ed[(size_t)a * n];
        int v[2], c = 0, deg = 0;
        for (int j = 0; j < n; ++j)
            for (int t = 0; t < e[j]; ++t) v[c++] = j;
        deg = c;
        for (; c < 2; ++c) v[c] = n;          // the dehomogenised variable x_nf = 1
        if (deg > 2) return fail(SOS_E_INVALID, "first layer: plan rows of degree > 2");
        rows[(size_t)v[0] * nf + v[1]] = (int32_t)a;
        rows[(size_t)v[1] * nf + v[0]] = (int32_t)a;
        pairs[a] = make_int2(v[0], v[1]);
    }
    for (int32_t r : rows)
        if (r < 0) return fail(SOS_E_INVALID, "first layer: plan rows do not cover the degree-2 forms");
    int32_t* d_rows = nullptr;
    int2* d_pairs = nullptr;
    cudaError_t e = cudaMalloc(&d_rows, rows.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_pairs, pairs.size() * sizeof(int2));
    if (e == cudaSuccess) e = cudaMemcpy(d_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_rows);
        cudaFree(d_pairs);
        return cuda_fail(e, "first layer: tables");
    }
    p->dev.form_rows = d_rows;
    p->dev.form_pairs = d_pairs;
    return SOS_OK;
}

template <typename T>
int launch_gemm(int64_t M, int64_t Ncol, int64_t K, int64_t kchunk, int splits, const T* A, int64_t as0, int64_t as1,
                const T* B, int64_t bs0, int64_t bs1, T* C, int64_t ldc, int64_t split_stride, cudaStream_t st) {
    if ((M + kBM - 1) / kBM > 65535 || (Ncol + kBN - 1) / kBN > 65535)
        return fail(SOS_E_UNSUPPORTED, "first layer: k (n + 1) or m too large for one GEMM grid");
    dim3 grid((unsigned)((Ncol + kBN - 1) / kBN), (unsigned)((M + kBM - 1) / kBM), (unsigned)splits);
    KernelScope ks_("layer_gemm", st);
    strided_gemm_kernel<T><<<grid, 256, 0, st>>>(M, Ncol, K, kchunk, A, as0, as1, B, bs0, bs1, C, ldc, split_stride);
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

// P_k = M_k A1 for every k, then A_hat.
template <typename T>
int expand(sos_plan_s* p, int m, const T* B, const T* A1, T* Ahat, const LayerLayout& w, void* ws, cudaStream_t st,
           bool b16_current = false) {
    const int64_t nf = p->n + 1, k = p->r;
    T* P = at<T>(ws, w.P);
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (w.tc) {   // BF16 step: bf16 copies of B and A1, then (k nf) x m times m x nf on tensor cores
            auto* B16 = at<__nv_bfloat16>(ws, w.B16);
            auto* A116 = at<__nv_bfloat16>(ws, w.A116);
            int2* tiles = at<int2>(ws, w.tilesP);
            {
                KernelScope ks_("layer_cast", st);
                if (!b16_current)   // else the previous step's update left the bf16 copy of B
                    cast_rows_bf16_kernel<<<grid_for(k * nf * m), 256, 0, st>>>(B, k * nf, m, B16, w.ldm);
                cast_rows_bf16_kernel<<<grid_for((int64_t)m * nf), 256, 0, st>>>(A1, m, nf, A116, w.ldnf);
                tile_grid_kernel<<<grid_for(w.ntP), 256, 0, st>>>((int)ceil_div(k * nf, 256), (int)ceil_div(nf, 256),
                                                                 tiles);
            }
            SOS_CUDA(cudaGetLastError());
            int32_t* status = at<int32_t>(ws, w.core + workspace_layout(p, SOS_BF16).status);
            SOS_CHECK(diag_gemm_pair(1, B16, A116, P, k * nf, nf, m, w.ldm, w.ldnf, tiles, w.ntP, status, st));
            done = true;
        }
    }
    if (!done)   // (k nf) x m times m x nf
        SOS_CHECK(launch_gemm<T>(k * nf, nf, m, m, 1, B, m, 1, A1, nf, 1, P, nf, 0, st));
    {
        KernelScope ks_("layer_expand", st);
        if (ceil_div(k, kTT) > 65535) return fail(SOS_E_UNSUPPORTED, "first layer: k too large for the expand grid");
        const dim3 grid((unsigned)ceil_div(p->N, kTT), (unsigned)ceil_div(k, kTT));
        form_expand_kernel<T><<<grid, dim3(kTT, 8), 0, st>>>(P, p->dev.form_pairs, p->N, k, (int)nf, Ahat);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

// dL/dB and dL/dA1 from dL/dA_hat (either output may be NULL).
template <typename T>
int pull_back(sos_plan_s* p, int m, const T* B, const T* A1, const T* gAhat, T* gB, T* gA1, const LayerLayout& w,
              void* ws, cudaStream_t st) {
    const int64_t nf = p->n + 1, k = p->r;
    T* S = at<T>(ws, w.P);
    // BF16 steps take dL/dB on the tensor cores from a bf16 copy of S, written by the same scatter
    const bool tc_gB = std::is_same<T, float>::value && w.tc && gB;
    {
        KernelScope ks_("layer_scatter", st);
        if (ceil_div(k, kTT) > 65535) return fail(SOS_E_UNSUPPORTED, "first layer: k too large for the scatter grid");
        const dim3 grid((unsigned)ceil_div(nf * nf, kTT), (unsigned)ceil_div(k, kTT));
        form_scatter_kernel<T><<<grid, dim3(kTT, 8), 0, st>>>(gAhat, p->dev.form_rows, k, (int)nf, S,
                                                              tc_gB ? at<__nv_bfloat16>(ws, w.S16) : nullptr, w.ldnf);
    }
    SOS_CUDA(cudaGetLastError());
    bool gb_done = false;
    if constexpr (std::is_same<T, float>::value) {
        if (tc_gB) {   // (k nf) x nf times (m x nf)^T on tensor cores
            auto* S16 = at<__nv_bfloat16>(ws, w.S16);
            auto* A116 = at<__nv_bfloat16>(ws, w.A116);   // cast by expand() in this pass
            int2* tiles = at<int2>(ws, w.tilesG);
            {
                KernelScope ks_("layer_scatter", st);
                tile_grid_kernel<<<grid_for(w.ntG), 256, 0, st>>>((int)ceil_div(k * nf, 256), (int)ceil_div(m, 256),
                                                                 tiles);
            }
            SOS_CUDA(cudaGetLastError());
            int32_t* status = at<int32_t>(ws, w.core + workspace_layout(p, SOS_BF16).status);
            SOS_CHECK(diag_gemm_pair(0, S16, A116, gB, k * nf, m, nf, w.ldnf, w.ldnf, tiles, w.ntG, status, st));
            gb_done = true;
        }
    }
    if (gB && !gb_done)   // S (k nf x nf) times A1^T (nf x m)
        SOS_CHECK(launch_gemm<T>(k * nf, m, nf, nf, 1, S, nf, 1, A1, 1, nf, gB, m, 0, st));
    if (gA1) {  // B^T (m x k nf) times S (k nf x nf), split along k nf
        T* part = at<T>(ws, w.part);
        SOS_CHECK(launch_gemm<T>(m, nf, k * nf, w.kchunk, w.splits, B, 1, m, S, nf, 1, part, nf, (int64_t)m * nf, st));
        KernelScope ks_("layer_split_sum", st);
        split_sum_kernel<T><<<grid_for((int64_t)m * nf), 256, 0, st>>>(part, w.splits, m, nf, gA1, nf);
        SOS_CUDA(cudaGetLastError());
    }
    return SOS_OK;
}

template <typename T>
int layer_loss_grad(sos_plan_s* p, int prec, int m, const void* B, const void* A1, const void* pv, void* gB, void* gA1,
                    void* loss, void* ws, cudaStream_t st, bool fp32_contraction, bool b16_current = false) {
    const LayerLayout w = layer_layout(p, prec, m);
    T* Ahat = at<T>(ws, w.Ahat);
    T* gAhat = (gB || gA1) ? at<T>(ws, w.gAhat) : nullptr;
    SOS_CHECK(expand<T>(p, m, static_cast<const T*>(B), static_cast<const T*>(A1), Ahat, w, ws, st, b16_current));
    SOS_CHECK(core_loss_grad(p, prec, Ahat, pv, gAhat, loss, at<char>(ws, w.core), st, fp32_contraction));
    if (gAhat)
        SOS_CHECK(pull_back<T>(p, m, static_cast<const T*>(B), static_cast<const T*>(A1), gAhat, static_cast<T*>(gB),
                               static_cast<T*>(gA1), w, ws, st));
    return SOS_OK;
}

}  // namespace
}  // namespace sos

using namespace sos;

extern "C" {

int sos_layer_workspace_size(sos_plan_t p, int prec, int m, size_t* bytes) {
    SOS_CHECK(check_layer(p, prec, m, "sos_layer_workspace_size"));
    if (!bytes) return fail(SOS_E_INVALID, "sos_layer_workspace_size: NULL output");
    *bytes = layer_layout(p, prec, m).total;
    return SOS_OK;
}

int sos_layer_expand(sos_plan_t p, int prec, int m, const void* B, const void* A1, void* A_hat, void* ws,
                     void* stream) {
    TraceRange trace_("sos_layer_expand");
    SOS_CHECK(check_layer(p, prec, m, "sos_layer_expand"));
    if (!B || !A1 || !A_hat || !ws) return fail(SOS_E_INVALID, "sos_layer_expand: NULL argument");
    SOS_CHECK(ensure_form_tables(p));
    cudaStream_t st = (cudaStream_t)stream;
    const LayerLayout w = layer_layout(p, prec, m);
    if (prec == SOS_FP64)
        return expand<double>(p, m, static_cast<const double*>(B), static_cast<const double*>(A1),
                              static_cast<double*>(A_hat), w, ws, st);
    return expand<float>(p, m, static_cast<const float*>(B), static_cast<const float*>(A1), static_cast<float*>(A_hat),
                         w, ws, st);
}

int sos_layer_loss_grad(sos_plan_t p, int prec, int m, const void* B, const void* A1, const void* pv, void* grad_B,
                        void* grad_A1, void* loss, void* ws, void* stream) {
    TraceRange trace_("sos_layer_loss_grad");
    SOS_CHECK(check_layer(p, prec, m, "sos_layer_loss_grad"));
    if (!B || !A1 || !pv || !ws) return fail(SOS_E_INVALID, "sos_layer_loss_grad: NULL argument");
    SOS_CHECK(ensure_form_tables(p));
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == SOS_FP64) return layer_loss_grad<double>(p, prec, m, B, A1, pv, grad_B, grad_A1, loss, ws, st, false);
    return layer_loss_grad<float>(p, prec, m, B, A1, pv, grad_B, grad_A1, loss, ws, st, false);
}

int sos_layer_step(sos_plan_t p, int prec, int m, sos_layer_state* s, const void* pv, const sos_step_opts* o,
                   void* loss, void* ws, void* stream) {
    TraceRange trace_("sos_layer_step");
    SOS_CHECK(check_layer(p, prec, m, "sos_layer_step"));
    if (!s || !o || !s->B || !s->A1 || !pv || !ws) return fail(SOS_E_INVALID, "sos_layer_step: NULL argument");
    if (o->optimizer != SOS_ADAM && o->optimizer != SOS_GD) return fail(SOS_E_INVALID, "sos_layer_step: bad optimizer");
    const bool fixed = (s->flags & SOS_LAYER_FIXED_A1) != 0;
    if (o->optimizer == SOS_ADAM && (!s->mB || !s->vB || (!fixed && (!s->mA1 || !s->vA1))))
        return fail(SOS_E_INVALID, "sos_layer_step: Adam needs m and v for every trained matrix");
    if (o->flags & ~SOS_STEP_FP32_ADJOINT) return fail(SOS_E_INVALID, "sos_layer_step: unknown flags");
    if (s->flags & ~(SOS_LAYER_FIXED_A1 | SOS_LAYER_BF16_CURRENT))
        return fail(SOS_E_INVALID, "sos_layer_step: unknown state flags");
    SOS_CHECK(ensure_form_tables(p));
    cudaStream_t st = (cudaStream_t)stream;
    const LayerLayout w = layer_layout(p, prec, m);
    const int64_t nf = p->n + 1, k = p->r, t = s->t + 1;
    const bool fp32c = prec == SOS_FP64 && (o->flags & SOS_STEP_FP32_ADJOINT);
    if (prec == SOS_FP64) {
        double* gB = at<double>(ws, w.gB);
        double* gA1 = fixed ? nullptr : at<double>(ws, w.gA1);
        SOS_CHECK(layer_loss_grad<double>(p, prec, m, s->B, s->A1, pv, gB, gA1, loss, ws, st, fp32c));
        SOS_CHECK(launch_update<double>(k, nf * m, static_cast<double*>(s->B), static_cast<double*>(s->mB),
                                        static_cast<double*>(s->vB), gB, o->optimizer, t, o->lr, o->beta1, o->beta2,
                                        o->eps, nullptr, 0, st));
        if (!fixed)
            SOS_CHECK(launch_update<double>(m, nf, static_cast<double*>(s->A1), static_cast<double*>(s->mA1),
                                            static_cast<double*>(s->vA1), gA1, o->optimizer, t, o->lr, o->beta1,
                                            o->beta2, o->eps, nullptr, 0, st));
    } else {
        float* gB = at<float>(ws, w.gB);
        float* gA1 = fixed ? nullptr : at<float>(ws, w.gA1);
        const bool b16 = w.tc != 0;   // BF16 step with the layer's GEMMs on tensor cores
        SOS_CHECK(layer_loss_grad<float>(p, prec, m, s->B, s->A1, pv, gB, gA1, loss, ws, st, false,
                                         b16 && (s->flags & SOS_LAYER_BF16_CURRENT)));
        // B as (k nf) x m, so that the update also writes the next step's bf16 copy in its padded rows
        SOS_CHECK(launch_update<float>(k * nf, m, static_cast<float*>(s->B), static_cast<float*>(s->mB),
                                       static_cast<float*>(s->vB), gB, o->optimizer, t, o->lr, o->beta1, o->beta2,
                                       o->eps, b16 ? at<char>(ws, w.B16) : nullptr, b16 ? w.ldm : 0, st));
        if (!fixed)
            SOS_CHECK(launch_update<float>(m, nf, static_cast<float*>(s->A1), static_cast<float*>(s->mA1),
                                           static_cast<float*>(s->vA1), gA1, o->optimizer, t, o->lr, o->beta1,
                                           o->beta2, o->eps, nullptr, 0, st));
    }
    if (prec == SOS_BF16 && w.tc)
        s->flags |= SOS_LAYER_BF16_CURRENT;
    else
        s->flags &= ~SOS_LAYER_BF16_CURRENT;
    s->t = t;
    return SOS_OK;
}

}  // extern "C"
