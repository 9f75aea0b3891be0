// CUDA-core kernels: plan tables, casts, the FP32/FP64 forward and adjoint,
// the residual/loss reduction and the optimiser update.
//
//   forward   c_g = sum_{a+b=g} w_ab (A A^T)_ab, w = 1 on the diagonal, 2 above
//             (Eq. 1 with B = A A^T; each unordered pair counted once)
//   residual  r = c - p, loss = 1/2 ||r||^2, ||p||^2         (Eq. 2)
//   adjoint   grad = 2 H(r) A, H[a][b] = r[idx(a, b)]        (chain rule of Eq. 2)
//   update    gradient descent or Adam (Sec. 3)
#include <cuda_bf16.h>

#include <cmath>
#include <mutex>
#include <string>

#include "internal.h"

namespace sos {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
    if (status) atomicCAS(status, 0, code);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T x) {
    return isfinite(x);
}

// ---- idx table ----------------------------------------------------------------

__global__ void build_idx_kernel(int n, int W, int64_t N, int64_t ld, const uint8_t* __restrict__ S,
                                 const int32_t* __restrict__ phi, int32_t* __restrict__ idx) {
    extern __shared__ int32_t sphi[];
    for (int i = threadIdx.x; i < n * W; i += blockDim.x) sphi[i] = phi[i];
    __syncthreads();
    for (int64_t a = blockIdx.y; a < N; a += gridDim.y) {
        const uint8_t* Sa = S + a * n;
        for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < ld;
             b += (int64_t)gridDim.x * blockDim.x) {
            int32_t g = 0;
            if (b < N) {
                const uint8_t* Sb = S + b * n;
                for (int j = 0; j < n; ++j) g += sphi[j * W + Sa[j] + Sb[j]];
            }
            idx[a * ld + b] = g;
        }
    }
}

// ---- bf16 copy of A -------------------------------------------------------------

__global__ void cast_bf16_kernel(const float* __restrict__ A, int64_t N, int64_t r,
                                 __nv_bfloat16* __restrict__ a16, int64_t ld) {
    const int64_t total = N * r;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / r, col = i - row * r;
        a16[row * ld + col] = __float2bfloat16_rn(A[i]);
    }
}

// Diagonal of A A^T from the bf16 copy, on CUDA cores: d[a] = sum_k bf16(A)[a][k]^2.
// Each product is exact in FP32 (a bf16 square needs 16 significand bits); the
// sums round to nearest.  One warp per row: each lane takes 16-byte vectors of
// 8 bf16, four vectors in flight per iteration, and keeps 8 partial sums
// (about r / 256 terms each), which it adds in a fixed order before a
// fixed-order shuffle reduction; a row's sum carries at most about
// (r / 256 + 8) 2^-24 of relative error, unbiased.
__device__ __forceinline__ void add_squares8(const uint4& v, float (&part)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(h[q]);
        part[2 * q] = fmaf(f.x, f.x, part[2 * q]);
        part[2 * q + 1] = fmaf(f.y, f.y, part[2 * q + 1]);
    }
}

__global__ void diag_sumsq_kernel(const __nv_bfloat16* __restrict__ a16, int64_t ld16, int64_t N, int64_t r,
                                  float* __restrict__ d) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const __nv_bfloat16* x = a16 + row * ld16;
    const uint4* xv = reinterpret_cast<const uint4*>(x);   // rows are 128-byte aligned (ld16 % 64 == 0)
    const int64_t nvec = r / 8;                             // whole vectors of the row
    float part[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int64_t v = lane;
    for (; v + 96 < nvec; v += 128) {
        const uint4 a = __ldg(xv + v), b = __ldg(xv + v + 32), c = __ldg(xv + v + 64), e = __ldg(xv + v + 96);
        add_squares8(a, part);
        add_squares8(b, part);
        add_squares8(c, part);
        add_squares8(e, part);
    }
    for (; v < nvec; v += 32) add_squares8(__ldg(xv + v), part);
    for (int64_t j = nvec * 8 + lane; j < r; j += 32) {
        const float f = __bfloat162float(x[j]);
        part[j & 7] = fmaf(f, f, part[j & 7]);
    }
    float s = ((part[0] + part[1]) + (part[2] + part[3])) + ((part[4] + part[5]) + (part[6] + part[7]));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) d[row] = s;
}

// ---- forward: upper-triangle tiles of A A^T, segment-summed into c ------------------
// 64 x 64 tile (I, J), J >= I; 256 threads, 4 x 4 outputs each at rows
// ty + 16 i and columns tx + 16 j; K in chunks of 16 staged in shared memory.

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(kThreads)
simt_forward_kernel(const Tin* __restrict__ A, int64_t N, int64_t r, const int32_t* __restrict__ idx,
                    int64_t ld_idx, Tacc* __restrict__ c, int64_t strideA, int64_t strideC) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J < I) return;
    A += (int64_t)blockIdx.z * strideA;
    c += (int64_t)blockIdx.z * strideC;
    __shared__ Tacc As[16][65];   // padded: staged with k fastest across threads
    __shared__ Tacc Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)I * 64, col0 = (int64_t)J * 64;
    Tacc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Tacc(0);
    for (int64_t k0 = 0; k0 < r; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * kThreads, rr = e >> 4, kk = e & 15;
            const int64_t gk = k0 + kk, ga = row0 + rr, gb = col0 + rr;
            As[kk][rr] = (ga < N && gk < r) ? (Tacc)A[ga * r + gk] : Tacc(0);
            Bs[kk][rr] = (gb < N && gk < r) ? (Tacc)A[gb * r + gk] : Tacc(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            Tacc a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = row0 + ty + 16 * i;
        if (a >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t b = col0 + tx + 16 * j;
            if (b < N && b >= a) {
                const Tacc w = (b == a) ? Tacc(1) : Tacc(2);
                atomicAdd(&c[idx[a * ld_idx + b]], w * acc[i][j]);
            }
        }
    }
}

// ---- the same with 128 x 128 tiles, for large plans ----------------------------------
// 256 threads, 8 x 8 outputs each (rows ty + 16 u, columns tx + 16 v), K in
// slices of 8 staged in shared memory (padded against bank conflicts); the next
// slice is read from global memory into registers while the current one is
// multiplied.  64 multiply-adds per 16 shared-memory loads.

template <typename Tin, typename Tacc>
__global__ void __launch_bounds__(kThreads)
simt_forward128_kernel(const Tin* __restrict__ A, int64_t N, int64_t r, const int32_t* __restrict__ idx,
                       int64_t ld_idx, Tacc* __restrict__ c, int64_t strideA, int64_t strideC) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J < I) return;
    A += (int64_t)blockIdx.z * strideA;
    c += (int64_t)blockIdx.z * strideC;
    __shared__ Tacc As[8][129];
    __shared__ Tacc Bs[8][129];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)I * 128, col0 = (int64_t)J * 128;
    Tacc ra[4], rb[4];
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = tid + kThreads * e, rr = q >> 3, kk = q & 7;
            const int64_t gk = k0 + kk, ga = row0 + rr, gb = col0 + rr;
            ra[e] = (ga < N && gk < r) ? (Tacc)A[ga * r + gk] : Tacc(0);
            rb[e] = (gb < N && gk < r) ? (Tacc)A[gb * r + gk] : Tacc(0);
        }
    };
    Tacc acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = Tacc(0);
    fetch(0);
    for (int64_t k0 = 0; k0 < r; k0 += 8) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = tid + kThreads * e;
            As[q & 7][q >> 3] = ra[e];
            Bs[q & 7][q >> 3] = rb[e];
        }
        __syncthreads();
        if (k0 + 8 < r) fetch(k0 + 8);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            Tacc a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t a = row0 + ty + 16 * i;
        if (a >= N) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t b = col0 + tx + 16 * j;
            if (b < N && b >= a) {
                const Tacc w = (b == a) ? Tacc(1) : Tacc(2);
                atomicAdd(&c[idx[a * ld_idx + b]], w * acc[i][j]);
            }
        }
    }
}

// ---- residual and loss ----------------------------------------------------------
// grid.y = instance.  With one block per instance the block reduces alone;
// with several, the last block to finish (ticket counter) sums the per-block
// partials in block order, so the result does not depend on timing.

template <typename T>
__global__ void __launch_bounds__(kThreads)
residual_kernel(const T* __restrict__ c, const T* __restrict__ p, T* __restrict__ resid, int64_t M,
                double* __restrict__ loss, double* __restrict__ partials, int32_t* __restrict__ status,
                int32_t* __restrict__ counter) {
    const int64_t inst = blockIdx.y;
    c += inst * M;
    p += inst * M;
    if (resid) resid += inst * M;
    loss += inst * 2;
    partials += inst * 2 * gridDim.x;
    // Each thread sums its few (about M / (blocks * 256)) terms in T; the block
    // and grid levels add in double.
    // The loop is unrolled four ways so that each thread has eight independent
    // loads in flight.
    T tr_t = T(0), tp_t = T(0);
    int bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < M; i += 4 * stride) {
        T cv[4], pv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            cv[u] = c[i + u * stride];
            pv[u] = p[i + u * stride];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const T e = cv[u] - pv[u];
            if (resid) resid[i + u * stride] = e;
            if (!finite_val(cv[u]) || !finite_val(pv[u]) || !finite_val(e)) bad = 1;
            tr_t += e * e;
            tp_t += pv[u] * pv[u];
        }
    }
    for (; i < M; i += stride) {
        const T cv = c[i], pv = p[i];
        const T e = cv - pv;
        if (resid) resid[i] = e;
        if (!finite_val(cv) || !finite_val(pv) || !finite_val(e)) bad = 1;
        tr_t += e * e;
        tp_t += pv * pv;
    }
    double sr = (double)tr_t, sp = (double)tp_t;
    __shared__ double red_r[kThreads / 32], red_p[kThreads / 32];
    __shared__ int red_bad;
    __shared__ bool is_last;
    if (threadIdx.x == 0) red_bad = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_down_sync(0xffffffffu, sr, o);
        sp += __shfl_down_sync(0xffffffffu, sp, o);
    }
    if (bad) red_bad = 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red_r[warp] = sr;
        red_p[warp] = sp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, tp = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            tr += red_r[w];
            tp += red_p[w];
        }
        if (red_bad) set_status(status, SOS_E_NONFINITE);
        if (gridDim.x == 1) {
            loss[0] = 0.5 * tr;
            loss[1] = tp;
            is_last = false;
        } else {
            partials[2 * blockIdx.x] = tr;
            partials[2 * blockIdx.x + 1] = tp;
            __threadfence();
            const int ticket = atomicAdd(counter + inst, 1);
            is_last = (ticket == (int)gridDim.x - 1);
        }
    }
    __syncthreads();
    if (is_last) {
        // The last block adds the per-block partials: each thread a fixed
        // stride of blocks, then the same warp and block tree as above, so the
        // order never depends on which block finished last.
        __threadfence();
        double tr = 0.0, tp = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            tr += __ldcg(partials + 2 * b);
            tp += __ldcg(partials + 2 * b + 1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            tr += __shfl_down_sync(0xffffffffu, tr, o);
            tp += __shfl_down_sync(0xffffffffu, tp, o);
        }
        __syncthreads();
        if (lane == 0) {
            red_r[warp] = tr;
            red_p[warp] = tp;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sr2 = 0.0, sp2 = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) {
                sr2 += red_r[w];
                sp2 += red_p[w];
            }
            loss[0] = 0.5 * sr2;
            loss[1] = sp2;
            counter[inst] = 0;
        }
    }
}

// ---- adjoint on CUDA cores: grad = 2 H(r) A, H gathered from r in the loader ----------
// Output tile 64 (rows a) x 64 (columns k); the contraction runs over b in
// chunks of 16.  H[a][b] = r[idx[a][b]] is read straight from the residual
// while staging, so H is never stored.

// Tc is the arithmetic type of the contraction: T, or float for FP64 steps
// that take their gradient in FP32 from the FP64 residual and iterate.
template <typename T, typename Tc>
__global__ void __launch_bounds__(kThreads)
simt_adjoint_kernel(const T* __restrict__ A, const T* __restrict__ resid, const int32_t* __restrict__ idx,
                    int64_t ld_idx, int64_t N, int64_t r, T* __restrict__ grad, int64_t strideA,
                    int64_t strideR) {
    A += (int64_t)blockIdx.z * strideA;
    grad += (int64_t)blockIdx.z * strideA;
    resid += (int64_t)blockIdx.z * strideR;
    __shared__ Tc Hs[16][65];     // padded: staged with b fastest across threads
    __shared__ Tc Bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * 64, col0 = (int64_t)blockIdx.x * 64;
    Tc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Tc(0);
    for (int64_t b0 = 0; b0 < N; b0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = tid + l * kThreads;
            {   // H tile: 64 rows a x 16 columns b
                const int rr = e >> 4, kk = e & 15;
                const int64_t a = row0 + rr, b = b0 + kk;
                Hs[kk][rr] = (a < N && b < N) ? (Tc)resid[idx[a * ld_idx + b]] : Tc(0);
            }
            {   // A tile: 16 rows b x 64 columns k
                const int kk = e >> 6, cc = e & 63;
                const int64_t b = b0 + kk, k = col0 + cc;
                Bs[kk][cc] = (b < N && k < r) ? (Tc)A[b * r + k] : Tc(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            Tc a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = Hs[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t a = row0 + ty + 16 * i;
        if (a >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t k = col0 + tx + 16 * j;
            if (k < r) grad[a * r + k] = T(2) * (T)acc[i][j];
        }
    }
}

// 128 x 128 output tiles (rows a, columns k) for large plans; the contraction
// over b in slices of 8, H gathered from the residual while staging.
template <typename T, typename Tc>
__global__ void __launch_bounds__(kThreads)
simt_adjoint128_kernel(const T* __restrict__ A, const T* __restrict__ resid, const int32_t* __restrict__ idx,
                       int64_t ld_idx, int64_t N, int64_t r, T* __restrict__ grad, int64_t strideA,
                       int64_t strideR) {
    A += (int64_t)blockIdx.z * strideA;
    grad += (int64_t)blockIdx.z * strideA;
    resid += (int64_t)blockIdx.z * strideR;
    __shared__ Tc Hs[8][129];
    __shared__ Tc Bs[8][129];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.y * 128, col0 = (int64_t)blockIdx.x * 128;
    Tc rh[4], rb[4];
    auto fetch = [&](int64_t b0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = tid + kThreads * e;
            {   // H: 128 rows a x 8 columns b (b fastest: index rows are contiguous in b)
                const int rr = q >> 3, kk = q & 7;
                const int64_t a = row0 + rr, b = b0 + kk;
                rh[e] = (a < N && b < N) ? (Tc)resid[idx[a * ld_idx + b]] : Tc(0);
            }
            {   // A: 8 rows b x 128 columns k (k fastest)
                const int kk = q >> 7, cc = q & 127;
                const int64_t b = b0 + kk, k = col0 + cc;
                rb[e] = (b < N && k < r) ? (Tc)A[b * r + k] : Tc(0);
            }
        }
    };
    Tc acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = Tc(0);
    fetch(0);
    for (int64_t b0 = 0; b0 < N; b0 += 8) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = tid + kThreads * e;
            Hs[q & 7][q >> 3] = rh[e];
            Bs[q >> 7][q & 127] = rb[e];
        }
        __syncthreads();
        if (b0 + 8 < N) fetch(b0 + 8);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            Tc a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = Hs[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t a = row0 + ty + 16 * i;
        if (a >= N) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t k = col0 + tx + 16 * j;
            if (k < r) grad[a * r + k] = T(2) * (T)acc[i][j];
        }
    }
}

// ---- optimiser update ---------------------------------------------------------------

template <typename T>
__global__ void update_kernel(int64_t N, int64_t r, T* __restrict__ A, T* __restrict__ m,
                              T* __restrict__ v, const T* __restrict__ g, int optimizer, T lr, T b1,
                              T b2, T eps, T c1, T c2, __nv_bfloat16* __restrict__ a16, int64_t ld16) {
    const int64_t total = N * r;
    const T one = T(1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T gi = g[i];
        T a = A[i];
        if (optimizer == SOS_GD) {
            a -= lr * gi;
        } else {
            const T mi = b1 * m[i] + (one - b1) * gi;
            const T vi = b2 * v[i] + (one - b2) * gi * gi;
            m[i] = mi;
            v[i] = vi;
            const T mhat = mi / c1;
            const T vhat = vi / c2;
            a -= lr * mhat / (sqrt(vhat) + eps);
        }
        A[i] = a;
        if (a16) {
            const int64_t row = i / r, col = i - row * r;
            a16[row * ld16 + col] = __float2bfloat16_rn((float)a);
        }
    }
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        y[i] = (Tout)x[i];
}

template <typename T>
__global__ void fill_kernel(T* x, int64_t count, T value) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = value;
}

int grid_for(int64_t work, int cap = 152 * 16) {
    int64_t g = (work + kThreads - 1) / kThreads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------

int launch_build_idx(const sos_plan_s* p, int32_t* idx, const uint8_t* d_S, const int32_t* d_phi,
                     cudaStream_t st) {
    const int W = p->two_d + 1;
    const size_t smem = (size_t)p->n * W * sizeof(int32_t);
    if (smem > 48 * 1024) return fail(SOS_E_UNSUPPORTED, "build_idx: n * (2d+1) too large");
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(p->ld_idx, kThreads), 64),
              (unsigned)std::min<int64_t>(p->N, 65535));
    {
        KernelScope ks_("build_idx", st);
        build_idx_kernel<<<grid, kThreads, smem, st>>>(p->n, W, p->N, p->ld_idx, d_S, d_phi, idx);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

int launch_diag_sumsq(const void* a16, int64_t ld16, int64_t N, int64_t r, float* d, cudaStream_t st) {
    const int64_t blocks = ceil_div(N * 32, kThreads);
    if (blocks > INT32_MAX) return fail(SOS_E_UNSUPPORTED, "diag_sumsq: too many rows");
    {
        KernelScope ks_("diag_sumsq", st);
        diag_sumsq_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(static_cast<const __nv_bfloat16*>(a16), ld16, N, r,
                                                                 d);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

int launch_cast_bf16(const float* A, int64_t N, int64_t r, void* a16, int64_t ld16, cudaStream_t st) {
    {
        KernelScope ks_("cast_bf16", st);
        cast_bf16_kernel<<<grid_for(N * r), kThreads, 0, st>>>(A, N, r, (__nv_bfloat16*)a16, ld16);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

// 128 x 128 tiles once a single problem fills a wave of them on 152 SMs
// (N >= about 2100); 64 x 64 tiles otherwise.
static bool use_simt128(int64_t N, int64_t batch) {
    const int64_t t128 = ceil_div(N, 128);
    return batch == 1 && t128 * (t128 + 1) / 2 >= 152;
}

template <typename Tin, typename Tacc>
int launch_simt_forward(const sos_plan_s* p, const Tin* A, Tacc* c, int64_t batch, cudaStream_t st) {
    if (batch > 65535) return fail(SOS_E_UNSUPPORTED, "simt_forward: batch too large");
    if (use_simt128(p->N, batch)) {
        const int64_t T = ceil_div(p->N, 128);
        if (T > 65535) return fail(SOS_E_UNSUPPORTED, "simt_forward: too many tiles");
        dim3 grid((unsigned)T, (unsigned)T, (unsigned)batch);
        KernelScope ks_("simt_forward", st);
        simt_forward128_kernel<Tin, Tacc><<<grid, kThreads, 0, st>>>(A, p->N, p->r, p->dev.idx, p->ld_idx, c,
                                                                     p->N * p->r, p->M);
    } else {
        const int64_t T = ceil_div(p->N, 64);
        if (T > 65535) return fail(SOS_E_UNSUPPORTED, "simt_forward: too many tiles");
        dim3 grid((unsigned)T, (unsigned)T, (unsigned)batch);
        KernelScope ks_("simt_forward", st);
        simt_forward_kernel<Tin, Tacc><<<grid, kThreads, 0, st>>>(A, p->N, p->r, p->dev.idx, p->ld_idx, c,
                                                                  p->N * p->r, p->M);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template <typename T>
int launch_residual(const sos_plan_s* p, const T* c, const T* pv, T* resid, double* loss,
                    double* partials, int32_t* status, int64_t batch, cudaStream_t st) {
    if (batch > 65535) return fail(SOS_E_UNSUPPORTED, "residual: batch too large");
    int blocks = 1;
    if (batch == 1) blocks = (int)std::min<int64_t>(kResidBlocks, std::max<int64_t>(1, ceil_div(p->M, 4 * kThreads)));
    dim3 grid(blocks, (unsigned)batch);
    {
        KernelScope ks_("residual", st);
        residual_kernel<T><<<grid, kThreads, 0, st>>>(c, pv, resid, p->M, loss, partials, status, status + 1);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template <typename T>
int launch_simt_adjoint(const sos_plan_s* p, const T* A, const T* resid, T* grad, int64_t batch, cudaStream_t st,
                        bool fp32_contraction) {
    if (use_simt128(p->N, batch)) {
        const int64_t TI = ceil_div(p->N, 128), TK = ceil_div(p->r, 128);
        if (TI > 65535 || batch > 65535 || TK > INT32_MAX)
            return fail(SOS_E_UNSUPPORTED, "simt_adjoint: too many tiles");
        dim3 grid((unsigned)TK, (unsigned)TI, (unsigned)batch);
        KernelScope ks_(fp32_contraction ? "simt_adjoint_fp32c" : "simt_adjoint", st);
        if (fp32_contraction)
            simt_adjoint128_kernel<T, float><<<grid, kThreads, 0, st>>>(A, resid, p->dev.idx, p->ld_idx, p->N, p->r,
                                                                        grad, p->N * p->r, p->M);
        else
            simt_adjoint128_kernel<T, T><<<grid, kThreads, 0, st>>>(A, resid, p->dev.idx, p->ld_idx, p->N, p->r,
                                                                    grad, p->N * p->r, p->M);
        SOS_CUDA(cudaGetLastError());
        return SOS_OK;
    }
    const int64_t TI = ceil_div(p->N, 64), TK = ceil_div(p->r, 64);
    if (TI > 65535 || batch > 65535 || TK > INT32_MAX) return fail(SOS_E_UNSUPPORTED, "simt_adjoint: too many tiles");
    dim3 grid((unsigned)TK, (unsigned)TI, (unsigned)batch);
    {
        KernelScope ks_(fp32_contraction ? "simt_adjoint_fp32c" : "simt_adjoint", st);
        if (fp32_contraction)
            simt_adjoint_kernel<T, float><<<grid, kThreads, 0, st>>>(A, resid, p->dev.idx, p->ld_idx, p->N, p->r,
                                                                     grad, p->N * p->r, p->M);
        else
            simt_adjoint_kernel<T, T><<<grid, kThreads, 0, st>>>(A, resid, p->dev.idx, p->ld_idx, p->N, p->r, grad,
                                                                 p->N * p->r, p->M);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template <typename T>
int launch_update(int64_t N, int64_t r, T* A, T* m, T* v, const T* grad, int optimizer, int64_t t,
                  double lr, double b1, double b2, double eps, void* a16, int64_t ld16, cudaStream_t st) {
    const double c1 = 1.0 - std::pow(b1, (double)t);
    const double c2 = 1.0 - std::pow(b2, (double)t);
    {
        KernelScope ks_("update", st);
        update_kernel<T><<<grid_for(N * r), kThreads, 0, st>>>(N, r, A, m, v, grad, optimizer, (T)lr, (T)b1,
                                                               (T)b2, (T)eps, (T)c1, (T)c2,
                                                               (__nv_bfloat16*)a16, ld16);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template <typename T>
int launch_fill(T* x, int64_t count, T value, cudaStream_t st) {
    {
        KernelScope ks_("fill", st);
        fill_kernel<T><<<grid_for(count), kThreads, 0, st>>>(x, count, value);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template <typename Tin, typename Tout>
int launch_convert(const Tin* x, Tout* y, int64_t count, cudaStream_t st) {
    {
        KernelScope ks_("convert", st);
        convert_kernel<Tin, Tout><<<grid_for(count), kThreads, 0, st>>>(x, y, count);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

template int launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template int launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template int launch_simt_forward<float, float>(const sos_plan_s*, const float*, float*, int64_t, cudaStream_t);
template int launch_simt_forward<double, double>(const sos_plan_s*, const double*, double*, int64_t, cudaStream_t);
template int launch_simt_forward<float, double>(const sos_plan_s*, const float*, double*, int64_t, cudaStream_t);
template int launch_residual<float>(const sos_plan_s*, const float*, const float*, float*, double*, double*,
                                    int32_t*, int64_t, cudaStream_t);
template int launch_residual<double>(const sos_plan_s*, const double*, const double*, double*, double*,
                                     double*, int32_t*, int64_t, cudaStream_t);
template int launch_simt_adjoint<float>(const sos_plan_s*, const float*, const float*, float*, int64_t,
                                        cudaStream_t, bool);
template int launch_simt_adjoint<double>(const sos_plan_s*, const double*, const double*, double*, int64_t,
                                         cudaStream_t, bool);
template int launch_update<float>(int64_t, int64_t, float*, float*, float*, const float*, int, int64_t, double,
                                  double, double, double, void*, int64_t, cudaStream_t);
template int launch_update<double>(int64_t, int64_t, double*, double*, double*, const double*, int, int64_t,
                                   double, double, double, double, void*, int64_t, cudaStream_t);
template int launch_fill<float>(float*, int64_t, float, cudaStream_t);
template int launch_fill<double>(double*, int64_t, double, cudaStream_t);

}  // namespace sos

// ---- loss from given coefficients, without any allocation ---------------------------
//
// For callers that cannot allocate device memory at call time (for example a
// host framework that hands a library only the buffers it allocated itself, or
// a loop that runs under a fixed memory budget), this variant of the residual
// and loss reduction keeps its scratch -- the status word, one ticket counter
// per problem and the per-block partial sums -- in a fixed array in the
// library's own device memory instead of a caller workspace.  Every GPU that
// loads the library holds the array (1 MiB) until the process exits.

namespace sos {
namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;
constexpr size_t kStaticHeaderBytes = 4096;   // status word + ticket counters
constexpr int64_t kStaticMaxBatch = (kStaticHeaderBytes - 64) / sizeof(int32_t);
constexpr int64_t kStaticMaxPartials = (kStaticScratchBytes - kStaticHeaderBytes) / (2 * sizeof(double));

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {};

// Host code cannot use g_static_scratch's name as a device address; look the
// address up once per device, with that device current.
int static_scratch(void** out) {
    int dev = -1;
    SOS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(SOS_E_UNSUPPORTED, "static scratch: device index out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return SOS_OK;
}

template <typename T>
int loss_from_coeffs_static(int64_t batch, int64_t M, const T* c, const T* p, T* resid, double* loss,
                            cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(kResidBlocks, std::max<int64_t>(1, ceil_div(M, 4 * kThreads)));
    if (batch > kStaticMaxBatch || batch * blocks > kStaticMaxPartials)
        return fail(SOS_E_INVALID, "sos_loss_from_coeffs_static: batch * blocks exceeds the fixed scratch (at most " +
                                       std::to_string(kStaticMaxBatch) + " problems and " +
                                       std::to_string(kStaticMaxPartials) + " block partials)");
    void* base = nullptr;
    SOS_CHECK(static_scratch(&base));
    int32_t* status = static_cast<int32_t*>(base);
    double* partials = reinterpret_cast<double*>(static_cast<char*>(base) + kStaticHeaderBytes);
    // Ticket counters must start at zero; the array keeps the previous call's contents.
    SOS_CUDA(cudaMemsetAsync(base, 0, kStaticHeaderBytes, st));
    dim3 grid(blocks, (unsigned)batch);
    {
        KernelScope ks_("residual_static", st);
        residual_kernel<T><<<grid, kThreads, 0, st>>>(c, p, resid, M, loss, partials, status, status + 16);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

}  // namespace

}  // namespace sos

extern "C" int sos_loss_from_coeffs_static(int prec, int64_t batch, int64_t M, const void* c, const void* p,
                                           void* resid, double* loss, void* stream) {
    using namespace sos;
    if ((prec != SOS_FP32 && prec != SOS_FP64) || batch < 1 || M < 1 || !c || !p || !loss)
        return fail(SOS_E_INVALID, "sos_loss_from_coeffs_static: FP32 or FP64, batch >= 1, M >= 1, c, p, loss");
    if (batch > 65535) return fail(SOS_E_INVALID, "sos_loss_from_coeffs_static: batch too large");
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == SOS_FP64)
        return loss_from_coeffs_static<double>(batch, M, static_cast<const double*>(c), static_cast<const double*>(p),
                                               static_cast<double*>(resid), loss, st);
    return loss_from_coeffs_static<float>(batch, M, static_cast<const float*>(c), static_cast<const float*>(p),
                                          static_cast<float*>(resid), loss, st);
}

