// Grouped steps over many independent problems (serving).
//
// A group holds up to `capacity` problems, each with its own plan (n, 2d),
// r = N, and its own buffers.  One step of the group runs three kernels whose
// work lists span every active problem, so large and small problems share the
// GPU the way a grouped GEMM shares it:
//   forward   64 x 64 tiles of G = A A^T on or above the diagonal, written
//             to the problem's G (no atomics)                  (Eq. 1)
//   residual  chunks of 512 coefficients: c_g is gathered from G through the
//             plan's pair lists, r = c - p, partial sums of ||r||^2, ||p||^2;
//             one thread also advances the group's step counter, which the
//             forward reads before it and the adjoint (as counter - 1) after it
//   adjoint   64 x 64 tiles of grad = 2 H(r) A with H gathered from r through
//             the index table, fused with the GD / Adam update (Sec. 3); the
//             operand A is read from one buffer of a ping-pong pair and the
//             update written to the other
// Every result is computed by one thread in a fixed order, so a problem's
// iterates do not depend on which other problems share the group.  The work
// lists and counters live in device memory, so the captured graph of K steps
// stays valid while problems join and leave.
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include <type_traits>

#include "internal.h"

namespace sos {
namespace grp {

constexpr int kT = 256;
constexpr int kChunk = 512;

template <typename T>
struct Inst {
    int N, M, r, active;
    int64_t ld_idx;
    const int32_t* idx;
    const int32_t* pair_ptr;
    const int32_t* pair_pos;
    T* A0;
    T* A1;
    T* m;
    T* v;
    const T* p;
    T* G;
    T* resid;
    double* partials;
    long long join;   // group step at which the problem entered this group
    long long t0;     // optimiser steps it had taken before (Adam's bias correction continues)
    double lr;
};

struct Item {
    int inst, i, j, pad;
};

// counts[0..2]: forward, residual, adjoint items; items laid out as three
// arrays of `cap` entries.
//
// The forward and the adjoint run 128 threads per 64 x 64 tile: thread (tx, ty),
// tx = 0..15 and ty = 0..7, owns rows 8 ty .. 8 ty + 7 and columns 4 tx .. 4 tx
// + 3, so each 16-deep step reads 8 + 4 staged values (three 16-byte shared
// loads) for 32 multiply-adds.  The values of the next step (and, for the
// adjoint, the index entries of the step after) are loaded into registers
// while the current step computes.  Every entry of the tile still accumulates
// its products one k at a time in increasing k, as one fused multiply-add each.
constexpr int kT2 = 128;
constexpr int kHP = 68;       // staged row length: 64 + 4 keeps rows 16-byte aligned and spreads the stores

template <typename T>
__global__ void __launch_bounds__(kT2)
group_forward(const int* __restrict__ counts, const Item* __restrict__ items, const Inst<T>* __restrict__ insts,
              const long long* __restrict__ step) {
    __shared__ __align__(16) T As[16][kHP];     // [k][row of the tile]
    __shared__ __align__(16) T Bs[16][kHP];     // [k][column of the tile]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n_items = counts[0];
    const long long now = *step;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const Item it = items[w];
        const Inst<T>& in = insts[it.inst];
        const int N = in.N, r = in.r;
        const T* A = ((now - in.join) & 1) ? in.A1 : in.A0;
        const int row0 = it.i * 64, col0 = it.j * 64;
        T acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
        // staged element l of this thread: k = k0 + (e & 15), tile row or column e >> 4, e = tid + 128 l
        T ra[8], rb[8];
        auto load = [&](int k0) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int e = tid + l * kT2, kk = e & 15, rr = e >> 4;
                const int gk = k0 + kk, ga = row0 + rr, gb = col0 + rr;
                ra[l] = (ga < N && gk < r) ? A[(int64_t)ga * r + gk] : T(0);
                rb[l] = (gb < N && gk < r) ? A[(int64_t)gb * r + gk] : T(0);
            }
        };
        load(0);
        for (int k0 = 0; k0 < r; k0 += 16) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int e = tid + l * kT2, kk = e & 15, rr = e >> 4;
                As[kk][rr] = ra[l];
                Bs[kk][rr] = rb[l];
            }
            __syncthreads();
            if (k0 + 16 < r) load(k0 + 16);
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                T a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = As[kk][8 * ty + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][4 * tx + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int a = row0 + 8 * ty + i;
            if (a >= N) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int b = col0 + 4 * tx + j;
                if (b < N) in.G[(int64_t)a * N + b] = acc[i][j];
            }
        }
    }
}

// FP64 groups with SOS_GROUP_FAST_FP64: the same forward in double-float
// arithmetic on the FP32 pipes (the FP64 pipe is slow on this GPU).  Each entry
// x of A is split into hi = float(x) and lo = float(x - hi) (48 of its 53
// bits).  A product a b is hi_a hi_b, taken exactly as p + e with
// e = fma(hi_a, hi_b, -p), plus the cross terms hi_a lo_b + lo_a hi_b; the sum
// runs as a pair (s, t): s by a two-sum of s and p, whose rounding error goes
// into t with e and the cross terms.  G = s + t in double is accurate to about
// 2^-46 of the sum of |products|.  The explicit _rn intrinsics keep the compiler
// from fusing the error-free steps into other multiply-adds.
__global__ void __launch_bounds__(kT)
group_forward_df(const int* __restrict__ counts, const Item* __restrict__ items,
                 const Inst<double>* __restrict__ insts, const long long* __restrict__ step) {
    __shared__ float Ah[16][65], Al[16][65], Bh[16][65], Bl[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n_items = counts[0];
    const long long now = *step;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const Item it = items[w];
        const Inst<double>& in = insts[it.inst];
        const int N = in.N, r = in.r;
        const double* A = ((now - in.join) & 1) ? in.A1 : in.A0;
        const int row0 = it.i * 64, col0 = it.j * 64;
        float sh[4][4], sl[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) sh[i][j] = sl[i][j] = 0.0f;
        for (int k0 = 0; k0 < r; k0 += 16) {
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int e = tid + l * kT, rr = e >> 4, kk = e & 15;
                const int gk = k0 + kk, ga = row0 + rr, gb = col0 + rr;
                const double xa = (ga < N && gk < r) ? A[(int64_t)ga * r + gk] : 0.0;
                const double xb = (gb < N && gk < r) ? A[(int64_t)gb * r + gk] : 0.0;
                const float ha = __double2float_rn(xa), hb = __double2float_rn(xb);
                Ah[kk][rr] = ha;
                Al[kk][rr] = __double2float_rn(xa - (double)ha);
                Bh[kk][rr] = hb;
                Bl[kk][rr] = __double2float_rn(xb - (double)hb);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < 16; ++kk) {
                float ah[4], al[4], bh[4], bl[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    ah[i] = Ah[kk][ty + 16 * i];
                    al[i] = Al[kk][ty + 16 * i];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    bh[j] = Bh[kk][tx + 16 * j];
                    bl[j] = Bl[kk][tx + 16 * j];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float p = __fmul_rn(ah[i], bh[j]);
                        const float e = __fmaf_rn(ah[i], bh[j], -p);
                        const float q = __fmaf_rn(ah[i], bl[j], __fmaf_rn(al[i], bh[j], e));
                        const float t = __fadd_rn(sh[i][j], p);
                        const float z = __fsub_rn(t, sh[i][j]);
                        const float err = __fadd_rn(__fsub_rn(sh[i][j], __fsub_rn(t, z)), __fsub_rn(p, z));
                        sh[i][j] = t;
                        sl[i][j] = __fadd_rn(sl[i][j], __fadd_rn(err, q));
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int a = row0 + ty + 16 * i;
            if (a >= N) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int b = col0 + tx + 16 * j;
                if (b < N) in.G[(int64_t)a * N + b] = (double)sh[i][j] + (double)sl[i][j];
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kT)
group_residual(const int* __restrict__ counts, const Item* __restrict__ items, int cap,
               const Inst<T>* __restrict__ insts, long long* __restrict__ step) {
    __shared__ double red[2][kT / 32];
    // the forward of this step has read the counter and the adjoint reads it
    // after this kernel: advancing it here saves a launch per step
    if (blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
    const int n_items = counts[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const Item it = items[cap + w];
        const Inst<T>& in = insts[it.inst];
        const int g0 = it.i * kChunk;
        const int g1 = min(in.M, g0 + kChunk);
        T sr = T(0), sp = T(0);
        for (int g = g0 + threadIdx.x; g < g1; g += kT) {
            T c = T(0);
            const int k1 = in.pair_ptr[g + 1];
            for (int k = in.pair_ptr[g]; k < k1; ++k) {
                const int32_t pos = in.pair_pos[k];
                const T v = in.G[pos & INT32_MAX];
                c += pos < 0 ? v : T(2) * v;
            }
            const T pv = in.p[g];
            const T e = c - pv;
            in.resid[g] = e;
            sr += e * e;
            sp += pv * pv;
        }
        double dr = (double)sr, dp = (double)sp;
        for (int o = 16; o > 0; o >>= 1) {
            dr += __shfl_down_sync(0xffffffffu, dr, o);
            dp += __shfl_down_sync(0xffffffffu, dp, o);
        }
        if (lane == 0) {
            red[0][warp] = dr;
            red[1][warp] = dp;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double tr = 0.0, tp = 0.0;
            for (int q = 0; q < kT / 32; ++q) {
                tr += red[0][q];
                tp += red[1][q];
            }
            in.partials[2 * it.i] = tr;
            in.partials[2 * it.i + 1] = tp;
        }
        __syncthreads();
    }
}

// Tc is the type of the contraction (T, or float for an FP64 group that
// takes its gradient from the FP64 residual in FP32 arithmetic); the update
// and the iterate stay in T.  H is gathered from the residual through the
// index table: the table entries two steps ahead and the gathered values and
// A one step ahead are in registers while a step computes.
template <typename T, typename Tc, typename U = T>
__global__ void __launch_bounds__(kT2)
group_adjoint(const int* __restrict__ counts, const Item* __restrict__ items, int cap,
              const Inst<T>* __restrict__ insts, const long long* __restrict__ step, int optimizer, double b1,
              double b2, double eps) {
    __shared__ __align__(16) Tc Hs[16][kHP];    // [b][row a of the tile]
    __shared__ __align__(16) Tc Bs[16][kHP];    // [b][column k of the tile]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int n_items = counts[2];
    const long long now = *step - 1;     // the residual kernel has advanced the counter
    for (int w = blockIdx.x; w < n_items; w += gridDim.x) {
        const Item it = items[2 * cap + w];
        const Inst<T>& in = insts[it.inst];
        const int N = in.N, r = in.r;
        const long long taken = now - in.join;
        const T* A = (taken & 1) ? in.A1 : in.A0;
        T* A_next = (taken & 1) ? in.A0 : in.A1;
        const int row0 = it.i * 64, col0 = it.j * 64;
        Tc acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = Tc(0);
        // staged element l, e = tid + 128 l: H entry (row0 + (e >> 4), b0 + (e & 15)),
        // A entry (b0 + (e >> 6), col0 + (e & 63))
        int ix[8];
        Tc hv[8], bv[8];
        auto load_idx = [&](int b0) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int e = tid + l * kT2, a = row0 + (e >> 4), b = b0 + (e & 15);
                ix[l] = (a < N && b < N) ? in.idx[(int64_t)a * in.ld_idx + b] : -1;
            }
        };
        auto gather = [&]() {
#pragma unroll
            for (int l = 0; l < 8; ++l) hv[l] = ix[l] >= 0 ? (Tc)in.resid[ix[l]] : Tc(0);
        };
        auto load_b = [&](int b0) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int e = tid + l * kT2, b = b0 + (e >> 6), k = col0 + (e & 63);
                bv[l] = (b < N && k < r) ? (Tc)A[(int64_t)b * r + k] : Tc(0);
            }
        };
        load_idx(0);
        gather();
        load_b(0);
        load_idx(16);
        for (int b0 = 0; b0 < N; b0 += 16) {
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int e = tid + l * kT2;
                Hs[e & 15][e >> 4] = hv[l];
                Bs[e >> 6][e & 63] = bv[l];
            }
            __syncthreads();
            if (b0 + 16 < N) {
                gather();                 // the entries of step b0 + 16, loaded one step ago
                load_b(b0 + 16);
                load_idx(b0 + 32);
            }
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                Tc a[8], b[4];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = Hs[kk][8 * ty + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][4 * tx + j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
        // the update's arithmetic runs in U (T, or float for SOS_GROUP_FAST_FP64);
        // the iterate and the moments are stored in T
        const double t = (double)(taken + in.t0 + 1);
        const U c1 = (U)(1.0 - pow(b1, t)), c2 = (U)(1.0 - pow(b2, t));
        const U lr = (U)in.lr, B1 = (U)b1, B2 = (U)b2, EPS = (U)eps, one = U(1);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int a = row0 + 8 * ty + i;
            if (a >= N) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = col0 + 4 * tx + j;
                if (k >= r) continue;
                const int64_t e = (int64_t)a * r + k;
                const U g = U(2) * (U)acc[i][j];
                U step_;
                if (optimizer == SOS_GD) {
                    step_ = lr * g;
                } else {
                    const U mi = B1 * (U)in.m[e] + (one - B1) * g;
                    const U vi = B2 * (U)in.v[e] + (one - B2) * g * g;
                    in.m[e] = (T)mi;
                    in.v[e] = (T)vi;
                    step_ = lr * (mi / c1) / (sqrt(vi / c2) + EPS);
                }
                A_next[e] = A[e] - (T)step_;
            }
        }
    }
}


template <typename T>
__global__ void group_collect(const Inst<T>* __restrict__ insts, int capacity, double* __restrict__ out) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < capacity; s += gridDim.x * blockDim.x) {
        const Inst<T>& in = insts[s];
        double tr = 0.0, tp = 0.0;
        if (in.active) {
            const int chunks = (in.M + kChunk - 1) / kChunk;
            for (int c = 0; c < chunks; ++c) {
                tr += in.partials[2 * c];
                tp += in.partials[2 * c + 1];
            }
        }
        out[2 * s] = 0.5 * tr;
        out[2 * s + 1] = tp;
    }
}

struct Slot {
    bool active = false;
    sos_plan_s* plan = nullptr;
    void *A = nullptr, *m = nullptr, *v = nullptr, *scratch = nullptr;
    const void* p = nullptr;
    double lr = 0.0;
    long long join = 0;
    long long t0 = 0;
};

size_t scratch_bytes(const sos_plan_s* p, int prec) {
    const size_t elt = prec == SOS_FP64 ? 8 : 4;
    const size_t NR = (size_t)p->N * p->r, NN = (size_t)p->N * p->N, M = (size_t)p->M;
    const size_t chunks = (M + kChunk - 1) / kChunk;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return up(NR * elt) + up(NN * elt) + up(M * elt) + up(chunks * 2 * sizeof(double));
}

}  // namespace grp
}  // namespace sos

using namespace sos;
using namespace sos::grp;

struct sos_group_s {
    int prec = SOS_FP32;
    bool fp32_adjoint = false;    // FP64 group: contraction of the adjoint in FP32
    bool fast_fp64 = false;       // FP64 group: double-float forward, FP32 update arithmetic
    int capacity = 0;
    int optimizer = SOS_ADAM;
    double b1 = 0.9, b2 = 0.999, eps = 1e-8;
    int device = -1;
    int grid = 0;
    int item_cap = 0;
    std::vector<Slot> slots;
    bool dirty = true;
    long long steps = 0;          // host copy of the device step counter
    // device
    void* d_insts = nullptr;      // capacity x Inst<T>
    int* d_counts = nullptr;      // 3 ints
    Item* d_items = nullptr;      // 3 x item_cap
    long long* d_step = nullptr;
    double* d_losses = nullptr;   // capacity x 2
    // pinned host staging
    void* h_insts = nullptr;
    int* h_counts = nullptr;
    Item* h_items = nullptr;
    double* h_losses = nullptr;
    cudaStream_t stream = nullptr;   // private stream for capture and replay
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<int, cudaGraphExec_t> graphs;   // steps -> executable graph
};

namespace {

int free_group(sos_group_s* g) {
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
    cudaFree(g->d_insts);
    cudaFree(g->d_counts);
    cudaFree(g->d_items);
    cudaFree(g->d_step);
    cudaFree(g->d_losses);
    cudaFreeHost(g->h_insts);
    cudaFreeHost(g->h_counts);
    cudaFreeHost(g->h_items);
    cudaFreeHost(g->h_losses);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->stream) cudaStreamDestroy(g->stream);
    return SOS_OK;
}

size_t inst_bytes(int prec) { return prec == SOS_FP64 ? sizeof(Inst<double>) : sizeof(Inst<float>); }

int alloc_items(sos_group_s* g, int cap) {
    cudaFree(g->d_items);
    cudaFreeHost(g->h_items);
    g->d_items = nullptr;
    g->h_items = nullptr;
    SOS_CUDA(cudaMalloc(&g->d_items, 3 * (size_t)cap * sizeof(Item)));
    SOS_CUDA(cudaMallocHost(&g->h_items, 3 * (size_t)cap * sizeof(Item)));
    g->item_cap = cap;
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);   // they name the old buffer
    g->graphs.clear();
    return SOS_OK;
}

template <typename T>
void fill_inst(const sos_group_s* g, int s, Inst<T>* out) {
    const Slot& sl = g->slots[s];
    Inst<T> in{};
    in.active = sl.active ? 1 : 0;
    if (sl.active) {
        const sos_plan_s* p = sl.plan;
        const size_t NR = (size_t)p->N * p->r, NN = (size_t)p->N * p->N, M = (size_t)p->M;
        auto up = [](size_t b) { return (b + 255) / 256 * 256; };
        char* sc = static_cast<char*>(sl.scratch);
        in.N = (int)p->N;
        in.M = (int)p->M;
        in.r = (int)p->r;
        in.ld_idx = p->ld_idx;
        in.idx = p->dev.idx;
        in.pair_ptr = p->dev.pair_ptr;
        in.pair_pos = p->dev.pair_pos;
        in.A0 = static_cast<T*>(sl.A);
        in.A1 = reinterpret_cast<T*>(sc);
        in.G = reinterpret_cast<T*>(sc + up(NR * sizeof(T)));
        in.resid = reinterpret_cast<T*>(sc + up(NR * sizeof(T)) + up(NN * sizeof(T)));
        in.partials =
            reinterpret_cast<double*>(sc + up(NR * sizeof(T)) + up(NN * sizeof(T)) + up(M * sizeof(T)));
        in.m = static_cast<T*>(sl.m);
        in.v = static_cast<T*>(sl.v);
        in.p = static_cast<const T*>(sl.p);
        in.join = sl.join;
        in.t0 = sl.t0;
        in.lr = sl.lr;
    }
    out[s] = in;
}

template <typename T>
int launch_step(sos_group_s* g, cudaStream_t st) {
    const Inst<T>* insts = static_cast<const Inst<T>*>(g->d_insts);
    {
        KernelScope ks_("group_forward", st);
        if constexpr (std::is_same<T, double>::value) {
            if (g->fast_fp64)
                group_forward_df<<<g->grid, kT, 0, st>>>(g->d_counts, g->d_items, insts, g->d_step);
            else
                group_forward<T><<<2 * g->grid, kT2, 0, st>>>(g->d_counts, g->d_items, insts, g->d_step);
        } else {
            group_forward<T><<<2 * g->grid, kT2, 0, st>>>(g->d_counts, g->d_items, insts, g->d_step);
        }
    }
    {
        KernelScope ks_("group_residual", st);
        group_residual<T><<<g->grid, kT, 0, st>>>(g->d_counts, g->d_items, g->item_cap, insts, g->d_step);
    }
    {
        KernelScope ks_("group_adjoint", st);
        const int blocks = 2 * g->grid;
        if (g->fp32_adjoint && g->fast_fp64)
            group_adjoint<T, float, float><<<blocks, kT2, 0, st>>>(g->d_counts, g->d_items, g->item_cap, insts,
                                                                   g->d_step, g->optimizer, g->b1, g->b2, g->eps);
        else if (g->fp32_adjoint)
            group_adjoint<T, float><<<blocks, kT2, 0, st>>>(g->d_counts, g->d_items, g->item_cap, insts, g->d_step,
                                                            g->optimizer, g->b1, g->b2, g->eps);
        else
            group_adjoint<T, T><<<blocks, kT2, 0, st>>>(g->d_counts, g->d_items, g->item_cap, insts, g->d_step,
                                                        g->optimizer, g->b1, g->b2, g->eps);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

}  // namespace

extern "C" {

int sos_group_scratch_size(sos_plan_t p, int prec, size_t* bytes) {
    if (!p || !bytes || (prec != SOS_FP32 && prec != SOS_FP64))
        return fail(SOS_E_INVALID, "sos_group_scratch_size: bad argument");
    if (p->r != p->N) return fail(SOS_E_UNSUPPORTED, "sos_group_scratch_size: groups need r = N");
    *bytes = scratch_bytes(p, prec);
    return SOS_OK;
}

int sos_group_create(int prec, int capacity, int optimizer, double beta1, double beta2, double eps, int flags,
                     sos_group_t* out) {
    if (!out || (prec != SOS_FP32 && prec != SOS_FP64) || capacity < 1 || capacity > (1 << 20) ||
        (optimizer != SOS_ADAM && optimizer != SOS_GD) || (flags & ~(SOS_GROUP_FP32_ADJOINT | SOS_GROUP_FAST_FP64)))
        return fail(SOS_E_INVALID, "sos_group_create: bad argument");
    *out = nullptr;
    sos_group_s* g = new sos_group_s();
    g->prec = prec;
    g->fp32_adjoint = prec == SOS_FP64 && (flags & SOS_GROUP_FP32_ADJOINT);
    g->fast_fp64 = prec == SOS_FP64 && (flags & SOS_GROUP_FAST_FP64);
    g->capacity = capacity;
    g->optimizer = optimizer;
    g->b1 = beta1;
    g->b2 = beta2;
    g->eps = eps;
    g->slots.resize(capacity);
    int rc = SOS_OK;
    cudaError_t e = cudaGetDevice(&g->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    g->grid = sms * 4;
    if (e == cudaSuccess) e = cudaMalloc(&g->d_insts, (size_t)capacity * inst_bytes(prec));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_counts, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_step, sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_losses, (size_t)capacity * 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_insts, (size_t)capacity * inst_bytes(prec));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_counts, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_losses, (size_t)capacity * 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemset(g->d_step, 0, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(g->d_counts, 0, 4 * sizeof(int));
    if (e != cudaSuccess) rc = cuda_fail(e, "sos_group_create");
    if (rc == SOS_OK) rc = alloc_items(g, std::max(1024, capacity * 64));
    if (rc != SOS_OK) {
        free_group(g);
        delete g;
        return rc;
    }
    *out = g;
    return SOS_OK;
}

int sos_group_destroy(sos_group_t g) {
    if (!g) return SOS_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    free_group(g);
    delete g;
    return SOS_OK;
}

int sos_group_set(sos_group_t g, int slot, sos_plan_t plan, void* A, void* m, void* v, const void* p,
                  void* scratch, double lr, int64_t t0) {
    if (!g || !plan || slot < 0 || slot >= g->capacity || !A || !p || !scratch)
        return fail(SOS_E_INVALID, "sos_group_set: bad argument");
    if (g->optimizer == SOS_ADAM && (!m || !v)) return fail(SOS_E_INVALID, "sos_group_set: Adam needs m and v");
    if (plan->r != plan->N) return fail(SOS_E_UNSUPPORTED, "sos_group_set: groups need r = N");
    SOS_CHECK(ensure_pair_lists(plan));
    Slot& s = g->slots[slot];
    s.active = true;
    s.plan = plan;
    s.A = A;
    s.m = m;
    s.v = v;
    s.p = p;
    s.scratch = scratch;
    s.lr = lr;
    s.join = g->steps;
    s.t0 = t0 < 0 ? 0 : t0;
    g->dirty = true;
    return SOS_OK;
}

int sos_group_set_lr(sos_group_t g, int slot, double lr) {
    if (!g || slot < 0 || slot >= g->capacity || !g->slots[slot].active)
        return fail(SOS_E_INVALID, "sos_group_set_lr: bad slot");
    g->slots[slot].lr = lr;
    g->dirty = true;
    return SOS_OK;
}

int sos_group_clear(sos_group_t g, int slot) {
    if (!g || slot < 0 || slot >= g->capacity) return fail(SOS_E_INVALID, "sos_group_clear: bad argument");
    g->slots[slot] = Slot{};
    g->dirty = true;
    return SOS_OK;
}

int sos_group_state(sos_group_t g, int slot, void** A_current, void** A_previous, int64_t* steps_taken) {
    if (!g || slot < 0 || slot >= g->capacity || !g->slots[slot].active)
        return fail(SOS_E_INVALID, "sos_group_state: bad slot");
    const Slot& s = g->slots[slot];
    const long long taken = g->steps - s.join;
    if (steps_taken) *steps_taken = taken;
    // A1 is the first region of the scratch; odd step counts leave A there
    if (A_current) *A_current = (taken & 1) ? s.scratch : s.A;
    if (A_previous) *A_previous = (taken & 1) ? s.A : s.scratch;
    return SOS_OK;
}

int sos_group_sync(sos_group_t g, void* stream) {
    TraceRange trace_("sos_group_sync");
    if (!g) return fail(SOS_E_INVALID, "sos_group_sync: NULL group");
    if (!g->dirty) return SOS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the staging buffers may still feed an earlier copy
    SOS_CUDA(cudaStreamSynchronize(st));
    SOS_CUDA(cudaStreamSynchronize(g->stream));
    int nf = 0, nr = 0, na = 0;
    for (int s = 0; s < g->capacity; ++s) {
        const Slot& sl = g->slots[s];
        if (!sl.active) continue;
        const int T = (int)ceil_div(sl.plan->N, 64);
        nf += T * (T + 1) / 2;
        nr += (int)ceil_div(sl.plan->M, kChunk);
        na += T * T;
    }
    const int need = std::max(nf, std::max(nr, na));
    if (need > g->item_cap) SOS_CHECK(alloc_items(g, need + need / 2));
    const int cap = g->item_cap;
    Item* fwd = g->h_items;
    Item* res = g->h_items + cap;
    Item* adj = g->h_items + 2 * cap;
    nf = nr = na = 0;
    for (int s = 0; s < g->capacity; ++s) {
        if (g->prec == SOS_FP64)
            fill_inst<double>(g, s, static_cast<Inst<double>*>(g->h_insts));
        else
            fill_inst<float>(g, s, static_cast<Inst<float>*>(g->h_insts));
        const Slot& sl = g->slots[s];
        if (!sl.active) continue;
        const int T = (int)ceil_div(sl.plan->N, 64);
        for (int i = 0; i < T; ++i)
            for (int j = i; j < T; ++j) fwd[nf++] = Item{s, i, j, 0};
        const int chunks = (int)ceil_div(sl.plan->M, kChunk);
        for (int c = 0; c < chunks; ++c) res[nr++] = Item{s, c, 0, 0};
        for (int i = 0; i < T; ++i)
            for (int j = 0; j < T; ++j) adj[na++] = Item{s, i, j, 0};
    }
    g->h_counts[0] = nf;
    g->h_counts[1] = nr;
    g->h_counts[2] = na;
    g->h_counts[3] = 0;
    SOS_CUDA(cudaMemcpyAsync(g->d_insts, g->h_insts, (size_t)g->capacity * inst_bytes(g->prec),
                             cudaMemcpyHostToDevice, st));
    SOS_CUDA(cudaMemcpyAsync(g->d_items, g->h_items, 3 * (size_t)cap * sizeof(Item), cudaMemcpyHostToDevice, st));
    SOS_CUDA(cudaMemcpyAsync(g->d_counts, g->h_counts, 4 * sizeof(int), cudaMemcpyHostToDevice, st));
    g->dirty = false;
    return SOS_OK;
}

// Runs `steps` steps of every active problem: a graph of steps x 3 kernels,
// captured on the group's private stream the first time and replayed after,
// ordered after and before the caller's stream with events.
int sos_group_run(sos_group_t g, int steps, void* stream) {
    TraceRange trace_("sos_group_run");
    if (!g || steps < 1 || steps > 100000) return fail(SOS_E_INVALID, "sos_group_run: bad argument");
    if (g->dirty) return fail(SOS_E_INVALID, "sos_group_run: call sos_group_sync after changing slots");
    cudaStream_t st = (cudaStream_t)stream;
    auto it = g->graphs.find(steps);
    if (it == g->graphs.end()) {
        cudaGraph_t graph = nullptr;
        SOS_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        int rc = SOS_OK;
        for (int s = 0; s < steps && rc == SOS_OK; ++s)
            rc = g->prec == SOS_FP64 ? launch_step<double>(g, g->stream) : launch_step<float>(g, g->stream);
        cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
        if (rc != SOS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "sos_group_run: capture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "sos_group_run: instantiate");
        it = g->graphs.emplace(steps, exec).first;
    }
    SOS_CUDA(cudaEventRecord(g->ev_in, st));
    SOS_CUDA(cudaStreamWaitEvent(g->stream, g->ev_in, 0));
    SOS_CUDA(cudaGraphLaunch(it->second, g->stream));
    SOS_CUDA(cudaEventRecord(g->ev_out, g->stream));
    SOS_CUDA(cudaStreamWaitEvent(st, g->ev_out, 0));
    g->steps += steps;
    return SOS_OK;
}

// losses[2 s] = 1/2 ||c - p||^2 and losses[2 s + 1] = ||p||^2 of slot s after
// the last step (0 for empty slots).  Host array of 2 x capacity; synchronous.
int sos_group_losses(sos_group_t g, double* losses, void* stream) {
    if (!g || !losses) return fail(SOS_E_INVALID, "sos_group_losses: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    {
        KernelScope ks_("group_collect", st);
        if (g->prec == SOS_FP64)
            group_collect<double><<<(g->capacity + 255) / 256, 256, 0, st>>>(
                static_cast<const Inst<double>*>(g->d_insts), g->capacity, g->d_losses);
        else
            group_collect<float><<<(g->capacity + 255) / 256, 256, 0, st>>>(
                static_cast<const Inst<float>*>(g->d_insts), g->capacity, g->d_losses);
    }
    SOS_CUDA(cudaGetLastError());
    SOS_CUDA(cudaMemcpyAsync(g->h_losses, g->d_losses, (size_t)g->capacity * 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, st));
    SOS_CUDA(cudaStreamSynchronize(st));
    std::memcpy(losses, g->h_losses, (size_t)g->capacity * 2 * sizeof(double));
    return SOS_OK;
}

}  // extern "C"
