// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <functional>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sos_gb300.h"

namespace sos {

// ---- error state ---------------------------------------------------------

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define SOS_CUDA(...)                                                   \
    do {                                                                \
        cudaError_t e_ = (__VA_ARGS__);                                 \
        if (e_ != cudaSuccess) return ::sos::cuda_fail(e_, #__VA_ARGS__); \
    } while (0)

#define SOS_CHECK(...)                  \
    do {                                \
        int s_ = (__VA_ARGS__);         \
        if (s_ != SOS_OK) return s_;    \
    } while (0)

// Counts every kernel launch and, when timing is on, brackets it with CUDA
// events on the launching stream (see timing.cpp).  Construct it right
// before the launch; it records the closing event when it goes out of scope.
class KernelScope {
   public:
    KernelScope(const char* name, cudaStream_t st);
    ~KernelScope();
    KernelScope(const KernelScope&) = delete;
    KernelScope& operator=(const KernelScope&) = delete;

   private:
    const char* name_;
    cudaStream_t st_;
    cudaEvent_t start_ = nullptr;
};

// Host-side NVTX range over an API call: shows up under Nsight tools, and
// costs one pointer test when no tool is attached.
class TraceRange {
   public:
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Kernel attributes (the dynamic shared-memory limit) and occupancy figures
// belong to a device: a process-wide "done" flag would skip them on a second
// GPU, and the first calls of two threads would race on it.  Runs
// setup(value) once per (key, current device) under a lock and hands back
// the value it produced on later calls.  Returns setup's status.
int per_device_value(const void* key, int* value, const std::function<int(int*)>& setup);

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

// ---- workspace -----------------------------------------------------------

constexpr int kResidBlocks = 512;     // blocks of the residual reduction

struct Workspace {
    size_t status = 0;     // int32[64]: [0] status word, [1..] reduction counters
    size_t partials = 0;   // double[2 * kResidBlocks]
    size_t loss = 0;       // double[2] when the caller passes no loss buffer
    size_t c = 0;          // M accumulators (float or double)
    size_t resid = 0;      // M residuals (float or double)
    size_t grad = 0;       // N x r gradient (float or double)
    size_t a16 = 0;        // 2 x N x ld16 bf16 copies of A, ping-pong (SOS_BF16 only)
    size_t diag = 0;       // N floats: the diagonal of A A^T from the bf16 copy (SOS_BF16 only)
    size_t h16 = 0;        // N x ld16h bf16 H(resid)   (SOS_BF16 without the ring, SOS_FP64_TC)
    size_t ring = 0;       // S x 256 x ld16h bf16 panels of H(resid) (SOS_BF16 with the ring)
    size_t ring_flags = 0; // abort word, built and consumed counters of the ring
    size_t resid32 = 0;    // M float residuals         (SOS_FP64_TC only)
    size_t slices = 0;     // max_slices x NP slice matrices of A, NP = N rounded up to 256 (SOS_FP64_TC)
    size_t ex = 0;         // N int32 row exponents     (SOS_FP64_TC only)
    size_t total = 0;
};

constexpr int kMaxSlices = 8;     // SOS_FP64_TC: 5-bit slices of A (the count the API takes)
constexpr int kSliceBits = 5;
constexpr int kMaxSlices8 = 10;   // E4M3 slices: 4-bit digits, ceil(5 s / 4) of them for s 5-bit slices
constexpr int kMaxSlicePairs = 36; // pairs (i <= j) with i + j below kMaxSlices8 (30), rounded up

// How SOS_FP64_TC cuts A into slices: bf16 slices of 5-bit digits (|d| <= 31),
// or with SOS_SLICE_FP8 = 1 E4M3 slices of 4-bit digits (|d| <= 15, exact in
// E4M3's three fraction bits), whose products run at twice the K per byte.
struct SliceFormat {
    bool fp8 = false;
    int bits = kSliceBits;       // bits per digit
    int dmax = 31;               // largest digit magnitude
    int max_slices = kMaxSlices;
    int64_t ld = 0;              // row stride of a slice matrix in elements (bf16) or bytes (E4M3)
    int elem_bytes = 2;
    // slices of this format that carry at least the bits of s 5-bit slices
    int slices_for(int s) const { return (kSliceBits * s + bits - 1) / bits; }
    // every inner sum of digit products, r dmax^2, stays below 2^24 (exact in FP32)
    bool exact_for(int64_t r) const { return r * dmax * dmax < ((int64_t)1 << 24); }
};

// SOS_FP64_TC with r 31^2 k < 2^24 (k >= 2): slice products of one order summed
// in one accumulator, as the segments sa[s] x sb[s] of one product (symmetric:
// (i, i) alone or (i, j) with (j, i)).
constexpr int kMaxGroupSeg = 8;
struct SliceGroup {
    int nseg, order;
    int sa[kMaxGroupSeg], sb[kMaxGroupSeg];
};

// ---- plan ----------------------------------------------------------------

struct DeviceTables {
    int device = -1;
    int num_sms = 0;
    int32_t* idx = nullptr;     // N x ld_idx, idx[a][b] = rank of x^a x^b
    int2* fwd_tiles = nullptr;  // (I, J) tiles of the upper triangle of A A^T
    int2* adj_tiles = nullptr;  // (alpha block, column block) tiles of 2 H A
    int num_fwd_tiles = 0;
    int num_adj_tiles = 0;
    int2* fwd_tiles2 = nullptr;  // the same in 256 x 256 tiles, for CTA pairs
    int2* adj_tiles2 = nullptr;  // entries with y < 0: narrow tiles, 128 columns from 128 (-y - 1)
    int32_t* panel_tiles = nullptr;  // per 256-row block: the adjoint tiles (of adj_tiles2) that read it
    // units of two 256 x 256 tiles sharing a column block, for clusters of two
    // pairs that multicast the B operand (a second tile with x < 0 stands in)
    int2* fwd_units = nullptr;
    int2* adj_units = nullptr;
    int num_fwd_units = 0;
    int num_adj_units = 0;
    int num_fwd_tiles2 = 0;
    int num_adj_tiles2 = 0;
    // pair lists of the Gram identity, grouped by coefficient (built on demand):
    // pairs of coefficient g are pair_pos[pair_ptr[g] .. pair_ptr[g+1]), each
    // a * N + b with a <= b, the top bit set when a == b
    int32_t* pair_ptr = nullptr;
    int32_t* pair_pos = nullptr;
    // first layer (two_d = 4 only, built on demand): form_rows[i * nf + j] is
    // the row of the form's monomial x_i x_j (nf = n + 1 form variables, the
    // last one dehomogenised to 1); form_pairs[a] = (i, j), i <= j, of row a
    int32_t* form_rows = nullptr;
    int2* form_pairs = nullptr;
    // SOS_FP64_TC, built on demand: the 256 x 256 tiles of every slice pair in
    // the stacked coordinates, ordered by i + j; the pairs with i + j < s are
    // the first slice_tile_count[s] entries
    int2* slice_tiles2 = nullptr;
    int slice_tile_count[kMaxSlices8 + 1] = {0};
    int slice_pairs = 0;                // pairs (i <= j) with i + j < the format's max_slices
    int slice_pair_offset[kMaxSlicePairs + 1] = {0};  // tiles of the u-th pair: [offset[u], offset[u + 1])
    // grouped form (r 31^2 2 < 2^24): groups by order, tiles (g * TP + I, J)
    // with J >= I; groups of order < s own the first slice_tile_count[s] tiles
    SliceGroup* slice_groups = nullptr;
    bool slice_grouped = false;
};

}  // namespace sos

struct sos_plan_s {
    int n = 0, two_d = 0, d = 0;
    int64_t N = 0, M = 0, r = 0;
    int64_t ld_idx = 0;   // row stride of the device idx table (multiple of 8)
    int64_t ld16 = 0;     // row stride of the bf16 copy of A (multiple of 64)
    int64_t ld16h = 0;    // row stride of the bf16 H (multiple of 64)
    std::vector<uint8_t> Ed, E2d;   // exponent tables, canonical order
    std::vector<uint8_t> Sd;        // suffix sums S_j(a) of the rows of Ed, N x n
    std::vector<int32_t> phi;       // n x (2d+1): rank(g) = sum_j phi[j][S_j(g)]
    sos::DeviceTables dev;
    std::mutex mu;
};

namespace sos {

Workspace workspace_layout(const sos_plan_s* plan, int prec);

// Whether the BF16 adjoint reads H(r) from band-local panels that the kernel
// builds itself instead of a materialised H (environment variable SOS_H_RING
// = 1, read once; only with the CTA-pair kernels).  Off by default: measured
// on the large workload it is about 9% slower than materialising H, and it
// holds a few bands of panels instead of the whole N x N H.
bool use_h_ring();
// Whether the CTA-pair contractions run in clusters of two pairs that share
// the B operand by TMA multicast (environment variable SOS_MCAST = 1, read
// once; only with the CTA-pair kernels, not with the H ring).
bool use_mcast();
// Whether the BF16 forward takes the diagonal of A A^T from a CUDA-core sum of
// the bf16 squares (FP32, round to nearest) instead of the tensor-core
// accumulator, which truncates once per 16-deep step (environment variable
// SOS_EXACT_DIAG = 1, read once; off by default).
bool use_exact_diag();
// The SOS_FP64_TC slice format the environment asks for (SOS_SLICE_FP8, read
// once): 1 E4M3 bytes of 4-bit digits, 0 bf16 5-bit digits, -1 (unset) chosen
// per plan.
int slice_fp8_setting();
// The slice format of SOS_FP64_TC for this plan: the one SOS_SLICE_FP8 names,
// else bf16 slices where their products are exact (r <= 17,458) and E4M3
// slices above (they are exact up to r = 74,565).
SliceFormat slice_format(const sos_plan_s* plan);
// Row-block band height of the adjoint's tile list (SOS_BAND_ADJ, default 8).
int adjoint_band();
// The ring of H panels: G = band height, S = slots (D G for a depth of D bands,
// SOS_RING_DEPTH, default 3; at most the number of 256-row panels), panels =
// ceil(N / 256).
struct RingGeometry {
    int band, slots, panels;
};
RingGeometry ring_geometry(const sos_plan_s* plan);
int ensure_device(sos_plan_s* plan);
int ensure_pair_lists(sos_plan_s* plan);

// ---- kernel launchers (kernels_simt.cu) ------------------------------------

int launch_build_idx(const sos_plan_s* plan, int32_t* idx, const uint8_t* d_S, const int32_t* d_phi,
                     cudaStream_t st);
int launch_cast_bf16(const float* A, int64_t N, int64_t r, void* a16, int64_t ld16,
                     cudaStream_t st);
// d[a] = sum_k bf16(A)[a][k]^2 from the bf16 copy, FP32 on CUDA cores (the exact
// diagonal of the BF16 forward).
int launch_diag_sumsq(const void* a16, int64_t ld16, int64_t N, int64_t r, float* d, cudaStream_t st);
template <typename Tin, typename Tacc>
int launch_simt_forward(const sos_plan_s* plan, const Tin* A, Tacc* c, int64_t batch,
                        cudaStream_t st);
template <typename T>
int launch_residual(const sos_plan_s* plan, const T* c, const T* p, T* resid, double* loss,
                    double* partials, int32_t* status, int64_t batch, cudaStream_t st);
template <typename T>
int launch_simt_adjoint(const sos_plan_s* plan, const T* A, const T* resid, T* grad,
                        int64_t batch, cudaStream_t st, bool fp32_contraction = false);
// H(resid) in bf16 (h16.cu); a timed-out wait sets *status to SOS_E_TIMEOUT.
int launch_build_h16(const sos_plan_s* plan, const float* resid, void* h16, int32_t* status, cudaStream_t st);
template <typename T>
int launch_update(int64_t N, int64_t r, T* A, T* m, T* v, const T* grad, int optimizer,
                  int64_t t, double lr, double b1, double b2, double eps, void* a16,
                  int64_t ld16, cudaStream_t st);
template <typename T>
int launch_fill(T* x, int64_t count, T value, cudaStream_t st);
template <typename Tin, typename Tout>
int launch_convert(const Tin* x, Tout* y, int64_t count, cudaStream_t st);

// ---- tensor-core kernels (kernels_tc.cu) ------------------------------------

int launch_tc_forward(const sos_plan_s* plan, const void* a16, float* c, int32_t* status,
                      cudaStream_t st);
int launch_tc_adjoint(const sos_plan_s* plan, const void* h16, const void* a16, float* grad,
                      int32_t* status, cudaStream_t st);
int launch_tc_adjoint_update(const sos_plan_s* plan, const void* h16, const void* a16_cur, void* a16_next,
                             float* A, float* m, float* v, int optimizer, int64_t t, double lr, double b1,
                             double b2, double eps, int32_t* status, cudaStream_t st);

// ---- the same on CTA pairs (kernels_tc2.cu) ---------------------------------------

// diag (N floats, or NULL): when given, the segment-sum takes the diagonal of
// A A^T from it instead of from the tensor-core accumulator.
int launch_tc_forward_pair(const sos_plan_s* plan, const void* a16, float* c, int32_t* status, cudaStream_t st,
                           const float* diag = nullptr);
int launch_tc_adjoint_pair(const sos_plan_s* plan, const void* h16, const void* a16, float* grad,
                           int32_t* status, cudaStream_t st);
// The same two adjoints reading H(resid) from the ring in the workspace
// (`ring`, `flags`): a prologue kernel builds the first band of panels and
// zeroes the flags, the adjoint's builder warps build the rest.
int launch_tc_adjoint_ring_pair(const sos_plan_s* plan, const float* resid, void* ring, uint32_t* flags,
                                const void* a16, float* grad, int32_t* status, cudaStream_t st);
int launch_tc_adjoint_update_ring_pair(const sos_plan_s* plan, const float* resid, void* ring, uint32_t* flags,
                                       const void* a16_cur, void* a16_next, float* A, float* m, float* v,
                                       int optimizer, int64_t t, double lr, double b1, double b2, double eps,
                                       int32_t* status, cudaStream_t st);
int launch_tc_adjoint_update_pair(const sos_plan_s* plan, const void* h16, const void* a16_cur, void* a16_next,
                                  float* A, float* m, float* v, int optimizer, int64_t t, double lr, double b1,
                                  double b2, double eps, int32_t* status, cudaStream_t st);
// How many CTA pairs of the adjoint kernel are resident on the current GPU at
// once (the persistent grid of its launches).
int adjoint_pair_capacity(int* pairs);

// ---- one pass of the objective (api.cu), shared with the first layer ----------

// loss = 1/2 ||c(A) - p||^2 into `loss` (or the workspace), gradient 2 H(c - p) A
// into `grad` when it is not NULL; `ws` is a workspace of workspace_layout(plan, prec).
int core_loss_grad(sos_plan_s* plan, int prec, const void* A, const void* p, void* grad, void* loss, void* ws,
                   cudaStream_t st, bool fp32_contraction);

// ---- SOS_FP64_TC (slices.cu, kernels_tc2.cu) ----------------------------------------

// c (FP64, zeroed here) = c(A) from slices of A on tensor cores, as many as
// carry the bits of `slices` 5-bit slices in the plan's slice format; also
// leaves the bf16 copy of A in the workspace's a16.
int forward_tc64(sos_plan_s* plan, const double* A, void* ws, double* c, int slices, cudaStream_t st);
// Every slice pair of the stacked slices S (slice i in rows i * NP .., in format
// f) listed in `tiles` (stacked 256 x 256 tile coordinates), in one launch.
int launch_tc_slices_pair(const sos_plan_s* plan, const SliceFormat& f, const void* S, int64_t NP,
                          const int2* tiles, int num_tiles, const int32_t* ex, double* c, int32_t* status,
                          cudaStream_t st);
// The grouped form: `groups` is a device array of SliceGroup.
int launch_tc_slice_groups_pair(const sos_plan_s* plan, const SliceFormat& f, const void* S, int64_t NP,
                                const int2* tiles, int num_tiles, const void* groups, const int32_t* ex, double* c,
                                int32_t* status, cudaStream_t st);
int launch_update_mixed(int64_t N, int64_t r, double* A, float* m, float* v, const float* grad, int optimizer,
                        int64_t t, double lr, double b1, double b2, double eps, cudaStream_t st);

// Whether the tensor-core contractions run on CTA pairs (environment variable
// SOS_CTA_PAIRS = 0 or 1, read once; pairs by default).
bool use_cta_pairs();

}  // namespace sos
