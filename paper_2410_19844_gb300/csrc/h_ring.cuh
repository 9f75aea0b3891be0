// H(r) for the tensor-core adjoint without materialising it: band-local panels
// in a ring (chain rule of Eq. 2: grad = 2 H(r) A, H[a][b] = r[idx(a, b)]).
//
// Panel P holds rows 256 P .. 256 P + 255 of H over all N columns, in bf16, in
// ring slot P mod S (S slots of 256 x ldh).  The adjoint's tile list walks
// bands of G row blocks (K-outer, rows inner) and S = D G for a depth of D >= 2
// bands, so every tile that reads panel P precedes, in the list and hence in
// each CTA pair's sequence, every tile that reads panel P + S, which reuses the
// slot.  A band's panels are all read until the band ends, so with depth D the
// builders may fill band b + D - 1 once band b - 1 is done.
//
// Who writes and who waits (all waits bounded; a timeout sets the abort word
// and the status word, and every waiter gives up when it sees the abort word):
//   * before the adjoint launch, a stand-alone kernel builds the first band
//     (panels 0 .. G-1) and zeroes the flags;
//   * inside the adjoint, builder warps of every CTA build panels G, G+1, ...
//     in order, each CTA its share of 64 x 64 units; before writing panel P a
//     CTA waits until every tile of panel P - S has finished with its slot
//     (consumed[P - S] reaches that panel's tile count); after writing it the
//     CTA fences its stores for the async proxy and adds 1 to built[P];
//   * the TMA producer of a tile of panel P >= G waits for built[P] to reach
//     the number of CTAs, fences, and loads the operand from the ring;
//   * when a tile's MMAs have completed (its accumulator is full, so both
//     CTAs' loads of the ring have landed), the leader's epilogue adds 1 to
//     consumed[P].
// Every CTA of the grid must be resident at once for the builders' shares to
// arrive; the launch is cooperative.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace sos {
namespace tc {

constexpr int kRingFlagsHeader = 64;   // words before the counters: [0] is the abort word

struct RingArgs {
    const int32_t* idx;          // N x ld_idx index table
    int64_t ld_idx;
    const float* resid;          // M residuals
    __nv_bfloat16* ring;         // S slots x 256 rows x ldh
    int64_t ldh;
    int N;
    int S;                       // slots
    int first_panel;             // panels below it are built before the launch
    int num_panels;              // ceil(N / 256)
    const int32_t* panel_tiles;  // number of tiles that read each panel
    uint32_t* flags;             // abort word, built[num_panels], consumed[num_panels]

    __device__ __forceinline__ uint32_t* abort_word() const { return flags; }
    __device__ __forceinline__ uint32_t* built(int P) const { return flags + kRingFlagsHeader + P; }
    __device__ __forceinline__ uint32_t* consumed(int P) const {
        return flags + kRingFlagsHeader + num_panels + P;
    }
    // 64 x 64 units of one panel: four row quarters times the column blocks
    __host__ __device__ __forceinline__ int units_per_panel() const { return 4 * ((N + 63) / 64); }
};

// Rows r0 .. r0 + RPW - 1 of the 64 rows of unit u of panel P, one warp:
// lane j covers columns 2j and 2j + 1 of the unit's 64.  All index loads
// (streamed: the table is read once per step) are issued before the gathers
// of r, and all gathers before the stores.
template <int RPW>
__device__ __forceinline__ void ring_build_rows(const RingArgs& g, int P, int u, int r0, int lane) {
    const int CB = (g.N + 63) / 64;
    const int rq = u / CB, cb = u - rq * CB;
    const int b = cb * 64 + 2 * lane;
    const int local0 = rq * 64 + r0;             // first row of the warp within the panel
    const int a0 = P * 256 + local0;
    int2 gi[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        gi[i] = make_int2(-1, -1);
        const int a = a0 + i;
        if (a < g.N && b < g.N) {
            const int32_t* src = g.idx + (int64_t)a * g.ld_idx + b;
            if (b + 1 < g.N)
                gi[i] = __ldcs(reinterpret_cast<const int2*>(src));
            else
                gi[i].x = __ldcs(src);
        }
    }
    float v0[RPW], v1[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        v0[i] = gi[i].x >= 0 ? __ldg(g.resid + gi[i].x) : 0.0f;
        v1[i] = gi[i].y >= 0 ? __ldg(g.resid + gi[i].y) : 0.0f;
    }
    __nv_bfloat16* dst = g.ring + ((int64_t)(P % g.S) * 256 + local0) * g.ldh + b;
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        if (a0 + i < g.N && b < g.N)
            *reinterpret_cast<__nv_bfloat162*>(dst + (int64_t)i * g.ldh) = __floats2bfloat162_rn(v0[i], v1[i]);
    }
}

// Prefetches into L2 the index-table rows that unit u of panel P reads (64
// rows of 64 int32, at most three 128-byte lines each), spread over nthreads
// threads (this one is t).  Every address stays inside the table.
__device__ __forceinline__ void ring_prefetch_unit(const RingArgs& g, int P, int u, int t, int nthreads) {
    const int CB = (g.N + 63) / 64;
    const int rq = u / CB, cb = u - rq * CB;
    for (int i = t; i < 64 * 3; i += nthreads) {
        const int row = i / 3, part = i - 3 * row;
        const int a = P * 256 + rq * 64 + row;
        const int b = min(cb * 64 + (part == 2 ? 63 : 32 * part), g.N - 1);
        if (a < g.N) asm volatile("prefetch.global.L2 [%0];" ::"l"(g.idx + (int64_t)a * g.ld_idx + b));
    }
}

// Zeroes the ring's flags and builds panels 0 .. g.first_panel - 1 (h16.cu),
// stream-ordered before the adjoint that builds the rest.
int launch_ring_prologue(const RingArgs& g, int num_sms, cudaStream_t st);

}  // namespace tc
}  // namespace sos
