// Tensor-core kernels on CTA pairs (tcgen05.mma.cta_group::2).
//
// Same contractions and epilogues as kernels_tc.cu, but two CTAs on two SMs
// compute one 256 x 256 tile together: each CTA stages its own 128 rows of the
// A operand and half (128 rows or columns) of the B operand, the leader CTA
// issues M = 256, N = 256, K = 16 MMAs that read both CTAs' shared memory and
// write 128 accumulator lanes in each CTA's TMEM.  Per CTA that halves the B
// traffic: 32 KB per 64-deep K-block instead of 48 KB, and each SM's shared
// memory serves 8 KB per MMA instead of 12 KB.
//
//   warp 0, one lane (both CTAs) : TMA producer; completion is counted on the
//                                  leader's mbarrier
//   warp 1, one lane (leader)    : MMA issuer; commits are multicast to both CTAs
//   warps 2-5 (both CTAs)        : epilogue on the CTA's own 128 rows; each warp
//                                  signals the leader when its TMEM buffer is free
// Every mbarrier wait is bounded by the global timer; a role that gives up sets
// the status word and unwinds, and both CTAs still meet at the final cluster
// barrier before TMEM is released.
//
// With RING (the BF16 adjoint), the A operand is H(r) read from band-local
// panels in a ring instead of a materialised H, and two more warps build the
// panels while the MMAs run (h_ring.cuh):
//   warps 6-7 (both CTAs)        : builders of the CTA's share of later panels
//
// With MC, a cluster of four CTAs runs two pairs on two tiles that share the
// B operand (the same column block): pair 0's CTAs load each half of B once and
// multicast it into both pairs' shared memory, which cuts the operand bytes each
// SM pulls from L2 by a quarter.  A stage is then refilled only when both pairs'
// MMAs are done with it: every empty barrier counts both leaders' commits.
// Tiles come in units of two (one per pair); a unit whose second tile has
// x < 0 runs a copy of the first tile (row block -1 - x) whose results are
// dropped.
//
// With F8 the operands are E4M3 bytes (the 4-bit slices of SOS_FP64_TC): the
// shared-memory layout is the same byte for byte (128-byte rows, so an atom is
// 128 K elements instead of 64) and each MMA is kind::f8f6f4 with K = 32.
//
// A tile entry (x, y) is row block x of 256 and column block y of 256.  An
// entry with y < 0 is a narrow tile: columns 128 (-y - 1) onwards, 128 wide,
// computed with N = 128 MMAs (each CTA supplies 64 columns of B).  The tile
// lists use narrow tiles to even out the last round of a persistent launch.
// The producer still loads the full B boxes for a narrow tile (the MMAs read
// only their first 64 columns or rows), so every stage expects the same bytes.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>

#include "h_ring.cuh"
#include "internal.h"
#include "tc_epilogues.cuh"
#include "tc_ptx.cuh"

namespace sos {
namespace tc2 {

using namespace tc;

constexpr int BM = 128;          // rows per CTA; the pair covers 256
constexpr int PAIR_M = 256;
constexpr int BN = 256;          // columns of the pair tile; each CTA stages 128
constexpr int BK = 64;
// A stage holds KATOMS consecutive 64-deep K-blocks ("atoms", one 128-byte
// swizzle span each) of both operands and is released by one commit: a
// tcgen05.commit costs the tensor pipe on the order of a hundred
// nanoseconds, so committing per atom wastes a sizeable share of the
// mainloop.  Three stages of two atoms keep the same 192 KB in flight as six
// stages of one.
constexpr int KATOMS = 2;
constexpr int STAGES = 3;
constexpr int ATOM_A = BM * BK * 2;               // 16 KB
constexpr int ATOM_B = (BN / 2) * BK * 2;         // 16 KB
constexpr int A_BYTES = KATOMS * ATOM_A;          // per stage
constexpr int B_BYTES = KATOMS * ATOM_B;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;    // 64 KB per CTA
constexpr int BAR_BYTES = 256;
constexpr int EPI_STAGE_BYTES = 4 * STAGE_FLOATS * 4;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + BAR_BYTES + EPI_STAGE_BYTES;
constexpr int THREADS = 192;
constexpr int RING_BUILDER_WARPS = 2;
constexpr int RING_THREADS = THREADS + 32 * RING_BUILDER_WARPS;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__host__ __device__ constexpr int threads_of(bool ring) { return ring ? RING_THREADS : THREADS; }

template <bool B_MN_MAJOR, class Epilogue, bool RING = false, bool MC = false, bool F8 = false>
__global__ void __launch_bounds__(threads_of(RING), 1)
tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int nkb,
                    const int2* __restrict__ tiles, int num_tiles, Epilogue epi, int32_t* __restrict__ status,
                    RingArgs ring) {
    static_assert(!(Epilogue::kSegmented && B_MN_MAJOR), "segmented K runs with K-major operands only");
    static_assert(!(Epilogue::kSegmented && RING), "the H ring serves the adjoint only");
    static_assert(!(MC && (RING || Epilogue::kSegmented)), "multicast runs plain tiles only");
    static_assert(!(F8 && (B_MN_MAJOR || RING || MC)), "E4M3 operands are K-major slices only");
    constexpr int BKE = F8 ? 2 * BK : BK;        // K elements of one 128-byte atom
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* base = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    uint8_t* sA = base;
    uint8_t* sB = base + STAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile uint32_t* err = tmem_slot + 1;
    volatile uint32_t* bstop = tmem_slot + 2;     // the ring builders' common decision to stop
    float* epi_stage = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES + BAR_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t crank = cluster_ctarank();
    const uint32_t rank = crank & 1u;            // rank within the CTA pair
    const uint32_t lead_rank = crank & ~1u;      // cluster rank of this pair's leader
    const bool leader = rank == 0;
    const int pc = MC ? (int)(crank >> 1) : 0;   // pair within the cluster
    // Work items: tiles, or with MC units of one tile per pair of the cluster.
    const int pair = MC ? (int)(blockIdx.x >> 2) : (int)(blockIdx.x >> 1);
    const int num_pairs = MC ? (int)(gridDim.x >> 2) : (int)(gridDim.x >> 1);
    auto tile_at = [&](int t) { return MC ? tiles[2 * t + pc] : tiles[t]; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], MC ? 2 : 1);     // with MC both pairs' leaders release a stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 8);     // 4 epilogue warps in each CTA
        }
        mbar_init(drain, 1);
        *err = 0;
        *bstop = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc_pair(tmem_slot, TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();                   // barriers initialised and TMEM allocated in both CTAs
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer (both CTAs) ----------------
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
        int s = 0;
        uint32_t ph = 0;
        int64_t issued = 0;
        bool ok = true;
        for (int t = pair; t < num_tiles && ok; t += num_pairs) {
            const int2 tile = tile_at(t);
            const bool narrow = tile.y < 0;
            const int tx = (MC && tile.x < 0) ? -1 - tile.x : tile.x;
            int arow = tx * PAIR_M + (int)rank * BM;
            if constexpr (RING) {
                // the tile's rows of H are panel tile.x, in its ring slot
                if (tile.x >= ring.first_panel) {
                    if (!wait_counter(ring.built(tile.x), gridDim.x, ring.abort_word(), WAIT_LIMIT_NS)) {
                        ok = false;
                        break;
                    }
                    fence_proxy_async_global();
                }
                arow = (tile.x % ring.S) * PAIR_M + (int)rank * BM;
            }
            const int bcol = narrow ? (-tile.y - 1) * (BN / 2) + (int)rank * (BN / 4)
                                    : tile.y * BN + (int)rank * (BN / 2);
            int nkbt = nkb;       // K blocks of this tile (all its segments)
            if constexpr (Epilogue::kSegmented) nkbt = epi.segments(tile) * nkb;
            for (int kb = 0; kb < nkbt; kb += KATOMS) {
                if (*err || !mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                if (leader) mbar_arrive_expect_tx(&full[s], 2 * STAGE_BYTES);
                const uint32_t bar = mapa_shared(smem_u32(&full[s]), lead_rank);
#pragma unroll
                for (int at = 0; at < KATOMS; ++at) {
                    int kx = (kb + at) * BKE;           // beyond K: zero fill, still counted
                    int ar = arow, bc = bcol;
                    if constexpr (Epilogue::kSegmented) {
                        // atom q of the tile: K block q % nkb of segment q / nkb; past the
                        // last segment, a block beyond K (zero fill)
                        const int q = kb + at;
                        const int seg = q < nkbt ? q / nkb : 0;
                        kx = q < nkbt ? (q - seg * nkb) * BKE : nkb * BKE;
                        ar = epi.seg_arow(tile, seg) + (int)rank * BM;
                        bc = epi.seg_brow(tile, seg) + (int)rank * (BN / 2);
                    }
                    tma_load_2d_pair(sA + s * A_BYTES + at * ATOM_A, &mapA, bar, kx, ar);
                    if constexpr (MC) {
                        // pair 0 loads B for both pairs; pair 1's bytes arrive on its own leader
                        const uint16_t mask = (uint16_t)((1u << crank) | (1u << (crank + 2)));
                        if (pc == 0) {
                            if (B_MN_MAJOR) {
#pragma unroll
                                for (int j = 0; j < BN / 2 / 64; ++j)
                                    tma_load_2d_pair_multicast(sB + s * B_BYTES + at * ATOM_B + j * (64 * BK * 2),
                                                               &mapB, bar, bcol + 64 * j, kx, mask);
                            } else {
                                tma_load_2d_pair_multicast(sB + s * B_BYTES + at * ATOM_B, &mapB, bar, kx, bc, mask);
                            }
                        }
                    } else if (B_MN_MAJOR) {
#pragma unroll
                        for (int j = 0; j < BN / 2 / 64; ++j)
                            tma_load_2d_pair(sB + s * B_BYTES + at * ATOM_B + j * (64 * BK * 2), &mapB, bar,
                                             bcol + 64 * j, kx);
                    } else {
                        tma_load_2d_pair(sB + s * B_BYTES + at * ATOM_B, &mapB, bar, kx, bc);
                    }
                }
                ++issued;
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        if (!ok) {
            *err = 1;
            atomicCAS(status, 0, SOS_E_TIMEOUT);
            if constexpr (RING) atomicExch(ring.abort_word(), 1u);
        }
        // The leader's full barriers count both CTAs' copies: let them land.
        if (leader)
            for (int64_t i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
                mbar_wait(&full[i % STAGES], (uint32_t)((i / STAGES) & 1), WAIT_LIMIT_NS);
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------- MMA issuer (leader) ----------------
        constexpr uint32_t idesc_full =
            F8 ? idesc_e4m3_f32(PAIR_M, BN) : idesc_bf16_f32(PAIR_M, BN, 0, B_MN_MAJOR ? 1 : 0);
        constexpr uint32_t idesc_narrow =
            F8 ? idesc_e4m3_f32(PAIR_M, BN / 2) : idesc_bf16_f32(PAIR_M, BN / 2, 0, B_MN_MAJOR ? 1 : 0);
        int s = 0;
        uint32_t ph = 0;
        int it = 0;
        bool ok = true;
        // the next tile's entry is loaded one tile ahead, off the issue path
        int2 next = pair < num_tiles ? tile_at(pair) : make_int2(0, 0);
        for (int t = pair; t < num_tiles && ok; t += num_pairs, ++it) {
            const int2 tile = next;
            if (t + num_pairs < num_tiles) next = tile_at(t + num_pairs);
            const int buf = it & 1;
            const uint32_t tph = (uint32_t)(it >> 1) & 1u;
            if (*err || !mbar_wait(&tempty[buf], tph ^ 1u, WAIT_LIMIT_NS)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t dtm = tmem_base + (uint32_t)(buf * BN);
            const uint32_t idesc = tile.y < 0 ? idesc_narrow : idesc_full;
            int nkbt = nkb;
            if constexpr (Epilogue::kSegmented) nkbt = epi.segments(tile) * nkb;
            for (int kb = 0; kb < nkbt; kb += KATOMS) {
                if (*err || !mbar_wait(&full[s], ph, WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA + s * A_BYTES);
                const uint32_t b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
                for (int at = 0; at < KATOMS; ++at) {
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ad = smem_desc_sw128(a_addr + at * ATOM_A + kk * 32, 16, 1024);
                        const uint64_t bd =
                            B_MN_MAJOR ? smem_desc_sw128(b_addr + at * ATOM_B + kk * 16 * 128, 64 * BK * 2, 1024)
                                       : smem_desc_sw128(b_addr + at * ATOM_B + kk * 32, 16, 1024);
                        if constexpr (F8)
                            umma_e4m3_pair(dtm, ad, bd, idesc, (kb | at | kk) != 0 ? 1u : 0u);
                        else
                            umma_bf16_pair(dtm, ad, bd, idesc, (kb | at | kk) != 0 ? 1u : 0u);
                    }
                }
                umma_commit_pair_multicast(&empty[s], MC ? 0xF : 0x3);
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            umma_commit_pair_multicast(&tfull[buf], (uint16_t)(0x3u << lead_rank));
        }
        if (!ok) {
            *err = 1;
            atomicCAS(status, 0, SOS_E_TIMEOUT);
            if constexpr (RING) atomicExch(ring.abort_word(), 1u);
        }
        umma_commit_pair_multicast(drain, (uint16_t)(1u << lead_rank));
        mbar_wait(drain, 0, WAIT_LIMIT_NS);
    } else if (warp >= 2 && warp < 6) {
        // ---------------- epilogue (both CTAs) ----------------
        const int q = warp & 3;
        const uint32_t tempty_leader0 = mapa_shared(smem_u32(&tempty[0]), lead_rank);
        int it = 0;
        for (int t = pair; t < num_tiles; t += num_pairs, ++it) {
            const int buf = it & 1;
            const uint32_t tph = (uint32_t)(it >> 1) & 1u;
            const bool ready = (*err == 0) && mbar_wait(&tfull[buf], tph, WAIT_LIMIT_NS);
            if (!__all_sync(0xffffffffu, ready)) {
                if (lane == 0) {
                    *err = 1;
                    atomicCAS(status, 0, SOS_E_TIMEOUT);
                    if constexpr (RING) atomicExch(ring.abort_word(), 1u);
                }
                break;
            }
            tc_fence_after();
            const int2 tile = tile_at(t);
            if constexpr (RING) {
                // the tile's MMAs are done, so both CTAs' loads of its panel have landed
                if (leader && warp == 2 && lane == 0) red_release_gpu_add(ring.consumed(tile.x), 1u);
            }
            float* stage = epi_stage + (warp - 2) * STAGE_FLOATS;
            const int row0 = tile.x * PAIR_M + (int)rank * BM + q * 32;
            const int col0 = tile.y < 0 ? (-tile.y - 1) * (BN / 2) : tile.y * BN;
            // a unit's stand-in tile (x < 0, with MC) computes but stores nothing
            const int nch = (MC && tile.x < 0) ? 0 : (tile.y < 0 ? BN / 64 : BN / 32);
#pragma unroll 1
            for (int ch = 0; ch < nch; ++ch) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + ch * 32), v);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) stage[stage_idx(lane, j)] = __uint_as_float(v[j]);
                __syncwarp();
                epi(row0, col0 + ch * 32, stage, lane);
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(tempty_leader0 + (uint32_t)(buf * sizeof(uint64_t)));
        }
    }
    if constexpr (RING) {
        if (warp >= 6) {
            // ---------------- panel builders (both CTAs) ----------------
            const int w = warp - 6, bt = threadIdx.x - THREADS;
            const int units = ring.units_per_panel();
            const int cta = (int)blockIdx.x, nctas = (int)gridDim.x;
            bool ok = true;
            // the index rows of the next panel go to L2 while this one is built,
            // so the builders' loads hit L2 instead of waiting on DRAM
            if (ring.first_panel < ring.num_panels)
                for (int u = cta; u < units; u += nctas) ring_prefetch_unit(ring, ring.first_panel, u, bt, 32 * RING_BUILDER_WARPS);
            for (int P = ring.first_panel; P < ring.num_panels && ok; ++P) {
                if (P + 1 < ring.num_panels)
                    for (int u = cta; u < units; u += nctas) ring_prefetch_unit(ring, P + 1, u, bt, 32 * RING_BUILDER_WARPS);
                if (P >= ring.S) {
                    // Slot P mod S is free once every tile of panel P - S is done with
                    // it.  One thread waits and writes the builders' common decision
                    // before the barrier; every builder reads it after the barrier, so
                    // all of them leave together or none does (the next write comes
                    // only after the barrier that ends this panel).
                    if (threadIdx.x == THREADS) {
                        bool freed = wait_counter(ring.consumed(P - ring.S), (uint32_t)ring.panel_tiles[P - ring.S],
                                                  ring.abort_word(), WAIT_LIMIT_NS);
                        *bstop = (!freed || *err) ? 1u : 0u;
                    }
                    named_bar_sync(1, 32 * RING_BUILDER_WARPS);
                    if (*bstop) {
                        ok = false;
                        break;
                    }
                }
                for (int u = cta; u < units; u += nctas)
                    for (int r0 = 32 * w; r0 < 64; r0 += 32 * RING_BUILDER_WARPS)
                        ring_build_rows<32>(ring, P, u, r0, lane);
                fence_proxy_async_global();
                named_bar_sync(1, 32 * RING_BUILDER_WARPS);
                if (threadIdx.x == THREADS) {
                    __threadfence();
                    red_release_gpu_add(ring.built(P), 1u);
                }
            }
            if (!ok && threadIdx.x == THREADS) {
                atomicCAS(status, 0, SOS_E_TIMEOUT);
                atomicExch(ring.abort_word(), 1u);
            }
        }
    }
    if (*err) {
        // give copies that may still be landing a moment before the CTAs part
        const uint64_t t0 = global_timer_ns();
        while (global_timer_ns() - t0 < 20000) {
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();                   // the leader's MMAs read the peer's shared memory
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, TMEM_COLS);
    }
}

}  // namespace tc2

namespace {

// Clusters of two CTAs; with `cooperative` the launch also guarantees that
// every CTA of the grid is resident at once (the H ring's builders and
// producers wait on one another across CTAs).
void pair_launch_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, cudaStream_t st, int threads,
                        bool cooperative, int cluster = 2) {
    using namespace tc2;
    cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeCooperative;
    attr[1].val.cooperative = 1;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = cooperative ? 2 : 1;
}

// How many clusters (of two CTAs by default) of `kern` fit on the current GPU at once.
int resident_pairs(const void* kern, int threads, int* out, int cluster = 2) {
    using namespace tc2;
    SOS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    int dev = 0, sms = 0;
    SOS_CUDA(cudaGetDevice(&dev));
    SOS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    pair_launch_config(cfg, attr, 0, threads, false, cluster);
    cfg.gridDim = dim3(sms / cluster * cluster);
    int clusters = 0;
    SOS_CUDA(cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg));
    if (clusters < 1) return fail(SOS_E_UNSUPPORTED, "CTA pairs: no cluster fits on this GPU");
    *out = clusters;
    return SOS_OK;
}

// With MC, `tiles` holds units of two tiles (num_tiles units) and the grid is
// made of clusters of four CTAs (two pairs).
template <bool B_MN, class Epi, bool RING = false, bool MC = false, bool F8 = false>
int launch_pair_gemm(const CUtensorMap& mA, const CUtensorMap& mB, int nkb, const int2* tiles, int num_tiles,
                     const Epi& epi, int32_t* status, cudaStream_t st, const tc::RingArgs& ring = tc::RingArgs{}) {
    using namespace tc2;
    auto kern = tc_gemm_pair_kernel<B_MN, Epi, RING, MC, F8>;
    const int threads = threads_of(RING);
    constexpr int cluster = MC ? 4 : 2;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[2];
    pair_launch_config(cfg, attr, st, threads, RING, cluster);
    // every cluster resident at once: the tile loop assumes it
    int max_clusters = 0;
    SOS_CHECK(per_device_value((const void*)kern, &max_clusters, [kern, threads](int* v) -> int {
        return resident_pairs((const void*)kern, threads, v, cluster);
    }));
    if (num_tiles <= 0) return SOS_OK;
    // the ring's producers wait for every CTA's builders: the whole persistent
    // grid runs even when there are fewer tiles than pairs
    const int clusters = RING ? max_clusters : (num_tiles < max_clusters ? num_tiles : max_clusters);
    cfg.gridDim = dim3(cluster * clusters);
    const char* name = Epi::kName;
    if constexpr (RING) name = Epi::kRingName;
    if constexpr (F8) name = Epi::kF8Name;
    {
        KernelScope ks_(name, st);
        SOS_CUDA(cudaLaunchKernelEx(&cfg, kern, mA, mB, nkb, tiles, num_tiles, epi, status, ring));
    }
    return SOS_OK;
}

}  // namespace

int adjoint_pair_capacity(int* pairs) {
    // the tile lists are cut for the grid of the adjoint that sos_step runs
    const bool ring = use_h_ring();
    const void* kern = ring ? (const void*)tc2::tc_gemm_pair_kernel<true, tc::UpdateEpilogue, true>
                            : (const void*)tc2::tc_gemm_pair_kernel<true, tc::UpdateEpilogue, false>;
    const int threads = tc2::threads_of(ring);
    return per_device_value(kern, pairs, [kern, threads](int* v) -> int { return resident_pairs(kern, threads, v); });
}

int launch_tc_forward_pair(const sos_plan_s* p, const void* a16, float* c, int32_t* status, cudaStream_t st,
                           const float* diag) {
    using namespace tc2;
    CUtensorMap mA, mB;
    SOS_CHECK(make_bf16_map(&mA, a16, p->r, p->N, p->ld16, BK, BM));
    SOS_CHECK(make_bf16_map(&mB, a16, p->r, p->N, p->ld16, BK, BN / 2));
    tc::SegmentSumEpilogue epi{(int)p->N, p->dev.idx, p->ld_idx, c, diag};
    if (use_mcast())
        return launch_pair_gemm<false, tc::SegmentSumEpilogue, false, true>(
            mA, mB, (int)ceil_div(p->r, BK), p->dev.fwd_units, p->dev.num_fwd_units, epi, status, st);
    return launch_pair_gemm<false>(mA, mB, (int)ceil_div(p->r, BK), p->dev.fwd_tiles2, p->dev.num_fwd_tiles2, epi,
                                   status, st);
}

int launch_tc_adjoint_update_pair(const sos_plan_s* p, const void* h16, const void* a16_cur, void* a16_next,
                                  float* A, float* m, float* v, int optimizer, int64_t t, double lr, double b1,
                                  double b2, double eps, int32_t* status, cudaStream_t st) {
    using namespace tc2;
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, h16, p->N, p->N, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16_cur, p->r, p->N, p->ld16, 64, BK));
    tc::UpdateEpilogue epi;
    epi.rows = (int)p->N;
    epi.cols = (int)p->r;
    epi.optimizer = optimizer;
    epi.lr = (float)lr;
    epi.b1 = (float)b1;
    epi.b2 = (float)b2;
    epi.eps = (float)eps;
    epi.c1 = (float)(1.0 - std::pow(b1, (double)t));
    epi.c2 = (float)(1.0 - std::pow(b2, (double)t));
    epi.A = A;
    epi.m = m;
    epi.v = v;
    epi.a16_next = static_cast<__nv_bfloat16*>(a16_next);
    epi.ld16 = p->ld16;
    if (use_mcast())
        return launch_pair_gemm<true, tc::UpdateEpilogue, false, true>(
            mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_units, p->dev.num_adj_units, epi, status, st);
    return launch_pair_gemm<true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles2, p->dev.num_adj_tiles2, epi,
                                  status, st);
}

namespace {

tc::RingArgs ring_args(const sos_plan_s* p, const float* resid, void* ring, uint32_t* flags) {
    const RingGeometry g = ring_geometry(p);
    tc::RingArgs a;
    a.idx = p->dev.idx;
    a.ld_idx = p->ld_idx;
    a.resid = resid;
    a.ring = static_cast<__nv_bfloat16*>(ring);
    a.ldh = p->ld16h;
    a.N = (int)p->N;
    a.S = g.slots;
    a.first_panel = g.band;
    a.num_panels = g.panels;
    a.panel_tiles = p->dev.panel_tiles;
    a.flags = flags;
    return a;
}

}  // namespace

int launch_tc_adjoint_update_ring_pair(const sos_plan_s* p, const float* resid, void* ring, uint32_t* flags,
                                       const void* a16_cur, void* a16_next, float* A, float* m, float* v,
                                       int optimizer, int64_t t, double lr, double b1, double b2, double eps,
                                       int32_t* status, cudaStream_t st) {
    using namespace tc2;
    const tc::RingArgs ra = ring_args(p, resid, ring, flags);
    SOS_CHECK(tc::launch_ring_prologue(ra, p->dev.num_sms, st));
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, ring, p->N, (uint64_t)ra.S * PAIR_M, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16_cur, p->r, p->N, p->ld16, 64, BK));
    tc::UpdateEpilogue epi;
    epi.rows = (int)p->N;
    epi.cols = (int)p->r;
    epi.optimizer = optimizer;
    epi.lr = (float)lr;
    epi.b1 = (float)b1;
    epi.b2 = (float)b2;
    epi.eps = (float)eps;
    epi.c1 = (float)(1.0 - std::pow(b1, (double)t));
    epi.c2 = (float)(1.0 - std::pow(b2, (double)t));
    epi.A = A;
    epi.m = m;
    epi.v = v;
    epi.a16_next = static_cast<__nv_bfloat16*>(a16_next);
    epi.ld16 = p->ld16;
    return launch_pair_gemm<true, tc::UpdateEpilogue, true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles2,
                                                            p->dev.num_adj_tiles2, epi, status, st, ra);
}

int launch_tc_adjoint_ring_pair(const sos_plan_s* p, const float* resid, void* ring, uint32_t* flags,
                                const void* a16, float* grad, int32_t* status, cudaStream_t st) {
    using namespace tc2;
    const tc::RingArgs ra = ring_args(p, resid, ring, flags);
    SOS_CHECK(tc::launch_ring_prologue(ra, p->dev.num_sms, st));
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, ring, p->N, (uint64_t)ra.S * PAIR_M, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16, p->r, p->N, p->ld16, 64, BK));
    tc::StoreEpilogue epi{(int)p->N, (int)p->r, p->r, 2.0f, grad};
    return launch_pair_gemm<true, tc::StoreEpilogue, true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles2,
                                                           p->dev.num_adj_tiles2, epi, status, st, ra);
}

int launch_tc_adjoint_pair(const sos_plan_s* p, const void* h16, const void* a16, float* grad, int32_t* status,
                           cudaStream_t st) {
    using namespace tc2;
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, h16, p->N, p->N, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16, p->r, p->N, p->ld16, 64, BK));
    tc::StoreEpilogue epi{(int)p->N, (int)p->r, p->r, 2.0f, grad};
    if (use_mcast())
        return launch_pair_gemm<true, tc::StoreEpilogue, false, true>(
            mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_units, p->dev.num_adj_units, epi, status, st);
    return launch_pair_gemm<true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles2, p->dev.num_adj_tiles2, epi,
                                  status, st);
}

// Tensor maps of the stacked slices: bf16 rows of 64-element atoms, or E4M3
// bytes of 128-element atoms (128 bytes either way); nkb = K blocks of one row.
static int slice_maps(const sos_plan_s* p, const SliceFormat& f, const void* S, int64_t NP, CUtensorMap* mA,
                      CUtensorMap* mB, int* nkb) {
    using namespace tc2;
    const int64_t rows = (int64_t)f.max_slices * NP;
    if (f.fp8) {
        SOS_CHECK(make_u8_map(mA, S, p->r, rows, f.ld, 2 * BK, BM));
        SOS_CHECK(make_u8_map(mB, S, p->r, rows, f.ld, 2 * BK, BN / 2));
        *nkb = (int)ceil_div(p->r, 2 * BK);
    } else {
        SOS_CHECK(make_bf16_map(mA, S, p->r, rows, f.ld, BK, BM));
        SOS_CHECK(make_bf16_map(mB, S, p->r, rows, f.ld, BK, BN / 2));
        *nkb = (int)ceil_div(p->r, BK);
    }
    return SOS_OK;
}

int launch_tc_slices_pair(const sos_plan_s* p, const SliceFormat& f, const void* S, int64_t NP, const int2* tiles,
                          int num_tiles, const int32_t* ex, double* c, int32_t* status, cudaStream_t st) {
    CUtensorMap mA, mB;
    int nkb = 0;
    SOS_CHECK(slice_maps(p, f, S, NP, &mA, &mB, &nkb));
    tc::SliceSumEpilogue epi{(int)p->N, (int)NP, p->dev.idx, p->ld_idx, c, ex, f.bits};
    if (f.fp8)
        return launch_pair_gemm<false, tc::SliceSumEpilogue, false, false, true>(mA, mB, nkb, tiles, num_tiles, epi,
                                                                                  status, st);
    return launch_pair_gemm<false>(mA, mB, nkb, tiles, num_tiles, epi, status, st);
}

int launch_tc_slice_groups_pair(const sos_plan_s* p, const SliceFormat& f, const void* S, int64_t NP,
                                const int2* tiles, int num_tiles, const void* groups, const int32_t* ex, double* c,
                                int32_t* status, cudaStream_t st) {
    CUtensorMap mA, mB;
    int nkb = 0;
    SOS_CHECK(slice_maps(p, f, S, NP, &mA, &mB, &nkb));
    tc::SliceGroupEpilogue epi{(int)p->N, (int)NP, (int)(NP / 256), p->dev.idx, p->ld_idx, c, ex,
                               static_cast<const SliceGroup*>(groups), f.bits};
    if (f.fp8)
        return launch_pair_gemm<false, tc::SliceGroupEpilogue, false, false, true>(mA, mB, nkb, tiles, num_tiles,
                                                                                    epi, status, st);
    return launch_pair_gemm<false>(mA, mB, nkb, tiles, num_tiles, epi, status, st);
}

int diag_gemm_pair(int b_mn_major, const void* X, const void* Y, float* D, int64_t m, int64_t n, int64_t k,
                   int64_t ldx, int64_t ldy, const int2* tiles, int num_tiles, int32_t* status, cudaStream_t st) {
    using namespace tc2;
    CUtensorMap mA, mB;
    SOS_CHECK(make_bf16_map(&mA, X, k, m, ldx, BK, BM));
    if (b_mn_major)
        SOS_CHECK(make_bf16_map(&mB, Y, n, k, ldy, 64, BK));
    else
        SOS_CHECK(make_bf16_map(&mB, Y, k, n, ldy, BK, BN / 2));
    tc::DiagEpilogue epi;
    epi.rows = (int)m;
    epi.cols = (int)n;
    epi.ld = n;
    epi.scale = 1.0f;
    epi.out = D;
    return b_mn_major ? launch_pair_gemm<true>(mA, mB, (int)ceil_div(k, BK), tiles, num_tiles, epi, status, st)
                      : launch_pair_gemm<false>(mA, mB, (int)ceil_div(k, BK), tiles, num_tiles, epi, status, st);
}

}  // namespace sos
