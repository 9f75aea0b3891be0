// H(r) in bf16 for the tensor-core adjoint: H[a][b] = r[idx(a, b)] (the
// residual gathered through the index table; chain rule of Eq. 2).
//
// H is symmetric, so each 64 x 64 tile on or above the diagonal is built once
// and stored twice, as itself and as its transpose.  The work reads the upper
// half of the index table and writes all of H from HBM, and gathers r (L1/L2
// resident) 4096 times per tile.  It is staged through shared memory with TMA
// in both directions:
//   * a persistent grid walks the upper-triangle tiles row by row; thread 0
//     loads the next tile's index block (64 x 64 int32, 16 KB) with a TMA
//     tile load while the block works on the current one;
//   * each warp gathers 4 x 8 patches of the tile: entries (a, b) and
//     (a + 1, b - 1) often share the monomial a + b, so a compact patch touches
//     about half the 32-byte sectors of r that a 1 x 32 row does;
//   * the bf16 tile and its transpose go to two 128-byte-swizzled smem tiles,
//     which thread 0 stores with TMA tile stores (out-of-range rows and
//     columns are clipped by the tensor map).
// Every mbarrier wait is bounded; a block that gives up sets the status word
// to SOS_E_TIMEOUT and leaves.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "h_ring.cuh"
#include "internal.h"
#include "tc_epilogues.cuh"
#include "tc_ptx.cuh"

namespace sos {

namespace {

using namespace tc;

constexpr int TILE = 64;
constexpr int THREADS = 256;
constexpr int IDX_BYTES = TILE * TILE * 4;     // 16 KB per index block
constexpr int IDX_STAGES = 2;                  // index blocks in flight: one tile ahead
constexpr int H_BYTES = TILE * TILE * 2;       // 8 KB each: the tile and its transpose
constexpr int BAR_OFFSET = IDX_STAGES * IDX_BYTES + 2 * H_BYTES;
constexpr int SMEM_BYTES = BAR_OFFSET + 1024 + 64;
constexpr int BLOCKS_PER_SM = 4;
constexpr int PER_THREAD = TILE * TILE / THREADS;   // 16: one 4 x 8 patch per warp each
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(src)), "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Until at most N committed store groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Shared-memory writes of the threads become visible to the TMA (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Byte offset of element (row, col) in a 64 x 64 bf16 tile stored with the
// 128-byte swizzle of the tensor map: the 16-byte chunk index within each
// 128-byte row is XORed with row % 8 (tile base 1024-byte aligned).
__device__ __forceinline__ uint32_t sw128_offset(int row, int col) {
    const uint32_t cb = (uint32_t)col * 2;
    return (uint32_t)row * 128 + ((((cb >> 4) ^ (uint32_t)(row & 7)) << 4) | (cb & 15));
}

// Upper-triangle tile t (row-major: row I holds tiles J = I .. T-1) -> (I, J).
__device__ __forceinline__ int2 upper_tile(int64_t t, int T) {
    const double b = 2.0 * T + 1.0;
    int I = (int)floor((b - sqrt(b * b - 8.0 * (double)t)) * 0.5);
    auto start = [T](int i) { return (int64_t)i * T - (int64_t)i * (i - 1) / 2; };
    if (I < 0) I = 0;
    while (I > 0 && start(I) > t) --I;
    while (I + 1 < T && start(I + 1) <= t) ++I;
    return make_int2(I, I + (int)(t - start(I)));
}

__global__ void __launch_bounds__(THREADS)
build_h16_tma_kernel(const __grid_constant__ CUtensorMap map_idx, const __grid_constant__ CUtensorMap map_h,
                     const float* __restrict__ resid, int T, int32_t* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    uint8_t* base = smem_raw + (((raw_addr + 1023u) & ~1023u) - raw_addr);
    uint8_t* sh = base + IDX_STAGES * IDX_BYTES;
    uint8_t* sht = sh + H_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + BAR_OFFSET);
    volatile int* stop = reinterpret_cast<volatile int*>(full + IDX_STAGES);

    const int64_t total = (int64_t)T * (T + 1) / 2;
    if (threadIdx.x == 0) {
        for (int i = 0; i < IDX_STAGES; ++i) mbar_init(&full[i], 1);
        *stop = 0;
        fence_mbar_init();
        tma_prefetch_desc(&map_idx);
        tma_prefetch_desc(&map_h);
        for (int i = 0; i + 1 < IDX_STAGES; ++i) {
            const int64_t tn = (int64_t)blockIdx.x + (int64_t)i * gridDim.x;
            if (tn >= total) break;
            const int2 tl = upper_tile(tn, T);
            mbar_arrive_expect_tx(&full[i], IDX_BYTES);
            tma_load_2d(base + i * IDX_BYTES, &map_idx, &full[i], tl.y * TILE, tl.x * TILE);
        }
    }
    __syncthreads();

    // Warp w gathers the 4 x 8 patches in columns 8w .. 8w + 7, rows 4k .. 4k + 3.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = warp * 8 + (lane & 7), row0 = lane >> 3;
    int it = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++it) {
        const int s = it % IDX_STAGES;
        const int32_t* sidx = reinterpret_cast<const int32_t*>(base + s * IDX_BYTES);
        if (threadIdx.x == 0) {
            // tile it + IDX_STAGES - 1 goes to the index buffer that tile it - 1 used
            const int64_t tn = t + (int64_t)(IDX_STAGES - 1) * gridDim.x;
            if (tn < total) {
                const int sn = (it + IDX_STAGES - 1) % IDX_STAGES;
                const int2 tl = upper_tile(tn, T);
                mbar_arrive_expect_tx(&full[sn], IDX_BYTES);
                tma_load_2d(base + sn * IDX_BYTES, &map_idx, &full[sn], tl.y * TILE, tl.x * TILE);
            }
            if (!mbar_wait(&full[s], (uint32_t)(it / IDX_STAGES) & 1u, WAIT_LIMIT_NS)) {
                atomicCAS(status, 0, SOS_E_TIMEOUT);
                *stop = 1;
            }
        }
        __syncthreads();
        if (*stop) {
            // the next index block may still be landing: give it a moment
            if (threadIdx.x == 0) {
                const uint64_t t0 = global_timer_ns();
                while (global_timer_ns() - t0 < 20000) {
                }
            }
            break;
        }
        int g[PER_THREAD];
#pragma unroll
        for (int k = 0; k < PER_THREAD; ++k) g[k] = sidx[(4 * k + row0) * TILE + col];
        float v[PER_THREAD];
#pragma unroll
        for (int k = 0; k < PER_THREAD; ++k) v[k] = __ldg(resid + g[k]);
        // While the gathers are in flight: the previous tile's stores must have
        // read the H tiles before they are written again.
        if (threadIdx.x == 0) bulk_wait_read<0>();
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER_THREAD; ++k) {
            const int row = 4 * k + row0;
            const __nv_bfloat16 hv = __float2bfloat16_rn(v[k]);
            *reinterpret_cast<__nv_bfloat16*>(sh + sw128_offset(row, col)) = hv;
            *reinterpret_cast<__nv_bfloat16*>(sht + sw128_offset(col, row)) = hv;
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int2 tl = upper_tile(t, T);
            tma_store_2d(&map_h, sh, tl.y * TILE, tl.x * TILE);
            if (tl.x != tl.y) tma_store_2d(&map_h, sht, tl.x * TILE, tl.y * TILE);
            bulk_commit();
        }
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of the int32 index table (N x N, row stride ld entries), 64 x 64
// boxes, no swizzle.
int make_idx_map(CUtensorMap* m, const int32_t* idx, int64_t N, int64_t ld) {
    auto fn = encode_tiled();
    if (!fn) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((reinterpret_cast<uintptr_t>(idx) & 15) || ((ld * 4) & 15))
        return fail(SOS_E_INVALID, "index map: base or row stride not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)N};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {TILE, TILE};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_INT32, 2, const_cast<int32_t*>(idx), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SOS_OK;
}

// First band of the H ring, and the ring's flags zeroed (h_ring.cuh): a grid
// of 8-warp blocks walks the 64 x 64 units of panels 0 .. first_panel - 1,
// each warp 8 rows of a unit.
__global__ void __launch_bounds__(256) ring_prologue_kernel(RingArgs g, int flag_words) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < flag_words; i += stride) g.flags[i] = 0u;
    const int units = g.units_per_panel();
    const int64_t total = (int64_t)g.first_panel * units;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
        const int P = (int)(t / units);
        ring_build_rows<8>(g, P, (int)(t - (int64_t)P * units), 8 * warp, lane);
    }
}

}  // namespace

namespace tc {

int launch_ring_prologue(const RingArgs& g, int num_sms, cudaStream_t st) {
    const int flag_words = kRingFlagsHeader + 2 * g.num_panels;
    const int64_t total = (int64_t)g.first_panel * g.units_per_panel();
    const int64_t want = std::max<int64_t>(total, 1);
    const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms * 8);
    {
        KernelScope ks_("ring_prologue", st);
        ring_prologue_kernel<<<grid, 256, 0, st>>>(g, flag_words);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

}  // namespace tc

int launch_build_h16(const sos_plan_s* p, const float* resid, void* h16, int32_t* status, cudaStream_t st) {
    int configured = 0;
    SOS_CHECK(per_device_value((const void*)build_h16_tma_kernel, &configured, [](int* v) -> int {
        SOS_CUDA(cudaFuncSetAttribute(build_h16_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      SMEM_BYTES));
        *v = 1;
        return SOS_OK;
    }));
    const int64_t T = ceil_div(p->N, TILE);
    if (T > 65535) return fail(SOS_E_UNSUPPORTED, "build_h16: too many tiles");
    CUtensorMap mi, mh;
    SOS_CHECK(make_idx_map(&mi, p->dev.idx, p->N, p->ld_idx));
    SOS_CHECK(make_bf16_map(&mh, h16, p->N, p->N, p->ld16h, TILE, TILE));
    const int64_t total = T * (T + 1) / 2;
    const int64_t cap = (int64_t)p->dev.num_sms * BLOCKS_PER_SM;
    const int grid = (int)(total < cap ? total : cap);
    {
        KernelScope ks_("build_h16", st);
        build_h16_tma_kernel<<<grid, THREADS, SMEM_BYTES, st>>>(mi, mh, resid, (int)T, status);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

}  // namespace sos
