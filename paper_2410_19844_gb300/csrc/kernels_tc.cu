// Tensor-core (tcgen05 / TMEM / TMA) kernels for the BF16 stage.
//
//   forward  G = A A^T over the upper-triangle tiles only; the epilogue
//            segment-sums every G_ab with b >= a into c[idx(a, b)] with weight
//            1 on the diagonal and 2 above it (Eq. 1 with B = A A^T).
//   adjoint  grad = 2 H(r) A (the chain rule of Eq. 2) with H[a][b] = r[idx(a, b)]
//            stored in bf16 by build_h16.
//
// One persistent CTA per SM (192 threads) walks a tile list:
//   warp 0, one lane : TMA producer, 4-stage ring of 48 KB (A 128x64, B 256x64)
//   warp 1, one lane : tcgen05.mma issuer, M = 128, N = 256, K = 16 per step
//   warps 2-5        : epilogue; each reads its 32 TMEM lanes (warp % 4)
// TMEM holds two 128 x 256 FP32 accumulators (512 columns), so the epilogue
// of one tile overlaps the mainloop of the next.  Operands are staged with the
// 128-byte swizzle; A is K-major, B is K-major (forward: rows of A) or
// MN-major (adjoint: the bf16 copy of A read as [b][k] with k contiguous).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cmath>

#include "internal.h"
#include "tc_epilogues.cuh"
#include "tc_ptx.cuh"

namespace sos {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;             // 16 KB
constexpr int B_BYTES = BN * BK * 2;             // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;   // 48 KB
constexpr int BAR_BYTES = 256;
constexpr int EPI_WARPS = 4;
constexpr int EPI_STAGE_BYTES = EPI_WARPS * STAGE_FLOATS * 4;   // transposition buffers
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + BAR_BYTES + EPI_STAGE_BYTES;
constexpr int THREADS = 192;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait, then give up

// ---- the GEMM core ---------------------------------------------------------------

template <bool B_MN_MAJOR, class Epilogue>
__global__ void __launch_bounds__(THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int nkb,
               const int2* __restrict__ tiles, int num_tiles, Epilogue epi, int32_t* __restrict__ status) {
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
    float* epi_stage = reinterpret_cast<float*>(base + STAGES * STAGE_BYTES + BAR_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4);
        }
        mbar_init(drain, 1);
        *err = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
        int s = 0;
        uint32_t ph = 0;
        int64_t issued = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            const int2 tile = tiles[t];
            for (int kb = 0; kb < nkb; ++kb) {
                if (*err || !mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(sA + s * A_BYTES, &mapA, &full[s], kb * BK, tile.x * BM);
                if (B_MN_MAJOR) {
#pragma unroll
                    for (int j = 0; j < BN / 64; ++j)
                        tma_load_2d(sB + s * B_BYTES + j * (64 * BK * 2), &mapB, &full[s], tile.y * BN + 64 * j,
                                    kb * BK);
                } else {
                    tma_load_2d(sB + s * B_BYTES, &mapB, &full[s], kb * BK, tile.y * BN);
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
        }
        // Let every copy this thread started land before the CTA can exit.
        for (int64_t i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
            mbar_wait(&full[i % STAGES], (uint32_t)((i / STAGES) & 1), WAIT_LIMIT_NS);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        constexpr uint32_t idesc = idesc_bf16_f32(BM, BN, 0, B_MN_MAJOR ? 1 : 0);
        int s = 0;
        uint32_t ph = 0;
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x, ++it) {
            const int buf = it & 1;
            const uint32_t tph = (uint32_t)(it >> 1) & 1u;
            if (*err || !mbar_wait(&tempty[buf], tph ^ 1u, WAIT_LIMIT_NS)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t dtm = tmem_base + (uint32_t)(buf * BN);
            for (int kb = 0; kb < nkb; ++kb) {
                if (*err || !mbar_wait(&full[s], ph, WAIT_LIMIT_NS)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA + s * A_BYTES);
                const uint32_t b_addr = smem_u32(sB + s * B_BYTES);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint64_t ad = smem_desc_sw128(a_addr + kk * 32, 16, 1024);
                    const uint64_t bd = B_MN_MAJOR ? smem_desc_sw128(b_addr + kk * 16 * 128, 64 * BK * 2, 1024)
                                                   : smem_desc_sw128(b_addr + kk * 32, 16, 1024);
                    umma_bf16(dtm, ad, bd, idesc, (kb | kk) != 0 ? 1u : 0u);
                }
                umma_commit(&empty[s]);
                if (++s == STAGES) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            umma_commit(&tfull[buf]);
        }
        if (!ok) {
            *err = 1;
            atomicCAS(status, 0, SOS_E_TIMEOUT);
        }
        // Every MMA this thread issued is complete before TMEM is released.
        umma_commit(drain);
        mbar_wait(drain, 0, WAIT_LIMIT_NS);
    } else if (warp >= 2) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;   // TMEM lane quarter this warp may read
        int it = 0;
        for (int t = blockIdx.x; t < num_tiles; t += gridDim.x, ++it) {
            const int buf = it & 1;
            const uint32_t tph = (uint32_t)(it >> 1) & 1u;
            const bool ready = (*err == 0) && mbar_wait(&tfull[buf], tph, WAIT_LIMIT_NS);
            if (!__all_sync(0xffffffffu, ready)) {
                if (lane == 0) {
                    *err = 1;
                    atomicCAS(status, 0, SOS_E_TIMEOUT);
                }
                break;
            }
            tc_fence_after();
            const int2 tile = tiles[t];
            float* stage = epi_stage + (warp - 2) * STAGE_FLOATS;
#pragma unroll 1
            for (int ch = 0; ch < BN / 32; ++ch) {
                uint32_t v[32];
                tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + ch * 32), v);
                tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) stage[stage_idx(lane, j)] = __uint_as_float(v[j]);
                __syncwarp();
                epi(tile.x * BM + q * 32, tile.y * BN + ch * 32, stage, lane);
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[buf]);
        }
    }
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---- host side -----------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

}  // namespace tc

// bf16 matrix of `outer` rows x `inner` columns, row stride ld elements,
// 128-byte swizzle, zero fill outside the matrix.
int make_bf16_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld,
                  uint32_t box_inner, uint32_t box_outer) {
    using namespace tc;
    auto fn = encode_fn();
    if (!fn) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15))
        return fail(SOS_E_INVALID, "tensor map: base or row stride not 16-byte aligned");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SOS_OK;
}

// uint8 matrix (the E4M3 slices) of `outer` rows x `inner` bytes, row stride
// ld bytes, 128-byte swizzle, zero fill outside the matrix.
int make_u8_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_inner,
                uint32_t box_outer) {
    using namespace tc;
    auto fn = encode_fn();
    if (!fn) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld & 15))
        return fail(SOS_E_INVALID, "tensor map: base or row stride not 16-byte aligned");
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(SOS_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SOS_OK;
}

namespace tc {

template <bool B_MN, class Epi>
static int launch_gemm(const CUtensorMap& mA, const CUtensorMap& mB, int nkb, const int2* tiles, int num_tiles,
                       int num_sms, const Epi& epi, int32_t* status, cudaStream_t st) {
    auto kern = tc_gemm_kernel<B_MN, Epi>;
    int configured = 0;
    SOS_CHECK(per_device_value((const void*)kern, &configured, [kern](int* v) -> int {
        SOS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        *v = 1;
        return SOS_OK;
    }));
    if (num_tiles <= 0) return SOS_OK;
    const int grid = num_tiles < num_sms ? num_tiles : num_sms;
    {
        KernelScope ks_(Epi::kName, st);
        kern<<<grid, THREADS, SMEM_BYTES, st>>>(mA, mB, nkb, tiles, num_tiles, epi, status);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

}  // namespace tc

int launch_tc_forward(const sos_plan_s* p, const void* a16, float* c, int32_t* status, cudaStream_t st) {
    using namespace tc;
    CUtensorMap mA, mB;
    SOS_CHECK(make_bf16_map(&mA, a16, p->r, p->N, p->ld16, BK, BM));
    SOS_CHECK(make_bf16_map(&mB, a16, p->r, p->N, p->ld16, BK, BN));
    SegmentSumEpilogue epi{(int)p->N, p->dev.idx, p->ld_idx, c};
    return launch_gemm<false>(mA, mB, (int)ceil_div(p->r, BK), p->dev.fwd_tiles, p->dev.num_fwd_tiles,
                              p->dev.num_sms, epi, status, st);
}

int launch_tc_adjoint(const sos_plan_s* p, const void* h16, const void* a16, float* grad, int32_t* status,
                      cudaStream_t st) {
    using namespace tc;
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, h16, p->N, p->N, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16, p->r, p->N, p->ld16, 64, BK));
    StoreEpilogue epi{(int)p->N, (int)p->r, p->r, 2.0f, grad};
    return launch_gemm<true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles, p->dev.num_adj_tiles,
                             p->dev.num_sms, epi, status, st);
}

int launch_tc_adjoint_update(const sos_plan_s* p, const void* h16, const void* a16_cur, void* a16_next, float* A,
                             float* m, float* v, int optimizer, int64_t t, double lr, double b1, double b2,
                             double eps, int32_t* status, cudaStream_t st) {
    using namespace tc;
    CUtensorMap mH, mA;
    SOS_CHECK(make_bf16_map(&mH, h16, p->N, p->N, p->ld16h, BK, BM));
    SOS_CHECK(make_bf16_map(&mA, a16_cur, p->r, p->N, p->ld16, 64, BK));
    UpdateEpilogue epi;
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
    return launch_gemm<true>(mH, mA, (int)ceil_div(p->N, BK), p->dev.adj_tiles, p->dev.num_adj_tiles,
                             p->dev.num_sms, epi, status, st);
}

}  // namespace sos

// ---- diagnostic: a bounded wait that runs out ------------------------------------------

namespace sos {
namespace tc {

// One thread waits, with the same bounded mbarrier wait the GEMM roles use, on
// a barrier that nothing arrives at; when the limit passes it records
// SOS_E_TIMEOUT and the kernel returns normally.
__global__ void bounded_wait_kernel(uint64_t limit_ns, int32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait(&bar, 0, limit_ns)) atomicCAS(status, 0, SOS_E_TIMEOUT);
    }
}

}  // namespace tc
}  // namespace sos

extern "C" int sos_diag_bounded_wait(uint64_t limit_ns, int32_t* status, void* stream) {
    using namespace sos;
    if (!status || limit_ns > 5000000000ull) return fail(SOS_E_INVALID, "sos_diag_bounded_wait: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    {
        KernelScope ks_("bounded_wait", st);
        tc::bounded_wait_kernel<<<1, 32, 0, st>>>(limit_ns, status);
    }
    SOS_CUDA(cudaGetLastError());
    return SOS_OK;
}

// ---- diagnostic entry point: a plain tcgen05 BF16 GEMM ------------------------------

extern "C" int sos_diag_gemm_bf16(int mode, const void* X, const void* Y, float* D, int64_t m, int64_t n, int64_t k,
                                  int64_t ldx, int64_t ldy, int32_t* status, void* stream) {
    using namespace sos;
    using namespace sos::tc;
    if (!X || !Y || !D || !status || m < 1 || n < 1 || k < 1 || m > INT32_MAX || n > INT32_MAX ||
        k > INT32_MAX || (mode & ~3))
        return fail(SOS_E_INVALID, "sos_diag_gemm_bf16: bad argument");
    const int b_mn_major = mode & 1;
    const bool pairs = (mode & 2) != 0;
    int dev = 0, sms = 0;
    SOS_CUDA(cudaGetDevice(&dev));
    SOS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tm = pairs ? 256 : BM;
    const int TI = (int)ceil_div(m, tm), TJ = (int)ceil_div(n, BN);
    std::vector<int2> tiles;
    for (int i = 0; i < TI; ++i)
        for (int j = 0; j < TJ; ++j) tiles.push_back(make_int2(i, j));
    int2* d_tiles = nullptr;
    SOS_CUDA(cudaMalloc(&d_tiles, tiles.size() * sizeof(int2)));
    cudaStream_t st = (cudaStream_t)stream;
    int rc = SOS_OK;
    cudaError_t e = cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "sos_diag_gemm_bf16: copy tiles");
    if (rc == SOS_OK && pairs) {
        rc = diag_gemm_pair(b_mn_major, X, Y, D, m, n, k, ldx, ldy, d_tiles, (int)tiles.size(), status, st);
    } else if (rc == SOS_OK) {
        CUtensorMap mA, mB;
        rc = make_bf16_map(&mA, X, k, m, ldx, BK, BM);
        if (rc == SOS_OK)
            rc = b_mn_major ? make_bf16_map(&mB, Y, n, k, ldy, 64, BK) : make_bf16_map(&mB, Y, k, n, ldy, BK, BN);
        DiagEpilogue epi;
        epi.rows = (int)m;
        epi.cols = (int)n;
        epi.ld = n;
        epi.scale = 1.0f;
        epi.out = D;
        if (rc == SOS_OK)
            rc = b_mn_major ? launch_gemm<true>(mA, mB, (int)ceil_div(k, BK), d_tiles, (int)tiles.size(), sms, epi,
                                                status, st)
                            : launch_gemm<false>(mA, mB, (int)ceil_div(k, BK), d_tiles, (int)tiles.size(), sms, epi,
                                                 status, st);
    }
    e = cudaStreamSynchronize(st);
    if (rc == SOS_OK && e != cudaSuccess) rc = cuda_fail(e, "sos_diag_gemm_bf16: run");
    cudaFree(d_tiles);
    return rc;
}
