// tc_gemm.cu - BF16 x BF16 -> FP32 matrix products on the 5th-generation
// tensor cores (tcgen05) for the learned warm start and the split-BF16 DFT.
//
//   C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k]  (+ C[b][m][n] if beta)
//
// A and B are row-major with k contiguous ("K-major" operands), bf16; C is
// row-major fp32.  One CTA computes a 128 x BN tile of one batch entry:
//   * one thread streams 128 x 64 tiles of A and BN x 64 tiles of B into a
//     STAGES-deep ring of shared-memory buffers with TMA
//     (cp.async.bulk.tensor, 128-byte swizzle, zero fill past the edges), each
//     buffer guarded by a "full" mbarrier (TMA transaction bytes) and an
//     "empty" mbarrier (tcgen05.commit of the products that read it);
//   * the same thread issues tcgen05.mma (M = 128, N = BN, K = 16 per
//     instruction) with the fp32 accumulator in tensor memory (TMEM);
//   * after the last k tile, all four warps read their 32 accumulator rows
//     back with tcgen05.ld and store them.
// Every wait is bounded: a wait that runs out sets the error word and the CTA
// stops issuing, waits (bounded) for the copies and products it has in
// flight, frees its TMEM and returns.
#include "mm_internal.cuh"

#include <cuda.h>
#include <cstdint>
#include <cstring>

namespace mm {
namespace tc {

constexpr int BM = 128, BK = 64, STAGES = 4, NTHREADS = 128;
constexpr unsigned long long WAIT_LIMIT = 1ull << 24;   // polls of one mbarrier wait

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// true when the phase with the given parity has completed; false after WAIT_LIMIT polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_u32(bar);
    for (unsigned long long i = 0; i < WAIT_LIMIT; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, groups of 8 rows 1024 bytes apart
// (stride byte offset), descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile) {
    const uint64_t addr = smem_u32(tile);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;                 // start address
    d |= (uint64_t)1 << 16;                       // leading byte offset (unused with 128-B swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;             // stride byte offset
    d |= (uint64_t)1 << 46;                       // descriptor version
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}
// Instruction descriptor of kind::f16: D fp32, A and B bf16, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN>
struct Smem {
    static constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int TOTAL = STAGES * STAGE + 1024 /* alignment */ + 256 /* barriers */;
    static constexpr int TMEM_COLS = BN < 32 ? 32 : BN;
};

struct GemmArgs {
    float* c;
    long long ldc, c_batch;      // elements
    int m, n, k;
    float alpha;
    int beta;                    // 1: accumulate into C
    unsigned* err;               // set non-zero when a wait ran out
};

template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b, GemmArgs g) {
    using S = Smem<BN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * S::STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(accum + 1);
    unsigned* abort_flag = tmem_slot + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, bz = blockIdx.z;
    const int nk = (g.k + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // producer and MMA issuer in one thread: TMA runs STAGES tiles ahead
        int issued = 0, committed = 0;
        bool ok = true;
        auto issue = [&](int kb) {
            const int s = kb % STAGES;
            unsigned char* a_dst = smem + s * S::STAGE;
            unsigned char* b_dst = a_dst + S::A_BYTES;
            mbar_expect_tx(&full[s], S::STAGE);
            tma_load_3d(a_dst, &map_a, &full[s], kb * BK, m0, bz);
            tma_load_3d(b_dst, &map_b, &full[s], kb * BK, n0, bz);
        };
        for (; issued < nk && issued < STAGES; ++issued) issue(issued);
        constexpr uint32_t idesc = idesc_bf16(BN);
        for (int kb = 0; kb < nk && ok; ++kb) {
            const int s = kb % STAGES;
            const unsigned ph = (kb / STAGES) & 1;
            if (!mbar_wait(&full[s], ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned char* a_t = smem + s * S::STAGE;
            const unsigned char* b_t = a_t + S::A_BYTES;
            const uint64_t da = smem_desc_sw128(a_t), db = smem_desc_sw128(b_t);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // advance 16 bf16 (32 bytes) along k inside the swizzle atom
                const uint64_t off = (uint64_t)((kk * 32) >> 4);
                const unsigned acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(da + off), "l"(db + off), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
            committed = kb + 1;
            if (issued < nk) {
                // the buffer of stage s is free once the products just issued have read it
                if (!mbar_wait(&empty[s], ph)) { ok = false; break; }
                issue(issued++);
            }
        }
        if (ok) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(accum))
                         : "memory");
        } else {
            // a wait ran out: record it, then let every copy and product in
            // flight land before the shared memory and TMEM are released
            atomicOr(g.err, 1u);
            *abort_flag = 1;
            for (int kb = committed; kb < issued; ++kb) mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1);
            if (committed > 0) {
                const int kb = committed - 1;
                mbar_wait(&empty[kb % STAGES], (kb / STAGES) & 1);
            }
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(accum)) : "memory");
        }
    }
    __syncwarp();
    // epilogue: every warp waits for the accumulator, then reads its 32 rows
    const bool acc_ok = mbar_wait(accum, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!acc_ok && lane == 0) atomicOr(g.err, 2u);
    __syncthreads();
    if (acc_ok && *abort_flag == 0) {
        const int row = m0 + warp * 32 + lane;
        float* crow = g.c + (long long)bz * g.c_batch + (long long)row * g.ldc;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
            unsigned r[32];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.m) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < g.n) {
                        const float v = g.alpha * __uint_as_float(r[j]);
                        crow[col] = g.beta ? crow[col] + v : v;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::TMEM_COLS)
                     : "memory");
    }
}

// ---- host side --------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 3-D map over a bf16 array [batch][rows][k] (row stride ld, batch stride bs,
// in elements), box 64 (k) x box_rows, 128-byte swizzle, zero fill outside
static cudaError_t make_map(CUtensorMap* map, const void* base, int k, int rows, int batch, long long ld,
                            long long bs, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(batch > 1 ? bs : ld * rows) * 2};
    const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
static cudaError_t configure_bn() {
    static bool configured[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Smem<BN>::TOTAL);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    return cudaSuccess;
}

template <int BN>
static cudaError_t launch_bn(const CUtensorMap& ma, const CUtensorMap& mb, const GemmArgs& g, int batch,
                             cudaStream_t s) {
    cudaError_t e = configure_bn<BN>();
    if (e != cudaSuccess) return e;
    const dim3 grid((g.m + BM - 1) / BM, (g.n + BN - 1) / BN, batch);
    k_gemm_bf16<BN><<<grid, NTHREADS, Smem<BN>::TOTAL, s>>>(ma, mb, g);
    return cudaGetLastError();
}

}  // namespace tc

// kernel attributes and the tensor-map encoder, set up once outside any stream
// capture (a step graph may contain the products)
cudaError_t gemm_configure() {
    using namespace tc;
    if (!encode_fn()) return cudaErrorNotSupported;
    cudaError_t e;
    if ((e = configure_bn<32>())) return e;
    if ((e = configure_bn<64>())) return e;
    if ((e = configure_bn<128>())) return e;
    return configure_bn<256>();
}

// C[b] = alpha A[b] B[b]^T (+ C[b] when beta); declared in mm_internal.cuh
cudaError_t gemm_bf16(const void* a, long long lda, long long a_batch, const void* b, long long ldb,
                      long long b_batch, float* c, long long ldc, long long c_batch, int m, int n, int k, int batch,
                      float alpha, int beta, unsigned* err, cudaStream_t s) {
    using namespace tc;
    if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return cudaSuccess;
    // TMA: 16-byte aligned base and row/batch strides
    if ((reinterpret_cast<uintptr_t>(a) & 15) || (reinterpret_cast<uintptr_t>(b) & 15) || (lda & 7) || (ldb & 7) ||
        (batch > 1 && ((a_batch & 7) || (b_batch & 7))) || lda < k || ldb < k)
        return cudaErrorInvalidValue;
    const int bn = n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256;
    CUtensorMap ma, mb;
    cudaError_t e = make_map(&ma, a, k, m, batch, lda, a_batch, BM);
    if (e != cudaSuccess) return e;
    e = make_map(&mb, b, k, n, batch, ldb, b_batch, bn);
    if (e != cudaSuccess) return e;
    GemmArgs g{c, ldc, c_batch, m, n, k, alpha, beta, err};
    switch (bn) {
        case 32: return launch_bn<32>(ma, mb, g, batch, s);
        case 64: return launch_bn<64>(ma, mb, g, batch, s);
        case 128: return launch_bn<128>(ma, mb, g, batch, s);
        default: return launch_bn<256>(ma, mb, g, batch, s);
    }
}

}  // namespace mm
