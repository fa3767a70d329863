// Tensor-core trailing update of the u_f LU on sm_103a: C[M x N] (FP32) -= A[M x K] B[K x N]
// with bf16/fp16 operands, FP32 accumulation in tensor memory (tcgen05).
//
// Operands are K-major in global memory: A = L21 rows of the stored factor (row-major, K
// contiguous) and Bt = U12^T (N x K, K contiguous, written by the TRSM). TMA copies 128-byte
// swizzled tiles (64 elements of K) into a 2-stage shared-memory ring; one thread issues
// tcgen05.mma (M = 128, N = 256, K = 16 per instruction) into a 128 x 256 FP32 accumulator in
// tensor memory; tcgen05.commit arrives on the stage's "empty" barrier so TMA can refill it.
// Two CTAs share an SM (2 x 256 of the 512 TMEM columns).
// The epilogue (4 warps, one TMEM lane quarter each) reads the accumulator with tcgen05.ld
// and subtracts it from C. Every mbarrier wait is bounded; a timeout raises a device flag.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "k_lu.cuh"

namespace gir {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;                   // one 128-byte swizzle atom of 16-bit elements
constexpr int STAGES = 2;                // ~100 KB shared memory: two CTAs per SM, so one
                                         // CTA's epilogue overlaps the other's main loop
constexpr int A_BYTES = BM * BK * 2;     // 16 KB
constexpr int B_BYTES = BN * BK * 2;     // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int THREADS = 128;
constexpr int TMEM_COLS = 256;
constexpr long long WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// bounded wait on the given phase parity; returns false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    uint32_t addr = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}
// K-major operand, 128-byte swizzle: rows of 128 B, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    uint64_t addr = smem_u32(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;
    d |= (uint64_t)(16 >> 4) << 16;     // leading-dimension byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset between 8-row groups
    d |= (uint64_t)1 << 46;             // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// instruction descriptor: D = F32, A = B = bf16 (fmt 1) or f16 (fmt 0), both K-major, M = 128, N = 256
__host__ __device__ constexpr uint32_t make_idesc(int bf16) {
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

__global__ void __launch_bounds__(THREADS, 2)
k_tc_gemm_sub(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float* __restrict__ Cm,
              int64_t ldc, int M, int N, int K, uint32_t idesc, int* __restrict__ flags) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the stage buffers (required by the 128-byte swizzle pattern)
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;
    unsigned char* sB = base + STAGES * A_BYTES;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_s = reinterpret_cast<int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int nk = (K + BK - 1) / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (kb >= STAGES) {
                if (!mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) { atomicExch(abort_s, 1); break; }
            }
            if (*(volatile int*)abort_s) break;
            mbar_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(sA + s * A_BYTES, &mapA, &full[s], kb * BK, m0);
            tma_load_2d(sB + s * B_BYTES, &mapB, &full[s], kb * BK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % STAGES;
            if (!mbar_wait(&full[s], (kb / STAGES) & 1)) { atomicExch(abort_s, 1); break; }
            if (*(volatile int*)abort_s) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t ad = smem_desc(sA + s * A_BYTES);
            const uint64_t bd = smem_desc(sB + s * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                // advance 16 elements (32 bytes) along K inside the swizzle atom
                mma_f16(tmem, ad + (uint64_t)((kk * 32) >> 4), bd + (uint64_t)((kk * 32) >> 4), idesc,
                        (kb > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    }
    __syncwarp();
    // epilogue: wait for the accumulator, then C -= acc (warp w owns TMEM lanes 32w..32w+31)
    bool ok = mbar_wait(done, 0);
    ok = __all_sync(0xffffffffu, ok && !*(volatile int*)abort_s);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(flags, DEV_TIMEOUT);
    } else {
        const int row = m0 + warp * 32 + lane;
        float* crow = Cm + (int64_t)row * ldc;
#pragma unroll 1
        for (int cb = 0; cb < BN / 32; ++cb) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int c0 = n0 + cb * 32;
            if (row < M) {
                if (c0 + 32 <= N && ((reinterpret_cast<uintptr_t>(crow + c0) & 15) == 0)) {
                    float4* p = reinterpret_cast<float4*>(crow + c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 c = p[q];
                        c.x -= __uint_as_float(v[4 * q + 0]);
                        c.y -= __uint_as_float(v[4 * q + 1]);
                        c.z -= __uint_as_float(v[4 * q + 2]);
                        c.w -= __uint_as_float(v[4 * q + 3]);
                        p[q] = c;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q)
                        if (c0 + q < N) crow[c0 + q] -= __uint_as_float(v[q]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;

}  // namespace tc

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 lookup_encode() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
}
static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encode();   // thread-safe one-time init
    return fn;
}

// 2-D K-major map: rows x k (k contiguous), row pitch ld elements, box {64, box_rows}.
static bool encode_map(CUtensorMap* map, const uint16_t* base, int64_t rows, int64_t k, int64_t ld, int box_rows,
                       int fmt) {
    auto enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, fmt == FF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<uint16_t*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool tc_gemm_supported(int64_t M, int64_t N, int64_t K, int64_t lda, int64_t ldb, int64_t ldc) {
    (void)ldc;
    if (M <= 0 || N <= 0 || K <= 0) return false;
    if (lda % 8 != 0 || ldb % 8 != 0) return false;  // 16-byte row pitch for TMA
    if (M > (1LL << 31) || N > (1LL << 31)) return false;
    return get_encode() != nullptr;
}

gir_status launch_tc_gemm_sub(float* C, int64_t ldc, const uint16_t* A, int64_t lda, const uint16_t* Bt, int64_t ldbt,
                              int64_t M, int64_t N, int64_t K, int fmt, int* flags, cudaStream_t s) {
    if (((uintptr_t)A & 15) || ((uintptr_t)Bt & 15)) return GIR_UNSUPPORTED;
    CUtensorMap ma, mb;
    if (!encode_map(&ma, A, M, K, lda, tc::BM, fmt) || !encode_map(&mb, Bt, N, K, ldbt, tc::BN, fmt))
        return GIR_UNSUPPORTED;
    static std::atomic<unsigned> attr_done{0};
    GIR_CUDA_TRY(ensure_dyn_smem((const void*)tc::k_tc_gemm_sub, (int)tc::SMEM_BYTES, attr_done));
    dim3 grid((unsigned)((N + tc::BN - 1) / tc::BN), (unsigned)((M + tc::BM - 1) / tc::BM));
    count_launch(), tc::k_tc_gemm_sub<<<grid, tc::THREADS, tc::SMEM_BYTES, s>>>(ma, mb, C, ldc, (int)M, (int)N, (int)K,
                                                                tc::make_idesc(fmt == FF_BF16 ? 1 : 0), flags);
    GIR_CUDA_TRY(cudaGetLastError());
    return GIR_OK;
}

}  // namespace gir
