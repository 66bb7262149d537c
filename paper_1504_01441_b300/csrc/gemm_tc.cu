// Row a-L: dense bfloat16 contractions on the fifth-generation tensor cores.
//
// C[M x N] = A[M x K] * B[N x K]^T with A and B bfloat16, K contiguous (K-major),
// accumulated in FP32. Every convolution of the displacement predictor is one such
// product: forward = im2col(x) * W^T, data gradient = dY * (W^T)^T, weight gradient =
// im2col(x)^T * dY^T (split over K, partial sums reduced in a fixed order).
//
// One CTA computes a 128 x BN tile (BN = 16..128). Tiles of A (128 x 64) and B
// (BN x 64) move by TMA with 128-byte swizzle into a four-stage ring (full / empty
// mbarriers); one thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16)
// into a TMEM accumulator of BN columns and commits each stage back to the
// producer; after the last stage all four warps read their 32 TMEM lanes with
// tcgen05.ld and apply the epilogue. Every wait is bounded: a timeout sets the
// error word, the CTA still frees its TMEM and returns.
#include <cuda_bf16.h>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kBM = 128, kBK = 64, kStages = 4, kGemmThreads = 128;
constexpr uint32_t kGemmWaitIters = 1u << 22;

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity)
{
    for (uint32_t i = 0; i < kGemmWaitIters; i++) {
        if (bar_try(b, parity)) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
        "{%2, %3}], [%4];" ::"r"(s32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(s32(b))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with 128-byte
// swizzle: rows of 64 bf16 (128 bytes), 8-row atoms 1024 bytes apart (stride byte
// offset), descriptor version 1, layout "128-byte swizzle".
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, both K-major.
template <int BN>
constexpr uint32_t idesc_bf16()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     s32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_bf16(const __grid_constant__ CUtensorMap mapA,
                                                               const __grid_constant__ CUtensorMap mapB,
                                                               int M, int N, int K, int k_split,
                                                               GemmEpi epi, int* err)
{
    constexpr int kCols = BN < 32 ? 32 : BN;  // TMEM columns (a power of two >= 32)
    constexpr uint32_t kBytesA = kBM * kBK * 2, kBytesB = BN * kBK * 2;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int bad;
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sA = base;
    uint8_t* sB = base + kStages * kBytesA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kbeg = blockIdx.z * k_split;
    const int kend = min(K, kbeg + k_split);
    const int KT = kend > kbeg ? (kend - kbeg + kBK - 1) / kBK : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) {
            bar_init(&full[s]);
            bar_init(&empty[s]);
        }
        bar_init(&done);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         s32(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {  // producer
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % kStages;
            if (kt >= kStages && !bar_wait(&empty[s], ((kt / kStages) - 1) & 1)) {
                bad = 1;
                break;
            }
            bar_expect(&full[s], kBytesA + kBytesB);
            tma_2d(sA + s * kBytesA, &mapA, kbeg + kt * kBK, m0, &full[s]);
            tma_2d(sB + s * kBytesB, &mapB, kbeg + kt * kBK, n0, &full[s]);
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % kStages;
            if (!bar_wait(&full[s], (kt / kStages) & 1)) {
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = desc_sw128(s32(sA + s * kBytesA));
            const uint64_t db = desc_sw128(s32(sB + s * kBytesB));
#pragma unroll
            for (int k = 0; k < kBK / 16; k++)  // +32 bytes along K = +2 in the address field
                mma_bf16(tmem, da + 2 * k, db + 2 * k, idesc_bf16<BN>(), (kt | k) != 0);
            mma_commit(&empty[s]);
        }
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = bar_wait(&done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        if (row < M && ok && !bad) {
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int col = n0 + c0 + j;
                if (col >= N) break;
                float v = KT > 0 ? __uint_as_float(r[j]) : 0.f;
                const size_t o = (size_t)row * epi.ldc + col;
                if (epi.mode == kEpiF32) {
                    epi.out[(size_t)blockIdx.z * epi.split_stride + o] = v;
                } else if (epi.mode == kEpiBiasF32) {
                    epi.out[o] = v + epi.bias[col];
                } else {  // kEpiBiasReluBf16
                    v += epi.bias[col];
                    epi.out_bf16[o] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
    }
    if (threadIdx.x == 0 && (!ok || bad)) atomicExch(err, 1);
}

// 2D tensor map over a rows x cols bf16 matrix (cols contiguous, row stride ld elements),
// boxes of 64 columns x box_rows rows, 128-byte swizzle, zero fill outside.
bool make_bf16_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows)
{
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int BN>
size_t gemm_smem()
{
    return 1024 + (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2);
}

template <int BN>
bool launch_bn(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, int splits,
               int k_split, const GemmEpi& epi, int* err, cudaStream_t s)
{
    const size_t smem = gemm_smem<BN>();
    ensure_smem((const void*)k_gemm_bf16<BN>, smem);
    dim3 grid((M + kBM - 1) / kBM, (N + BN - 1) / BN, splits);
    note_launch();
    k_gemm_bf16<BN><<<grid, kGemmThreads, smem, s>>>(a, b, M, N, K, k_split, epi, err);
    return true;
}

}  // namespace

int gemm_bn_for(int N)
{
    if (N <= 16) return 16;
    if (N <= 32) return 32;
    if (N <= 64) return 64;
    return 128;
}

bool gemm_supported(const void* A, int lda, const void* B, int ldb)
{
    return tensor_map_encoder() != nullptr && ((uintptr_t)A & 15u) == 0 &&
           ((uintptr_t)B & 15u) == 0 && (lda % 8) == 0 && (ldb % 8) == 0;
}

bool launch_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                      int splits, const GemmEpi& epi, int* err, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0 || splits < 1) return false;
    if (!gemm_supported(A, lda, B, ldb)) return false;
    const int BN = gemm_bn_for(N);
    int k_split = (K + splits - 1) / splits;
    k_split = (k_split + kBK - 1) / kBK * kBK;
    splits = (K + k_split - 1) / k_split;
    CUtensorMap ma, mb;
    if (!make_bf16_map(&ma, A, M, K, lda, kBM)) return false;
    if (!make_bf16_map(&mb, B, N, K, ldb, BN)) return false;
    switch (BN) {
    case 16: return launch_bn<16>(ma, mb, M, N, K, splits, k_split, epi, err, s);
    case 32: return launch_bn<32>(ma, mb, M, N, K, splits, k_split, epi, err, s);
    case 64: return launch_bn<64>(ma, mb, M, N, K, splits, k_split, epi, err, s);
    default: return launch_bn<128>(ma, mb, M, N, K, splits, k_split, epi, err, s);
    }
}

int gemm_splits_used(int K, int splits)
{
    int k_split = (K + splits - 1) / splits;
    k_split = (k_split + kBK - 1) / kBK * kBK;
    return (K + k_split - 1) / k_split;
}

}  // namespace hdrreg
