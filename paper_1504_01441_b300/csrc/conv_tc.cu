// Row a-L, inference: the predictor's 3x3 convolutions as implicit GEMMs on the
// fifth-generation tensor cores, with no im2col matrix in memory.
//
// out[m][co] = relu(b[co] + sum_k A[m][k] W[co][k]) for output pixel m and
// k = (ky * 3 + kx) * CIN + c, A[m][k] = x(s i + ky - 1, s j + kx - 1, c) (0 outside).
// One CTA computes 128 output pixels x BN (= cout) channels:
//  * the weights of the layer (FP32 parameters, rounded to bfloat16 here) are written
//    once into shared memory in the 128-byte-swizzled K-major layout the MMA reads,
//    and stay there for every K block;
//  * four producer warps gather A: each 16-byte chunk (8 channels of one tap of one
//    pixel) is one cp.async with zero fill for taps outside the image, written at its
//    swizzled place; groups complete two K blocks behind the issue front, and each
//    producer fences the async proxy before it arrives on the stage's barrier;
//  * one thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16) into a TMEM
//    accumulator and commits each stage back to the producers;
//  * the four producer warps read their 32 TMEM lanes and write bias + ReLU as bfloat16.
// Every wait is bounded: a timeout sets the error word; producers drain their copies and
// the CTA frees its TMEM before it returns.
#include <cuda_bf16.h>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kCM = 128, kCK = 64, kCStages = 4, kLag = 2;
constexpr int kProducers = 128, kConvThreads = kProducers + 32;
constexpr uint32_t kConvWaitIters = 1u << 22;

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void cbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sa(b)) : "memory");
}

__device__ __forceinline__ bool cbar_wait(uint64_t* b, uint32_t parity)
{
    for (uint32_t i = 0; i < kConvWaitIters; i++) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(sa(b)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (i > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t cdesc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

template <int BN>
constexpr uint32_t cidesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(kCM >> 4) << 24);
}

// byte offset of the 16-byte chunk j of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t swz(int r, int j) { return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4)); }

template <int CIN, int STRIDE, int BN>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv3x3(const __nv_bfloat16* __restrict__ x, int h, int w, int ho, int wo, int M,
              const float* __restrict__ W, int cin_src, int cout, const float* __restrict__ bias,
              __nv_bfloat16* __restrict__ out, int* err)
{
    constexpr int K = 9 * CIN, KT = (K + kCK - 1) / kCK;
    constexpr int kCols = BN < 32 ? 32 : (BN <= 32 ? 32 : 64);  // TMEM columns, power of two
    constexpr uint32_t kBytesA = kCM * kCK * 2, kBytesB = BN * kCK * 2;
    static_assert(CIN % 8 == 0 && kBytesB % 1024 == 0 && BN <= 64, "layout");
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kCStages], empty[kCStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ int bad;
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sB = base;                       // KT blocks of BN x 64, resident
    uint8_t* sA = base + KT * kBytesB;        // kCStages blocks of 128 x 64
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kCM;

    if (tid == 0) {
        for (int s = 0; s < kCStages; s++) {
            cbar_init(&full[s], kProducers);
            cbar_init(&empty[s], 1);
        }
        cbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        bad = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         sa(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // resident weights: chunk (row n, block kt, chunk j) = 8 consecutive k of output channel n
    for (int e = tid; e < KT * BN * 8; e += kConvThreads) {
        const int j = e & 7, n = (e >> 3) % BN, kt = (e >> 3) / BN;
        uint32_t packed[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float v2[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int k = kt * kCK + j * 8 + 2 * q + u;
                const int tap = k / CIN, c = k - tap * CIN;
                v2[u] = (n < cout && tap < 9 && c < cin_src) ? W[((size_t)n * 9 + tap) * cin_src + c]
                                                             : 0.f;
            }
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v2[0], v2[1]);
            packed[q] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(sB + kt * kBytesB + swz(n, j)) =
            make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid < kProducers) {
        // this thread's chunk j of rows r = tid / 8 + 16 i, i = 0..7
        const int j = tid & 7;
        long long pix[8];
        int iy0[8], ix0[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int m = m0 + (tid >> 3) + 16 * i;
            if (m < M) {
                const int ox = m % wo, t = m / wo, oy = t % ho, b = t / ho;
                iy0[i] = STRIDE * oy - 1;
                ix0[i] = STRIDE * ox - 1;
                pix[i] = (((long long)b * h + iy0[i]) * w + ix0[i]) * CIN;
            } else {
                iy0[i] = -(1 << 20);  // every tap outside
                ix0[i] = 0;
                pix[i] = 0;
            }
        }
        bool ok = true;
        for (int it = 0; it < KT + kLag; it++) {
            if (it < KT && ok) {
                const int s = it % kCStages;
                if (it >= kCStages && !cbar_wait(&empty[s], ((it / kCStages) - 1) & 1)) {
                    ok = false;
                    bad = 1;
                }
                if (ok) {
                    const int k = it * kCK + j * 8;
                    const int tap = k / CIN, c = k - tap * CIN;
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const uint32_t dst0 = sa(sA + s * kBytesA);
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const int r = (tid >> 3) + 16 * i;
                        const int iy = iy0[i] + ky, ix = ix0[i] + kx;
                        const bool in = tap < 9 && iy >= 0 && iy < h && ix >= 0 && ix < w;
                        const __nv_bfloat16* src =
                            in ? x + pix[i] + ((long long)ky * w + kx) * CIN + c : x;
                        cp16(dst0 + swz(r, j), src, in ? 16u : 0u);
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            const int jb = it - kLag;
            if (jb >= 0 && jb < KT) {
                asm volatile("cp.async.wait_group %0;" ::"n"(kLag) : "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                if (ok) cbar_arrive(&full[jb % kCStages]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (tid == kProducers) {  // MMA issuer
        for (int kt = 0; kt < KT; kt++) {
            const int s = kt % kCStages;
            if (!cbar_wait(&full[s], (kt / kCStages) & 1)) {
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = cdesc_sw128(sa(sA + s * kBytesA));
            const uint64_t db = cdesc_sw128(sa(sB + kt * kBytesB));
#pragma unroll
            for (int k = 0; k < kCK / 16; k++) {
                const uint32_t acc = (kt | k) != 0;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da + 2 * k), "l"(db + 2 * k), "r"(cidesc<BN>()), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    sa(&empty[s]))
                : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                sa(&done))
            : "memory");
    }
    __syncwarp();
    if (tid < kProducers) {
        const bool ok = cbar_wait(&done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M && ok && !bad && c0 < cout) {
                uint32_t packed[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int col = c0 + 2 * q;
                    float v0 = __uint_as_float(r[2 * q]) + bias[col];
                    float v1 = __uint_as_float(r[2 * q + 1]) + bias[col + 1];
                    const __nv_bfloat162 b2 =
                        __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
                    packed[q] = *reinterpret_cast<const uint32_t*>(&b2);
                }
                uint4* o = reinterpret_cast<uint4*>(out + (size_t)row * cout + c0);
                o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
        }
        if (!ok && lane == 0) bad = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
    }
    if (tid == 0 && bad) atomicExch(err, 1);
}

template <int CIN, int STRIDE, int BN>
size_t conv_smem()
{
    constexpr int KT = (9 * CIN + kCK - 1) / kCK;
    return 1024 + (size_t)KT * BN * kCK * 2 + (size_t)kCStages * kCM * kCK * 2;
}

template <int CIN, int STRIDE, int BN>
void launch_one(const ConvArgs& a, cudaStream_t s)
{
    const size_t smem = conv_smem<CIN, STRIDE, BN>();
    ensure_smem((const void*)k_conv3x3<CIN, STRIDE, BN>, smem);
    note_launch();
    k_conv3x3<CIN, STRIDE, BN><<<(a.M + kCM - 1) / kCM, kConvThreads, smem, s>>>(
        a.x, a.h, a.w, a.ho, a.wo, a.M, a.W, a.cin_src, a.cout, a.bias, a.out, a.err);
}

}  // namespace

// The eight 3x3 layers of the predictor: (padded input channels, stride, output channels).
bool launch_conv3x3(const ConvArgs& a, cudaStream_t s)
{
    if (a.M <= 0) return true;
    const int key = a.cin * 1000 + a.stride * 100 + a.cout;
    switch (key) {
    case 32116: launch_one<32, 1, 16>(a, s); return true;
    case 16116: launch_one<16, 1, 16>(a, s); return true;
    case 16232: launch_one<16, 2, 32>(a, s); return true;
    case 32132: launch_one<32, 1, 32>(a, s); return true;
    case 32248: launch_one<32, 2, 48>(a, s); return true;
    case 48148: launch_one<48, 1, 48>(a, s); return true;
    case 48264: launch_one<48, 2, 64>(a, s); return true;
    case 64164: launch_one<64, 1, 64>(a, s); return true;
    default: return false;
    }
}

}  // namespace hdrreg
