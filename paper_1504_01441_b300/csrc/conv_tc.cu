// Row a-L, inference: the predictor's 3x3 convolutions as implicit GEMMs on the
// fifth-generation tensor cores, with no im2col matrix in memory.
//
// out[m][co] = relu(b[co] + sum_k A[m][k] W[co][k]) for output pixel m and
// k = (ky * 3 + kx) * CIN + c, A[m][k] = x(s i + ky - 1, s j + kx - 1, c) (0 outside).
// A small kernel first writes the layer's weights (FP32 parameters rounded to bfloat16)
// as the shared-memory image the MMA reads: 128-byte-swizzled K-major blocks of 64 K.
// Then persistent CTAs (one or two per SM) walk 128-pixel tiles with warp roles:
//  * warps 0-7 gather A: each 16-byte chunk (8 channels of one tap of one pixel) is one
//    cp.async (L1-cached: the nine taps of neighbouring pixels overlap) with zero fill
//    for taps outside the image, written at its swizzled place in a six-stage ring;
//    copy groups complete four K blocks behind the issue front, and each producer
//    fences the async proxy before it arrives on the stage's barrier;
//  * one thread of warp 8 issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16) into
//    one of two TMEM accumulators and commits each stage back to the producers;
//  * warps 9-12 read their 32 TMEM lanes and write bias + ReLU as bfloat16 while the
//    MMAs of the next tile fill the other accumulator.
// The weights arrive by bulk copy into shared memory once per CTA and stay there. Every wait is
// bounded: a timeout sets the error word; producers drain their copies and the CTA
// frees its TMEM before it returns.
#include <cuda_bf16.h>

#include "hdrreg_internal.cuh"

namespace hdrreg {

namespace {

constexpr int kCM = 128, kCK = 64, kCStages = 6, kLag = 4;
constexpr int kProducers = 256, kConvThreads = kProducers + 32 + 128;
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
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes)
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

// Weights of a layer as the convolution kernel's shared-memory image: KT blocks of
// BN rows x 64 K (bfloat16, 128-byte rows, 128-byte swizzle), k = (ky * 3 + kx) * CIN + c,
// zero past the layer's K and cin_src.
// All layers' images in one launch: blockIdx.y = layer (runtime shapes).
__global__ void k_pack_conv_all(ConvPack p)
{
    const int l = blockIdx.y;
    const int CIN = p.cin[l], BN = p.cout[l], cin_src = p.cin_src[l];
    const int KT = (9 * CIN + kCK - 1) / kCK;
    const float* __restrict__ W = p.W[l];
    uint4* __restrict__ img = reinterpret_cast<uint4*>(p.img[l]);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < KT * BN * 8;
         e += gridDim.x * blockDim.x) {
        const int j = e & 7, n = (e >> 3) % BN, kt = (e >> 3) / BN;
        uint32_t packed[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            float v2[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int k = kt * kCK + j * 8 + 2 * q + u;
                const int tap = k / CIN, c = k - tap * CIN;
                v2[u] = (tap < 9 && c < cin_src) ? W[((size_t)n * 9 + tap) * cin_src + c] : 0.f;
            }
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v2[0], v2[1]);
            packed[q] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        img[(kt * BN * 128 + swz(n, j)) / 16] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
}

// Persistent CTAs over 128-pixel tiles. Warps 0-7 gather A, warp 8 (one thread) issues
// the MMAs, warps 9-12 drain the accumulator: two TMEM accumulators, so the MMAs of the
// next tile run while the previous one is written out.
template <int CIN, int STRIDE, int BN>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv3x3(const __nv_bfloat16* __restrict__ x, int h, int w, int ho, int wo, int M,
              const uint4* __restrict__ wimg, int cout, const float* __restrict__ bias,
              __nv_bfloat16* __restrict__ out, int* err)
{
    constexpr int K = 9 * CIN, KT = (K + kCK - 1) / kCK;
    constexpr int kCols = 2 * BN <= 32 ? 32 : (2 * BN <= 64 ? 64 : 128);
    constexpr uint32_t kBytesA = kCM * kCK * 2, kBytesB = BN * kCK * 2;
    static_assert(CIN % 8 == 0 && kBytesB % 1024 == 0 && BN <= 64, "layout");
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kCStages], empty[kCStages], tfull[2], tempty[2], done, wbar;
    __shared__ uint32_t tmem_base;
    __shared__ int bad;
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint8_t* sB = base;                       // KT blocks of BN x 64, resident
    uint8_t* sA = base + KT * kBytesB;        // kCStages blocks of 128 x 64
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (M + kCM - 1) / kCM;

    if (tid == 0) {
        for (int s = 0; s < kCStages; s++) {
            cbar_init(&full[s], kProducers);
            cbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; a++) {
            cbar_init(&tfull[a], 1);
            cbar_init(&tempty[a], 4);
        }
        cbar_init(&done, 1);
        cbar_init(&wbar, 1);
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
    __syncthreads();  // barriers initialized
    if (tid == 0) {   // the weight image: bulk copies of at most 16 KB onto one barrier
        constexpr uint32_t kW = KT * kBytesB;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(&wbar)),
                     "r"(kW)
                     : "memory");
        for (uint32_t o = 0; o < kW; o += 16384) {
            const uint32_t n = kW - o < 16384 ? kW - o : 16384;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
                "[%3];" ::"r"(sa(sB + o)),
                "l"(reinterpret_cast<const uint8_t*>(wimg) + o), "r"(n), "r"(sa(&wbar))
                : "memory");
        }
    }
    if (!cbar_wait(&wbar, 0)) bad = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (bad) {  // the weights did not arrive in time: wait once more (bounded) so that no
                // copy is left in flight, free the TMEM and return
        if (tid == 0) {
            atomicExch(err, 1);
            cbar_wait(&wbar, 0);
        }
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                         "r"(kCols)
                         : "memory");
        return;
    }

    if (warp < kProducers / 32) {
        // producers: chunk j of rows r = tid / 8 + kRowStep i (i < kRowsPer) of every K
        // block; per tile and row the element offset of the tap (0, 0) pixel and a 9-bit
        // mask of the taps inside the image
        constexpr int kRowStep = kProducers / 8, kRowsPer = kCM / kRowStep;
        const int j = tid & 7;
        const uint32_t swz0 = (uint32_t)((tid >> 3) * 128 + ((j ^ ((tid >> 3) & 7)) << 4));
        int off[kRowsPer];
        uint32_t vmask[kRowsPer];
        bool ok = true;
        int g = 0;  // K blocks issued by this CTA
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int m0 = tile * kCM;
#pragma unroll
            for (int i = 0; i < kRowsPer; i++) {
                const int m = m0 + (tid >> 3) + kRowStep * i;
                const int mm = m < M ? m : 0;
                const int ox = mm % wo, t = mm / wo, oy = t % ho, b = t / ho;
                const int iy0 = STRIDE * oy - 1, ix0 = STRIDE * ox - 1;
                off[i] = ((b * h + iy0) * w + ix0) * CIN;
                const uint32_t rv = (uint32_t)(iy0 >= 0) | 2u | ((uint32_t)(iy0 + 2 < h) << 2);
                const uint32_t cv = (uint32_t)(ix0 >= 0) | 2u | ((uint32_t)(ix0 + 2 < w) << 2);
                const uint32_t rm = ((rv & 1u) ? 0x7u : 0u) | ((rv & 4u) ? 0x1C0u : 0u) | 0x38u;
                vmask[i] = m < M ? (rm & (cv * 0x49u)) : 0u;
            }
            for (int kt = 0; kt < KT; kt++, g++) {
                const int s = g % kCStages;
                if (ok && g >= kCStages && !cbar_wait(&empty[s], ((g / kCStages) - 1) & 1)) {
                    ok = false;
                    bad = 1;
                }
                if (ok) {
                    const int k = kt * kCK + j * 8;
                    const int tap = k / CIN, c = k - tap * CIN;
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const uint32_t tbit = tap < 9 ? 1u << tap : 0u;
                    const int toff = (ky * w + kx) * CIN + c;
                    const uint32_t dst0 = sa(sA + s * kBytesA) + swz0;
#pragma unroll
                    for (int i = 0; i < kRowsPer; i++) {
                        const bool in = (vmask[i] & tbit) != 0;
                        cp16(dst0 + (uint32_t)(i * kRowStep * 128), x + (in ? off[i] + toff : 0),
                             in ? 16u : 0u);
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (g >= kLag) {
                    asm volatile("cp.async.wait_group %0;" ::"n"(kLag) : "memory");
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (ok) cbar_arrive(&full[(g - kLag) % kCStages]);
                }
            }
        }
        // the last kLag blocks
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int q = g - kLag < 0 ? 0 : g - kLag; q < g; q++)
            if (ok) cbar_arrive(&full[q % kCStages]);
    } else if (warp == kProducers / 32) {
        if (lane == 0) {  // MMA issuer
            int g = 0, i = 0;
            for (int tile = blockIdx.x; tile < ntiles && !bad; tile += gridDim.x, i++) {
                const int acc = i & 1;
                if (i >= 2 && !cbar_wait(&tempty[acc], ((i >> 1) - 1) & 1)) {
                    bad = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)(acc * BN);
                for (int kt = 0; kt < KT; kt++, g++) {
                    const int s = g % kCStages;
                    if (!cbar_wait(&full[s], (g / kCStages) & 1)) {
                        bad = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = cdesc_sw128(sa(sA + s * kBytesA));
                    const uint64_t db = cdesc_sw128(sa(sB + kt * kBytesB));
#pragma unroll
                    for (int k = 0; k < kCK / 16; k++) {
                        const uint32_t accum = (kt | k) != 0;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dacc),
                            "l"(da + 2 * k), "l"(db + 2 * k), "r"(cidesc<BN>()), "r"(accum)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            sa(&empty[s]))
                        : "memory");
                }
                if (bad) break;
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        sa(&tfull[acc]))
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    sa(&done))
                : "memory");
            if (!cbar_wait(&done, 0)) bad = 1;
        }
        __syncwarp();
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 = tile rows of that range
        const int q4 = warp & 3;
        int i = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, i++) {
            const int acc = i & 1;
            bool ok = !bad && cbar_wait(&tfull[acc], (i >> 1) & 1);
            if (!ok) {
                bad = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int row = tile * kCM + q4 * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                    "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * BN + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M && c0 < cout) {
                    uint32_t packed[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int col = c0 + 2 * q;
                        const float v0 = __uint_as_float(r[2 * q]) + bias[col];
                        const float v1 = __uint_as_float(r[2 * q + 1]) + bias[col + 1];
                        const __nv_bfloat162 b2 =
                            __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
                        packed[q] = *reinterpret_cast<const uint32_t*>(&b2);
                    }
                    uint4* o = reinterpret_cast<uint4*>(out + (size_t)row * cout + c0);
                    o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
                    o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) cbar_arrive(&tempty[acc]);
        }
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

template <int CIN, int BN>
constexpr size_t conv_wimg_bytes()
{
    return (size_t)((9 * CIN + kCK - 1) / kCK) * BN * kCK * 2;
}

template <int CIN, int STRIDE, int BN>
void launch_one(const ConvArgs& a, cudaStream_t s)
{
    const uint4* img = reinterpret_cast<const uint4*>(a.wimg);
    const size_t smem = conv_smem<CIN, STRIDE, BN>();
    ensure_smem((const void*)k_conv3x3<CIN, STRIDE, BN>, smem);
    const int ntiles = (a.M + kCM - 1) / kCM;
    const int per_sm = smem <= 110 * 1024 ? 2 : 1;
    const int grid = ntiles < 148 * per_sm ? ntiles : 148 * per_sm;
    note_launch();
    k_conv3x3<CIN, STRIDE, BN><<<grid, kConvThreads, smem, s>>>(
        a.x, a.h, a.w, a.ho, a.wo, a.M, img, a.cout, a.bias, a.out, a.err);
}

}  // namespace

size_t conv_wimg_size(int cin, int cout)
{
    return (size_t)((9 * cin + kCK - 1) / kCK) * cout * kCK * 2;
}

void launch_pack_conv(const ConvPack& p, cudaStream_t s)
{
    if (p.layers <= 0) return;
    note_launch();
    k_pack_conv_all<<<dim3(8, p.layers), 256, 0, s>>>(p);
}

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
