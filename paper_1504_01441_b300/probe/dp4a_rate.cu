// Measurement aid of the benchmark, built as its own library (libhdrreg_probe.so) and
// not part of the registration library or its C ABI.
//
// Measured integer dot-product rate: the denominator of the SSD search's ALU roofline
// (Sec. 2.2's search is 8-bit products summed in 32-bit integers; the search kernel
// issues them as __dp4a). Every thread runs `iters` rounds of eight independent chains
// acc_k <- dp4a(acc_k, b + k, acc_k): each product depends on the chain's previous
// value, so the compiler can neither fold nor hoist them, and the eight chains give
// the scheduler independent work. The xor of the chains is compared with a value the
// caller never passes, so the chains stay live and `sink` is written only then.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__global__ void __launch_bounds__(256) k_probe_dp4a(int iters, uint32_t b, uint32_t never,
                                                    uint32_t* __restrict__ sink)
{
    uint32_t acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = threadIdx.x * 0x01010101u + blockIdx.x + (uint32_t)k;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k] = __dp4a(acc[k], b + (uint32_t)k, acc[k]);
    }
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s ^= acc[k];
    if (s == never) sink[0] = s;
}

}  // namespace

// Enqueue blocks x 256 threads, each issuing 8 * iters __dp4a, on `stream` (a
// cudaStream_t, or NULL for the legacy default stream). sink: device, one uint32.
// Returns 0 when enqueued, 1 for arguments out of range (blocks in [1, 2^20], iters in
// [1, 2^24], sink not NULL; nothing is launched), 2 when the launch failed.
extern "C" int hdrreg_probe_dp4a(int blocks, int iters, uint32_t* sink, void* stream)
{
    if (blocks <= 0 || blocks > (1 << 20) || iters <= 0 || iters > (1 << 24) || !sink) return 1;
    k_probe_dp4a<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0x03050709u,
                                                                       0xFFFFFFFFu, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
