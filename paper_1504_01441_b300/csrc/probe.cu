// Measured integer dot-product rate: the denominator of the SSD search's ALU roofline
// (Sec. 2.2's search is 8-bit products summed in 32-bit integers; the kernel issues them
// as __dp4a). Every thread runs `iters` rounds of eight independent chains
// acc_k <- dp4a(acc_k, b + k, acc_k): each product depends on the chain's previous
// value, so the compiler can neither fold nor hoist them, and the eight chains give
// the scheduler independent work. The xor of the chains is compared with a value the
// caller never passes, so the chains stay live and `sink` is written only then.
#include "hdrreg_internal.cuh"

namespace hdrreg {

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

}  // namespace hdrreg

using namespace hdrreg;

extern "C" hdrreg_status hdrreg_probe_dp4a(int blocks, int iters, uint32_t* sink, void* stream)
{
    if (blocks <= 0 || blocks > (1 << 20) || iters <= 0 || iters > (1 << 24))
        return fail(HDRREG_E_INVALID_ARG, "probe_dp4a: blocks in [1, 2^20], iters in [1, 2^24]");
    if (!sink) return fail(HDRREG_E_INVALID_ARG, "probe_dp4a: NULL sink");
    note_launch();
    k_probe_dp4a<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0x03050709u,
                                                                       0xFFFFFFFFu, sink);
    return launch_status("probe_dp4a");
}
