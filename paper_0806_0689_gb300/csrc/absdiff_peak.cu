// absdiff_peak.cu -- measures how many byte absolute differences per second
// the SMs sustain with each encoding of the 4-byte SIMD sum of absolute
// differences (me::sadacc).  The best measured rate is the compute roofline
// of the SAD kernels (full search is bound by it; DCDS is compared with it).
//
// Each thread keeps 16 independent accumulators over 8 changing operands:
// per loop trip, 32 accumulations (128 byte-absdiffs) and 8 operand updates
// that stop the compiler from hoisting anything out of the loop.
#include "me_internal.cuh"

namespace me {
namespace {

template <int V>
__global__ void __launch_bounds__(256) absdiff_peak_kernel(int iters, unsigned* __restrict__ sink)
{
    uint32_t x[8], y[4], acc[16];
    const uint32_t seed = 0x9e3779b9u * (blockIdx.x * blockDim.x + threadIdx.x + 1u);
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed ^ (0x01234567u * (i + 1));
#pragma unroll
    for (int i = 0; i < 4; ++i) y[i] = seed * (2u * i + 3u);
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j & 15] = sadacc<V>(x[j & 7], y[(j >> 3) & 3], acc[j & 15]);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] += 0x01010101u;
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += acc[i];
    if (s == 0x7fffffffu) sink[0] = s;  // keeps the work alive; practically never stores
}

}  // namespace

cudaError_t launch_absdiff_peak(int variant, int iters, int blocks, int threads, unsigned* sink,
                                cudaStream_t st)
{
    switch (variant) {
    case SAD_VSADU4: absdiff_peak_kernel<SAD_VSADU4><<<blocks, threads, 0, st>>>(iters, sink); break;
    case SAD_PTX_ADD: absdiff_peak_kernel<SAD_PTX_ADD><<<blocks, threads, 0, st>>>(iters, sink); break;
    case SAD_DP4A: absdiff_peak_kernel<SAD_DP4A><<<blocks, threads, 0, st>>>(iters, sink); break;
    case SAD_MINMAX: absdiff_peak_kernel<SAD_MINMAX><<<blocks, threads, 0, st>>>(iters, sink); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace me
