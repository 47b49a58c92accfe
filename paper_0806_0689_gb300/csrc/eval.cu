// eval.cu -- motion compensation and the six measures of Sec. IV on sm_103a.
//
// The prediction of pixel (x, y) of block k is ref(x + dx_k, y + dy_k).  The
// kernel accumulates exact integer sums per frame: sum |e|, sum e^2, sum of
// search points, number of blocks whose MV equals the FS MV, and the sum of
// round(2^24 * |mv - mv_fs|).  Integer atomics make the sums independent of
// scheduling.  The ratios and the PSNR are formed on the host.
#include "me_internal.cuh"

namespace me {
namespace {

template <int B>
__global__ void __launch_bounds__(256) eval_kernel(const EvalDev* __restrict__ frames,
                                                   unsigned long long* __restrict__ sums)
{
    constexpr int BW = B / 4;
    constexpr int ITEMS = B * BW;  // (row, word) items per block
    const EvalDev& F = frames[blockIdx.y];
    unsigned long long* out = sums + (size_t)blockIdx.y * 8;
    const int nb = F.nbx * F.nby;
    const long total = (long)nb * ITEMS;

    unsigned long long s_abs = 0, s_sq = 0, s_nsp = 0, s_eq = 0, s_dist = 0, s_pix = 0;
    for (long it = (long)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += (long)gridDim.x * blockDim.x) {
        const int k = (int)(it / ITEMS);
        const int rem = (int)(it - (long)k * ITEMS);
        const int r = rem / BW, w = rem - r * BW;
        const int bx = k % F.nbx, by = k / F.nbx;
        const uint32_t mvw = __ldg(reinterpret_cast<const uint32_t*>(F.mv) + k);
        const int dx = (int)(int16_t)(mvw & 0xffffu), dy = (int)(int16_t)(mvw >> 16);
        const int x = bx * B + 4 * w, y = by * B + r;
        const bool ok = bx * B + dx >= 0 && bx * B + dx <= F.w - B && by * B + dy >= 0 && by * B + dy <= F.h - B;
        if (ok) {
            const uint32_t c = __ldg(reinterpret_cast<const uint32_t*>(F.cur + (size_t)y * F.pitch + x));
            const long g = (long)(y + dy) * F.pitch + x + dx;
            const long a = g & ~3l;
            const unsigned sh = (unsigned)(g & 3) * 8u;
            const uint32_t lo = __ldg(reinterpret_cast<const uint32_t*>(F.ref + a));
            const uint32_t hi = sh ? __ldg(reinterpret_cast<const uint32_t*>(F.ref + a + 4)) : 0u;
            const uint32_t p = __funnelshift_r(lo, hi, sh);
            const uint32_t ad = __vabsdiffu4(c, p);
            s_abs += __dp4a(ad, 0x01010101u, 0u);
            s_sq += __dp4a(ad, ad, 0u);
            s_pix += 4;
        }
        if (rem == 0) {
            if (F.nsp) s_nsp += F.nsp[k];
            if (F.mv_fs) {
                const uint32_t fw = __ldg(reinterpret_cast<const uint32_t*>(F.mv_fs) + k);
                const int ex = dx - (int)(int16_t)(fw & 0xffffu), ey = dy - (int)(int16_t)(fw >> 16);
                s_eq += (ex == 0 && ey == 0);
                s_dist += (unsigned long long)__double2ll_rn(sqrt((double)(ex * ex + ey * ey)) * 16777216.0);
            }
        }
    }
    // an MV that moves its block out of the frame is not compensated; its
    // pixels are left out of ME_SUM_PIXELS and of the error sums
    unsigned long long v[6] = {s_abs, s_sq, s_nsp, s_eq, s_dist, s_pix};
    __shared__ unsigned long long red[6][8];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 6; ++i) red[i][warp] = v[i];
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned long long a = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) a += red[threadIdx.x][j];
        // sums layout: ABS, SQ, NSP, EQUAL, DIST_Q24, BLOCKS, PIXELS, HAS_FS
        const int slot = threadIdx.x < 5 ? threadIdx.x : 6;
        if (a) atomicAdd(out + slot, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[5] = (unsigned long long)nb;
        out[7] = F.mv_fs ? 1ull : 0ull;
    }
}

}  // namespace

cudaError_t launch_eval(const EvalDev* frames, int nframes, int block, int max_blocks,
                        unsigned long long* sums, cudaStream_t st)
{
    const int items = block * (block / 4);
    long total = (long)max_blocks * items;
    int gx = (int)((total + 255) / 256);
    if (gx > 2048) gx = 2048;
    if (gx < 1) gx = 1;
    dim3 grid(gx, nframes);
    if (block == 16) eval_kernel<16><<<grid, 256, 0, st>>>(frames, sums);
    else eval_kernel<8><<<grid, 256, 0, st>>>(frames, sums);
    return cudaGetLastError();
}

}  // namespace me
