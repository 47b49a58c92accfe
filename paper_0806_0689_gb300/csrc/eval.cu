// eval.cu -- motion compensation and the six measures of Sec. IV on sm_103a.
//
// The prediction of pixel (x, y) of block k is ref(x + dx_k, y + dy_k).  The
// kernel accumulates exact integer sums per frame: sum |e|, sum e^2, sum of
// search points, number of blocks whose MV equals the FS MV, and the sum of
// round(2^24 * |mv - mv_fs|).  Integer atomics make the sums independent of
// scheduling.  The ratios and the PSNR are formed on the host.
//
// Mapping: one item = one B-pixel row segment of one block.  Consecutive
// threads take consecutive blocks of the same pixel row, so a warp reads 32
// neighbouring segments of cur (one coalesced span) and of ref.  Each thread
// walks many items (grid-stride) and the CTA reduces once at the end.  An MV
// that moves its block out of the frame is not compensated; its pixels are
// left out of ME_SUM_PIXELS and of the error sums.
#include "me_internal.cuh"

#include <algorithm>

namespace me {
namespace {

template <int B>
__global__ void __launch_bounds__(256) eval_kernel(const EvalDev* __restrict__ frames,
                                                   unsigned long long* __restrict__ sums)
{
    constexpr int BW = B / 4;  // words per segment
    const EvalDev& F = frames[blockIdx.y];
    unsigned long long* out = sums + (size_t)blockIdx.y * 8;
    const int nbx = F.nbx, W = F.w, H = F.h, P = F.pitch;
    const int total = F.h * nbx;  // (pixel row, block column) items
    const uint32_t* mvw = reinterpret_cast<const uint32_t*>(F.mv);
    const uint32_t* fsw = reinterpret_cast<const uint32_t*>(F.mv_fs);

    unsigned long long s_abs = 0, s_sq = 0, s_nsp = 0, s_eq = 0, s_dist = 0, s_pix = 0;
    constexpr int U = 4;  // items per thread per trip: their loads are issued together
    const int stride = gridDim.x * blockDim.x;
    for (int it0 = blockIdx.x * blockDim.x + threadIdx.x; it0 < total; it0 += U * stride) {
        uint32_t m[U];
        int yv[U], bxv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int it = it0 + u * stride;
            const int itc = it < total ? it : it0;
            yv[u] = itc / nbx;
            bxv[u] = itc - yv[u] * nbx;
            m[u] = __ldg(mvw + (yv[u] / B) * nbx + bxv[u]);
        }
        uint32_t c[U][BW], wv[U][BW + 1];
        bool okv[U];
        long gv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int y = yv[u], bx = bxv[u], by = y / B;
            const int dx = (int)(int16_t)(m[u] & 0xffffu), dy = (int)(int16_t)(m[u] >> 16);
            const int x = bx * B;
            okv[u] = (it0 + u * stride < total) && x + dx >= 0 && x + dx <= W - B && by * B + dy >= 0 &&
                     by * B + dy <= H - B;
            gv[u] = (long)(y + dy) * P + x + dx;
            if (okv[u]) {
                const uint8_t* cp = F.cur + (size_t)y * P + x;
                if constexpr (BW == 4) {
                    const uint4 v = __ldg(reinterpret_cast<const uint4*>(cp));
                    c[u][0] = v.x; c[u][1] = v.y; c[u][2] = v.z; c[u][3] = v.w;
                } else {
                    const uint2 v = __ldg(reinterpret_cast<const uint2*>(cp));
                    c[u][0] = v.x; c[u][1] = v.y;
                }
                const uint32_t* rp = reinterpret_cast<const uint32_t*>(F.ref + (gv[u] & ~3l));
#pragma unroll
                for (int i = 0; i < BW; ++i) wv[u][i] = __ldg(rp + i);
                // the word after the segment is read only when the segment is unaligned,
                // and then it still lies inside the row
                wv[u][BW] = (gv[u] & 3) ? __ldg(rp + BW) : 0u;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (it0 + u * stride >= total) continue;
            const int y = yv[u], bx = bxv[u], by = y / B, r = y - by * B;
            const int k = by * nbx + bx;
            const int dx = (int)(int16_t)(m[u] & 0xffffu), dy = (int)(int16_t)(m[u] >> 16);
            if (okv[u]) {
                const unsigned sh = (unsigned)(gv[u] & 3) * 8u;
                uint32_t a = 0, q = 0;
#pragma unroll
                for (int i = 0; i < BW; ++i) {
                    const uint32_t d = __vabsdiffu4(c[u][i], __funnelshift_r(wv[u][i], wv[u][i + 1], sh));
                    a = __dp4a(d, 0x01010101u, a);
                    q = __dp4a(d, d, q);
                }
                s_abs += a;
                s_sq += q;
                s_pix += B;
            }
            if (r == 0) {
                if (F.nsp) s_nsp += F.nsp[k];
                if (fsw) {
                    const uint32_t fw = __ldg(fsw + k);
                    const int ex = dx - (int)(int16_t)(fw & 0xffffu), ey = dy - (int)(int16_t)(fw >> 16);
                    if (ex == 0 && ey == 0) s_eq += 1;
                    else s_dist += dist_q24(ex, ey);
                }
            }
        }
    }
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
        out[5] = (unsigned long long)F.nbx * F.nby;
        out[7] = F.mv_fs ? 1ull : 0ull;
    }
}

}  // namespace

cudaError_t launch_eval(const EvalDev* frames, int nframes, int block, int max_blocks, int num_sms,
                        unsigned long long* sums, cudaStream_t st)
{
    // enough CTAs to fill the GPU a few times over, and at least ~16 items per thread
    const long items = (long)max_blocks * block;
    const long by_items = (items + 256 * 32 - 1) / (256 * 32);
    const long by_gpu = (long)num_sms * 8 / std::max(nframes, 1) + 1;
    int gx = (int)std::max(1l, std::min(by_items, by_gpu));
    dim3 grid(gx, nframes);
    if (block == 16) eval_kernel<16><<<grid, 256, 0, st>>>(frames, sums);
    else eval_kernel<8><<<grid, 256, 0, st>>>(frames, sums);
    return cudaGetLastError();
}

}  // namespace me
