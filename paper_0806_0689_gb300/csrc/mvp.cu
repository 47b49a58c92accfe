// mvp.cu -- motion-vector probability statistics of Sec. II-C over full-search
// fields (the counts behind Tables II-V): the 2-D histogram of the global
// best-matched points (the FS motion vectors), the prior distribution D1 of
// eq. (4) -- the global BMP given the current BMP found in the first-step
// point set S1 of CDS (the cross of radius 2) -- and the posterior
// distribution D2 of eq. (6) -- the current BMP in the 5x5 square S2 given the
// global BMP.  Counts are exact integers (atomics); the ratios, the folded
// tables and the fits are host arithmetic.
//
// One warp per block: lane l holds 8 current pixels (row l / 2, half l % 2);
// each candidate's SAD is two byte-SIMD differences per lane and a warp sum.
// The current BMP of a set is its strict minimum with the points compared in
// the set's order (the centre first), over the points inside the search window
// and the frame.
#include "me_internal.cuh"

#include <algorithm>

namespace me {
namespace {

// S1: the centre, then the CDS first step as printed in Sec. II-C-2.
__constant__ int8_t kS1[9][2] = {{0, 0}, {-2, 0}, {-1, 0}, {1, 0}, {2, 0}, {0, 2}, {0, 1}, {0, -1}, {0, -2}};

__device__ __forceinline__ uint32_t warp_sad16(const EvalDev& F, int px, int py, int dx, int dy, uint32_t c0,
                                               uint32_t c1, int lane)
{
    const int r = lane >> 1, hh = lane & 1;
    const long g = (long)(py + dy + r) * F.pitch + px + dx + 8 * hh;
    const uint32_t* wp = reinterpret_cast<const uint32_t*>(F.ref + (g & ~3l));
    const unsigned sh = (unsigned)(g & 3) * 8u;
    const uint32_t w0 = __ldg(wp), w1 = __ldg(wp + 1);
    const uint32_t w2 = sh ? __ldg(wp + 2) : 0u;  // inside the row whenever the segment is unaligned
    uint32_t s = sadacc<kSadVariant>(__funnelshift_r(w0, w1, sh), c0, 0u);
    s = sadacc<kSadVariant>(__funnelshift_r(w1, w2, sh), c1, s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// frames[i].mv holds the FS field; ranges[i] the frame's search range.
__global__ void __launch_bounds__(256) mvp_kernel(const EvalDev* __restrict__ frames, const int* __restrict__ ranges,
                                                  const long* __restrict__ bases, int nframes, long total, int R,
                                                  unsigned long long* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int side = 2 * R + 1, nq = side * side;
    unsigned long long* hist = out;
    unsigned long long* d1 = out + nq;
    unsigned long long* d2 = out + 10 * (size_t)nq;
    const long nwarps = (long)gridDim.x * (blockDim.x >> 5);
    for (long b = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); b < total; b += nwarps) {
        int f = 0;
        {
            int lo = 0, hi = nframes - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bases[mid] <= b) lo = mid; else hi = mid - 1;
            }
            f = lo;
        }
        const EvalDev& F = frames[f];
        const int Rf = ranges[f];
        const int k = (int)(b - bases[f]);
        const int px = (k % F.nbx) * 16, py = (k / F.nbx) * 16;
        const int dxlo = max(-Rf, -px), dxhi = min(Rf, F.w - 16 - px);
        const int dylo = max(-Rf, -py), dyhi = min(Rf, F.h - 16 - py);
        const uint32_t q = __ldg(reinterpret_cast<const uint32_t*>(F.mv) + k);
        const int qx = (int)(int16_t)(q & 0xffffu), qy = (int)(int16_t)(q >> 16);
        const uint32_t* cp = reinterpret_cast<const uint32_t*>(F.cur + (size_t)(py + (lane >> 1)) * F.pitch + px +
                                                               8 * (lane & 1));
        const uint32_t c0 = __ldg(cp), c1 = __ldg(cp + 1);
        // current BMP in S1 (the centre is always a candidate)
        const uint32_t s0 = warp_sad16(F, px, py, 0, 0, c0, c1, lane);
        int p1 = 0;
        uint32_t b1 = s0;
        for (int i = 1; i < 9; ++i) {
            const int dx = kS1[i][0], dy = kS1[i][1];
            if (dx < dxlo || dx > dxhi || dy < dylo || dy > dyhi) continue;
            const uint32_t s = warp_sad16(F, px, py, dx, dy, c0, c1, lane);
            if (s < b1) { b1 = s; p1 = i; }
        }
        // current BMP in S2: the centre, then the 5x5 square row by row
        int p2 = 12;
        uint32_t b2 = s0;
        for (int i = 0; i < 25; ++i) {
            if (i == 12) continue;
            const int dx = i % 5 - 2, dy = i / 5 - 2;
            if (dx < dxlo || dx > dxhi || dy < dylo || dy > dyhi) continue;
            const uint32_t s = warp_sad16(F, px, py, dx, dy, c0, c1, lane);
            if (s < b2) { b2 = s; p2 = i; }
        }
        if (lane == 0 && qx >= -R && qx <= R && qy >= -R && qy <= R) {
            const int qi = (qy + R) * side + (qx + R);
            atomicAdd(hist + qi, 1ull);
            atomicAdd(d1 + (size_t)p1 * nq + qi, 1ull);
            atomicAdd(d2 + (size_t)qi * 25 + p2, 1ull);
        }
    }
}

}  // namespace

cudaError_t launch_mvp(const EvalDev* frames, const int* ranges, const long* bases, int nframes, long total, int R,
                       int num_sms, unsigned long long* out, cudaStream_t st)
{
    const int grid = (int)std::min<long>((total + 7) / 8, (long)num_sms * 16);
    mvp_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>(frames, ranges, bases, nframes, total, R, out);
    return cudaGetLastError();
}

}  // namespace me
