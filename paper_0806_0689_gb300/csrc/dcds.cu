// dcds.cu -- Directional Cross Diamond Search on sm_103a.
//
// Algorithm: Jia & Zhang, Sec. III-B (steps 1-4, switching strategies one
// and two) with the patterns of Sec. III-A (HCSP, HDSP, VDSP and the middle
// points); DCDS^S of Sec. IV-C as a compile-time variant.
//
// GPU mapping
//   * A CTA owns a tile of tx x ty blocks of one frame.  The reference window
//     the tile can reach (the tile grown by R rows and by R rounded up to 16
//     columns) is staged once in shared memory with 16-byte loads.
//   * One group of G = B/4 lanes searches one block; lane w keeps column w
//     (4 pixels) of the B rows of the current block in registers.  A SAD is
//     B unaligned 4-byte shared-memory reads per lane (two aligned words and
//     a funnel shift), B SIMD absolute-difference accumulations and a
//     log2(G)-step shuffle reduction.
//   * Groups pull blocks of the tile from a shared counter, so a group that
//     stops after the HCSP (the half-way stop) immediately takes another
//     block.  Each group runs a flat state machine: every iteration of the
//     warp loop first advances each group to its next unvisited candidate
//     (pattern transitions, fetching a new block) and then evaluates one SAD
//     for all active groups together, so the SAD code never runs diverged.
//   * Persistent CTAs pull tiles from a global counter (the work queue), so
//     a single launch covers any number of frames of any sizes.
//   * Visited points: one bit per (dx, dy) of the window in a per-group
//     shared-memory bitmap.  A point evaluated earlier always has a SAD no
//     smaller than the current centre's (every move lowers the best SAD
//     strictly), so skipping it leaves the path unchanged; the bitmap only
//     decides what is counted and recomputed.
#include "me_internal.cuh"

#include <climits>

namespace me {
namespace {

enum { PH_FETCH = 0, PH_HCSP = 1, PH_DDSP = 2, PH_SIDE = 3, PH_MID = 4, PH_DONE = 5 };
enum { PAT_H = 0, PAT_V = 1 };

// Offsets packed 6 bits each: (dx + 2) | (dy + 2) << 3, in evaluation order.
constexpr uint64_t enc(int dx, int dy, int k) { return (uint64_t)((dx + 2) | ((dy + 2) << 3)) << (6 * k); }
// HCSP (Sec. III-A): centre, (-1,0), (+1,0), (0,-1), (0,+1), (-2,0), (+2,0)
constexpr uint64_t kHcsp = enc(0, 0, 0) | enc(-1, 0, 1) | enc(1, 0, 2) | enc(0, -1, 3) | enc(0, 1, 4) |
                           enc(-2, 0, 5) | enc(2, 0, 6);
// HDSP: near points (0,-1), (0,+1) then distant points (-2,0), (+2,0)
constexpr uint64_t kDdspH = enc(0, -1, 0) | enc(0, 1, 1) | enc(-2, 0, 2) | enc(2, 0, 3);
// VDSP: near points (-1,0), (+1,0) then distant points (0,-2), (0,+2)
constexpr uint64_t kDdspV = enc(-1, 0, 0) | enc(1, 0, 1) | enc(0, -2, 2) | enc(0, 2, 3);
// Middle points of the long wing
constexpr uint64_t kMidH = enc(-1, 0, 0) | enc(1, 0, 1);
constexpr uint64_t kMidV = enc(0, -1, 0) | enc(0, 1, 1);

constexpr uint32_t kUnknown = 0xfffffffeu;  // distant-point SAD not produced this round
constexpr uint32_t kInvalid = 0xffffffffu;  // distant point outside window/frame

__device__ __forceinline__ void decode(uint64_t code, int k, int& ox, int& oy)
{
    const unsigned v = (unsigned)(code >> (6 * k)) & 63u;
    ox = (int)(v & 7u) - 2;
    oy = (int)(v >> 3) - 2;
}

template <int B, bool SIMPL>
__global__ void __launch_bounds__(128) dcds_kernel(const FrameDev* __restrict__ frames, int nframes,
                                                   int ntiles, int tx, int ty, int max_range, int sp,
                                                   int* __restrict__ head)
{
    constexpr int G = B / 4;
    constexpr int V = kSadVariant;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_tile, s_next, s_frame;

    const int win_rows = ty * B + 2 * max_range;
    uint8_t* win = smem;
    const int nwr = bm_words_per_row(max_range);
    const int bm_stride = (2 * max_range + 1) * nwr;
    uint32_t* bm_all = reinterpret_cast<uint32_t*>(smem + (size_t)win_rows * sp);

    const int lane = threadIdx.x & 31;
    const int lig = lane & (G - 1);
    const int gid = threadIdx.x / G;
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    uint32_t* bm = bm_all + (size_t)gid * bm_stride;
    const int ngroups = blockDim.x / G;

    for (int i = threadIdx.x; i < ngroups * bm_stride; i += blockDim.x) bm_all[i] = 0u;

    for (;;) {
        __syncthreads();  // the previous tile is finished and its bitmaps are clean
        if (threadIdx.x == 0) {
            const int t = atomicAdd(head, 1);
            int f = 0;
            if (t < ntiles) {
                int lo = 0, hi = nframes - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (frames[mid].tile_base <= t) lo = mid; else hi = mid - 1;
                }
                f = lo;
            }
            s_tile = t;
            s_frame = f;
            s_next = 0;
        }
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const FrameDev& F = frames[s_frame];
        const int W = F.w, H = F.h, P = F.pitch, R = F.range, NBX = F.nbx;
        const int lt = t - F.tile_base;
        const int tile_y = lt / F.tiles_x, tile_x = lt - tile_y * F.tiles_x;
        const int bx0 = tile_x * tx, by0 = tile_y * ty;
        const int nbx_t = min(tx, NBX - bx0), nby_t = min(ty, F.nby - by0);
        const int nmb = nbx_t * nby_t;
        const int rx = (R + 15) & ~15;
        const int x_lo = bx0 * B - rx, y_lo = by0 * B - R;

        // ---- stage the reference window (zeros outside the frame) ----
        {
            const int cpr = (((nbx_t * B + 15) & ~15) + 2 * rx) >> 4;
            const int win_h = nby_t * B + 2 * R;
            const int total = cpr * win_h;
            for (int i = threadIdx.x; i < total; i += blockDim.x) {
                const int row = i / cpr, c = i - row * cpr;
                const int gy = y_lo + row, gx = x_lo + (c << 4);
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                    v = __ldg(reinterpret_cast<const uint4*>(F.ref + (size_t)gy * P + gx));
                *reinterpret_cast<uint4*>(win + (size_t)row * sp + (c << 4)) = v;
            }
        }
        __syncthreads();

        // ---- per-group search state (replicated in the G lanes) ----
        int phase = PH_FETCH, pat = PAT_H, k = 0, nsp = 0, slot = 0;
        int wx0 = 0, wy0 = 0, blk = 0;
        int dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0;
        int cx = 0, cy = 0, bxp = 0, byp = 0;
        uint32_t bsad = 0xffffffffu;
        int tmin = INT_MAX, tmax = -1;  // bitmap rows touched (lane 0 only)
        uint32_t ds0 = kUnknown, ds1 = kUnknown;
        int nmid = 2;
        uint64_t midcode = kMidH;
        uint32_t cb[B];
#pragma unroll
        for (int r = 0; r < B; ++r) cb[r] = 0u;

        for (;;) {
            bool have = false, counted = false;
            int qx = 0, qy = 0;
            // Advance to the next candidate; bounded by the number of
            // transitions one step can chain (list ends, a block finish and a
            // fetch), far below the guard.
            for (int guard = 0; guard < 40; ++guard) {
                if (phase == PH_DONE) break;
                if (phase == PH_FETCH) {
                    int m = 0;
                    if (lig == 0) m = atomicAdd(&s_next, 1);
                    m = __shfl_sync(gmask, m, 0, G);
                    if (m >= nmb) { phase = PH_DONE; break; }
                    const int bxl = m % nbx_t, byl = m / nbx_t;
                    const int bxg = bx0 + bxl, byg = by0 + byl;
                    const int px = bxg * B, py = byg * B;
                    blk = byg * NBX + bxg;
                    wx0 = bxl * B + rx;
                    wy0 = byl * B + R;
                    dxlo = max(-R, -px); dxhi = min(R, W - B - px);
                    dylo = max(-R, -py); dyhi = min(R, H - B - py);
                    const uint8_t* cp = F.cur + (size_t)py * P + px + 4 * lig;
#pragma unroll
                    for (int r = 0; r < B; ++r) cb[r] = __ldg(reinterpret_cast<const uint32_t*>(cp + (size_t)r * P));
                    cx = cy = 0; bxp = byp = 0; bsad = 0xffffffffu; nsp = 0; pat = PAT_H;
                    phase = PH_HCSP; k = 0;
                    continue;
                }
                int n;
                uint64_t code;
                if (phase == PH_HCSP) { n = 7; code = kHcsp; }
                else if (phase == PH_DDSP) { n = 4; code = pat ? kDdspV : kDdspH; }
                else if (phase == PH_SIDE) { n = 2; code = (pat ? kDdspV : kDdspH) >> 12; }
                else { n = nmid; code = midcode; }
                if (k < n) {
                    int ox, oy;
                    decode(code, k, ox, oy);
                    const int x = cx + ox, y = cy + oy;
                    slot = k;
                    ++k;
                    const bool valid = x >= dxlo && x <= dxhi && y >= dylo && y <= dyhi;
                    if (SIMPL && phase == PH_SIDE) {
                        // recompute a distant point visited in an earlier round
                        const uint32_t d = slot ? ds1 : ds0;
                        if (!valid || d != kUnknown) continue;
                        qx = x; qy = y; have = true; counted = false;
                        break;
                    }
                    if (!valid) {
                        if (SIMPL && phase == PH_DDSP && slot >= 2) { if (slot == 2) ds0 = kInvalid; else ds1 = kInvalid; }
                        continue;
                    }
                    int vis = 0;
                    if (lig == 0) {
                        uint32_t* wp = bm + (y + R) * nwr + ((x + R) >> 5);
                        const uint32_t bit = 1u << ((x + R) & 31);
                        const uint32_t wv = *wp;
                        vis = (wv & bit) != 0u;
                        if (!vis) {
                            *wp = wv | bit;
                            tmin = min(tmin, y + R);
                            tmax = max(tmax, y + R);
                        }
                    }
                    vis = __shfl_sync(gmask, vis, 0, G);
                    if (vis) continue;
                    ++nsp;
                    qx = x; qy = y; have = true; counted = true;
                    break;
                }
                // ---- list exhausted: pattern transitions (Sec. III-B) ----
                bool finish = false;
                if (phase == PH_HCSP) {
                    if (bxp == 0 && byp == 0) {
                        finish = true;  // step 1 half-way stop
                    } else {
                        pat = (byp == 0) ? PAT_H : PAT_V;  // switching strategy one
                        cx = bxp; cy = byp;
                        phase = PH_DDSP; k = 0; ds0 = ds1 = kUnknown;
                    }
                } else if (phase == PH_DDSP) {
                    if (bxp == cx && byp == cy) {
                        k = 0;
                        if (SIMPL) { phase = PH_SIDE; }
                        else { phase = PH_MID; nmid = 2; midcode = pat ? kMidV : kMidH; }
                    } else {
                        const int ddx = bxp - cx, ddy = byp - cy;
                        if (abs(ddx) + abs(ddy) == 1) pat ^= 1;  // switching strategy two
                        cx = bxp; cy = byp;
                        k = 0; ds0 = ds1 = kUnknown;
                    }
                } else if (SIMPL && phase == PH_SIDE) {
                    const uint64_t mc = pat ? kMidV : kMidH;
                    if (ds0 == kInvalid && ds1 == kInvalid) { nmid = 2; midcode = mc; }
                    else {
                        const int side = (ds0 == kInvalid) ? 1 : (ds1 == kInvalid) ? 0 : (ds1 < ds0 ? 1 : 0);
                        nmid = 1; midcode = mc >> (6 * side);
                    }
                    phase = PH_MID; k = 0;
                } else {
                    finish = true;  // step 4 done
                }
                if (finish) {
                    if (lig == 0) {
                        *reinterpret_cast<uint32_t*>(F.mv + 2 * (size_t)blk) =
                            (uint32_t)(uint16_t)bxp | ((uint32_t)(uint16_t)byp << 16);
                        F.sad[blk] = bsad;
                        if (F.nsp) F.nsp[blk] = (uint16_t)nsp;
                        for (int r = tmin; r <= tmax; ++r)
                            for (int w = 0; w < nwr; ++w) bm[r * nwr + w] = 0u;
                        tmin = INT_MAX; tmax = -1;
                    }
                    phase = PH_FETCH;
                }
            }
            if (!__any_sync(0xffffffffu, phase != PH_DONE)) break;

            // ---- one SAD per active group ----
            uint32_t part = 0u;
            if (have) {
                const int col = wx0 + qx + 4 * lig;
                const uint8_t* base = win + (size_t)(wy0 + qy) * sp + (col & ~3);
                const unsigned sh = (unsigned)(col & 3) * 8u;
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const uint32_t lo = *reinterpret_cast<const uint32_t*>(base + r * sp);
                    const uint32_t hi = *reinterpret_cast<const uint32_t*>(base + r * sp + 4);
                    part = sadacc<V>(__funnelshift_r(lo, hi, sh), cb[r], part);
                }
            }
#pragma unroll
            for (int o = 1; o < G; o <<= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (have) {
                if (counted && part < bsad) { bsad = part; bxp = qx; byp = qy; }
                if (SIMPL) {
                    if (phase == PH_DDSP && slot >= 2) { if (slot == 2) ds0 = part; else ds1 = part; }
                    else if (phase == PH_SIDE) { if (slot == 0) ds0 = part; else ds1 = part; }
                }
            }
        }
    }
}

template <int B, bool SIMPL>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s,
                     int* head, int num_sms, cudaStream_t st)
{
    const size_t smem = dcds_smem_bytes(B, max_range, s);
    auto kern = dcds_kernel<B, SIMPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = ntiles;
    if (s.ctas_per_sm > 0) grid = min(ntiles, s.ctas_per_sm * num_sms);
    if (grid < 1) grid = 1;
    const int rxm = (max_range + 15) & ~15;
    const int sp = ((s.tx * B + 15) & ~15) + 2 * rxm + 16;
    kern<<<grid, s.threads, smem, st>>>(frames, nframes, ntiles, s.tx, s.ty, max_range, sp, head);
    return cudaGetLastError();
}

}  // namespace

size_t dcds_smem_bytes(int block, int max_range, const Shape& s)
{
    const int rxm = (max_range + 15) & ~15;
    const int sp = ((s.tx * block + 15) & ~15) + 2 * rxm + 16;
    const size_t win = (size_t)(s.ty * block + 2 * max_range) * sp;
    const int groups = s.threads / (block / 4);
    const size_t bm = (size_t)groups * (2 * max_range + 1) * bm_words_per_row(max_range) * 4;
    return win + bm;
}

cudaError_t launch_dcds(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                        bool simplified, const Shape& s, int* head, unsigned* /*status*/, int num_sms,
                        cudaStream_t st)
{
    if (block == 16) {
        return simplified ? launch_t<16, true>(frames, nframes, ntiles, max_range, s, head, num_sms, st)
                          : launch_t<16, false>(frames, nframes, ntiles, max_range, s, head, num_sms, st);
    }
    return simplified ? launch_t<8, true>(frames, nframes, ntiles, max_range, s, head, num_sms, st)
                      : launch_t<8, false>(frames, nframes, ntiles, max_range, s, head, num_sms, st);
}

}  // namespace me
