// dcds_common.cuh -- device helpers shared by the two DCDS kernels: the
// search patterns of Sec. III-A in evaluation order, and the TMA / mbarrier
// primitives that stage a tile.
#pragma once

#include "me_internal.cuh"

namespace me {
namespace dcds {

enum { PH_FETCH = 0, PH_DDSP = 1, PH_SIDE = 2, PH_MID = 3, PH_DONE = 4 };
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
constexpr uint32_t kWaitLimit = 1u << 20;   // bounded mbarrier waits (each try_wait call suspends briefly)
constexpr uint32_t kShortWait = 1u << 12;   // the limit under the failure-detection test hook

__device__ __forceinline__ void decode(uint64_t code, int k, int& ox, int& oy)
{
    const unsigned v = (unsigned)(code >> (6 * k)) & 63u;
    ox = (int)(v & 7u) - 2;
    oy = (int)(v >> 3) - 2;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity.  try_wait suspends the thread in
// hardware for a bounded time per call; after kWaitLimit calls the wait gives
// up and the caller reports a timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kWaitLimit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 2-D tiled TMA load of a box at element coordinates (x, y); x*1 byte must be
// a multiple of 16 (it is: tile origins are multiples of 128, margins of 16).
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ int find_frame(const FrameDev* frames, int nframes, int t)
{
    const int u = frames[0].uniform_tiles;
    if (u > 0) return min(t / u, nframes - 1);
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (frames[mid].tile_base <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__host__ __device__ inline int round128(int v) { return (v + 127) & ~127; }

__host__ __device__ inline int win_bytes_max(int max_range, int tile_h)
{
    const int rxm = (max_range + 15) & ~15;
    return round128((kTile + 2 * rxm) * (tile_h + 2 * max_range));
}

// The fields of a tile's frame that the search reads, copied into shared
// memory by the thread that claims the tile, so that the CTA does not wait on
// the frame table's global loads when the tile arrives.
struct TileDesc {
    uint32_t* mv;
    uint32_t* sad;
    uint16_t* nsp;
    const uint32_t* mv_fs;
    unsigned long long* sums;
    int w, h, range, nbx, nby, tile_x, tile_y, first;  // first: the frame's first tile (writes its counts)
};

// Thread 0: take tile t into stage `st`: publish its index and descriptor,
// then arm the stage's mbarrier with the byte count and start the two TMA
// copies.  A tile index past the end completes the phase with no data.
// extra_tx > 0 arms the barrier for more bytes than the copies deliver (the
// failure-detection test hook: the wait on this stage then runs out).
__device__ inline void issue_tile(int t, const FrameDev* frames, int nframes, int ntiles, uint8_t* stage,
                           int cur_off, int tile_h, uint64_t* bar, int* s_tile, TileDesc* desc,
                           uint32_t extra_tx = 0)
{
    *s_tile = t;
    if (t >= ntiles) {
        mbar_arrive(bar);
        return;
    }
    const int f = find_frame(frames, nframes, t);
    const FrameDev& F = frames[f];
    const int lt = t - F.tile_base;
    const int ty = lt / F.tiles_x, tx = lt - ty * F.tiles_x;
    const int rx = (F.range + 15) & ~15;
    desc->mv = reinterpret_cast<uint32_t*>(F.mv);
    desc->sad = F.sad;
    desc->nsp = F.nsp;
    desc->mv_fs = reinterpret_cast<const uint32_t*>(F.mv_fs);
    desc->sums = F.sums;
    desc->w = F.w; desc->h = F.h; desc->range = F.range; desc->nbx = F.nbx; desc->nby = F.nby;
    desc->tile_x = tx; desc->tile_y = ty; desc->first = lt == 0;
    const uint32_t bytes = (uint32_t)((kTile + 2 * rx) * (tile_h + 2 * F.range) + kTile * tile_h) + extra_tx;
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_2d(stage, &F.tm_ref, tx * kTile - rx, ty * tile_h - F.range, bar);
    tma_load_2d(stage + cur_off, &F.tm_cur, tx * kTile, ty * tile_h, bar);
}


}  // namespace dcds
}  // namespace me
