// dcds_cross.cu -- Directional Cross Diamond Search on sm_103a as one uniform
// per-block state machine over a 9-point cross.
//
// Algorithm: Jia & Zhang, Sec. III-B (steps 1-4, switching strategies one
// and two) with the patterns of Sec. III-A; DCDS^S of Sec. IV-C as a
// compile-time variant; the Sec. IV measures optionally fused.
//
// The primitive.  Every pattern of the method lies inside the cross of
// radius 2 around the current centre c: the HCSP (c, c+(+-1,0), c+(+-2,0),
// c+(0,+-1)), the HDSP (c+(0,+-1), c+(+-2,0)), the VDSP (c+(+-1,0),
// c+(0,+-2)) and both pairs of middle points.  One pass over the reference
// rows c.y-2 .. c.y+B+1 gives the SADs of all nine cross points: five
// horizontal offsets share each row (three aligned words realigned by two
// funnel shifts, then three more shifts), and the four vertical offsets
// reuse the neighbouring rows.  A point evaluated earlier never has a SAD
// below the current centre's (every move lowers the best SAD strictly), so
// recomputing it changes no decision; a per-block bitmap of visited points
// decides only what is counted.  So one pass decides one step of the search:
// step 1 at the origin, then each step of steps 2-3 -- and when the centre
// wins, step 4's middle points are already in the same pass.
//
// The schedule.  Persistent CTAs of 128 threads.  Each CTA keeps two tile
// stages in shared memory (a tile is 128 x 64 pixels: the reference window,
// grown by R rows and R rounded up to 16 columns and zero-filled outside the
// frame, and the current tile), copied by the TMA unit with mbarrier
// completion.  Groups of B/4 lanes (one 4-byte column of the block each) take
// blocks one at a time from a CTA-wide sequence: block q is block q % NMB of
// the CTA's tile q / NMB, which lives in stage (q / NMB) & 1.  Every round,
// each group runs one cross pass for its block and one step of its state
// machine; a finished group takes the next block at once, from the same tile
// or the next, so there is no barrier between phases and no tile tail.  When
// the last block of a tile is done, that lane claims the next tile from the
// global counter and copies it into the freed stage (claims are made in
// sequence order under a small lock, so a claim past the end is never
// followed by a real one).  A group whose tile has not landed yet tests its
// barrier once per round instead of waiting, so a warp never blocks while it
// holds unfinished blocks.  Waits are bounded: a group that has tested its
// barrier too often records a time-out and stops.
#include "dcds_common.cuh"

#include <climits>

namespace me {
namespace {

using namespace dcds;

constexpr int kTileH = 64;  // tile height in pixels (width kTile)
constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t kInf = 0xffffffffu;

// cross points: 0 (0,0), 1 (-1,0), 2 (+1,0), 3 (0,-1), 4 (0,+1), 5 (-2,0), 6 (+2,0), 7 (0,-2), 8 (0,+2)
__device__ __forceinline__ int cx_of(int i) { return i == 1 ? -1 : i == 2 ? 1 : i == 5 ? -2 : i == 6 ? 2 : 0; }
__device__ __forceinline__ int cy_of(int i) { return i == 3 ? -1 : i == 4 ? 1 : i == 7 ? -2 : i == 8 ? 2 : 0; }
// evaluation orders (Sec. III-A patterns; ties keep the earlier point), cross indices 4 bits each
constexpr uint32_t kOrdHcsp = 1 | 2 << 4 | 3 << 8 | 4 << 12 | 5 << 16 | 6 << 20;  // 6 points
constexpr uint32_t kOrdH = 3 | 4 << 4 | 5 << 8 | 6 << 12;                           // HDSP: near, then distant
constexpr uint32_t kOrdV = 1 | 2 << 4 | 7 << 8 | 8 << 12;                           // VDSP
constexpr uint32_t kMidH = 1 | 2 << 4;
constexpr uint32_t kMidV = 3 | 4 << 4;

enum { S_NONE = 0, S_WAIT = 1, S_HCSP = 2, S_DDSP = 3, S_FIN = 4, S_EXIT = 5 };

// The best of the centre (cross point 0) and the listed cross points, in the
// listed order with a strict "<" (ties keep the earlier point); points not in
// `mask` are skipped.  Compile-time lists keep the SADs in registers.
template <int... I>
__device__ __forceinline__ int pick(const uint32_t (&sd)[9], uint32_t mask, uint32_t& bv)
{
    int best = 0;
    bv = sd[0];
    ((((mask >> I) & 1u) && sd[I] < bv ? (bv = sd[I], best = I) : 0), ...);
    return best;
}

// What a group needs of its tile, written by the lane that issues the tile.
struct StageInfo {
    int32_t tile;  // global tile index, or -1: no more tiles
    int32_t seq;   // the CTA's tile sequence number held by the stage
    int32_t frame;
    int32_t w, h, range, nbx, nby, pitch;
    int32_t bx0, by0;  // first block of the tile
    int32_t first;     // 1: the frame's first tile (writes its block count)
    int16_t* mv;
    uint32_t* sad;
    uint16_t* nsp;
    const uint32_t* mv_fs;
    unsigned long long* sums;
};

template <int B>
struct Geo {
    static constexpr int TXB = kTile / B;    // blocks per tile row
    static constexpr int TYB = kTileH / B;   // block rows per tile
    static constexpr int NMB = TXB * TYB;    // blocks per tile
    static constexpr int GL = B / 4;         // lanes per group
};

__host__ __device__ inline int cross_win_bytes(int max_range)
{
    const int rxm = (max_range + 15) & ~15;
    return round128((kTile + 2 * rxm) * (kTileH + 2 * max_range));
}
__host__ __device__ inline int cross_stage_bytes(int max_range) { return cross_win_bytes(max_range) + kTile * kTileH; }

// Claim the next global tile and start its copy into `stage` (one lane).
__device__ void issue_stage(int s, int seq, const FrameDev* frames, int nframes, int ntiles, int* head,
                            uint8_t* stage, int cur_off, uint64_t* bar, StageInfo* si, uint32_t extra_tx)
{
    const int t = atomicAdd(head, 1);
    StageInfo& I = si[s];
    I.seq = seq;
    if (t >= ntiles) {
        I.tile = -1;
        mbar_arrive(bar);
        return;
    }
    const int f = find_frame(frames, nframes, t);
    const FrameDev& F = frames[f];
    const int lt = t - F.tile_base;
    const int ty = lt / F.tiles_x, tx = lt - ty * F.tiles_x;
    const int rx = (F.range + 15) & ~15;
    I.tile = t;
    I.frame = f;
    I.w = F.w; I.h = F.h; I.range = F.range; I.nbx = F.nbx; I.nby = F.nby; I.pitch = F.pitch;
    I.bx0 = tx * (kTile / (F.w / F.nbx));
    I.by0 = ty * (kTileH / (F.w / F.nbx));
    I.first = lt == 0;
    I.mv = F.mv; I.sad = F.sad; I.nsp = F.nsp;
    I.mv_fs = reinterpret_cast<const uint32_t*>(F.mv_fs);
    I.sums = F.sums;
    const uint32_t bytes = (uint32_t)((kTile + 2 * rx) * (kTileH + 2 * F.range) + kTile * kTileH) + extra_tx;
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_2d(stage, &F.tm_ref, tx * kTile - rx, ty * kTileH - F.range, bar);
    tma_load_2d(stage + cur_off, &F.tm_cur, tx * kTile, ty * kTileH, bar);
}

template <int B, bool SIMPL, bool EVAL>
__global__ void __launch_bounds__(128, 4) dcds_cross_kernel(const FrameDev* __restrict__ frames, int nframes,
                                                            int ntiles, int max_range, int* __restrict__ head,
                                                            unsigned* __restrict__ status)
{
    using G = Geo<B>;
    constexpr int V = kSadVariant;
    constexpr int GL = G::GL, NMB = G::NMB, TXB = G::TXB;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ StageInfo s_info[2];
    __shared__ int s_next;      // next block sequence number of this CTA
    __shared__ int s_done[2];   // blocks of the stage's tile finished
    __shared__ int s_free[2];   // stage free for the next tile (its tile is done)
    __shared__ int s_issued;    // tile sequence numbers claimed so far
    __shared__ int s_lock;
    __shared__ unsigned long long s_sums[2][6];  // EVAL: ABS SQ NSP EQUAL DIST PIXELS of the stage's tile

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int cur_off = cross_win_bytes(max_range);
    const int stage_bytes = cur_off + kTile * kTileH;
    const int side_max = 2 * max_range + 1;
    const int nwb = (side_max * side_max + 31) / 32;
    uint32_t* bm_all = reinterpret_cast<uint32_t*>(smem + 2 * stage_bytes);

    const int tid = threadIdx.x, lane = tid & 31;
    const int gq = tid / GL, gl = lane % GL;          // group in the CTA, lane in the group
    const int glead = lane - gl;                      // first lane of the group
    const unsigned gmask = ((1u << GL) - 1u) << glead;
    uint32_t* bm = bm_all + gq * nwb;

    for (int i = tid; i < (blockDim.x / GL) * nwb; i += blockDim.x) bm_all[i] = 0u;
    // failure-detection test hook (last counter word): the first copy is armed
    // for 16 bytes that never arrive and the waits are shortened
    const bool starve = head[kCounterInts - 1] != 0;
    const uint32_t wait_limit = starve ? kShortWait : kWaitLimit;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        s_next = 0;
        s_done[0] = s_done[1] = 0;
        s_free[0] = s_free[1] = 0;
        s_issued = 2;
        s_lock = 0;
        for (int i = 0; i < 12; ++i) (&s_sums[0][0])[i] = 0ull;
        issue_stage(0, 0, frames, nframes, ntiles, head, smem, cur_off, &s_bar[0], s_info, starve ? 16u : 0u);
        issue_stage(1, 1, frames, nframes, ntiles, head, smem + stage_bytes, cur_off, &s_bar[1], s_info, 0u);
    }
    __syncthreads();

    // ---- group state (identical in the GL lanes of a group) ----
    int state = S_NONE;
    int q = 0, st = 0;
    uint32_t waits = 0;
    int R = 0, W = 0, H = 0, NBX = 0, WP = 0, rx = 0;
    int bxg = 0, byg = 0, px = 0, py = 0;
    int dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0;
    int wx0 = 0, wy0 = 0;  // window column of this lane's word and window row of the block's row 0, at (0,0)
    const uint8_t* win = smem;
    int cx = 0, cy = 0, pat = PAT_H, nsp = 0;
    uint32_t bsad = 0;           // SAD of the current centre
    uint32_t fw = 0;             // EVAL: the block's full-search MV
    int wmin = INT_MAX, wmax = -1;
    uint32_t cb[B];
#pragma unroll
    for (int r = 0; r < B; ++r) cb[r] = 0u;

    // the lane that finishes a tile frees its stage and issues the tiles whose turn has come
    auto release = [&](int s) {
        __threadfence_block();  // the finished blocks' outputs and sums are visible
        const StageInfo& I = s_info[s];
        if (EVAL) {
            unsigned long long* fs = I.sums;
            const unsigned long long* ss = s_sums[s];
            // ABS SQ NSP EQUAL -> sums 0..3, DIST -> 4, PIXELS -> 6
            if (ss[0]) atomicAdd(fs + 0, ss[0]);
            if (ss[1]) atomicAdd(fs + 1, ss[1]);
            if (ss[2]) atomicAdd(fs + 2, ss[2]);
            if (ss[3]) atomicAdd(fs + 3, ss[3]);
            if (ss[4]) atomicAdd(fs + 4, ss[4]);
            if (ss[5]) atomicAdd(fs + 6, ss[5]);
            if (I.first) {
                fs[5] = (unsigned long long)I.nbx * I.nby;
                fs[7] = I.mv_fs ? 1ull : 0ull;
            }
            for (int i = 0; i < 6; ++i) s_sums[s][i] = 0ull;
        }
        s_done[s] = 0;
        __threadfence_block();
        // the lock orders the claims: tile sequence numbers are issued in order
        uint32_t it = 0;
        while (atomicCAS(&s_lock, 0, 1) != 0)
            if (++it > kWaitLimit) { if (status) atomicOr(status, STATUS_TIMEOUT); return; }
        __threadfence_block();
        s_free[s] = 1;
        for (;;) {
            const int k = s_issued, ks = k & 1;
            if (!s_free[ks]) break;
            s_free[ks] = 0;
            s_issued = k + 1;
            fence_proxy_async();  // the stage's earlier reads come before the copy's writes
            issue_stage(ks, k, frames, nframes, ntiles, head, smem + ks * stage_bytes, cur_off, &s_bar[ks], s_info, 0u);
        }
        __threadfence_block();
        atomicExch(&s_lock, 0);
    };

    for (int round = 0;; ++round) {
        // ---- (1) groups without a block take the next sequence numbers (one atomic per warp) ----
        const unsigned need = __ballot_sync(FULL, state == S_NONE && gl == 0);
        if (need) {
            const int first = __ffs(need) - 1;
            int base = 0;
            if (lane == first) base = atomicAdd(&s_next, __popc(need));
            base = __shfl_sync(FULL, base, first);
            const int mine = __shfl_sync(FULL, base + __popc(need & ((1u << lane) - 1u)), glead);
            if (state == S_NONE) {
                q = mine;
                st = (q / NMB) & 1;
                state = S_WAIT;
                waits = 0;
            }
        }
        // ---- (2) groups whose tile has landed set up their block ----
        if (state == S_WAIT) {
            const int k = q / NMB;
            bool ready = false;
            if (gl == 0) ready = mbar_try(&s_bar[st], (uint32_t)((k >> 1) & 1)) && s_info[st].seq == k;
            ready = __shfl_sync(gmask, ready, glead);
            if (!ready) {
                if (++waits > wait_limit) {
                    if (gl == 0 && status) atomicOr(status, STATUS_TIMEOUT);
                    state = S_EXIT;
                }
            } else if (s_info[st].tile < 0) {
                state = S_EXIT;  // no more tiles
            } else {
                const StageInfo& I = s_info[st];
                const int b = q % NMB, bxl = b % TXB, byl = b / TXB;
                bxg = I.bx0 + bxl;
                byg = I.by0 + byl;
                if (bxg >= I.nbx || byg >= I.nby) {
                    // a block slot of a partial tile: nothing to search
                    state = S_NONE;
                    if (gl == 0) {
                        __threadfence_block();
                        if (atomicAdd(&s_done[st], 1) == NMB - 1) release(st);
                    }
                } else {
                    R = I.range; W = I.w; H = I.h; NBX = I.nbx;
                    rx = (R + 15) & ~15;
                    WP = kTile + 2 * rx;
                    px = bxg * B; py = byg * B;
                    dxlo = max(-R, -px); dxhi = min(R, W - B - px);
                    dylo = max(-R, -py); dyhi = min(R, H - B - py);
                    win = smem + st * stage_bytes;
                    wx0 = rx + bxl * B + 4 * gl;
                    wy0 = R + byl * B;
                    const uint8_t* cp = win + cur_off + (byl * B) * kTile + bxl * B + 4 * gl;
#pragma unroll
                    for (int r = 0; r < B; ++r) cb[r] = *reinterpret_cast<const uint32_t*>(cp + r * kTile);
                    if (EVAL) fw = I.mv_fs ? __ldg(I.mv_fs + (size_t)byg * NBX + bxg) : 0u;
                    cx = cy = 0;
                    nsp = 0;
                    state = S_HCSP;
                }
            }
        }
        const bool active = state == S_HCSP || state == S_DDSP || state == S_FIN;
        if (!__any_sync(FULL, state != S_EXIT)) break;
        if (!__any_sync(FULL, active)) continue;

        // ---- (3) one cross pass per group at its centre ----
        uint32_t sd[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) sd[i] = 0u;
        uint32_t sq = 0u;
        // fast pass: every read of the cross stays inside the staged window
        const bool fast = !active || (cx >= 2 - rx && cx <= rx - 6 && cy >= 2 - R && cy <= R - 2);
        if (__any_sync(FULL, fast)) {
            const int ccx = (active && fast) ? cx : 0, ccy = (active && fast) ? cy : 0;
            // an inactive group reads the middle of its stage (always inside)
            const uint8_t* wb = active ? win : smem;
            const int x0 = (active ? wx0 : 16 + 4 * gl) + ccx;
            const int y0 = (active ? wy0 : 8) + ccy;
            const int ab = (x0 - 2) & ~3;
            const unsigned s8 = (unsigned)((x0 - 2) & 3) * 8u;
            const int wp = active ? WP : kTile;
            const uint8_t* rp = wb + (y0 - 2) * wp + ab;
#pragma unroll
            for (int rr = -2; rr < B + 2; ++rr) {
                const uint32_t* p = reinterpret_cast<const uint32_t*>(rp + (rr + 2) * wp);
                const uint32_t w0 = p[0], w1 = p[1], w2 = p[2];
                const uint32_t r0 = __funnelshift_r(w0, w1, s8);  // bytes x0-2 .. x0+1
                const uint32_t r1 = __funnelshift_r(w1, w2, s8);  // bytes x0+2 .. x0+5
                const uint32_t h0 = __funnelshift_r(r0, r1, 16);  // bytes x0 .. x0+3
                if (rr >= 0 && rr < B) {
                    const uint32_t c = cb[rr];
                    if constexpr (EVAL) {
                        const uint32_t d = __vabsdiffu4(h0, c);
                        sd[0] = (uint32_t)__dp4a(d, 0x01010101u, sd[0]);
                        sq = (uint32_t)__dp4a(d, d, sq);
                    } else {
                        sd[0] = sadacc<V>(h0, c, sd[0]);
                    }
                    sd[5] = sadacc<V>(r0, c, sd[5]);
                    sd[1] = sadacc<V>(__funnelshift_r(r0, r1, 8), c, sd[1]);
                    sd[2] = sadacc<V>(__funnelshift_r(r0, r1, 24), c, sd[2]);
                    sd[6] = sadacc<V>(r1, c, sd[6]);
                }
                if (rr - 1 >= 0 && rr - 1 < B) sd[4] = sadacc<V>(h0, cb[rr - 1], sd[4]);  // (0,+1)
                if (rr + 1 >= 0 && rr + 1 < B) sd[3] = sadacc<V>(h0, cb[rr + 1], sd[3]);  // (0,-1)
                if (rr - 2 >= 0 && rr - 2 < B) sd[8] = sadacc<V>(h0, cb[rr - 2], sd[8]);  // (0,+2)
                if (rr + 2 >= 0 && rr + 2 < B) sd[7] = sadacc<V>(h0, cb[rr + 2], sd[7]);  // (0,-2)
            }
        }
        if (__any_sync(FULL, !fast)) {
            // near the window's edge: the valid cross points one at a time
            // (a valid point lies inside the window); the others read the block's own position
#pragma unroll 1
            for (int i = 0; i < 9; ++i) {
                const int qx = cx + cx_of(i), qy = cy + cy_of(i);
                const bool use = !fast && qx >= dxlo && qx <= dxhi && qy >= dylo && qy <= dyhi;
                const int ox = use ? qx : 0, oy = use ? qy : 0;
                const uint8_t* wb = active ? win : smem;
                const int wp = active ? WP : kTile;
                const int c0 = (active ? wx0 : 16 + 4 * gl) + ox;
                const uint8_t* p0 = wb + ((active ? wy0 : 8) + oy) * wp + (c0 & ~3);
                const unsigned sh = (unsigned)(c0 & 3) * 8u;
                uint32_t a = 0u, s2 = 0u;
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const uint32_t* p = reinterpret_cast<const uint32_t*>(p0 + r * wp);
                    const uint32_t v = __funnelshift_r(p[0], p[1], sh);
                    if (EVAL && i == 0) {
                        const uint32_t d = __vabsdiffu4(v, cb[r]);
                        a = (uint32_t)__dp4a(d, 0x01010101u, a);
                        s2 = (uint32_t)__dp4a(d, d, s2);
                    } else {
                        a = sadacc<V>(v, cb[r], a);
                    }
                }
                if (!fast) {
                    // written through selects: the sums stay in registers
#pragma unroll
                    for (int k = 0; k < 9; ++k) sd[k] = (k == i) ? a : sd[k];
                    if (EVAL && i == 0) sq = s2;
                }
            }
        }
        // complete the sums across the group
#pragma unroll
        for (int o = 1; o < GL; o <<= 1) {
#pragma unroll
            for (int i = 0; i < 9; ++i) sd[i] += __shfl_xor_sync(FULL, sd[i], o);
            if (EVAL) sq += __shfl_xor_sync(FULL, sq, o);
        }

        // ---- (4) one step of each active group's search (Sec. III-B) ----
        if (active) {
        unsigned valid = 0u;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int qx = cx + cx_of(i), qy = cy + cy_of(i);
            valid |= (unsigned)(qx >= dxlo && qx <= dxhi && qy >= dylo && qy <= dyhi) << i;
        }
        const int side = 2 * R + 1;
        // mark the listed valid points visited; returns how many of them are
        // new (the counted points).  Lane gl checks points gl, gl + GL, ...;
        // the count is completed across the group.
        auto visit = [&](uint32_t ord, int n) {
            int cnt = 0;
            for (int j = gl; j < n; j += GL) {
                const int i = (int)((ord >> (4 * j)) & 15u);
                if ((valid >> i) & 1u) {
                    const int bit = (cy + cy_of(i) + R) * side + (cx + cx_of(i) + R);
                    const uint32_t m = 1u << (bit & 31);
                    if (!(atomicOr(&bm[bit >> 5], m) & m)) ++cnt;
                    wmin = min(wmin, bit >> 5);
                    wmax = max(wmax, bit >> 5);
                }
            }
#pragma unroll
            for (int o = 1; o < GL; o <<= 1) cnt += __shfl_xor_sync(gmask, cnt, o);
            return cnt;
        };
        int fin = -1;  // cross index of the final MV once the search has ended
        if (state == S_HCSP) {
            // step 1: the HCSP at the origin (every valid point is new)
            nsp = visit(0u, 1);
            nsp += visit(kOrdHcsp, 6);
            uint32_t bv;
            const int best = pick<1, 2, 3, 4, 5, 6>(sd, valid, bv);
            bsad = bv;
            if (best == 0) {
                fin = 0;  // the half-way stop
            } else {
                pat = (cy_of(best) == 0) ? PAT_H : PAT_V;  // switching strategy one
                cx += cx_of(best);
                cy += cy_of(best);
                state = S_DDSP;
            }
        } else if (state == S_DDSP) {
            // steps 2-3: the HDSP or VDSP at the centre
            const uint32_t ord = pat ? kOrdV : kOrdH;
            nsp += visit(ord, 4);
            uint32_t bv;
            const int best = pat ? pick<1, 2, 7, 8>(sd, valid, bv) : pick<3, 4, 5, 6>(sd, valid, bv);
            if (best != 0) {
                const bool near = pat ? (best == 1 || best == 2) : (best == 3 || best == 4);
                if (near) pat ^= 1;  // switching strategy two
                cx += cx_of(best);
                cy += cy_of(best);
                bsad = bv;
            } else {
                // step 4: the middle points of the current pattern, from the same pass
                uint32_t mid = pat ? kMidV : kMidH;
                int nmid = 2;
                uint32_t mmask = valid;
                if (SIMPL) {
                    // DCDS^S: only the middle point on the side of the better distant point
                    const uint32_t s0 = pat ? (((valid >> 7) & 1u) ? sd[7] : kInf) : (((valid >> 5) & 1u) ? sd[5] : kInf);
                    const uint32_t s1 = pat ? (((valid >> 8) & 1u) ? sd[8] : kInf) : (((valid >> 6) & 1u) ? sd[6] : kInf);
                    if (!(s0 == kInf && s1 == kInf)) {
                        const int side_pick = (s0 == kInf) ? 1 : (s1 == kInf) ? 0 : (s1 < s0 ? 1 : 0);
                        mid = (mid >> (4 * side_pick)) & 15u;
                        nmid = 1;
                        mmask &= 1u << mid;  // the other middle point is not evaluated
                    }
                }
                nsp += visit(mid, nmid);
                uint32_t bv2;
                fin = pat ? pick<3, 4>(sd, mmask, bv2) : pick<1, 2>(sd, mmask, bv2);
                bsad = bv2;
            }
        } else {
            fin = 0;  // S_FIN: this pass was centred on the final MV for its squared error
        }
        bool finish = false;
        if (fin >= 0) {
            cx += cx_of(fin);
            cy += cy_of(fin);
            if (EVAL && fin != 0) state = S_FIN;  // the squared error at a middle point: one more pass
            else finish = true;
        }
        if (finish) {
            const StageInfo& I = s_info[st];
            const size_t blk = (size_t)byg * NBX + bxg;
            if (gl == 0) {
                reinterpret_cast<uint32_t*>(I.mv)[blk] = (uint32_t)(uint16_t)cx | ((uint32_t)(uint16_t)cy << 16);
                I.sad[blk] = bsad;
                if (I.nsp) I.nsp[blk] = (uint16_t)nsp;
                if constexpr (EVAL) {
                    unsigned long long* ss = s_sums[st];
                    atomicAdd(ss + 0, (unsigned long long)bsad);
                    atomicAdd(ss + 1, (unsigned long long)sq);
                    if (I.nsp) atomicAdd(ss + 2, (unsigned long long)nsp);
                    if (I.mv_fs) {
                        const int ex = cx - (int)(int16_t)(fw & 0xffffu), ey = cy - (int)(int16_t)(fw >> 16);
                        if (ex == 0 && ey == 0) atomicAdd(ss + 3, 1ull);
                        else atomicAdd(ss + 4, dist_q24(ex, ey));
                    }
                    atomicAdd(ss + 5, (unsigned long long)(B * B));
                }
            }
            for (int i = wmin; i <= wmax; ++i) bm[i] = 0u;
            wmin = INT_MAX;
            wmax = -1;
            state = S_NONE;
            __syncwarp(gmask);
            if (gl == 0) {
                __threadfence_block();
                if (atomicAdd(&s_done[st], 1) == NMB - 1) release(st);
            }
        }
        }  // active
        __syncwarp();  // bitmap updates and clears are ordered before the next round
    }
}

template <int B, bool SIMPL, bool EVAL>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, cudaStream_t st)
{
    const size_t smem = dcds_cross_smem_bytes(B, max_range, s);
    auto kern = dcds_cross_kernel<B, SIMPL, EVAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = s.ctas_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = std::max(1, std::min(ntiles, std::max(per_sm, 1) * num_sms));
    kern<<<grid, 128, smem, st>>>(frames, nframes, ntiles, max_range, head, status);
    return cudaGetLastError();
}

template <int B, bool SIMPL>
cudaError_t launch_b(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, bool eval, cudaStream_t st)
{
    if (eval) return launch_t<B, SIMPL, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
    return launch_t<B, SIMPL, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
}

}  // namespace

int cross_tile_h() { return kTileH; }

size_t dcds_cross_smem_bytes(int block, int max_range, const Shape& s)
{
    (void)s;
    const int side = 2 * max_range + 1;
    const int nwb = (side * side + 31) / 32;
    return 128 + 2 * (size_t)cross_stage_bytes(max_range) + (size_t)(128 / (block / 4)) * nwb * 4;
}

cudaError_t dcds_cross_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, dcds_cross_kernel<16, false, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_cross_kernel<16, true, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_cross_kernel<8, false, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_cross_kernel<8, true, false>);
    return e;
}

cudaError_t launch_dcds_cross(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                              bool simplified, const Shape& s, int* head, unsigned* status, int num_sms,
                              cudaStream_t st, bool eval)
{
    if (block == 16)
        return simplified ? launch_b<16, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st)
                          : launch_b<16, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st);
    return simplified ? launch_b<8, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st)
                      : launch_b<8, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st);
}

}  // namespace me
