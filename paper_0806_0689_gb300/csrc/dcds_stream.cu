// dcds_stream.cu -- Directional Cross Diamond Search, streaming kernel.
//
// Same algorithm and results as dcds.cu (Sec. III-B steps 1-4, switching
// strategies one and two, the patterns of Sec. III-A; DCDS^S of Sec. IV-C as
// a compile-time variant).  A different schedule, meant to remove the idle
// lanes at the end of every tile:
//
//   * One CTA per SM keeps NS tiles resident in a ring of shared-memory
//     stages.  A tile enters a free stage through the TMA unit (reference
//     window and current tile, as in dcds.cu) and stays until its last block
//     is finished; then the stage is refilled with the next tile of the
//     global tile counter.
//   * Work comes in two kinds and any warp takes either.  A "row" is step 1
//     (the HCSP, warp-uniform) for one tile row of blocks, claimed from the
//     oldest loaded tile; its continuing blocks go into a CTA-wide FIFO of
//     items.  An "item" is steps 2-4 for one block, run by a 4-lane group in
//     converged diamond rounds reading the tile's stage.  Groups take items
//     from the FIFO regardless of the tile they belong to, so the groups of
//     a warp stay busy across tile boundaries; the only tail is at the end of
//     the launch.
//   * Stage accounting: work[s] counts the rows not yet done plus the items
//     not yet finished of the tile in stage s.  A row adds its items before it
//     removes itself, so work[s] reaches zero exactly when the tile is done.
//   * All waits are polls inside the warp loop with a bounded count; a
//     time-out records STATUS_TIMEOUT and ends the CTA after its copies land.
#include "dcds_common.cuh"

#include <algorithm>
#include <climits>

namespace me {
namespace {

using namespace dcds;

constexpr uint32_t kIdleLimit = 1u << 22;  // warp-loop iterations without progress before a time-out

__device__ __forceinline__ int vld(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ unsigned vldu(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }
__device__ __forceinline__ void vst(int* p, int v) { *reinterpret_cast<volatile int*>(p) = v; }
__device__ __forceinline__ void vstu(unsigned* p, unsigned v) { *reinterpret_cast<volatile unsigned*>(p) = v; }

struct StreamShared {
    int tile, frame;
    int claim;     // (tile sequence << 8) | next row; sequence -1 before the first use
    int work;      // rows not done + items not finished
    int done_seq;  // sequence + 1 of the last tile completed in this stage
};

template <int B, bool SIMPL, int NS>
__global__ void __launch_bounds__(512, 1) dcds_stream_kernel(const FrameDev* __restrict__ frames, int nframes,
                                                             int ntiles, int max_range, int* __restrict__ head,
                                                             unsigned* __restrict__ status)
{
    constexpr int V = kSadVariant;
    constexpr int TXB = kTile / B;    // blocks per tile row
    constexpr int NMB = TXB * TXB;    // blocks per tile
    constexpr int GA = B / 4;         // HCSP lanes per block
    constexpr int WPB = B / 4;        // 4-byte words per block row
    constexpr int RPL = B * WPB / 4;  // diamond-round rows per lane (4 lanes per block)
    // FIFO entries: the items reserved since any unfinished item come from at most
    // 2*NS-1 tiles, so a slot is always free again when its index comes round
    constexpr int CAP = 2 * NS * NMB;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[NS];
    __shared__ StreamShared s_st[NS];
    __shared__ int s_k_issued, s_k_a, s_end_issued, s_no_more, s_rows_out, s_tail, s_head, s_fail;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int cur_off = win_bytes_max(max_range);
    const int stage_bytes = cur_off + kTile * kTile;
    uint2* items = reinterpret_cast<uint2*>(smem + NS * stage_bytes);
    unsigned* flags = reinterpret_cast<unsigned*>(items + CAP);
    const int side_max = 2 * max_range + 1;
    const int nwb = (side_max * side_max + 31) / 32;
    uint32_t* bm_all = reinterpret_cast<uint32_t*>(flags + CAP);

    const int tid = threadIdx.x, lane = tid & 31;
    const int ngroups = blockDim.x >> 2;

    for (int i = tid; i < ngroups * nwb; i += blockDim.x) bm_all[i] = 0u;
    for (int i = tid; i < CAP; i += blockDim.x) flags[i] = 0u;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&s_bar[s], 1);
            s_st[s].tile = 0;
            s_st[s].frame = 0;
            s_st[s].claim = -256;
            s_st[s].work = 0;
            s_st[s].done_seq = 0;
        }
        s_k_issued = 0; s_k_a = 0; s_end_issued = 0; s_no_more = 0;
        s_rows_out = 0; s_tail = 0; s_head = 0; s_fail = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // ---- group state (identical in the 4 lanes of a group) ----
    const int gq = tid >> 2, l4 = lane & 3, lead = lane & ~3;
    const int wb = l4 % WPB, rb = l4 / WPB;
    uint32_t* bm = bm_all + gq * nwb;
    int act = 0;  // 0: needs an item, 1: waiting for its publication, 2: searching, 3: done
    int idx = 0, gs = 0;
    int phase = PH_DDSP, pat = PAT_H, nsp = 0, pick = -1;
    int cx = 0, cy = 0, bxp = 0, byp = 0;
    uint32_t bsad = 0;
    int R = 1, side = 3, WP = 0, dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0, wx0 = 0, wy0 = 0;
    const uint8_t* win = smem;
    uint32_t* out_mv = nullptr;
    uint32_t* out_sad = nullptr;
    uint16_t* out_nsp = nullptr;
    size_t blk = 0;
    uint32_t ds0 = kUnknown, ds1 = kUnknown;
    int wmin = INT_MAX, wmax = -1;
    uint32_t cb[RPL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) cb[r] = 0u;
    uint32_t idle = 0;

    for (;;) {
        bool progress = false;

        // ---- (0) refill a free stage: lane 0 of any warp ----
        if (lane == 0 && !vld(&s_end_issued)) {
            const int j = vld(&s_k_issued);
            const int s = j % NS;
            if ((j < NS || vld(&s_st[s].done_seq) == j - NS + 1) && atomicCAS(&s_k_issued, j, j + 1) == j) {
                const int t = atomicAdd(head, 1);
                s_st[s].tile = t;
                if (t < ntiles) {
                    s_st[s].frame = find_frame(frames, nframes, t);
                    s_st[s].work = TXB;
                    atomicAdd(&s_rows_out, TXB);
                } else {
                    s_st[s].work = 0;
                    vst(&s_end_issued, 1);
                }
                __threadfence_block();
                vst(&s_st[s].claim, j << 8);  // armed for sequence j
                fence_proxy_async();          // the stage's earlier generic reads precede the copy
                if (t < ntiles)
                    issue_tile(t, frames, nframes, ntiles, smem + s * stage_bytes, cur_off, &s_bar[s], &s_st[s].tile,
                               &s_st[s].frame);
                else
                    mbar_arrive(&s_bar[s]);
                progress = true;
            }
        }

        // ---- (1) step 1 for one tile row when the FIFO runs short ----
        int row = -1, rk = 0;
        if (lane == 0 && vld(&s_tail) - vld(&s_head) < ngroups) {
            const int k = vld(&s_k_a);
            const int s = k % NS;
            if ((vld(&s_st[s].claim) >> 8) == k && mbar_try(&s_bar[s], (uint32_t)(k / NS) & 1u)) {
                __threadfence_block();
                if (vld(&s_st[s].tile) >= ntiles) {
                    vst(&s_no_more, 1);
                } else {
                    for (int tries = 0; tries < 32; ++tries) {
                        const int c = vld(&s_st[s].claim);
                        if ((c >> 8) != k || (c & 255) >= TXB) break;
                        if (atomicCAS(&s_st[s].claim, c, c + 1) == c) {
                            row = c & 255;
                            rk = k;
                            if (row == TXB - 1) {
                                __threadfence_block();
                                vst(&s_k_a, k + 1);
                            }
                            break;
                        }
                    }
                }
            }
        }
        row = __shfl_sync(FULL, row, 0);
        if (row >= 0) {
            rk = __shfl_sync(FULL, rk, 0);
            const int s = rk % NS;
            (void)mbar_try(&s_bar[s], (uint32_t)(rk / NS) & 1u);  // completed: every lane acquires the copy
            const int t = vld(&s_st[s].tile);
            const FrameDev* Fp = frames + vld(&s_st[s].frame);
            const int W = Fp->w, H = Fp->h, RA = Fp->range, NBX = Fp->nbx, NBY = Fp->nby;
            uint32_t* __restrict__ a_mv = reinterpret_cast<uint32_t*>(Fp->mv);
            uint32_t* __restrict__ a_sad = Fp->sad;
            uint16_t* __restrict__ a_nsp = Fp->nsp;
            const int lt = t - Fp->tile_base;
            const int txs = Fp->tiles_x;
            const int tile_y = lt / txs, tile_x = lt - tile_y * txs;
            const int bx0 = tile_x * TXB, by0 = tile_y * TXB;
            const int rxa = (RA + 15) & ~15;
            const int WPA = kTile + 2 * rxa;
            const uint8_t* awin = smem + s * stage_bytes;
            const uint8_t* curS = awin + cur_off;

            const int g = lane / GA, w = lane % GA;
            const int bxg = bx0 + g, byg = by0 + row;
            const bool exists = bxg < NBX && byg < NBY;
            uint32_t cw[B];
            const uint32_t* cp = reinterpret_cast<const uint32_t*>(curS + (row * B) * kTile + g * B + 4 * w);
#pragma unroll
            for (int r = 0; r < B; ++r) cw[r] = cp[r * (kTile / 4)];
            const uint8_t* base = awin + (row * B + RA - 1) * WPA + rxa + g * B + 4 * w - 4;
            uint32_t acc[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) acc[k] = 0u;
#pragma unroll
            for (int jj = -1; jj <= B; ++jj) {
                const uint32_t* rp = reinterpret_cast<const uint32_t*>(base + (jj + 1) * WPA);
                const uint32_t b = rp[1];
                if (jj >= 0 && jj < B) {
                    const uint32_t a = rp[0], c = rp[2];
                    acc[0] = sadacc<V>(b, cw[jj], acc[0]);
                    acc[1] = sadacc<V>(__funnelshift_r(a, b, 24), cw[jj], acc[1]);
                    acc[2] = sadacc<V>(__funnelshift_r(b, c, 8), cw[jj], acc[2]);
                    acc[5] = sadacc<V>(__funnelshift_r(a, b, 16), cw[jj], acc[5]);
                    acc[6] = sadacc<V>(__funnelshift_r(b, c, 16), cw[jj], acc[6]);
                }
                if (jj + 1 >= 0 && jj + 1 < B) acc[3] = sadacc<V>(b, cw[jj + 1], acc[3]);  // (0,-1)
                if (jj - 1 >= 0 && jj - 1 < B) acc[4] = sadacc<V>(b, cw[jj - 1], acc[4]);  // (0,+1)
            }
#pragma unroll
            for (int o = 1; o < GA; o <<= 1)
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[k] += __shfl_xor_sync(FULL, acc[k], o);
            const int px = bxg * B, py = byg * B;
            unsigned vmask = 0x7fu;
            if (RA < 2 || px < 2 || px > W - B - 2 || py < 1 || py > H - B - 1) {
                vmask = 0;
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    int ox, oy;
                    decode(kHcsp, k, ox, oy);
                    const bool v = abs(ox) <= RA && abs(oy) <= RA && px + ox >= 0 && px + ox <= W - B &&
                                   py + oy >= 0 && py + oy <= H - B;
                    vmask |= (unsigned)v << k;
                }
            }
            int best = 0;
            uint32_t bs = acc[0];
#pragma unroll
            for (int k = 1; k < 7; ++k)
                if (((vmask >> k) & 1u) && acc[k] < bs) { best = k; bs = acc[k]; }
            const bool leader = (w == 0) && exists;
            if (leader && best == 0) {
                const size_t b0 = (size_t)byg * NBX + bxg;
                a_mv[b0] = 0u;
                a_sad[b0] = bs;
                if (a_nsp) a_nsp[b0] = (uint16_t)__popc(vmask);
            }
            const bool cont = leader && best != 0;
            const unsigned bal = __ballot_sync(FULL, cont);
            if (bal) {
                const int first = __ffs(bal) - 1;
                int qbase = 0;
                if (lane == first) {
                    atomicAdd(&s_st[s].work, __popc(bal));  // before this row leaves the count
                    qbase = atomicAdd(&s_tail, __popc(bal));
                }
                qbase = __shfl_sync(FULL, qbase, first);
                if (cont) {
                    const int q = qbase + __popc(bal & ((1u << lane) - 1u));
                    const int slot = q % CAP;
                    // the slot's previous item was taken long ago; the wait is a safety bound
                    uint32_t spins = 0;
                    while (vldu(&flags[slot]) != 0u && ++spins < kWaitLimit) __nanosleep(32);
                    if (spins >= kWaitLimit) atomicOr(&s_fail, 1);
                    items[slot] = make_uint2((uint32_t)s | ((uint32_t)(row * TXB + g) << 2) | ((uint32_t)best << 10) |
                                                 ((uint32_t)__popc(vmask) << 13),
                                             bs);
                    __threadfence_block();
                    vstu(&flags[slot], (uint32_t)(q / CAP) + 1u);
                }
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicSub(&s_rows_out, 1);
                if (atomicSub(&s_st[s].work, 1) == 1) {
                    __threadfence_block();
                    vst(&s_st[s].done_seq, rk + 1);
                }
            }
            progress = true;
        }

        // ---- (2) one diamond round for the warp's groups ----
        // (a) groups without an item reserve the next FIFO entries (one atomic per warp)
        const unsigned need = __ballot_sync(FULL, act == 0 && l4 == 0);
        if (need) {
            const int first = __ffs(need) - 1;
            int base = 0;
            if (lane == first) base = atomicAdd(&s_head, __popc(need));
            base = __shfl_sync(FULL, base, first);
            const int mine = __shfl_sync(FULL, base + __popc(need & ((1u << lane) - 1u)), lead);
            if (act == 0) { idx = mine; act = 1; }
        }
        // (b) waiting groups: lane 0 polls the entry
        {
            uint2 e = make_uint2(0u, 0u);
            int got = 0;  // 1: item taken, 2: past the last item
            if (act == 1 && l4 == 0) {
                const int slot = idx % CAP;
                if (vldu(&flags[slot]) == (uint32_t)(idx / CAP) + 1u) {
                    __threadfence_block();
                    e = items[slot];
                    __threadfence_block();
                    vstu(&flags[slot], 0u);
                    got = 1;
                } else if (vld(&s_no_more) && vld(&s_rows_out) == 0) {
                    __threadfence_block();
                    if (idx >= vld(&s_tail)) got = 2;
                }
            }
            got = __shfl_sync(FULL, got, lead);
            e.x = __shfl_sync(FULL, e.x, lead);
            e.y = __shfl_sync(FULL, e.y, lead);
            if (act == 1 && got == 2) act = 3;
            if (act == 1 && got == 1) {
                gs = (int)(e.x & 3u);
                (void)mbar_try(&s_bar[gs], (uint32_t)((vld(&s_st[gs].claim) >> 8) / NS) & 1u);  // acquire the copy
                const int mb = (int)((e.x >> 2) & 255u), hb = (int)((e.x >> 10) & 7u);
                const int t = vld(&s_st[gs].tile);
                const FrameDev* Fp = frames + vld(&s_st[gs].frame);
                const int W = Fp->w, H = Fp->h, NBX = Fp->nbx;
                R = Fp->range;
                side = 2 * R + 1;
                const int rx = (R + 15) & ~15;
                WP = kTile + 2 * rx;
                out_mv = reinterpret_cast<uint32_t*>(Fp->mv);
                out_sad = Fp->sad;
                out_nsp = Fp->nsp;
                const int lt = t - Fp->tile_base;
                const int tile_y = lt / Fp->tiles_x, tile_x = lt - tile_y * Fp->tiles_x;
                const int bxl = mb % TXB, byl = mb / TXB;
                const int bxg = tile_x * TXB + bxl, byg = tile_y * TXB + byl;
                const int px = bxg * B, py = byg * B;
                blk = (size_t)byg * NBX + bxg;
                dxlo = max(-R, -px); dxhi = min(R, W - B - px);
                dylo = max(-R, -py); dyhi = min(R, H - B - py);
                win = smem + gs * stage_bytes;
                wx0 = rx + bxl * B + 4 * wb;
                wy0 = R + byl * B + rb * RPL;
                const uint32_t* cp = reinterpret_cast<const uint32_t*>(win + cur_off + (byl * B + rb * RPL) * kTile +
                                                                       bxl * B + 4 * wb);
#pragma unroll
                for (int r = 0; r < RPL; ++r) cb[r] = cp[r * (kTile / 4)];
                decode(kHcsp, hb, cx, cy);
                bxp = cx; byp = cy; bsad = e.y;
                nsp = (int)((e.x >> 13) & 7u);
                pat = (cy == 0) ? PAT_H : PAT_V;  // switching strategy one
                phase = PH_DDSP;
                pick = -1;
                act = 2;
                // every valid HCSP point is visited (lanes take points l4 and l4 + 4)
                for (int k = l4; k < 7; k += 4) {
                    int ox, oy;
                    decode(kHcsp, k, ox, oy);
                    if (ox >= dxlo && ox <= dxhi && oy >= dylo && oy <= dyhi) {
                        const int bit = (oy + R) * side + (ox + R);
                        atomicOr(&bm[bit >> 5], 1u << (bit & 31));
                        wmin = min(wmin, bit >> 5);
                        wmax = max(wmax, bit >> 5);
                    }
                }
                progress = true;
            }
        }
        __syncwarp();  // bitmap initialisation visible to the whole group
        if (__any_sync(FULL, vld(&s_fail) != 0)) break;
        if (!__any_sync(FULL, act != 3)) break;

        if (__any_sync(FULL, act == 2)) {
            // (c) this round's list: lane k checks point k
            uint64_t code;
            int npts;
            if (phase == PH_DDSP) { code = pat ? kDdspV : kDdspH; npts = 4; }
            else if (SIMPL && phase == PH_SIDE) { code = (pat ? kDdspV : kDdspH) >> 12; npts = 2; }
            else {
                code = pat ? kMidV : kMidH;
                npts = 2;
                if (SIMPL && pick >= 0) { code >>= 6 * pick; npts = 1; }
            }
            const bool counted = !(SIMPL && phase == PH_SIDE);
            bool valid = false, fresh = false;
            int bit = 0;
            if (act == 2 && l4 < npts) {
                int ox, oy;
                decode(code, l4, ox, oy);
                const int x = cx + ox, y = cy + oy;
                valid = x >= dxlo && x <= dxhi && y >= dylo && y <= dyhi;
                if (valid) {
                    if (counted) {
                        bit = (y + R) * side + (x + R);
                        fresh = ((bm[bit >> 5] >> (bit & 31)) & 1u) == 0u;
                    } else {
                        fresh = (l4 == 0 ? ds0 : ds1) == kUnknown;
                    }
                }
            }
            const unsigned vb = (__ballot_sync(FULL, valid) >> lead) & 15u;
            const unsigned nbm = (__ballot_sync(FULL, fresh) >> lead) & 15u;
            if (counted && fresh) {
                atomicOr(&bm[bit >> 5], 1u << (bit & 31));
                wmin = min(wmin, bit >> 5);
                wmax = max(wmax, bit >> 5);
            }
            if (SIMPL && phase == PH_DDSP) {
                ds0 = (vb & 4u) ? kUnknown : kInvalid;
                ds1 = (vb & 8u) ? kUnknown : kInvalid;
            }
            if (counted) nsp += __popc(nbm);
            int ncand = 0;
            uint32_t pack = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((nbm >> k) & 1u) { pack |= (uint32_t)k << (4 * ncand); ++ncand; }

            // (d) evaluate the new points, two at a time
            uint32_t sad[4] = {0u, 0u, 0u, 0u};
            int qx[4], qy[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int ox = 0, oy = 0;
                if (i < ncand) decode(code, (int)((pack >> (4 * i)) & 15u), ox, oy);
                qx[i] = cx + ox;  // unused slots read the centre: a valid address
                qy[i] = cy + oy;
            }
            const bool more = __any_sync(FULL, ncand > 2);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && !more) break;
                const int i0 = 2 * half;
                uint32_t a0 = 0u, a1 = 0u;
                if (act == 2) {
                    const int c0 = wx0 + qx[i0], c1 = wx0 + qx[i0 + 1];
                    const uint8_t* p0 = win + (wy0 + qy[i0]) * WP + (c0 & ~3);
                    const uint8_t* p1 = win + (wy0 + qy[i0 + 1]) * WP + (c1 & ~3);
                    const unsigned s0 = (unsigned)(c0 & 3) * 8u, s1 = (unsigned)(c1 & 3) * 8u;
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        const uint32_t l0 = *reinterpret_cast<const uint32_t*>(p0 + r * WP);
                        const uint32_t h0 = *reinterpret_cast<const uint32_t*>(p0 + r * WP + 4);
                        const uint32_t l1 = *reinterpret_cast<const uint32_t*>(p1 + r * WP);
                        const uint32_t h1 = *reinterpret_cast<const uint32_t*>(p1 + r * WP + 4);
                        a0 = sadacc<V>(__funnelshift_r(l0, h0, s0), cb[r], a0);
                        a1 = sadacc<V>(__funnelshift_r(l1, h1, s1), cb[r], a1);
                    }
                }
                a0 += __shfl_xor_sync(FULL, a0, 1);
                a1 += __shfl_xor_sync(FULL, a1, 1);
                a0 += __shfl_xor_sync(FULL, a0, 2);
                a1 += __shfl_xor_sync(FULL, a1, 2);
                sad[i0] = a0;
                sad[i0 + 1] = a1;
            }

            // (e) best point of the list, then the switching strategies (Sec. III-B)
            if (act == 2) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i < ncand) {
                        if (counted && sad[i] < bsad) { bsad = sad[i]; bxp = qx[i]; byp = qy[i]; }
                        if (SIMPL) {
                            const int slot = (int)((pack >> (4 * i)) & 15u);
                            if (phase == PH_DDSP && slot >= 2) { if (slot == 2) ds0 = sad[i]; else ds1 = sad[i]; }
                            else if (phase == PH_SIDE) { if (slot == 0) ds0 = sad[i]; else ds1 = sad[i]; }
                        }
                    }
                }
                if (phase == PH_DDSP) {
                    if (bxp == cx && byp == cy) {
                        phase = SIMPL ? PH_SIDE : PH_MID;  // the centre won: step 4 next
                    } else {
                        if (abs(bxp - cx) + abs(byp - cy) == 1) pat ^= 1;  // switching strategy two
                        cx = bxp; cy = byp;
                    }
                } else if (SIMPL && phase == PH_SIDE) {
                    phase = PH_MID;
                    pick = (ds0 == kInvalid && ds1 == kInvalid) ? -1
                         : (ds0 == kInvalid) ? 1 : (ds1 == kInvalid) ? 0 : (ds1 < ds0 ? 1 : 0);
                } else {  // step 4 evaluated: the block is done
                    if (l4 == 0) {
                        out_mv[blk] = (uint32_t)(uint16_t)bxp | ((uint32_t)(uint16_t)byp << 16);
                        out_sad[blk] = bsad;
                        if (out_nsp) out_nsp[blk] = (uint16_t)nsp;
                    }
                    for (int i = wmin; i <= wmax; ++i) bm[i] = 0u;
                    wmin = INT_MAX; wmax = -1;
                    act = 0;
                    if (l4 == 0) {
                        // the group's reads of the stage are done: release its share of the tile
                        __threadfence_block();
                        if (atomicSub(&s_st[gs].work, 1) == 1) {
                            __threadfence_block();
                            vst(&s_st[gs].done_seq, (vld(&s_st[gs].claim) >> 8) + 1);
                        }
                    }
                }
            }
            __syncwarp();  // bitmap updates and clears are ordered before the next round
            progress = true;
        }

        if (__any_sync(FULL, progress)) {
            idle = 0;
        } else {
            if (++idle > kIdleLimit) {
                if (lane == 0) atomicOr(&s_fail, 1);
                break;
            }
            __nanosleep(64);
        }
    }

    // ---- exit: report a time-out, and let every armed copy land before the CTA's memory goes away ----
    __syncthreads();
    if (tid == 0) {
        if (s_fail && status) atomicOr(status, STATUS_TIMEOUT);
        for (int s = 0; s < NS; ++s) {
            const int seq = s_st[s].claim >> 8;
            if (seq >= 0) (void)mbar_wait(&s_bar[s], (uint32_t)(seq / NS) & 1u);
        }
    }
}

template <int B, bool SIMPL, int NS>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, cudaStream_t st)
{
    const size_t smem = dcds_stream_smem_bytes(B, max_range, s);
    auto kern = dcds_stream_kernel<B, SIMPL, NS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(ntiles, num_sms));
    kern<<<grid, s.threads, smem, st>>>(frames, nframes, ntiles, max_range, head, status);
    return cudaGetLastError();
}

template <int B, bool SIMPL>
cudaError_t launch_b(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, cudaStream_t st)
{
    if (s.stages == 3) return launch_t<B, SIMPL, 3>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
    return launch_t<B, SIMPL, 2>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
}

}  // namespace

size_t dcds_stream_smem_bytes(int block, int max_range, const Shape& s)
{
    const int ns = s.stages == 3 ? 3 : 2;
    const int stage = win_bytes_max(max_range) + kTile * kTile;
    const int nmb = (kTile / block) * (kTile / block);
    const int side = 2 * max_range + 1;
    const int nwb = (side * side + 31) / 32;
    return 128 + (size_t)ns * stage + (size_t)2 * ns * nmb * 12 + (size_t)(s.threads / 4) * nwb * 4;
}

cudaError_t launch_dcds_stream(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                               bool simplified, const Shape& s, int* head, unsigned* status, int num_sms,
                               cudaStream_t st)
{
    if (s.threads % 32 || s.threads < 128 || s.threads > 512) return cudaErrorInvalidValue;
    if (s.stages != 2 && s.stages != 3) return cudaErrorInvalidValue;
    // a shape that does not fit this batch's range gives up a stage, then threads
    Shape f = s;
    while (dcds_stream_smem_bytes(block, max_range, f) > 227 * 1024) {
        if (f.stages == 3) f.stages = 2;
        else if (f.threads > 128) f.threads -= 128;
        else return cudaErrorInvalidValue;
    }
    if (block == 16)
        return simplified ? launch_b<16, true>(frames, nframes, ntiles, max_range, f, head, status, num_sms, st)
                          : launch_b<16, false>(frames, nframes, ntiles, max_range, f, head, status, num_sms, st);
    return simplified ? launch_b<8, true>(frames, nframes, ntiles, max_range, f, head, status, num_sms, st)
                      : launch_b<8, false>(frames, nframes, ntiles, max_range, f, head, status, num_sms, st);
}

}  // namespace me
