// dcds_ws.cu -- Directional Cross Diamond Search, warp-specialised kernel.
//
// Same algorithm and results as dcds.cu (Sec. III-B steps 1-4, switching
// strategies one and two, patterns of Sec. III-A; DCDS^S of Sec. IV-C as a
// compile-time variant); a different schedule:
//
//   * "A" warps own the tiles.  Each CTA pulls 128x128-pixel tiles from the
//     global tile counter; the TMA unit copies the reference window and the
//     current tile into one of two shared-memory stages while the A warps
//     run step 1 (the HCSP, warp-uniform, as in dcds.cu) on the other.  A
//     named barrier synchronises the A warps only.  Blocks whose centre wins
//     are finished; the others are appended to a global item queue (one atomic
//     per 8- or 16-block task) and published with a release flag.
//   * "B" warps run steps 2-4 on queue items: 4-lane groups take items (one
//     atomic per warp), wait for their publication, and run the diamond rounds
//     reading the frames through L1/L2 (the tile has just passed through L2
//     on its way to shared memory).  They never hold up the A warps, and the
//     A warps turn into B warps once the tile counter is exhausted, so no
//     warp waits at a tile barrier for the slowest search.
//   * Waits are bounded: a TMA stage (try_wait), an item not yet published
//     (flag polling with back-off).  On a time-out the kernel records
//     STATUS_TIMEOUT and finishes.  An item is published by writing the
//     launch's epoch (the queue header's epoch + 1) into its flag; the last CTA
//     to finish stores the new epoch.  Flags of an earlier launch, even one
//     that timed out, therefore never look published, and the queue needs no
//     reset between launches.  Item fields are checked before use.
#include "dcds_common.cuh"

#include <algorithm>
#include <climits>

namespace me {
namespace {

using namespace dcds;

enum { C_TILE = 0, C_TAIL = 1, C_HEAD = 2, C_DONE = 3, C_EXIT = 4 };  // counters (zeroed before each launch)
constexpr uint32_t kItemWait = 1u << 24;                  // polls of an unpublished item

__device__ __forceinline__ int ld_acq(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_rel(unsigned* p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void named_sync(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <int B, bool SIMPL>
__global__ void __launch_bounds__(256) dcds_ws_kernel(const FrameDev* __restrict__ frames, int nframes, int ntiles,
                                                      int max_range, int* __restrict__ counters,
                                                      unsigned* __restrict__ queue, int max_items,
                                                      unsigned* __restrict__ status, int a_warps)
{
    constexpr int V = kSadVariant;
    constexpr int TXB = kTile / B;
    constexpr int GA = B / 4;
    constexpr int WPB = B / 4;
    constexpr int RPL = B * WPB / 4;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_tile[2], s_frame[2], s_fail;
    __shared__ unsigned s_epoch;
    unsigned* const flags = queue + kQueueHeadWords;
    uint4* const items = reinterpret_cast<uint4*>(flags + max_items);

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int cur_off = win_bytes_max(max_range);
    const int stage_bytes = cur_off + kTile * kTile;
    const int side_max = 2 * max_range + 1;
    const int nwb = (side_max * side_max + 31) / 32;
    uint32_t* bm_all = reinterpret_cast<uint32_t*>(smem + 2 * stage_bytes);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ngroups = blockDim.x >> 2;
    const int a_threads = a_warps * 32;

    for (int i = tid; i < ngroups * nwb; i += blockDim.x) bm_all[i] = 0u;
    if (tid == 0) {
        s_fail = 0;
        s_epoch = *reinterpret_cast<volatile unsigned*>(queue) + 1u;  // queue[0]: epoch of the last launch
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        issue_tile(atomicAdd(counters + C_TILE, 1), frames, nframes, ntiles, smem, cur_off, &s_bar[0], &s_tile[0],
                   &s_frame[0]);
    }
    __syncthreads();

    const unsigned epoch = s_epoch;

    // ================================================================ A warps
    if (warp < a_warps) {
        for (int it = 0;; ++it) {
            const int st = it & 1;
            const uint32_t par = (it >> 1) & 1;
            if (!mbar_wait(&s_bar[st], par)) atomicOr(&s_fail, 1);
            named_sync(1, a_threads);
            if (s_fail) {
                if (tid == 0 && status) atomicOr(status, STATUS_TIMEOUT);
                if (tid == 0) (void)mbar_wait(&s_bar[st], par);  // bounded: let an outstanding copy land
                break;
            }
            const int t = s_tile[st];
            if (t >= ntiles) break;
            if (tid == 0) {
                // stage st^1 was last read in the previous tile, which ended with the A barrier
                fence_proxy_async();
                issue_tile(atomicAdd(counters + C_TILE, 1), frames, nframes, ntiles, smem + (st ^ 1) * stage_bytes,
                           cur_off, &s_bar[st ^ 1], &s_tile[st ^ 1], &s_frame[st ^ 1]);
            }
            const int f = s_frame[st];
            const FrameDev* Fp = frames + f;
            const int W = Fp->w, H = Fp->h, R = Fp->range, NBX = Fp->nbx, NBY = Fp->nby;
            uint32_t* __restrict__ out_mv = reinterpret_cast<uint32_t*>(Fp->mv);
            uint32_t* __restrict__ out_sad = Fp->sad;
            uint16_t* __restrict__ out_nsp = Fp->nsp;
            const int lt = t - Fp->tile_base;
            const int txs = Fp->tiles_x;
            const int tile_y = lt / txs, tile_x = lt - tile_y * txs;
            const int bx0 = tile_x * TXB, by0 = tile_y * TXB;
            const int rx = (R + 15) & ~15;
            const int WP = kTile + 2 * rx;
            const uint8_t* win = smem + st * stage_bytes;
            const uint8_t* curS = win + cur_off;

            for (int row = warp; row < TXB; row += a_warps) {
                const int g = lane / GA, w = lane % GA;
                const int bxg = bx0 + g, byg = by0 + row;
                const bool exists = bxg < NBX && byg < NBY;
                uint32_t cw[B];
                const uint32_t* cp = reinterpret_cast<const uint32_t*>(curS + (row * B) * kTile + g * B + 4 * w);
#pragma unroll
                for (int r = 0; r < B; ++r) cw[r] = cp[r * (kTile / 4)];
                const uint8_t* base = win + (row * B + R - 1) * WP + rx + g * B + 4 * w - 4;
                uint32_t acc[7];
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[k] = 0u;
#pragma unroll
                for (int jj = -1; jj <= B; ++jj) {
                    const uint32_t* rp = reinterpret_cast<const uint32_t*>(base + (jj + 1) * WP);
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
                if (R < 2 || px < 2 || px > W - B - 2 || py < 1 || py > H - B - 1) {
                    vmask = 0;
#pragma unroll
                    for (int k = 0; k < 7; ++k) {
                        int ox, oy;
                        decode(kHcsp, k, ox, oy);
                        const bool v = abs(ox) <= R && abs(oy) <= R && px + ox >= 0 && px + ox <= W - B &&
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
                const int blk = byg * NBX + bxg;
                if (leader && best == 0) {
                    out_mv[blk] = 0u;
                    out_sad[blk] = bs;
                    if (out_nsp) out_nsp[blk] = (uint16_t)__popc(vmask);
                }
                const bool cont = leader && best != 0;
                const unsigned bal = __ballot_sync(FULL, cont);
                if (bal) {
                    const int first = __ffs(bal) - 1;
                    int qbase = 0;
                    if (lane == first) qbase = atomicAdd(counters + C_TAIL, __popc(bal));
                    qbase = __shfl_sync(FULL, qbase, first);
                    if (cont) {
                        const int q = qbase + __popc(bal & ((1u << lane) - 1u));
                        if (q < max_items) {
                            items[q] = make_uint4((uint32_t)f, (uint32_t)blk,
                                                  (uint32_t)best | ((uint32_t)__popc(vmask) << 8), bs);
                            __threadfence();
                            st_rel(flags + q, epoch);
                        } else if (status) {
                            atomicOr(status, STATUS_BAD_ARG);
                        }
                    }
                }
            }
            named_sync(1, a_threads);  // every A read of this stage is done
            if (tid == 0) {
                __threadfence();  // this tile's queue reservations precede the count
                atomicAdd(counters + C_DONE, 1);
            }
        }
    }

    // ================================================================ B warps (and A warps when the tiles run out)
    {
        const int gq = tid >> 2, l4 = lane & 3, lead = lane & ~3;
        const int wb = l4 % WPB, rb = l4 / WPB;
        uint32_t* bm = bm_all + gq * nwb;

        int act = 0;  // 0: needs an item, 1: waiting for its publication, 2: searching, 3: done
        int idx = 0;
        uint32_t waited = 0;
        int phase = PH_DDSP, pat = PAT_H, nsp = 0, pick = -1;
        int cx = 0, cy = 0, bxp = 0, byp = 0;
        uint32_t bsad = 0;
        int R = 1, side = 3, dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0, px = 0, py = 0, pitch = 0;
        const uint8_t* ref = nullptr;
        uint32_t* out_mv = nullptr;
        uint32_t* out_sad = nullptr;
        uint16_t* out_nsp = nullptr;
        int blk = 0;
        uint32_t ds0 = kUnknown, ds1 = kUnknown;
        int wmin = INT_MAX, wmax = -1;
        uint32_t cb[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) cb[r] = 0u;

        for (;;) {
            // ---- claim: one atomic for all groups of the warp that need an item ----
            const unsigned need = __ballot_sync(FULL, act == 0 && l4 == 0);
            if (need) {
                const int first = __ffs(need) - 1;
                int base = 0;
                if (lane == first) base = atomicAdd(counters + C_HEAD, __popc(need));
                base = __shfl_sync(FULL, base, first);
                const int mine = __shfl_sync(FULL, base + __popc(need & ((1u << lane) - 1u)), lead);
                if (act == 0) { idx = mine; act = 1; waited = 0; }
            }
            // ---- waiting groups: lane 0 polls the flag, then takes the item ----
            uint4 e = make_uint4(0u, 0u, 0u, 0u);
            int got = 0;  // 1: item taken, 2: past the end of the queue
            if (act == 1 && l4 == 0) {
                if (idx >= max_items) {
                    got = 2;  // beyond the queue: the producer has recorded STATUS_BAD_ARG
                } else if (ld_acq(flags + idx) == epoch) {
                    e = items[idx];
                    got = 1;
                } else if (ld_acq(counters + C_DONE) >= ntiles && idx >= ld_acq(counters + C_TAIL)) {
                    got = 2;
                } else if (++waited > kItemWait) {
                    if (status) atomicOr(status, STATUS_TIMEOUT);
                    got = 2;
                }
            }
            got = __shfl_sync(FULL, got, lead);
            e.x = __shfl_sync(FULL, e.x, lead);
            e.y = __shfl_sync(FULL, e.y, lead);
            e.z = __shfl_sync(FULL, e.z, lead);
            e.w = __shfl_sync(FULL, e.w, lead);
            if (act == 1 && got == 2) act = 3;
            if (act == 1 && got == 1) {
                const int f = (int)e.x;
                const FrameDev* Fp = frames + (f < nframes ? f : 0);
                const int nb = Fp->nbx * Fp->nby;
                if (f >= nframes || (int)e.y >= nb || (e.z & 7u) > 6u) {
                    if (l4 == 0 && status) atomicOr(status, STATUS_BAD_ARG);
                    act = 0;
                } else {
                    blk = (int)e.y;
                    R = Fp->range;
                    side = 2 * R + 1;
                    pitch = Fp->pitch;
                    ref = Fp->ref;
                    out_mv = reinterpret_cast<uint32_t*>(Fp->mv);
                    out_sad = Fp->sad;
                    out_nsp = Fp->nsp;
                    px = (blk % Fp->nbx) * B;
                    py = (blk / Fp->nbx) * B;
                    dxlo = max(-R, -px); dxhi = min(R, Fp->w - B - px);
                    dylo = max(-R, -py); dyhi = min(R, Fp->h - B - py);
                    const uint8_t* cp = Fp->cur + (size_t)(py + rb * RPL) * pitch + px + 4 * wb;
#pragma unroll
                    for (int r = 0; r < RPL; ++r) cb[r] = __ldg(reinterpret_cast<const uint32_t*>(cp + (size_t)r * pitch));
                    decode(kHcsp, (int)(e.z & 7u), cx, cy);
                    bxp = cx; byp = cy; bsad = e.w;
                    nsp = (int)((e.z >> 8) & 15u);
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
                }
            }
            __syncwarp();  // bitmap initialisation visible to the whole group
            if (!__any_sync(FULL, act != 3)) break;
            if (!__any_sync(FULL, act == 2)) {  // nothing to search yet: back off
                __nanosleep(128);
                continue;
            }

            // ---- this round's list: lane k checks point k ----
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

            // ---- evaluate the new points (two at a time, from L1/L2) ----
            uint32_t sad[4] = {0u, 0u, 0u, 0u};
            int qx[4], qy[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int ox = 0, oy = 0;
                if (i < ncand) decode(code, (int)((pack >> (4 * i)) & 15u), ox, oy);
                qx[i] = cx + ox;  // unused slots read the centre: inside the frame
                qy[i] = cy + oy;
            }
            const bool more = __any_sync(FULL, ncand > 2);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && !more) break;
                const int i0 = 2 * half;
                uint32_t a0 = 0u, a1 = 0u;
                if (act == 2) {
                    const long g0 = (long)(py + qy[i0] + rb * RPL) * pitch + px + qx[i0] + 4 * wb;
                    const long g1 = (long)(py + qy[i0 + 1] + rb * RPL) * pitch + px + qx[i0 + 1] + 4 * wb;
                    const uint32_t* p0 = reinterpret_cast<const uint32_t*>(ref + (g0 & ~3l));
                    const uint32_t* p1 = reinterpret_cast<const uint32_t*>(ref + (g1 & ~3l));
                    const unsigned s0 = (unsigned)(g0 & 3) * 8u, s1 = (unsigned)(g1 & 3) * 8u;
                    const int pw = pitch >> 2;
#pragma unroll
                    for (int r = 0; r < RPL; ++r) {
                        // the second word is read only for an unaligned segment, and then it
                        // lies inside the row
                        const uint32_t l0 = __ldg(p0 + r * pw), h0 = s0 ? __ldg(p0 + r * pw + 1) : 0u;
                        const uint32_t l1 = __ldg(p1 + r * pw), h1 = s1 ? __ldg(p1 + r * pw + 1) : 0u;
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

            // ---- best point of the list, then switching strategies (Sec. III-B) ----
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
                }
            }
            __syncwarp();  // bitmap updates and clears are ordered before the next round
        }
    }

    // the last CTA to finish publishes this launch's epoch (every CTA read the old one at its start)
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(counters + C_EXIT, 1) == (int)gridDim.x - 1) {
            __threadfence();
            *reinterpret_cast<volatile unsigned*>(queue) = epoch;
        }
    }
}

template <int B, bool SIMPL>
cudaError_t launch_ws_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s,
                        int* counters, unsigned* queue, int max_items, unsigned* status, int num_sms,
                        cudaStream_t st)
{
    const size_t smem = dcds_ws_smem_bytes(B, max_range, s);
    auto kern = dcds_ws_kernel<B, SIMPL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = s.ctas_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.threads, smem);
        if (e != cudaSuccess) return e;
    }
    // the B warps may wait on items the A warps of other CTAs publish: every CTA must be resident
    const int grid = std::max(1, std::max(per_sm, 1) * num_sms);
    const int a_warps = std::min(std::max(1, s.a_warps), s.threads / 32);
    kern<<<grid, s.threads, smem, st>>>(frames, nframes, ntiles, max_range, counters, queue, max_items, status,
                                        a_warps);
    return cudaGetLastError();
}

}  // namespace

size_t dcds_ws_smem_bytes(int block, int max_range, const Shape& s)
{
    (void)block;
    const int stage = win_bytes_max(max_range) + kTile * kTile;
    const int side = 2 * max_range + 1;
    const int nwb = (side * side + 31) / 32;
    return 128 + 2 * (size_t)stage + (size_t)(s.threads / 4) * nwb * 4;
}

cudaError_t launch_dcds_ws(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                           bool simplified, const Shape& s, int* counters, void* queue, int max_items,
                           unsigned* status, int num_sms, cudaStream_t st)
{
    if (s.threads != 128 && s.threads != 256) return cudaErrorInvalidValue;
    if (max_items <= 0 || (max_items & 3)) return cudaErrorInvalidValue;  // items stay 16-byte aligned
    unsigned* q = reinterpret_cast<unsigned*>(queue);
    if (block == 16)
        return simplified ? launch_ws_t<16, true>(frames, nframes, ntiles, max_range, s, counters, q, max_items,
                                                  status, num_sms, st)
                          : launch_ws_t<16, false>(frames, nframes, ntiles, max_range, s, counters, q, max_items,
                                                   status, num_sms, st);
    return simplified ? launch_ws_t<8, true>(frames, nframes, ntiles, max_range, s, counters, q, max_items, status,
                                             num_sms, st)
                      : launch_ws_t<8, false>(frames, nframes, ntiles, max_range, s, counters, q, max_items, status,
                                              num_sms, st);
}

}  // namespace me
