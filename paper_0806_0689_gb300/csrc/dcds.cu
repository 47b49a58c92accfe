// dcds.cu -- Directional Cross Diamond Search on sm_103a.
//
// Algorithm: Jia & Zhang, Sec. III-B (steps 1-4, switching strategies one
// and two) with the patterns of Sec. III-A (HCSP, HDSP, VDSP and the middle
// points); DCDS^S of Sec. IV-C as a compile-time variant.
//
// GPU mapping
//   * Persistent CTAs pull 128x128-pixel tiles from a global counter (the work
//     queue over every frame pair of the launch; a CTA's first tile is its
//     own index).  For each tile the TMA unit
//     copies the reference window (the tile grown by R rows and by R rounded
//     up to 16 columns, zero-filled outside the frame) and the current tile
//     into shared memory (cp.async.bulk.tensor.2d, completion on an
//     mbarrier).  With two stages the next tile is fetched while this one is
//     searched.
//   * Phase A (step 1 for every block, warp-uniform): a warp takes one tile
//     row of blocks per pass (two rows for the search alone), B/4 lanes per
//     block, lane w holding 4-pixel column w of the block.  The five
//     horizontal HCSP points share each reference row (three aligned words
//     and four funnel shifts), the two vertical points
//     reuse the neighbouring rows, so the 7 SADs cost 18 rows of reads.
//     Blocks whose centre wins are finished (the half-way stop, Sec. III-C);
//     the others go to a per-tile ring in shared memory.
//   * Phase B (steps 2-4): groups of LPB lanes per block (2 for 16x16, 4
//     for 8x8) pull blocks from the ring and run the diamond rounds.  A round evaluates every new point of the
//     current pattern (at most 4) at once, then applies the switching
//     strategies.  A per-group bitmap of visited points (one bit per
//     displacement of the +-R window; for 8x8 blocks a 32 x 32 box of
//     displacements, a block whose path leaves it being searched again after
//     the pass with +-R bitmaps) keeps points from being evaluated or
//     counted twice.  A point evaluated earlier always has a SAD no smaller
//     than the current centre's (every move lowers the best SAD strictly), so
//     skipping it leaves the path unchanged.
//   * Ties: candidates are compared in the fixed pattern order with a strict
//     "<", so the centre and earlier points keep a tie (the oracle's order).
//   * With EVAL the measures of Sec. IV are fused in, from the staged tile,
//     so the frames are read once: sum |e| is the SAD at the final MV, sum e^2
//     takes one pass over the block at that MV (during the HCSP for blocks
//     whose centre wins; for the others in a dense pass over the ring after
//     the rounds, where phase B left each block's final MV, SAD and count),
//     the MV is compared with the full-search MV, and the tile's sums (the
//     warps' totals met in shared memory) go to the frame's eight counters
//     with one set of integer atomics per tile -- the same sums the
//     evaluation kernel computes.
#include "dcds_common.cuh"

#include <algorithm>
#include <climits>
#include <type_traits>

namespace me {
namespace {

using namespace dcds;

// Bounds-check build (-DME_CHECK, the stand-in for a memory sanitizer): every
// shared-memory word the search reads from a staged tile is checked against
// the region it belongs to (the tile's reference window, or its current
// blocks), and every ring and bitmap index against its array; an access
// outside is skipped (a read gives 0) and recorded in the status word
// (STATUS_BOUNDS).  The default build compiles the checks away.
struct Region {
#ifdef ME_CHECK
    const uint8_t* lo;
    const uint8_t* hi;
    unsigned* status;
#endif
};

__device__ __forceinline__ Region region(const uint8_t* lo, size_t bytes, unsigned* status)
{
#ifdef ME_CHECK
    return Region{lo, lo + bytes, status};
#else
    (void)lo; (void)bytes; (void)status;
    return Region{};
#endif
}

__device__ __forceinline__ bool index_ok(int i, int n, unsigned* status)
{
#ifdef ME_CHECK
    if (i >= 0 && i < n) return true;
    if (status) atomicOr(status, STATUS_BOUNDS);
    return false;
#else
    (void)i; (void)n; (void)status;
    return true;
#endif
}

__device__ __forceinline__ uint32_t ld_word(const uint8_t* p, const Region& g)
{
#ifdef ME_CHECK
    if (p < g.lo || p + 4 > g.hi || (reinterpret_cast<uintptr_t>(p) & 3u)) {
        if (g.status) atomicOr(g.status, STATUS_BOUNDS);
        return 0u;
    }
#else
    (void)g;
#endif
    return *reinterpret_cast<const uint32_t*>(p);
}

// Lanes per block in the diamond rounds (phase B).  Measured on the 1080p
// batch (16x16, +-16) and the 2160p 8x8 +-32 batch: 16x16 with 2 lanes 5 %
// faster than with 4 for the search alone, the same with the evaluation
// fused; 8x8 with 2 or 1 lanes 23 % and 35 % slower (the per-group bitmaps
// cost CTAs per SM), and with 1 lane and a 15 x 15 visited box per lane
// (blocks whose path leaves it searched again in an overflow pass) 56 %
// slower: 32 lanes reading 32 unrelated rows multiply the bank conflicts.
__host__ __device__ constexpr int dcds_lanes_per_block(int block) { return block == 16 ? 2 : 4; }

// Visited points of an 8x8 block in phase B, in the box variant (BOX): a
// 32 x 32 box of displacements (-16 .. 15 on each axis; word y + 16, bit
// x + 16) instead of the +-R bitmap, which at +-32 is four times larger and,
// over 64 groups, costs a CTA per SM.  A block that meets a point outside the
// box is dropped (its ring entry still holds the HCSP result) and searched
// again from the start after the main pass, by one warp with +-R bitmaps: the
// same path, the same count.  The groups' boxes lie 33 words apart, so that
// the same row of eight groups' boxes falls in eight banks.  The launcher
// takes this variant where it fits more CTAs per SM than the +-R bitmaps
// (2160p 8x8 +-32, 256 threads: three instead of two, 302 -> 275 us for
// DCDS, 442 -> 376 us for DCDS^S); where both fit as many, the box's extra
// registers (80 against 64) cost a CTA and it measured 10-12 % slower.
constexpr int kBoxWords = 33;

// Lanes of a phase-B group: a block of B x B pixels (B / 4 words per row) is
// split over LPB lanes, each holding CPL adjacent word columns of RPL rows:
// rows row0, row0 + RS, row0 + 2 RS, ... from column col0.  With more lanes
// than words per row the lanes of one column interleave their rows (RS > 1):
// lanes that read rows 4 apart would hit the same banks (a window row is 40
// or 48 words, so 4 rows are a multiple of 32 words), rows 1 apart do not.
template <int B, int LPB>
struct GroupMap {
    static constexpr int WPB = B / 4;
    static constexpr int CPL = WPB >= LPB ? WPB / LPB : 1;
    static constexpr int RPL = WPB >= LPB ? B : B * WPB / LPB;
    static constexpr int RS = WPB >= LPB ? 1 : LPB / WPB;
    __device__ static int col0(int lg) { return WPB >= LPB ? lg * CPL : lg % WPB; }
    __device__ static int row0(int lg) { return WPB >= LPB ? 0 : lg / WPB; }
};

// SADs of NP candidates (slots i0 .. i0 + NP - 1 of qx / qy; only those below
// nvalid are loaded, so groups with fewer candidates add no shared-memory
// traffic) of an LPB-lane group (a lane's rows RS apart).  Per row a lane loads the CPL + 1 aligned
// words that cover its CPL unaligned ones; the loads of all NP points are
// issued together, then each sum is completed across the group (every lane
// of the warp takes part in the shuffles).
template <int NP, int V, int RPL, int CPL, int LPB, int RS>
__device__ __forceinline__ void eval_points(const uint8_t* win, int WP, int wx0, int wy0, const int (&qx)[4],
                                            const int (&qy)[4], const uint32_t (&cb)[RPL][CPL],
                                            uint32_t (&sad)[4], int i0, int nvalid, const Region& gw)
{
    const uint8_t* p[NP];
    unsigned sh[NP];
    uint32_t a[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int c = wx0 + qx[i0 + k];
        p[k] = win + (wy0 + qy[i0 + k]) * WP + (c & ~3);
        sh[k] = (unsigned)(c & 3) * 8u;
        a[k] = 0u;
    }
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (i0 + k < nvalid) {
                uint32_t w[CPL + 1];
#pragma unroll
                for (int j = 0; j < CPL; ++j) w[j] = ld_word(p[k] + r * RS * WP + 4 * j, gw);
                // the word after them only when the columns are unaligned (at the
                // window's right edge an aligned block needs nothing beyond it)
                w[CPL] = ld_word(p[k] + r * RS * WP + 4 * CPL, gw);
#pragma unroll
                for (int j = 0; j < CPL; ++j) a[k] = sadacc<V>(__funnelshift_r(w[j], w[j + 1], sh[k]), cb[r][j], a[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) {
#pragma unroll
        for (int o = 1; o < LPB; o <<= 1) a[k] += __shfl_xor_sync(0xffffffffu, a[k], o);
        sad[i0 + k] = a[k];
    }
}

// Sec. IV sums of one finished block into the thread's tile sums e = {ABS, SQ,
// NSP, EQUAL, PIXELS} (32 bits hold a tile's worth) and dist.  fw: the block's
// full-search MV.
__device__ __forceinline__ void eval_block(int dx, int dy, uint32_t sad, uint32_t sq, int nsp, bool has_nsp,
                                           bool has_fs, uint32_t fw, int bb, uint32_t (&e)[5],
                                           unsigned long long& dist)
{
    e[0] += sad;
    e[1] += sq;
    if (has_nsp) e[2] += (unsigned)nsp;
    if (has_fs) {
        const int ex = dx - (int)(int16_t)(fw & 0xffffu), ey = dy - (int)(int16_t)(fw >> 16);
        if (ex == 0 && ey == 0) e[3] += 1u;
        else dist += dist_q24(ex, ey);
    }
    e[4] += (unsigned)bb;
}

template <int B, bool SIMPL, int NST, bool EVAL, bool BOX>
__device__ __forceinline__ void dcds_tiles(const FrameDev* __restrict__ frames, int nframes, int ntiles, int max_range,
                                           int* __restrict__ head, unsigned* __restrict__ status)
{
    constexpr int V = kSadVariant;
    constexpr int TH = kDcdsTileH;        // tile height in pixels (width kTile)
    constexpr int TXB = kTile / B;        // blocks per tile row
    constexpr int TYB = TH / B;           // block rows per tile
    constexpr int NMB = TXB * TYB;        // blocks per tile
    constexpr int GA = B / 4;             // phase-A lanes per block
    constexpr int LPB = dcds_lanes_per_block(B);  // phase-B lanes per block
    using GM = GroupMap<B, LPB>;
    constexpr int RPLB = GM::RPL, CPL = GM::CPL, RSB = GM::RS;
    constexpr unsigned FULL = 0xffffffffu;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[NST];
    __shared__ int s_tile[NST];
    __shared__ TileDesc s_desc[NST];
    __shared__ unsigned long long s_part[EVAL ? 8 : 1][6];  // EVAL: the warps' tile sums
    __shared__ int s_ring_n, s_ring_next, s_novf, s_ovf_next;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int cur_off = win_bytes_max(max_range, TH);
    const int stage_bytes = cur_off + kTile * TH;
    uint2* ring = reinterpret_cast<uint2*>(smem + NST * stage_bytes);
    const int side_max = 2 * max_range + 1;
    const int nwb = (side_max * side_max + 31) / 32;
    const int bw = BOX ? kBoxWords : nwb;  // visited words per group in the main pass
    // one +-R bitmap or visited box per group; BOX: then +-R bitmaps for
    // the overflow warp's groups and the tile's overflow list
    uint32_t* bm_all = reinterpret_cast<uint32_t*>(ring + NMB);
    uint32_t* bm_full = bm_all + (int)(blockDim.x / LPB) * bw;
    const int nclear = (int)(blockDim.x / LPB) * bw + (BOX ? (32 / LPB) * nwb : 0);
    int* ovf = reinterpret_cast<int*>(bm_all + nclear);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int i = tid; i < nclear; i += blockDim.x) bm_all[i] = 0u;
    // failure-detection test hook (last counter word, zero unless the host set it):
    // the first copy is armed for 16 bytes it never receives and the waits are shortened
    const bool starve = head[kCounterInts - 1] != 0;
    const uint32_t wait_limit = starve ? kShortWait : kWaitLimit;
    uint32_t esum[5] = {0u, 0u, 0u, 0u, 0u};  // EVAL: this tile's ABS SQ NSP EQUAL PIXELS
    unsigned long long edist = 0ull;          // EVAL: this tile's DIST_Q24
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&s_bar[s], 1);
        fence_mbar_init();
        // a CTA's first tile is its own index (the grid never exceeds the tile
        // count), later ones come from the counter: the launch does not open with
        // every CTA queueing on the counter's one word
        issue_tile((int)blockIdx.x, frames, nframes, ntiles, smem, cur_off, TH, &s_bar[0], &s_tile[0],
                   &s_desc[0], starve ? 16u : 0u);
    }
    __syncthreads();

    for (int it = 0;; ++it) {
        const int st = (NST == 2) ? (it & 1) : 0;
        const uint32_t par = (NST == 2) ? ((it >> 1) & 1) : (it & 1);
        if (tid == 0) { s_ring_n = 0; s_ring_next = 0; s_novf = 0; s_ovf_next = 0; }
        const bool ok = mbar_wait(&s_bar[st], par, wait_limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && status) atomicOr(status, STATUS_TIMEOUT);
            // give an outstanding copy a bounded chance to land before exiting
            if (tid == 0) (void)mbar_wait(&s_bar[st], par, wait_limit);
            break;
        }
        const int t = s_tile[st];
        if (t >= ntiles) break;
        uint8_t* stage = smem + st * stage_bytes;
        if (NST == 2 && tid == 0) {
            // stage st^1 was last read in the previous tile, which ended with a barrier
            fence_proxy_async();
            issue_tile((int)gridDim.x + atomicAdd(head, 1), frames, nframes, ntiles, smem + (st ^ 1) * stage_bytes,
                       cur_off, TH, &s_bar[st ^ 1], &s_tile[st ^ 1], &s_desc[st ^ 1]);
        }
        // descriptor fields in registers (from the claim's shared copy): the
        // output stores below cannot alias them
        const TileDesc& D = s_desc[st];
        const int W = D.w, H = D.h, R = D.range, NBX = D.nbx, NBY = D.nby;
        uint32_t* __restrict__ out_mv = D.mv;
        uint32_t* __restrict__ out_sad = D.sad;
        uint16_t* __restrict__ out_nsp = D.nsp;
        const uint32_t* __restrict__ mv_fs = EVAL ? D.mv_fs : nullptr;
        unsigned long long* const sums = EVAL ? D.sums : nullptr;
        const bool first_tile = D.first != 0;
        const int tile_y = D.tile_y, tile_x = D.tile_x;
        const int bx0 = tile_x * TXB, by0 = tile_y * TYB;
        const int rx = (R + 15) & ~15;
        const int WP = kTile + 2 * rx;  // window row pitch
        const uint8_t* win = stage;
        const uint8_t* curS = stage + cur_off;
        // this tile's window rows; the word after a lane's last needed byte is
        // always loaded (a shift of 0 discards it: loading it only when needed
        // measured 26 % slower), so at the window's last row a read may reach
        // 4 bytes past it, still inside the stage (the current tile follows)
        const Region gw = region(win, (size_t)WP * (TH + 2 * R) + 4, status);
        const Region gc = region(curS, (size_t)kTile * TH, status);       // its current blocks

        // ------------------------------------------------ phase A: HCSP
        // A warp takes NR tile rows of blocks per pass (the search alone: two
        // while the tile has at least two rows per warp left): the rows' loads
        // and SADs are independent, so one pass keeps twice as many in flight.
        auto hcsp_rows = [&](int row0, int rstep, auto nr_c) {
            constexpr int NR = decltype(nr_c)::value;
            const int g = lane / GA, w = lane % GA;
            const int bxg = bx0 + g;
            uint32_t fw0[NR];  // the FS vectors, fetched now so their latency hides behind the SADs
            uint32_t cw[NR][B];
            uint32_t acc[NR][7];
            uint32_t sq0[NR];  // sum of squared errors at (0,0), EVAL only
            const uint8_t* base[NR];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int row = row0 + q * rstep, byg = by0 + row;
                fw0[q] = 0u;
                if (EVAL && mv_fs && bxg < NBX && byg < NBY && w == 0) fw0[q] = __ldg(mv_fs + (size_t)byg * NBX + bxg);
                const uint32_t* cp = reinterpret_cast<const uint32_t*>(curS + (row * B) * kTile + g * B + 4 * w);
#pragma unroll
                for (int r = 0; r < B; ++r)
                    cw[q][r] = ld_word(reinterpret_cast<const uint8_t*>(cp + r * (kTile / 4)), gc);
                base[q] = win + (row * B + R - 1) * WP + rx + g * B + 4 * w - 4;
                sq0[q] = 0u;
#pragma unroll
                for (int k = 0; k < 7; ++k) acc[q][k] = 0u;
            }
#pragma unroll
            for (int jj = -1; jj <= B; ++jj) {
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    const uint8_t* rp = base[q] + (jj + 1) * WP;
                    const uint32_t b = ld_word(rp + 4, gw);
                    if (jj >= 0 && jj < B) {
                        const uint32_t a = ld_word(rp, gw), c = ld_word(rp + 8, gw);
                        if constexpr (EVAL) {
                            const uint32_t d0 = __vabsdiffu4(b, cw[q][jj]);
                            sq0[q] = __dp4a(d0, d0, sq0[q]);
                        }
                        acc[q][0] = sadacc<V>(b, cw[q][jj], acc[q][0]);
                        acc[q][1] = sadacc<V>(__funnelshift_r(a, b, 24), cw[q][jj], acc[q][1]);
                        acc[q][2] = sadacc<V>(__funnelshift_r(b, c, 8), cw[q][jj], acc[q][2]);
                        acc[q][5] = sadacc<V>(__funnelshift_r(a, b, 16), cw[q][jj], acc[q][5]);
                        acc[q][6] = sadacc<V>(__funnelshift_r(b, c, 16), cw[q][jj], acc[q][6]);
                    }
                    if (jj + 1 >= 0 && jj + 1 < B) acc[q][3] = sadacc<V>(b, cw[q][jj + 1], acc[q][3]);  // (0,-1)
                    if (jj - 1 >= 0 && jj - 1 < B) acc[q][4] = sadacc<V>(b, cw[q][jj - 1], acc[q][4]);  // (0,+1)
                }
            }
#pragma unroll
            for (int o = 1; o < GA; o <<= 1) {
#pragma unroll
                for (int q = 0; q < NR; ++q) {
#pragma unroll
                    for (int k = 0; k < 7; ++k) acc[q][k] += __shfl_xor_sync(FULL, acc[q][k], o);
                    if constexpr (EVAL) sq0[q] += __shfl_xor_sync(FULL, sq0[q], o);
                }
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int row = row0 + q * rstep, byg = by0 + row;
                const bool exists = bxg < NBX && byg < NBY;
                const int px = bxg * B, py = byg * B;
                unsigned vmask = 0x7fu;  // all 7 HCSP points inside the window and the frame
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
                uint32_t bs = acc[q][0];
#pragma unroll
                for (int k = 1; k < 7; ++k)
                    if (((vmask >> k) & 1u) && acc[q][k] < bs) { best = k; bs = acc[q][k]; }
                const bool leader = (w == 0) && exists;
                if (leader && best == 0) {
                    const size_t blk = (size_t)byg * NBX + bxg;
                    out_mv[blk] = 0u;
                    out_sad[blk] = bs;
                    if (out_nsp) out_nsp[blk] = (uint16_t)__popc(vmask);
                    if constexpr (EVAL)
                        eval_block(0, 0, bs, sq0[q], __popc(vmask), out_nsp != nullptr, mv_fs != nullptr, fw0[q],
                                   B * B, esum, edist);
                }
                const bool cont = leader && best != 0;
                const unsigned bal = __ballot_sync(FULL, cont);
                if (bal) {
                    const int first = __ffs(bal) - 1;
                    int rbase = 0;
                    if (lane == first) rbase = atomicAdd(&s_ring_n, __popc(bal));
                    rbase = __shfl_sync(FULL, rbase, first);
                    if (cont && index_ok(rbase + __popc(bal & ((1u << lane) - 1u)), NMB, status)) {
                        const int rank = __popc(bal & ((1u << lane) - 1u));
                        ring[rbase + rank] = make_uint2((uint32_t)(row * TXB + g) | ((uint32_t)best << 8) |
                                                            ((uint32_t)__popc(vmask) << 11),
                                                        bs);
                    }
                }
            }
        };
        {
            int row = warp;
            // two rows per pass measured faster for the search alone, slower with
            // the evaluation fused (its registers are at the four-CTA limit)
            if constexpr (!EVAL)
                for (; row + nwarps < TYB; row += 2 * nwarps)
                    hcsp_rows(row, nwarps, std::integral_constant<int, 2>{});
            for (; row < TYB; row += nwarps) hcsp_rows(row, 0, std::integral_constant<int, 1>{});
        }
        __syncthreads();

        // ------------------------------------------------ phase B: diamond rounds
        // Every iteration runs one round for every group of the warp, in
        // converged code: (1) groups without a block take the next ring entries
        // (one atomic per warp), (2) each group builds its round's list, lane lg
        // checking points lg, lg + LPB, ..., (3) the new points' SADs are
        // evaluated together, (4) the switching strategies pick the next list.
        // A group is LPB lanes: 2 for 16x16 blocks (a warp serves 16 blocks per
        // round, so a round's control costs half of what 4-lane groups pay per
        // block), 4 for 8x8 blocks.  The pass runs over the ring (list null)
        // with +-R bitmaps (FULLM) or, in the box variant, with visited boxes;
        // the box variant then runs it again over the ring entries of the
        // blocks that left their box (list; FULLM, warp 0 only).
        auto rounds = [&](const int* list, int nlist, int* next, auto full_c) {
            constexpr bool FULLM = decltype(full_c)::value;
            constexpr unsigned GMASK = (1u << LPB) - 1u;
            const int gq = tid / LPB, lg = lane % LPB, lead = lane & ~(LPB - 1);
            const int col0 = GM::col0(lg), row0 = GM::row0(lg);
            uint32_t* bm = (BOX && FULLM) ? bm_full + gq * nwb : bm_all + gq * bw;
            const int bmw = FULLM ? nwb : bw;  // words of this group's bitmap
            const int side = 2 * R + 1;
            // visited word and bit of displacement (x, y); false: outside the box
            auto vbit = [&](int x, int y, int& word, int& bitn) {
                if constexpr (FULLM) {
                    const int bit = (y + R) * side + (x + R);
                    word = bit >> 5;
                    bitn = bit & 31;
                    return true;
                } else {
                    word = y + 16;
                    bitn = x + 16;
                    return (unsigned)(word | bitn) < 32u;
                }
            };

            // group state, identical in the group's lanes
            int act = 0;  // 0: needs a block, 1: searching, 2: done
            int phase = PH_DDSP, pat = PAT_H, nsp = 0, pick = -1;
            int cx = 0, cy = 0, bxp = 0, byp = 0;
            uint32_t bsad = 0;
            int dxlo = 0, dxhi = 0, dylo = 0, dyhi = 0, wx0 = 0, wy0 = 0;
            size_t blk = 0;
            int ridx = 0, rmb = 0;                    // EVAL: the block's ring entry and tile position
            uint32_t ds0 = kUnknown, ds1 = kUnknown;  // distant-point SADs of this round (DCDS^S)
            int wmin = INT_MAX, wmax = -1;            // bitmap words this lane has set
            uint32_t cb[RPLB][CPL];
#pragma unroll
            for (int r = 0; r < RPLB; ++r)
#pragma unroll
                for (int j = 0; j < CPL; ++j) cb[r][j] = 0u;

            for (int iter = 0;; ++iter) {
                // ---- (1) fetch: one atomic for all groups of the warp that need a block ----
                const unsigned need = __ballot_sync(FULL, act == 0 && lg == 0);
                if (need) {
                    const int first = __ffs(need) - 1;
                    int base = 0;
                    if (lane == first) base = atomicAdd(next, __popc(need));
                    base = __shfl_sync(FULL, base, first);
                    int idx = base + __popc(need & ((1u << lane) - 1u));
                    idx = __shfl_sync(FULL, idx, lead);
                    if (act == 0) {
                        if (idx >= nlist || !index_ok(idx, NMB, status) ||
                            !index_ok(list ? list[idx] : idx, NMB, status)) {
                            act = 2;
                        } else {
                            if (list) idx = list[idx];
                            const uint2 e = ring[idx];
                            const int mb = (int)(e.x & 255u), hb = (int)((e.x >> 8) & 7u);
                            const int bxl = mb % TXB, byl = mb / TXB;
                            const int bxg = bx0 + bxl, byg = by0 + byl;
                            const int px = bxg * B, py = byg * B;
                            blk = (size_t)byg * NBX + bxg;
                            ridx = idx;
                            rmb = mb;
                            dxlo = max(-R, -px); dxhi = min(R, W - B - px);
                            dylo = max(-R, -py); dyhi = min(R, H - B - py);
                            wx0 = rx + bxl * B + 4 * col0;
                            wy0 = R + byl * B + row0;
                            const uint32_t* cp = reinterpret_cast<const uint32_t*>(
                                curS + (byl * B + row0) * kTile + bxl * B + 4 * col0);
#pragma unroll
                            for (int r = 0; r < RPLB; ++r)
#pragma unroll
                                for (int j = 0; j < CPL; ++j)
                                    cb[r][j] = ld_word(
                                        reinterpret_cast<const uint8_t*>(cp + r * RSB * (kTile / 4) + j), gc);
                            decode(kHcsp, hb, cx, cy);
                            bxp = cx; byp = cy; bsad = e.y;
                            nsp = (int)((e.x >> 11) & 7u);
                            pat = (cy == 0) ? PAT_H : PAT_V;  // switching strategy one
                            phase = PH_DDSP;
                            pick = -1;
                            act = 1;
                            // every valid HCSP point is visited (lane lg takes points lg, lg + LPB, ...)
                            for (int k = lg; k < 7; k += LPB) {
                                int ox, oy;
                                decode(kHcsp, k, ox, oy);
                                int wd, bn;
                                // the HCSP points (+-2) always fit the box
                                if (ox >= dxlo && ox <= dxhi && oy >= dylo && oy <= dyhi && vbit(ox, oy, wd, bn)) {
                                    if (index_ok(wd, bmw, status)) atomicOr(&bm[wd], 1u << bn);
                                    wmin = min(wmin, wd);
                                    wmax = max(wmax, wd);
                                }
                            }
                        }
                    }
                    __syncwarp();  // bitmap initialisation visible to the whole group
                }
                if (!__any_sync(FULL, act != 2)) break;

                // ---- (2) this round's list: lane lg checks points lg, lg + LPB, ... ----
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
                unsigned vb = 0u, nb = 0u;  // valid / new points of the list, bit k = point k
                bool outbox = false;        // a valid point of this lane's outside the visited box
#pragma unroll
                for (int i = 0; i < 4 / LPB; ++i) {
                    const int k = i * LPB + lg;
                    bool valid = false, fresh = false;
                    int wd = 0, bn = 0;
                    if (act == 1 && k < npts) {
                        int ox, oy;
                        decode(code, k, ox, oy);
                        const int x = cx + ox, y = cy + oy;
                        valid = x >= dxlo && x <= dxhi && y >= dylo && y <= dyhi;
                        if (valid) {
                            if (counted) {
                                if (vbit(x, y, wd, bn))
                                    fresh = index_ok(wd, bmw, status) && ((bm[wd] >> bn) & 1u) == 0u;
                                else
                                    outbox = true;
                            } else {
                                fresh = (k == 0 ? ds0 : ds1) == kUnknown;
                            }
                        }
                    }
                    if constexpr (LPB == 1) {
                        vb |= (unsigned)valid << i;
                        nb |= (unsigned)fresh << i;
                    } else {
                        vb |= ((__ballot_sync(FULL, valid) >> lead) & GMASK) << (i * LPB);
                        nb |= ((__ballot_sync(FULL, fresh) >> lead) & GMASK) << (i * LPB);
                    }
                    // the list's points are distinct: marking one leaves the others' checks unchanged
                    if (counted && fresh) {
                        if (index_ok(wd, bmw, status)) atomicOr(&bm[wd], 1u << bn);
                        wmin = min(wmin, wd);
                        wmax = max(wmax, wd);
                    }
                }
                // a point outside the box: the group drops the block this round
                bool drop = false;
                if constexpr (BOX && !FULLM) {
                    drop = ((__ballot_sync(FULL, outbox) >> lead) & GMASK) != 0u;
                    if (drop) nb = 0u;
                }
                if (SIMPL && phase == PH_DDSP) {
                    ds0 = (vb & 4u) ? kUnknown : kInvalid;
                    ds1 = (vb & 8u) ? kUnknown : kInvalid;
                }
                if (counted) nsp += __popc(nb);
                int ncand = 0;
                uint32_t pack = 0;  // slot indices of the new points, 4 bits each
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((nb >> k) & 1u) { pack |= (uint32_t)k << (4 * ncand); ++ncand; }

                // ---- (3) evaluate the new points (two at a time, all groups together) ----
                uint32_t sad[4] = {0u, 0u, 0u, 0u};
                int qx[4], qy[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int ox = 0, oy = 0;
                    if (i < ncand) decode(code, (int)((pack >> (4 * i)) & 15u), ox, oy);
                    qx[i] = cx + ox;  // unused slots read the centre: a valid address
                    qy[i] = cy + oy;
                }
                // a DDSP round after a move has 3 new points, a step-4 round at most 2:
                // evaluate them in one pass of 2 or 3 (a 4th, which the pattern
                // geometry rules out after the HCSP, would take one more pass)
                const bool three = __any_sync(FULL, ncand > 2);
                if (three) {
                    eval_points<3, V, RPLB, CPL, LPB, RSB>(win, WP, wx0, wy0, qx, qy, cb, sad, 0, ncand, gw);
                    if (__any_sync(FULL, ncand > 3))
                        eval_points<1, V, RPLB, CPL, LPB, RSB>(win, WP, wx0, wy0, qx, qy, cb, sad, 3, ncand, gw);
                } else {
                    eval_points<2, V, RPLB, CPL, LPB, RSB>(win, WP, wx0, wy0, qx, qy, cb, sad, 0, ncand, gw);
                }

                // ---- (4) best point of the list, then switching strategies (Sec. III-B) ----
                if (act == 1 && drop) {
                    // searched again from its HCSP result in the overflow pass
                    if (lg == 0) {
                        const int o = atomicAdd(&s_novf, 1);
                        if (index_ok(o, NMB, status)) ovf[o] = ridx;
                    }
                    for (int i = wmin; i <= wmax; ++i)
                        if (index_ok(i, bmw, status)) bm[i] = 0u;
                    wmin = INT_MAX; wmax = -1;
                    act = 0;
                } else if (act == 1) {
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
                        // DCDS^S: the middle point on the side of the better distant point
                        phase = PH_MID;
                        pick = (ds0 == kInvalid && ds1 == kInvalid) ? -1
                             : (ds0 == kInvalid) ? 1 : (ds1 == kInvalid) ? 0 : (ds1 < ds0 ? 1 : 0);
                    } else {  // step 4 evaluated: the block is done
                        if (lg == 0) {
                            out_mv[blk] = (uint32_t)(uint16_t)bxp | ((uint32_t)(uint16_t)byp << 16);
                            out_sad[blk] = bsad;
                            if (out_nsp) out_nsp[blk] = (uint16_t)nsp;
                        }
                        for (int i = wmin; i <= wmax; ++i)
                            if (index_ok(i, bmw, status)) bm[i] = 0u;
                        wmin = INT_MAX; wmax = -1;
                        act = 0;
                        // the ring entry now holds the final result for the evaluation pass
                        if (EVAL && lg == 0 && index_ok(ridx, NMB, status))
                            ring[ridx] = make_uint2((uint32_t)rmb | ((uint32_t)(bxp + 32) << 8) |
                                                        ((uint32_t)(byp + 32) << 16),
                                                    bsad | ((uint32_t)nsp << 16));
                    }
                }
                __syncwarp();  // bitmap updates and clears are ordered before the next round
            }
        };
        if constexpr (BOX) {
            rounds(nullptr, s_ring_n, &s_ring_next, std::false_type{});
            __syncthreads();  // every dropped block is on the overflow list
            const int novf = s_novf;
            if (novf > 0 && warp == 0) rounds(ovf, novf, &s_ovf_next, std::true_type{});
        } else {
            rounds(nullptr, s_ring_n, &s_ring_next, std::true_type{});
        }
        if constexpr (EVAL) {
            // ---- phase C: squared error of every ring block at its final MV (dense; lanes per
            // block and their words as in phase B) ----
            __syncthreads();
            const int nring = s_ring_n;
            const int gq = tid / LPB, lg = lane % LPB;
            const int col0 = GM::col0(lg), row0 = GM::row0(lg);
            const int ngroups_c = blockDim.x / LPB;
            for (int base = 0; base < nring; base += ngroups_c) {
                const int i = base + gq;
                const bool ok = i < nring;
                uint32_t q = 0u, fw = 0u, fsad = 0u;
                int dx = 0, dy = 0, fnsp = 0;
                if (ok && index_ok(i, NMB, status)) {
                    const uint2 e = ring[i];
                    const int mb = (int)(e.x & 255u);
                    dx = (int)((e.x >> 8) & 255u) - 32;
                    dy = (int)((e.x >> 16) & 255u) - 32;
                    fsad = e.y & 0xffffu;
                    fnsp = (int)(e.y >> 16);
                    const int bxl = mb % TXB, byl = mb / TXB;
                    if (mv_fs && lg == 0) fw = __ldg(mv_fs + (size_t)(by0 + byl) * NBX + bx0 + bxl);
                    const int c0 = rx + bxl * B + 4 * col0 + dx;
                    const uint8_t* p0 = win + (R + byl * B + row0 + dy) * WP + (c0 & ~3);
                    const unsigned s0 = (unsigned)(c0 & 3) * 8u;
                    const uint32_t* cp = reinterpret_cast<const uint32_t*>(curS + (byl * B + row0) * kTile +
                                                                           bxl * B + 4 * col0);
#pragma unroll
                    for (int r = 0; r < RPLB; ++r) {
                        uint32_t w[CPL + 1];
#pragma unroll
                        for (int j = 0; j <= CPL; ++j) w[j] = ld_word(p0 + r * RSB * WP + 4 * j, gw);
#pragma unroll
                        for (int j = 0; j < CPL; ++j) {
                            const uint32_t cw0 =
                                ld_word(reinterpret_cast<const uint8_t*>(cp + r * RSB * (kTile / 4) + j), gc);
                            const uint32_t d = __vabsdiffu4(__funnelshift_r(w[j], w[j + 1], s0), cw0);
                            q = __dp4a(d, d, q);
                        }
                    }
                }
#pragma unroll
                for (int o = 1; o < LPB; o <<= 1) q += __shfl_xor_sync(FULL, q, o);
                if (ok && lg == 0)
                    eval_block(dx, dy, fsad, q, fnsp, out_nsp != nullptr, mv_fs != nullptr, fw, B * B, esum, edist);
            }
            // this tile's sums: one atomic per warp and counter
            // (warp sums by redux.sync: one instruction each instead of a
            // five-step shuffle tree; the 64-bit distance in two 32-bit parts,
            // its low 16 bits and the rest, neither of which can overflow: a
            // lane adds at most four blocks' distances per tile, each below
            // 2^41).  The warps' sums meet in shared memory and one warp adds
            // the tile's total to the frame's counters after the barrier: a
            // quarter of the atomics, which all land on the frame's eight words.
            unsigned long long* fs = sums;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const uint32_t v = __reduce_add_sync(FULL, esum[k]);
                if (lane == 0) s_part[warp][k] = v;
                esum[k] = 0u;
            }
            {
                const uint32_t lo = __reduce_add_sync(FULL, (uint32_t)(edist & 0xffffu));
                const uint32_t hi = __reduce_add_sync(FULL, (uint32_t)(edist >> 16));
                if (lane == 0) s_part[warp][5] = ((unsigned long long)hi << 16) + lo;
                edist = 0ull;
            }
            if (tid == 0 && first_tile) {
                fs[5] = (unsigned long long)NBX * NBY;
                fs[7] = mv_fs ? 1ull : 0ull;
            }
        }
        __syncthreads();  // every read of this stage is done
        if constexpr (EVAL) {
            if (warp == nwarps - 1 && lane < 6) {
                unsigned long long v = 0ull;
                for (int w = 0; w < nwarps; ++w) v += s_part[w][lane];
                // sums order: ABS SQ NSP EQUAL, then DIST (slot 4) and PIXELS (slot 6)
                if (v) atomicAdd(sums + (lane < 4 ? lane : lane == 4 ? 6 : 4), v);
            }
        }
        if (NST == 1 && tid == 0) {
            fence_proxy_async();
            issue_tile((int)gridDim.x + atomicAdd(head, 1), frames, nframes, ntiles, smem, cur_off, TH, &s_bar[0],
                       &s_tile[0], &s_desc[0]);
        }
    }
}

// The +-R visited bitmaps (every block size, with or without the fused sums).
template <int B, bool SIMPL, int NST, bool EVAL>
__global__ void __launch_bounds__(256) dcds_kernel(const FrameDev* __restrict__ frames, int nframes, int ntiles,
                                                   int max_range, int* __restrict__ head,
                                                   unsigned* __restrict__ status)
{
    dcds_tiles<B, SIMPL, NST, EVAL, false>(frames, nframes, ntiles, max_range, head, status);
}

// 8x8 blocks with visited boxes (the search alone): at most 80 registers, so
// that three 256-thread CTAs fit an SM.
template <bool SIMPL, int NST>
__global__ void __launch_bounds__(256, 3) dcds_box_kernel(const FrameDev* __restrict__ frames, int nframes,
                                                          int ntiles, int max_range, int* __restrict__ head,
                                                          unsigned* __restrict__ status)
{
    dcds_tiles<8, SIMPL, NST, false, true>(frames, nframes, ntiles, max_range, head, status);
}

// Sets the attributes a launch of kern with smem bytes of dynamic shared
// memory needs; per_sm: its CTAs per SM.
template <typename K>
cudaError_t occupancy(K kern, size_t smem, int threads, int& per_sm)
{
    per_sm = 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    return e;
}

template <typename K>
cudaError_t launch_k(K kern, size_t smem, int per_sm, const FrameDev* frames, int nframes, int ntiles, int max_range,
                     const Shape& s, int* head, unsigned* status, int num_sms, cudaStream_t st)
{
    if (s.ctas_per_sm > 0) per_sm = s.ctas_per_sm;
    const int grid = std::max(1, std::min(ntiles, std::max(per_sm, 1) * num_sms));
    kern<<<grid, s.threads, smem, st>>>(frames, nframes, ntiles, max_range, head, status);
    return cudaGetLastError();
}

template <int B, bool SIMPL, int NST, bool EVAL>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, cudaStream_t st)
{
    auto kern = dcds_kernel<B, SIMPL, NST, EVAL>;
    const size_t smem = dcds_smem_bytes(B, max_range, s, false);
    int per_sm = 0;
    cudaError_t e = occupancy(kern, smem, s.threads, per_sm);
    if (e != cudaSuccess) return e;
    if constexpr (B == 8 && !EVAL) {
        // the visited-box variant where it fits more CTAs per SM
        auto kbox = dcds_box_kernel<SIMPL, NST>;
        const size_t smem_box = dcds_smem_bytes(B, max_range, s, true);
        int per_sm_box = 0;
        if (occupancy(kbox, smem_box, s.threads, per_sm_box) != cudaSuccess) {
            (void)cudaGetLastError();  // the bitmap variant runs instead
        } else if (per_sm_box > per_sm) {
            return launch_k(kbox, smem_box, per_sm_box, frames, nframes, ntiles, max_range, s, head, status, num_sms,
                            st);
        }
    }
    return launch_k(kern, smem, per_sm, frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
}

template <int B, bool SIMPL>
cudaError_t launch_b(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* head,
                     unsigned* status, int num_sms, bool eval, cudaStream_t st)
{
    if (eval) {
        if (s.stages == 2)
            return launch_t<B, SIMPL, 2, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
        return launch_t<B, SIMPL, 1, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
    }
    if (s.stages == 2)
        return launch_t<B, SIMPL, 2, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
    return launch_t<B, SIMPL, 1, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, st);
}

}  // namespace

size_t dcds_smem_bytes(int block, int max_range, const Shape& s, bool box)
{
    const int nst = s.stages == 2 ? 2 : 1;
    const int stage = win_bytes_max(max_range, kDcdsTileH) + kTile * kDcdsTileH;
    const int nmb = (kTile / block) * (kDcdsTileH / block);
    const int side = 2 * max_range + 1;
    const int nwb = (side * side + 31) / 32;
    const size_t groups = (size_t)(s.threads / dcds_lanes_per_block(block));
    const size_t visited = box ? groups * kBoxWords * 4 + (size_t)(32 / dcds_lanes_per_block(block)) * nwb * 4 +
                                     (size_t)nmb * 4
                               : groups * nwb * 4;
    return 128 + (size_t)nst * stage + (size_t)nmb * 8 + visited;
}

cudaError_t dcds_preload()
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, dcds_kernel<16, false, 1, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_kernel<16, true, 1, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_kernel<8, false, 1, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_kernel<8, true, 1, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_box_kernel<false, 1>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, dcds_box_kernel<true, 1>);
    return e;
}

cudaError_t launch_dcds(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                        bool simplified, const Shape& s, int* head, unsigned* status, int num_sms,
                        cudaStream_t st, bool eval)
{
    if (s.threads != 64 && s.threads != 128 && s.threads != 256) return cudaErrorInvalidValue;
    if (block == 16)
        return simplified ? launch_b<16, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st)
                          : launch_b<16, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st);
    return simplified ? launch_b<8, true>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st)
                      : launch_b<8, false>(frames, nframes, ntiles, max_range, s, head, status, num_sms, eval, st);
}

}  // namespace me
