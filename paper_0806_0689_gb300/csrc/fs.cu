// fs.cu -- full-search block matching on sm_103a (Sec. I; the FS rows of
// Table IX).  Every candidate of the +-R window whose block lies inside the
// frame is evaluated; the result is the argmin of the key
// (SAD, |dx|+|dy|, dy, dx).
//
// GPU mapping
//   * Persistent CTAs take tiles from a global counter.  A tile is a row of
//     tx blocks; its reference window (the rows the candidates touch, and the
//     columns tx*B + 2R plus a small margin) and its current blocks are
//     copied into shared memory by the TMA unit, double-buffered: the copy of
//     the next tile runs while the CTA searches the current one.  The window
//     is one copy through a 3-D view of the frame (16-byte chunks x chunk
//     columns x rows), so it may be wider than the 256-element limit of a box
//     dimension and still lands as contiguous rows.
//   * The raw window is expanded once per tile into E, where word c of a row
//     holds the four bytes starting at byte column c.  A candidate's
//     reference row is then four aligned 32-bit loads at any dx, and the
//     lanes of a warp (consecutive dx) hit 32 different banks.  The row pitch
//     P of E is chosen so that when a warp wraps from one group of dy to the
//     next, its lanes still land on distinct banks.
//   * A thread evaluates K vertically consecutive candidates (dx, dy0..dy0+K-1)
//     of one block.  Reference row j is read once and accumulated into every
//     candidate that uses it (rows j-K+1..j of the block), so a thread reads
//     K+B-1 reference rows for K*B rows of work.  The current block sits in
//     registers.
//   * A thread reduces its K candidates with 32-bit keys: dx is fixed within
//     the thread, so SAD * 2^14 + ((|dy| << 7) | (dy+32)) orders them like the
//     full key.  The dy part comes from a per-tile shared table that also
//     marks rows outside the frame or the range (bit 31), so the reduction is
//     one multiply-add and one min per candidate.  The block's candidates then
//     meet in a 64-bit shared-memory atomicMin on the packed key
//     (SAD << 21 | (|dx|+|dy|) << 14 | (dy+32) << 7 | (dx+32)).
//   * Every wait is bounded; a time-out sets STATUS_TIMEOUT and ends the CTA.
//   * DUAL (16x16 blocks): the accumulators are kept per 8x8 quadrant, so the
//     same sweep also yields the full search of the four 8x8 sub-blocks (their
//     SADs at every displacement of the +-R square; a 16x16 SAD is the sum of
//     its quadrants' at the same displacement), each with its own validity and
//     key -- both block sizes of a frame for the price of the 16x16 search.
#include "dcds_common.cuh"

#include <algorithm>

namespace me {
namespace {

using dcds::fence_mbar_init;
using dcds::fence_proxy_async;
using dcds::find_frame;
using dcds::mbar_arrive;
using dcds::mbar_arrive_expect_tx;
using dcds::mbar_init;
using dcds::mbar_wait;
using dcds::tma_load_2d;

constexpr int kMaxTx = 32;
constexpr int kDyTable = 96;               // dy + 32 for dy in [-32, 63]
constexpr uint32_t kDyInvalid = 0x80000000u;

struct FsArgs {
    int tx, rwb, raw_stride, cur_stride, P;
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dcds::smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z),
          "r"(dcds::smem_addr(bar))
        : "memory");
}

// Thread 0: claim tile t into stage buffers; a tile past the end completes
// the phase with no data.
__device__ __forceinline__ void fs_issue(int t, const FrameDev* frames, int nframes, int ntiles, const FsArgs& a,
                                         int B, int K, uint8_t* raw, uint8_t* cur, uint64_t* bar, int* s_tile,
                                         int* s_frame)
{
    *s_tile = t;
    if (t >= ntiles) {
        mbar_arrive(bar);
        return;
    }
    const int f = find_frame(frames, nframes, t);
    *s_frame = f;
    const FrameDev& F = frames[f];
    const int lt = t - F.tile_base;
    const int ty = lt / F.tiles_x, tx = lt - ty * F.tiles_x;
    const int R = F.range, rx = (R + 15) & ~15;
    const int rows = fs_rows(B, R, K);
    const int x0 = tx * a.tx * B, y0 = ty * B;
    mbar_arrive_expect_tx(bar, (uint32_t)(a.rwb * rows + a.tx * B * B));
    tma_load_3d(raw, &F.tm_ref, 0, (x0 - rx) >> 4, y0 - R, bar);  // x0 - rx is a multiple of 16
    tma_load_2d(cur, &F.tm_cur, x0, y0, bar);
}

template <int B, int K, bool DUAL>
__global__ void __launch_bounds__(256, 2) fs_kernel(const FrameDev* __restrict__ frames, int nframes, int ntiles,
                                                    int* __restrict__ counter, unsigned* __restrict__ status,
                                                    FsArgs a)
{
    static_assert(!DUAL || B == 16, "the two-size sweep runs over 16x16 blocks");
    constexpr int V = kSadVariant;
    constexpr int BW = B / 4;
    constexpr int NQ = DUAL ? 4 : 1;  // accumulators per candidate: the 8x8 quadrants, or the block
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ unsigned long long s_key[kMaxTx];
    __shared__ unsigned long long s_key8[DUAL ? 4 * kMaxTx : 1];  // DUAL: 8x8 blocks (2 rows x 2 tx)
    __shared__ uint32_t s_dkey[kDyTable];
    __shared__ uint32_t s_dkey8[DUAL ? 2 : 1][kDyTable];          // DUAL: rows of the upper / lower 8x8
    __shared__ int s_tile[2], s_frame[2], s_fail;

    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int raw_bytes = a.raw_stride;  // one stage of the reference window
    uint8_t* cur_base = smem + 2 * raw_bytes;
    uint32_t* E = reinterpret_cast<uint32_t*>(cur_base + 2 * a.cur_stride);
    const int tid = threadIdx.x;
    const int P = a.P;
    const int rww = a.rwb >> 2;  // words per raw window row
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int i = tid; i < kMaxTx; i += blockDim.x) s_key[i] = ~0ull;
    if constexpr (DUAL)
        for (int i = tid; i < 4 * kMaxTx; i += blockDim.x) s_key8[i] = ~0ull;
    if (tid == 0) {
        s_fail = 0;
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_mbar_init();
        fs_issue(atomicAdd(counter, 1), frames, nframes, ntiles, a, B, K, smem, cur_base, &s_bar[0], &s_tile[0],
                 &s_frame[0]);
    }
    __syncthreads();

    for (int it = 0;; ++it) {
        const int st = it & 1;
        const uint32_t par = (it >> 1) & 1;
        if (!mbar_wait(&s_bar[st], par)) atomicOr(&s_fail, 1);
        __syncthreads();  // stage st landed; the previous tile's reads of E and s_key are done
        if (s_fail) {
            if (tid == 0) {
                if (status) atomicOr(status, STATUS_TIMEOUT);
                (void)mbar_wait(&s_bar[st], par);  // bounded: let an outstanding copy land
            }
            break;
        }
        const int t = s_tile[st];
        if (t >= ntiles) break;
        if (tid == 0) {
            // stage st^1 was last read by the previous tile, which ended with a CTA barrier
            fence_proxy_async();
            fs_issue(atomicAdd(counter, 1), frames, nframes, ntiles, a, B, K, smem + (st ^ 1) * raw_bytes,
                     cur_base + (st ^ 1) * a.cur_stride, &s_bar[st ^ 1], &s_tile[st ^ 1], &s_frame[st ^ 1]);
        }

        const FrameDev& F = frames[s_frame[st]];
        const int W = F.w, H = F.h, R = F.range;
        const int rx = (R + 15) & ~15;
        const int lt = t - F.tile_base;
        const int tile_y = lt / F.tiles_x, tile_x = lt - tile_y * F.tiles_x;
        const int bx0 = tile_x * a.tx, by = tile_y;
        const int nbx_t = min(a.tx, F.nbx - bx0);
        const int ndx = 2 * R + 1;
        const int ndyg = (ndx + K - 1) / K;
        const int rows = ndyg * K + B - 1;
        const int py = by * B;
        const int dylo = max(-R, -py), dyhi = min(R, H - B - py);

        // dy part of the candidate key; bit 31 marks a row outside the frame or the range
        for (int i = tid; i < kDyTable; i += blockDim.x) {
            const int dy = i - 32;
            const uint32_t v = ((uint32_t)abs(dy) << 7) | (uint32_t)(dy + 32);
            s_dkey[i] = (dy >= dylo && dy <= dyhi) ? v : kDyInvalid;
            if constexpr (DUAL) {
#pragma unroll
                for (int qy = 0; qy < 2; ++qy) {
                    const int lo = max(-R, -(py + 8 * qy)), hi = min(R, H - 8 - (py + 8 * qy));
                    s_dkey8[qy][i] = (dy >= lo && dy <= hi) ? v : kDyInvalid;
                }
            }
        }

        // ---- expand the raw window: E[r][c] = bytes c..c+3 of window row r ----
        // A warp step covers 4 rows x 8 column quads: with P odd and the raw row
        // pitch = 8 (mod 32) words, its loads and stores hit 32 distinct banks.
        {
            const uint32_t* raw = reinterpret_cast<const uint32_t*>(smem + st * raw_bytes);
            const int nq = (a.tx * B + rx + R + 3) >> 2;  // column quads used by this frame
            const int nqg = (nq + 7) >> 3, nrg = (rows + 3) >> 2;
            const int lr = lane >> 3, lq = lane & 7;
            int rg = warp / nqg, qg = warp - rg * nqg;
            while (rg < nrg) {
                const int r = rg * 4 + lr, i = qg * 8 + lq;
                if (r < rows && i < nq) {
                    const uint32_t w0 = raw[r * rww + i], w1 = raw[r * rww + i + 1];
                    uint32_t* e = E + r * P + 4 * i;
                    e[0] = w0;
                    e[1] = __funnelshift_r(w0, w1, 8u);
                    e[2] = __funnelshift_r(w0, w1, 16u);
                    e[3] = __funnelshift_r(w0, w1, 24u);
                }
                qg += nwarps;
                while (qg >= nqg) { qg -= nqg; ++rg; }
            }
        }
        __syncthreads();

        // ---- search: thread = (block, dy group, dx) ----
        const uint32_t* curw = reinterpret_cast<const uint32_t*>(cur_base + st * a.cur_stride);
        const int cwpr = a.tx * BW;  // words per staged current row
        const int tpb = ndx * ndyg;
        const int ntasks = nbx_t * tpb;
        for (int task = tid; task < ntasks; task += blockDim.x) {
            const int b = task / tpb;
            const int rem = task - b * tpb;
            const int dyg = rem / ndx;
            const int dxi = rem - dyg * ndx;
            const int dx = dxi - R;
            const int dy0 = dyg * K - R;
            const int px = (bx0 + b) * B;

            uint32_t cb[B][BW];
#pragma unroll
            for (int r = 0; r < B; ++r)
#pragma unroll
                for (int w = 0; w < BW; ++w) cb[r][w] = curw[r * cwpr + b * BW + w];

            const uint32_t* ep = E + dyg * K * P + b * B + rx + dx;
            uint32_t acc[K][NQ];  // DUAL: quadrant (r / 8) * 2 + (w / 2) of the 16x16 block
#pragma unroll
            for (int i = 0; i < K; ++i)
#pragma unroll
                for (int q = 0; q < NQ; ++q) acc[i][q] = 0u;
#pragma unroll
            for (int j = 0; j < K + B - 1; ++j) {
                uint32_t rw[BW];
#pragma unroll
                for (int w = 0; w < BW; ++w) rw[w] = ep[4 * w];
                ep += P;
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const int r = j - i;
                    if (r >= 0 && r < B) {
#pragma unroll
                        for (int w = 0; w < BW; ++w) {
                            const int q = DUAL ? (r >> 3) * 2 + (w >> 1) : 0;
                            acc[i][q] = sadacc<V>(rw[w], cb[r][w], acc[i][q]);
                        }
                    }
                }
            }
            // dx is fixed within the thread: SAD * 2^14 + (|dy| << 7 | dy + 32) orders its candidates
            const uint32_t* dk = s_dkey + dy0 + 32;
            uint32_t best = 0xffffffffu;
#pragma unroll
            for (int i = 0; i < K; ++i) {
                uint32_t sum = acc[i][0];
#pragma unroll
                for (int q = 1; q < NQ; ++q) sum += acc[i][q];
                best = min(best, sum * 16384u + dk[i]);
            }
            if (best < kDyInvalid && px + dx >= 0 && px + dx <= W - B) {
                const uint32_t key = best + ((uint32_t)abs(dx) << 7);  // (SAD, |dx|+|dy|, dy)
                atomicMin(&s_key[b], ((unsigned long long)key << 7) | (unsigned long long)(dx + 32));
            }
            if constexpr (DUAL) {
                // the four 8x8 sub-blocks at the same displacements, each with its own window / frame limits
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int qy = q >> 1, qx = q & 1;
                    const uint32_t* dk8 = s_dkey8[qy] + dy0 + 32;
                    uint32_t b8 = 0xffffffffu;
#pragma unroll
                    for (int i = 0; i < K; ++i) b8 = min(b8, acc[i][q] * 16384u + dk8[i]);
                    const int px8 = px + 8 * qx;
                    if (b8 < kDyInvalid && px8 + dx >= 0 && px8 + dx <= W - 8) {
                        const uint32_t key = b8 + ((uint32_t)abs(dx) << 7);
                        atomicMin(&s_key8[(2 * b + qx) * 2 + qy],
                                  ((unsigned long long)key << 7) | (unsigned long long)(dx + 32));
                    }
                }
            }
        }
        __syncthreads();

        for (int b = tid; b < nbx_t; b += blockDim.x) {
            const unsigned long long key = s_key[b];
            s_key[b] = ~0ull;
            const int dx = (int)(key & 127ull) - 32;
            const int dy = (int)((key >> 7) & 127ull) - 32;
            const int px = (bx0 + b) * B;
            const int nx = min(R, W - B - px) - max(-R, -px) + 1;
            const int ny = dyhi - dylo + 1;
            const size_t blk = (size_t)by * F.nbx + bx0 + b;
            *reinterpret_cast<uint32_t*>(F.mv + 2 * blk) = (uint32_t)(uint16_t)dx | ((uint32_t)(uint16_t)dy << 16);
            F.sad[blk] = (uint32_t)(key >> 21);
            if (F.nsp) F.nsp[blk] = (uint16_t)(nx * ny);
        }
        if constexpr (DUAL) {
            // the 8x8 field: blocks (2 (bx0 + b) + qx, 2 by + qy) of a frame 2 * nbx blocks wide
            for (int i = tid; i < 4 * nbx_t; i += blockDim.x) {
                const int qy = i & 1, c8 = i >> 1;  // c8 = 2 b + qx
                const unsigned long long key = s_key8[i];
                s_key8[i] = ~0ull;
                const int dx = (int)(key & 127ull) - 32;
                const int dy = (int)((key >> 7) & 127ull) - 32;
                const int px8 = bx0 * B + 8 * c8, py8 = by * B + 8 * qy;
                const int nx = min(R, W - 8 - px8) - max(-R, -px8) + 1;
                const int ny = min(R, H - 8 - py8) - max(-R, -py8) + 1;
                const size_t blk8 = (size_t)(2 * by + qy) * (2 * F.nbx) + 2 * bx0 + c8;
                *reinterpret_cast<uint32_t*>(F.mv8 + 2 * blk8) =
                    (uint32_t)(uint16_t)dx | ((uint32_t)(uint16_t)dy << 16);
                F.sad8[blk8] = (uint32_t)(key >> 21);
                if (F.nsp8) F.nsp8[blk8] = (uint16_t)(nx * ny);
            }
        }
        // the next iteration's first barrier orders these resets before the next search
    }
}

int inv_mod32(int k)
{
    for (int p = 1; p < 32; p += 2)
        if ((k * p) % 32 == 1) return p;
    return 1;
}

template <int B, int K, bool DUAL>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s, int* counter,
                     unsigned* status, int num_sms, cudaStream_t st)
{
    const FsGeom g = fs_geom(B, max_range, s.tx, K);
    auto kern = fs_kernel<B, K, DUAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int per_sm = s.ctas_per_sm;
    if (per_sm <= 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, s.threads, g.smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = std::max(1, std::min(ntiles, std::max(per_sm, 1) * num_sms));
    FsArgs a{s.tx, g.rwb, g.raw_stride, g.cur_stride, g.P};
    kern<<<grid, s.threads, g.smem, st>>>(frames, nframes, ntiles, counter, status, a);
    return cudaGetLastError();
}

}  // namespace

FsGeom fs_geom(int block, int max_range, int tx, int k)
{
    FsGeom g{};
    const int rx = (max_range + 15) & ~15;
    const int raw_w = tx * block + rx + max_range + 8;  // bytes the expansion reads per row
    g.nch = (raw_w + 15) >> 4;
    g.nch += ((2 - g.nch) % 8 + 8) % 8;  // row pitch = 8 (mod 32) words: conflict-free expansion loads
    g.rwb = g.nch * 16;
    g.rows = fs_rows(block, max_range, k);
    g.raw_stride = dcds::round128(g.rows * g.rwb);
    g.cur_stride = dcds::round128(block * tx * block);
    g.ecols = (tx * block + rx + max_range + 3) & ~3;
    // P = (2R+1) / K (mod 32): a warp that wraps from dx = R of one dy group to
    // dx = -R of the next (K rows down) keeps its lanes on distinct banks
    const int target = ((2 * max_range + 1) * inv_mod32(k)) & 31;
    g.P = g.ecols + (((target - g.ecols) % 32) + 32) % 32;
    g.smem = 128 + (size_t)2 * g.raw_stride + (size_t)2 * g.cur_stride + (size_t)g.rows * g.P * 4;
    return g;
}

bool fs_shape_ok(int block, int max_range, const Shape& s)
{
    if (s.threads != 256 || s.tx < 1 || s.tx > kMaxTx || s.tx * block > 256) return false;
    if (fs_geom(block, max_range, s.tx, s.k).nch > 256) return false;
    if (block == 8 && (s.tx & 1)) return false;  // TMA x coordinates stay multiples of 16 bytes
    if (s.k != 9 && s.k != 11 && s.k != 13 && s.k != 15 && s.k != 33) return false;
    return fs_geom(block, max_range, s.tx, s.k).smem <= 227 * 1024;
}

size_t fs_smem_bytes(int block, int max_range, const Shape& s)
{
    return fs_geom(block, max_range, s.tx, s.k).smem;
}

cudaError_t launch_fs(const FrameDev* frames, int nframes, int ntiles, int block, int max_range, const Shape& s,
                      int* counter, unsigned* status, int num_sms, cudaStream_t st, bool dual)
{
    if (!fs_shape_ok(block, max_range, s)) return cudaErrorInvalidValue;
    if (dual) {
        if (block != 16) return cudaErrorInvalidValue;
        // quadrant accumulators: rows of work per thread kept small (registers)
        if (s.k == 9) return launch_t<16, 9, true>(frames, nframes, ntiles, max_range, s, counter, status, num_sms, st);
        if (s.k == 11) return launch_t<16, 11, true>(frames, nframes, ntiles, max_range, s, counter, status, num_sms, st);
        return cudaErrorInvalidValue;
    }
#define ME_FS_CASE(BB, KK) \
    if (block == BB && s.k == KK) return launch_t<BB, KK, false>(frames, nframes, ntiles, max_range, s, counter, status, num_sms, st);
    ME_FS_CASE(16, 9) ME_FS_CASE(16, 11) ME_FS_CASE(16, 13) ME_FS_CASE(16, 15)
    ME_FS_CASE(8, 9) ME_FS_CASE(8, 11) ME_FS_CASE(8, 13) ME_FS_CASE(8, 15)
    ME_FS_CASE(16, 33) ME_FS_CASE(8, 33)
#undef ME_FS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace me
