// fs.cu -- full-search block matching on sm_103a (Sec. I; the FS rows of
// Table IX).  Every candidate of the +-R window whose block lies inside the
// frame is evaluated; the result is the argmin of the key
// (SAD, |dx|+|dy|, dy, dx).
//
// GPU mapping
//   * A CTA owns a row of tx blocks.  The window of the row (B + 2R rows,
//     tx*B + 2R columns) is staged in shared memory four times, shifted by
//     0..3 bytes, so that a reference row at any column is read as aligned
//     32-bit words.  The current blocks are staged as well.
//   * A thread evaluates K vertically consecutive candidates (dx, dy0..dy0+K-1)
//     of one block.  Reference row j is read once and accumulated into every
//     candidate that uses it (rows j-K+1..j of the block), so a thread reads
//     K+B-1 reference rows for K*B rows of work.  The current block sits in
//     registers.
//   * Consecutive threads take consecutive dx; their reads land in the four
//     shifted copies, which are laid out so that the 32 lanes hit 32 banks.
//   * Candidates reduce through a 64-bit shared-memory atomicMin on the
//     packed key (SAD << 21 | (|dx|+|dy|) << 14 | (dy+32) << 7 | (dx+32)).
#include "me_internal.cuh"

namespace me {
namespace {

__device__ __forceinline__ uint32_t load_word_or_zero(const uint8_t* row, int a, int W)
{
    return (a >= 0 && a < W) ? __ldg(reinterpret_cast<const uint32_t*>(row + a)) : 0u;
}

template <int B, int K>
__global__ void __launch_bounds__(256) fs_kernel(const FrameDev* __restrict__ frames, int nframes, int tx,
                                                 int max_range, int spw, int copy_stride)
{
    constexpr int V = kSadVariant;
    constexpr int BW = B / 4;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int s_frame;
    __shared__ unsigned long long s_key[64];

    uint32_t* copies = reinterpret_cast<uint32_t*>(smem);
    uint32_t* curs = copies + 4 * (size_t)copy_stride;  // [B rows][tx*BW words]

    const int t = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nframes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (frames[mid].tile_base <= t) lo = mid; else hi = mid - 1;
        }
        s_frame = lo;
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s_key[i] = ~0ull;
    __syncthreads();
    const FrameDev& F = frames[s_frame];
    const int W = F.w, H = F.h, P = F.pitch, R = F.range;
    const int lt = t - F.tile_base;
    const int tile_y = lt / F.tiles_x, tile_x = lt - tile_y * F.tiles_x;
    const int bx0 = tile_x * tx, by = tile_y;
    const int nbx_t = min(tx, F.nbx - bx0);
    const int x_lo = bx0 * B - R, y_lo = by * B - R;
    const int ndx = 2 * R + 1;
    const int ndyg = (ndx + K - 1) / K;
    const int rows = ndyg * K + B - 1;
    const int wpr = (nbx_t * B + 2 * R + 3) / 4 + 1;

    // ---- stage 4 byte-shifted copies of the window: copy s, word i holds
    //      window bytes 4i+s .. 4i+s+3 (zeros outside the frame) ----
    for (int idx = threadIdx.x; idx < 4 * rows * wpr; idx += blockDim.x) {
        const int s = idx / (rows * wpr);
        const int rem = idx - s * rows * wpr;
        const int r = rem / wpr, i = rem - r * wpr;
        const int gy = y_lo + r;
        uint32_t v = 0u;
        if (gy >= 0 && gy < H) {
            const uint8_t* row = F.ref + (size_t)gy * P;
            const int g = x_lo + 4 * i + s;
            const int a = g & ~3;
            const uint32_t lo = load_word_or_zero(row, a, W);
            const uint32_t hi = load_word_or_zero(row, a + 4, W);
            v = __funnelshift_r(lo, hi, (unsigned)(g & 3) * 8u);
        }
        copies[(size_t)s * copy_stride + (size_t)r * spw + i] = v;
    }
    // ---- stage the current blocks of the row ----
    const int cw = nbx_t * BW;
    for (int idx = threadIdx.x; idx < B * cw; idx += blockDim.x) {
        const int r = idx / cw, i = idx - r * cw;
        curs[r * tx * BW + i] = __ldg(reinterpret_cast<const uint32_t*>(F.cur + (size_t)(by * B + r) * P + bx0 * B + 4 * i));
    }
    __syncthreads();

    const int tpb = ndx * ndyg;  // tasks per block
    const int ntasks = nbx_t * tpb;
    for (int task = threadIdx.x; task < ntasks; task += blockDim.x) {
        const int b = task / tpb;
        const int rem = task - b * tpb;
        const int dyg = rem / ndx;
        const int dxi = rem - dyg * ndx;
        const int dx = dxi - R;
        const int dy0 = dyg * K - R;
        const int px = (bx0 + b) * B, py = by * B;

        uint32_t cb[B][BW];
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
            for (int w = 0; w < BW; ++w) cb[r][w] = curs[r * tx * BW + b * BW + w];

        const int col = b * B + R + dx;  // window column of the candidate
        const uint32_t* cp = copies + (size_t)(col & 3) * copy_stride + (size_t)(dy0 + R) * spw + (col >> 2);
        uint32_t acc[K];
#pragma unroll
        for (int i = 0; i < K; ++i) acc[i] = 0u;
#pragma unroll
        for (int j = 0; j < K + B - 1; ++j) {
            uint32_t rw[BW];
#pragma unroll
            for (int w = 0; w < BW; ++w) rw[w] = cp[j * spw + w];
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int r = j - i;
                if (r >= 0 && r < B) {
#pragma unroll
                    for (int w = 0; w < BW; ++w) acc[i] = sadacc<V>(rw[w], cb[r][w], acc[i]);
                }
            }
        }
        unsigned long long best = ~0ull;
        const bool xok = (px + dx >= 0) && (px + dx <= W - B);
        if (xok) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int dy = dy0 + i;
                if (dy <= R && py + dy >= 0 && py + dy <= H - B) {
                    const unsigned long long key = ((unsigned long long)acc[i] << 21) |
                                                   ((unsigned long long)(abs(dx) + abs(dy)) << 14) |
                                                   ((unsigned long long)(dy + 32) << 7) |
                                                   (unsigned long long)(dx + 32);
                    best = key < best ? key : best;
                }
            }
        }
        if (best != ~0ull) atomicMin(&s_key[b], best);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbx_t; b += blockDim.x) {
        const unsigned long long key = s_key[b];
        const int dx = (int)(key & 127ull) - 32;
        const int dy = (int)((key >> 7) & 127ull) - 32;
        const int px = (bx0 + b) * B, py = by * B;
        const int nx = min(R, W - B - px) - max(-R, -px) + 1;
        const int ny = min(R, H - B - py) - max(-R, -py) + 1;
        const size_t blk = (size_t)by * F.nbx + bx0 + b;
        *reinterpret_cast<uint32_t*>(F.mv + 2 * blk) = (uint32_t)(uint16_t)dx | ((uint32_t)(uint16_t)dy << 16);
        F.sad[blk] = (uint32_t)(key >> 21);
        if (F.nsp) F.nsp[blk] = (uint16_t)(nx * ny);
    }
}

struct FsGeom { int spw, copy_stride, rows; };

FsGeom fs_geom(int block, int max_range, int tx, int k)
{
    FsGeom g;
    const int ndx = 2 * max_range + 1;
    g.rows = ((ndx + k - 1) / k) * k + block - 1;
    g.spw = (tx * block + 2 * max_range + 3) / 4 + 1;
    int cs = g.rows * g.spw;
    cs += ((8 - cs % 32) + 32) % 32;  // copy stride = 8 (mod 32) words: the four copies use disjoint banks
    g.copy_stride = cs;
    return g;
}

template <int B, int K>
cudaError_t launch_t(const FrameDev* frames, int nframes, int ntiles, int max_range, const Shape& s,
                     cudaStream_t st)
{
    const FsGeom g = fs_geom(B, max_range, s.tx, K);
    const size_t smem = fs_smem_bytes(B, max_range, s);
    auto kern = fs_kernel<B, K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, s.threads, smem, st>>>(frames, nframes, s.tx, max_range, g.spw, g.copy_stride);
    return cudaGetLastError();
}

}  // namespace

size_t fs_smem_bytes(int block, int max_range, const Shape& s)
{
    const FsGeom g = fs_geom(block, max_range, s.tx, s.k);
    return (size_t)4 * g.copy_stride * 4 + (size_t)block * s.tx * (block / 4) * 4;
}

cudaError_t launch_fs(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                      const Shape& s, cudaStream_t st)
{
    if (s.tx > 64) return cudaErrorInvalidValue;
#define ME_FS_CASE(BB, KK) \
    if (block == BB && s.k == KK) return launch_t<BB, KK>(frames, nframes, ntiles, max_range, s, st);
    ME_FS_CASE(16, 8) ME_FS_CASE(16, 11) ME_FS_CASE(16, 13) ME_FS_CASE(16, 15)
    ME_FS_CASE(8, 8) ME_FS_CASE(8, 11) ME_FS_CASE(8, 13) ME_FS_CASE(8, 15)
#undef ME_FS_CASE
    return cudaErrorInvalidValue;
}

}  // namespace me
