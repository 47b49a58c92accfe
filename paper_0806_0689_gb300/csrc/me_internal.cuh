// me_internal.cuh -- definitions shared by the sm_103a kernels and the C-ABI
// host code of libme.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace me {

// Pixel width of the tiles the DCDS kernel stages with TMA, and their height
// (tiles of 128 x 64 with 2-warp CTAs, 8 per SM, measured no faster for the
// search and 35 % slower with the evaluation fused).
constexpr int kTile = 128;
constexpr int kDcdsTileH = 128;

// Device-side view of one frame pair of a launch.  The two tensor maps
// describe the frames for the TMA unit.  DCDS: the reference window of a
// tile (box (kTile + 2*rx) x (kDcdsTileH + 2*R), rx = R rounded up to 16) and
// the current tile (box kTile x kDcdsTileH).  FS: see encode_fs_maps.
struct __align__(128) FrameDev {
    CUtensorMap tm_ref;
    CUtensorMap tm_cur;
    const uint8_t* cur;
    const uint8_t* ref;
    int16_t* mv;
    uint32_t* sad;
    uint16_t* nsp;
    int32_t w, h, pitch, range;
    int32_t nbx, nby;          // blocks per row / column
    int32_t tiles_x, tiles_y;  // tiles of this frame
    int32_t tile_base;         // first global tile index of this frame
    int32_t uniform_tiles;     // > 0: every frame of the table has this many tiles (tile t is in frame t / it)
    const int16_t* mv_fs;      // fused evaluation: the full-search field (may be null)
    unsigned long long* sums;  // fused evaluation: the frame's eight sums (null: no evaluation)
    int16_t* mv8;              // two-size full search: the 8x8 field (null: not requested)
    uint32_t* sad8;
    uint16_t* nsp8;
};

// Encode the two tensor maps of `f` (its pointers, sizes and range must be
// set) for tiles of kTile x tile_h pixels.  Host code; returns false if the
// CUDA driver rejects the description.
bool encode_frame_maps(FrameDev& f, int tile_h = kTile);

// Host code, after a table's tile counts and bases are set: mark the table
// uniform when every frame has the same number of tiles, so that the kernels
// find a tile's frame with one division instead of a binary search.
inline void set_uniform_tiles(FrameDev* table, int n)
{
    const int t0 = n > 0 ? table[0].tiles_x * table[0].tiles_y : 0;
    bool same = t0 > 0;
    for (int i = 1; i < n && same; ++i) same = table[i].tiles_x * table[i].tiles_y == t0;
    for (int i = 0; i < n; ++i) table[i].uniform_tiles = same ? t0 : 0;
}

// Device-side view of one frame of an evaluation batch.
struct __align__(64) EvalDev {
    const uint8_t* cur;
    const uint8_t* ref;
    const int16_t* mv;
    const int16_t* mv_fs;
    const uint16_t* nsp;
    int32_t w, h, pitch, nbx, nby;
};

// Launch shape of the search kernels.
struct Shape {
    int tx, ty;        // FS: a tile is tx blocks of one block row (ty unused)
    int threads;       // threads per CTA
    int ctas_per_sm;   // persistent grid = ctas_per_sm * SM count (0 = occupancy)
    int k;             // FS: candidate rows per thread
    int stages;        // DCDS: 1 = load each tile when needed, 2 = prefetch the next tile
};

// Status bits a kernel may record (read back by me_check_status).
enum : unsigned { STATUS_TIMEOUT = 1u, STATUS_BAD_ARG = 2u, STATUS_BOUNDS = 4u };

// Bitmap of visited points: one row per dy in [-R, R], this many 32-bit
// words per row (one bit per dx in [-R, R]).
__host__ __device__ inline int bm_words_per_row(int max_range) { return (2 * max_range + 1 + 31) / 32; }

// ---------------------------------------------------------------------------
// 4-byte SIMD sum of absolute differences, accumulated.  Several encodings of
// the same arithmetic; the byte-absdiff microbenchmark measures each and the
// kernels are instantiated with the fastest (kSadVariant).
// ---------------------------------------------------------------------------
enum { SAD_VSADU4 = 0, SAD_PTX_ADD = 1, SAD_DP4A = 2, SAD_MINMAX = 3, SAD_NVARIANTS = 4 };

template <int V>
__device__ __forceinline__ uint32_t sadacc(uint32_t a, uint32_t b, uint32_t c)
{
    if constexpr (V == SAD_VSADU4) {
        return __vsadu4(a, b) + c;
    } else if constexpr (V == SAD_PTX_ADD) {
        uint32_t d;
        asm("vabsdiff4.u32.u32.u32.add %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
        return d;
    } else if constexpr (V == SAD_DP4A) {
        return (uint32_t)__dp4a(__vabsdiffu4(a, b), 0x01010101u, c);
    } else {
        uint32_t d = __vsub4(__vmaxu4(a, b), __vminu4(a, b));
        return (uint32_t)__dp4a(d, 0x01010101u, c);
    }
}

// Variant the search kernels are compiled with: the PTX vabsdiff4 with
// accumulate measured fastest on GB300 (about 77 T byte-absdiffs/s against
// 68 T for dp4a and 52 T for __vsadu4 plus an add).
// round(sqrt(n) * 2^24) for 0 < n < 2^14 (the squared length of an MV
// difference; |dx|, |dy| <= 64 gives n <= 8192), in integer arithmetic: a
// single-precision estimate, one Newton step on the integer residual
// N - s^2 with N = n * 2^48, then exact integer corrections (one step at most
// over the whole range, checked exhaustively), and rounding from the
// residual: sqrt(N) >= s + 1/2 exactly when N - s^2 > s.  It keeps the
// GPU's slow double-precision units off the evaluation's path.
__device__ __forceinline__ unsigned long long sqrt_q24(unsigned n)
{
    const long long N = (long long)n << 48;
    long long s = (long long)(sqrtf((float)n) * 16777216.0f);
    s += (long long)rintf((float)(N - s * s) / (2.0f * (float)s));
    if (s * s > N) --s;
    if (s * s > N) --s;
    if ((s + 1) * (s + 1) <= N) ++s;
    if ((s + 1) * (s + 1) <= N) ++s;
    return (unsigned long long)(s + ((N - s * s > s) ? 1 : 0));
}

// Q24 length of an MV difference (ex, ey) != (0, 0); differences beyond the
// search ranges (a caller's out-of-range FS field) take the double path.
__device__ __forceinline__ unsigned long long dist_q24(int ex, int ey)
{
    const unsigned n = (unsigned)(ex * ex + ey * ey);
    if (n < (1u << 14)) return sqrt_q24(n);
    return (unsigned long long)__double2ll_rn(sqrt((double)n) * 16777216.0);
}

#ifndef ME_SAD_VARIANT
#define ME_SAD_VARIANT 1
#endif
constexpr int kSadVariant = ME_SAD_VARIANT;

// ---------------------------------------------------------------------------
// Host-side launchers (each .cu file owns its kernels).
// ---------------------------------------------------------------------------
// eval: fuse the evaluation sums of Sec. IV into the search (FrameDev::sums,
// zeroed before the launch; FrameDev::mv_fs optional).
cudaError_t launch_dcds(const FrameDev* frames, int nframes, int ntiles, int block, int max_range,
                        bool simplified, const Shape& s, int* head, unsigned* status, int num_sms,
                        cudaStream_t st, bool eval = false);
// dynamic shared memory of a DCDS launch; box: the 8x8 visited-box variant
size_t dcds_smem_bytes(int block, int max_range, const Shape& s, bool box = false);
// Load (under lazy module loading) the one-stage search-only DCDS kernels
// for both block sizes and both variants, without launching them.
cudaError_t dcds_preload();
// Failure-detection test hook of me_estimate_batch_noalloc (noalloc.cu).
void noalloc_inject_wait_timeout(int on);

// DCDS head: kCounterInts ints, zeroed before every launch (word 0: the tile
// counter; the last word: the failure-detection test hook).
constexpr int kCounterInts = 8;

// Full search.  counter: one int zeroed before every launch (the tile counter).
// Shape: threads 256, tx blocks per tile with tx*block <= 256 (tx even for
// block 8), k in {9, 11, 13, 15} candidate rows per thread.
cudaError_t launch_fs(const FrameDev* frames, int nframes, int ntiles, int block, int max_range, const Shape& s,
                      int* counter, unsigned* status, int num_sms, cudaStream_t st, bool dual = false);
size_t fs_smem_bytes(int block, int max_range, const Shape& s);
bool fs_shape_ok(int block, int max_range, const Shape& s);

// Reference-window rows of an FS tile: the candidate rows rounded up to
// whole groups of k, plus the block height.
__host__ __device__ inline int fs_rows(int block, int range, int k)
{
    const int n = 2 * range + 1;
    return ((n + k - 1) / k) * k + block - 1;
}

// Shared-memory geometry of an FS launch (for the largest range of the batch).
struct FsGeom {
    int nch;         // 16-byte chunks per reference window row (the TMA box's middle dimension)
    int rwb;         // bytes per staged window row (nch * 16)
    int rows;        // window rows
    int raw_stride;  // bytes per staged window
    int cur_stride;  // bytes per staged current tile
    int ecols;       // columns of the expanded window
    int P;           // words per row of the expanded window
    size_t smem;     // dynamic shared memory per CTA
};
FsGeom fs_geom(int block, int max_range, int tx, int k);

// Encode the FS tensor maps of `f`: the reference frame as a 3-D tensor
// (16 bytes x w/16 chunks x h rows, box 16 x nch x rows) and the current
// frame as 2-D (box cur_w x block).  Host code; false if the CUDA driver
// rejects the description.
bool encode_fs_maps(FrameDev& f, int nch, int rows, int cur_w, int block);

cudaError_t launch_eval(const EvalDev* frames, int nframes, int block, int max_blocks, int num_sms,
                        unsigned long long* sums, cudaStream_t st);

// Motion-vector statistics (16x16 blocks): frames[i].mv is the FS field,
// ranges[i] its search range, bases[i] its first block; out (zeroed) receives
// [(2R+1)^2] histogram, [9][(2R+1)^2] D1 counts, [(2R+1)^2][25] D2 counts.
cudaError_t launch_mvp(const EvalDev* frames, const int* ranges, const long* bases, int nframes, long total, int R,
                       int num_sms, unsigned long long* out, cudaStream_t st);

cudaError_t launch_absdiff_peak(int variant, int iters, int blocks, int threads, unsigned* sink,
                                cudaStream_t st);

}  // namespace me
