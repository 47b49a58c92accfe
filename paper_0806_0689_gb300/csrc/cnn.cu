// cnn.cu -- kernels of the learned start proposal (not in the paper; the
// task adds it): a 4-layer 3x3 stride-2 convolutional trunk over a block's
// 32x32 neighbourhood, and a linear head producing 33 dx, 33 dy and 2 H/V
// logits.  Training runs the convolutions as im2col + a BF16 tensor-core GEMM
// with FP32 accumulation (mma.sync m16n8k16); the small head, the loss and
// the optimiser run on the CUDA cores in FP32, every reduction in a fixed
// order.  Inference runs the fused trunk (trunk_tc_kernel, layer 2 on
// tcgen05) with each activation carried as two bf16 parts.
//
// Layouts: activations are NHWC ([sample][y][x][channel]); an im2col row is
// one output pixel, its column k = (ky * 3 + kx) * Cin + c, zero-padded to
// Kp = a multiple of 32.  GEMM weights are [32][Kp] in the same column order.
// The canonical parameter vector (the order the host sees) is
// conv1.w [32][2][3][3], conv1.b, conv2.w [32][32][3][3], conv2.b, conv3.*,
// conv4.*, fc.w [68][NFEAT], fc.b; the head's NFEAT = 136 inputs are the 128
// conv-4 outputs in (c, y, x) order followed by the NSCAL = 8 neighbour
// scalars (left, top and top-right MVs, then their component-wise median).
#include "me_cnn.cuh"

#include <algorithm>

namespace me {
namespace cnn {
namespace {

// ------------------------------------------------------------------ GEMM
// C[M][N] (fp32) = A[M][K] * B[N][K]^T, A and B bf16 with K contiguous
// (lda, ldb elements), K a multiple of 32 inside each split.  CTA tile 64x32,
// 4 warps of 16x32, k-step 32 through shared memory.  gridDim.z splits K;
// with more than one split, split z stores its partial product at
// C + z * M * ldc and a second kernel sums the splits in order (no atomics:
// the result does not depend on scheduling).
constexpr int GM = 64, GN = 32, GK = 32, GKP = 40;  // GKP: padded smem row (bank spread)

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) gemm_kernel(const __nv_bfloat16* __restrict__ A, int lda,
                                                   const __nv_bfloat16* __restrict__ B, int ldb,
                                                   float* __restrict__ Cm, int ldc, int M, int N, int K,
                                                   int k_per_split, const float* __restrict__ bias,
                                                   __nv_bfloat16* __restrict__ out_bf16, int mode)
{
    __shared__ __align__(16) __nv_bfloat16 sA[GM][GKP];
    __shared__ __align__(16) __nv_bfloat16 sB[GN][GKP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    const int k_begin = blockIdx.z * k_per_split;
    const int k_end = min(K, k_begin + k_per_split);
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    const int g = lane >> 2, t = lane & 3;
    for (int k0 = k_begin; k0 < k_end; k0 += GK) {
        // A tile: 64 rows x 32 k = 256 chunks of 8 bf16; B tile: 32 x 32 = 128 chunks
        for (int c = tid; c < GM * 4; c += 128) {
            const int r = c >> 2, kc = (c & 3) * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + r < M && k0 + kc < k_end)
                v = *reinterpret_cast<const uint4*>(A + (size_t)(m0 + r) * lda + k0 + kc);
            *reinterpret_cast<uint4*>(&sA[r][kc]) = v;
        }
        {
            const int r = tid >> 2, kc = (tid & 3) * 8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (n0 + r < N && k0 + kc < k_end)
                v = *reinterpret_cast<const uint4*>(B + (size_t)(n0 + r) * ldb + k0 + kc);
            *reinterpret_cast<uint4*>(&sB[r][kc]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t a[4];
            const int ar = warp * 16 + g;
            a[0] = *reinterpret_cast<const uint32_t*>(&sA[ar][ks + 2 * t]);
            a[1] = *reinterpret_cast<const uint32_t*>(&sA[ar + 8][ks + 2 * t]);
            a[2] = *reinterpret_cast<const uint32_t*>(&sA[ar][ks + 2 * t + 8]);
            a[3] = *reinterpret_cast<const uint32_t*>(&sA[ar + 8][ks + 2 * t + 8]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t b[2];
                b[0] = *reinterpret_cast<const uint32_t*>(&sB[j * 8 + g][ks + 2 * t]);
                b[1] = *reinterpret_cast<const uint32_t*>(&sB[j * 8 + g][ks + 2 * t + 8]);
                mma_bf16(acc[j], a, b);
            }
        }
        __syncthreads();
    }
    // epilogue: acc[j] holds rows (g, g+8) x cols (2t, 2t+1) of n-tile j
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = m0 + warp * 16 + g + 8 * h;
            if (r >= M) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int col = n0 + j * 8 + 2 * t + q;
                if (col >= N) continue;
                const float v = acc[j][2 * h + q];
                if (mode == GEMM_STORE) {
                    Cm[(size_t)r * ldc + col] = v;
                } else if (mode == GEMM_PARTIAL) {
                    Cm[(size_t)blockIdx.z * M * ldc + (size_t)r * ldc + col] = v;
                } else {  // GEMM_BIAS_RELU: bias + ReLU, stored as bf16
                    const float z = v + bias[col];
                    out_bf16[(size_t)r * ldc + col] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ fused trunk (inference)
// Features and all four convolutions without im2col.  Helpers shared by the
// layers that run on mma.sync: implicit-GEMM A fragments are gathered from
// the previous layer's activations in shared memory (NHWC, a pixel padded to
// PXW words so that the 8 output pixels of a fragment, two input pixels
// apart, fall on 8 different bank groups), B fragments are read from the
// GEMM-layout weights (L1-resident), bias + ReLU + bf16 rounding happen in
// the epilogue.  Operands are bf16 and sums fp32; each activation enters the
// next layer as two bf16 parts (split_relu), both multiplied by the same
// weights, so the trunk computes the network with bf16 weights and
// activations of about fp32 precision.  (The training path, on the im2col
// GEMMs, rounds each activation once to bf16.)
constexpr int PXW = 18;   // smem words per pixel of a 32-channel activation (16 + 2 padding)

struct TrunkW {
    const __nv_bfloat16* w[LAYERS];
    const float* b[LAYERS];
};

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 h) { return *reinterpret_cast<const uint32_t*>(&h); }

// Two ReLU outputs of the inference trunk as a pair of bf16 words, hi + lo:
// hi is the activation rounded to bf16, lo the remainder rounded to bf16, so
// that hi + lo carries 16 significant bits and a layer that multiplies both
// parts by the same bf16 weights sees the fp32 activation to within 2^-17.
__device__ __forceinline__ void split_relu(float v0, float v1, uint32_t& hi, uint32_t& lo)
{
    v0 = v0 > 0.f ? v0 : 0.f;
    v1 = v1 > 0.f ? v1 : 0.f;
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 f = __bfloat1622float2(h);
    hi = bf2_bits(h);
    lo = bf2_bits(__floats2bfloat162_rn(v0 - f.x, v1 - f.y));
}

// Output pixels of a warp's m-tiles: rows g and g + 8 (h = 0, 1) of m-tile i.
template <int NM>
struct Rows {
    int s[NM][2], oy[NM][2], ox[NM][2];
};

// One 3x3 stride-2 layer with 32 input channels (implicit GEMM, K = 9 taps x
// 32) over an activation held as hi and lo bf16 parts (the same layout twice,
// rows ROWP words apart), for NM m-tiles of n-tile n0 per warp, added to acc:
// each weight fragment is loaded once for both parts, and the taps are
// unrolled so that the weight loads of later taps issue early.
template <int HIN, int NM, int ROWP>
__device__ __forceinline__ void conv32_hl(const uint32_t* __restrict__ hi, const uint32_t* __restrict__ lo,
                                          const uint32_t* __restrict__ Wl, const Rows<NM> rw, int n0,
                                          float (&acc)[NM][1][4], int g, int t)
{
#pragma unroll 3
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap - 3 * ky;
        int pix[NM][2];  // word offset of the input pixel, -1 outside (zero padding)
#pragma unroll
        for (int i = 0; i < NM; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int y = 2 * rw.oy[i][h] + ky - 1, x = 2 * rw.ox[i][h] + kx - 1;
                pix[i][h] = (y >= 0 && y < HIN && x >= 0 && x < HIN) ? (rw.s[i][h] * HIN + y) * ROWP + x * PXW : -1;
            }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int w0 = half * 8 + t;  // channel pair 2*w0 (and +8 channels)
            const uint32_t* wr = Wl + (size_t)(n0 * 8 + g) * 144 + tap * 16 + half * 8 + t;
            const uint32_t bf[2] = {__ldg(wr), __ldg(wr + 4)};
#pragma unroll
            for (int i = 0; i < NM; ++i) {
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    const uint32_t* in = part ? lo : hi;
                    uint32_t a[4];
                    a[0] = pix[i][0] >= 0 ? in[pix[i][0] + w0] : 0u;
                    a[1] = pix[i][1] >= 0 ? in[pix[i][1] + w0] : 0u;
                    a[2] = pix[i][0] >= 0 ? in[pix[i][0] + w0 + 4] : 0u;
                    a[3] = pix[i][1] >= 0 ? in[pix[i][1] + w0 + 4] : 0u;
                    mma_bf16(acc[i][0], a, bf);
                }
            }
        }
    }
}

__device__ __forceinline__ int trunk_frame(const PropFrame* fr, int nframes, long gid)
{
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].base <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------ trunk with tcgen05 (inference)
// Two samples per iteration: their two feature planes are built from the
// frames straight into shared memory (the features of feat_kernel; values
// k/128, exact in bf16), then the four layers run back to back, each layer's
// input as its hi and lo bf16 parts.  Layer 1 runs twice, the first pass
// writing the hi parts of its output, the second the lo parts, into the same
// planes; layer 2 accumulates both passes in TMEM.  Layer 2 (64 % of the
// trunk's multiply-adds)
// runs on the 5th-generation tensor cores: one thread issues
// tcgen05.mma (M = 128 rows = 2 samples x 8 x 8 outputs, N = 32, K = 16 per
// instruction, bf16 x bf16 -> fp32 in TMEM) for the 9 taps x 2 channel
// halves, completion arrives on an mbarrier, and every warp reads its TMEM
// lane quarter back with tcgen05.ld for bias + ReLU.  The A operand needs no
// gather: layer 1 writes its output in a parity-split layout -- for each
// group of 8 channels and each (row parity, column parity) a plane of
// 9 x 9 pixels of 16 bytes, row 0 / column 0 of the odd planes being the
// zero padding at -1, the two samples' lines interleaved -- in which the
// pixels one tap reads for 8 consecutive outputs of one output row are 8
// consecutive 16-byte rows, i.e. one 8x16-byte core matrix of the canonical
// K-major layout without swizzle.  Shared-memory matrix descriptors then
// address every tap directly: the next 8 channels are one channel-group plane
// further (leading byte offset), the next output row of the tile one
// interleaved line further (stride byte offset).  Layers 1, 3 and 4 stay on
// mma.sync (K = 18 for layer 1, and too few rows per sample for M = 128 in
// layers 3-4).  The layer-2 and layer-3 outputs (hi and lo arrays) reuse the
// layer-1 planes, dead once the second layer-2 pass has completed; the cells
// of those planes that are zero padding are cleared again every iteration.
constexpr int TC_S = 2;                          // samples per iteration (one M = 128 tile in layer 2)
constexpr int TC_LINE = 9 * 16;                  // bytes per interleaved plane line (9 pixels)
constexpr int TC_PLANE = 9 * TC_S * TC_LINE;     // 9 rows x 2 samples
constexpr int TC_CG = 4 * TC_PLANE;              // the 4 parity planes of one channel group
constexpr int TC_A1 = 4 * TC_CG;                 // 4 channel groups
constexpr int TC_W2 = 9 * 2048;                  // layer-2 weights in core layout
constexpr uint32_t TC_WAIT = 1u << 22;

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle (sm_100 family format).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// row pitches (words) of the layer-2 and layer-3 outputs: a fragment's 8
// pixels then sit on 8 different groups of 4 banks (layer 3 reads rows 2
// apart: 2 * TC_R8 = 16 mod 32; layer 4 rows 2 and samples 4 rows apart:
// 2 * TC_R4 = 8 and 4 * TC_R4 = 16 mod 32, pixels 2 apart 4)
constexpr int TC_R8 = 8 * PXW + 8;
constexpr int TC_R4 = 4 * PXW + 12;
constexpr int TC_A23 = 2 * TC_S * (8 * TC_R8 + 4 * TC_R4);  // words of A2 and A3, hi and lo
static_assert(TC_A23 * 4 <= TC_A1, "the layer-2/3 outputs fit in the layer-1 planes");

__global__ void __launch_bounds__(256, 3) trunk_tc_kernel(const PropFrame* __restrict__ fr, int nframes, long sbase,
                                                          int n, TrunkW tw, float* __restrict__ a4,
                                                          unsigned* __restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t tcs[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tcs) + 1023) & ~uintptr_t(1023));
    uint8_t* A1 = base;                                                 // parity-split layer-1 output
    uint8_t* W2c = A1 + TC_A1;                                          // layer-2 weights, core layout
    uint32_t* X = reinterpret_cast<uint32_t*>(W2c + TC_W2);             // [TC_S][32][32] feature words
    uint32_t* A2h = reinterpret_cast<uint32_t*>(A1);                    // [TC_S][8] rows of TC_R8 words, in A1
    uint32_t* A2l = A2h + TC_S * 8 * TC_R8;
    uint32_t* A3h = A2l + TC_S * 8 * TC_R8;                             // [TC_S][4] rows of TC_R4 words
    uint32_t* A3l = A3h + TC_S * 4 * TC_R4;
    __shared__ float sb[LAYERS][CH];
    __shared__ int s_fr[TC_S], s_px[TC_S], s_py[TC_S];
    __shared__ const uint8_t* s_cur[TC_S];
    __shared__ const uint8_t* s_ref[TC_S];
    __shared__ int s_pitch[TC_S], s_w[TC_S], s_h[TC_S];
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t* W3 = reinterpret_cast<const uint32_t*>(tw.w[2]);
    const uint32_t* W4 = reinterpret_cast<const uint32_t*>(tw.w[3]);

#pragma unroll
    for (int l = 0; l < LAYERS; ++l)
        if (tid < CH) sb[l][tid] = tw.b[l][tid];
    // zero the layer-1 planes once: the padding (row / column 0 of odd planes) is never written
    for (int i = tid; i < TC_A1 / 16; i += blockDim.x) reinterpret_cast<uint4*>(A1)[i] = make_uint4(0u, 0u, 0u, 0u);
    // layer-2 weights [32][288] (k = tap * 32 + c) -> core matrices (n-group, k-group) of each tap
    {
        const __nv_bfloat16* w2 = tw.w[1];
        for (int i = tid; i < 32 * 288; i += blockDim.x) {
            const int nn = i / 288, k = i - nn * 288, tap = k >> 5, c = k & 31;
            *reinterpret_cast<__nv_bfloat16*>(W2c + tap * 2048 + ((c >> 3) * 4 + (nn >> 3)) * 128 + (nn & 7) * 16 +
                                              (c & 7) * 2) = w2[i];
        }
    }
    uint32_t b1[4][2][2];
    {
        const uint32_t* w1 = reinterpret_cast<const uint32_t*>(tw.w[0]);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                b1[j][kt][0] = w1[(j * 8 + g) * 16 + kt * 8 + t];
                b1[j][kt][1] = w1[(j * 8 + g) * 16 + kt * 8 + t + 4];
            }
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(tc_smem(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // D f32, A bf16, B bf16, both K-major, N = 32, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

    uint32_t phase = 0;
    for (int s0 = blockIdx.x * TC_S; s0 < n; s0 += gridDim.x * TC_S) {
        const int ns = min(TC_S, n - s0);
        if (tid < TC_S && tid < ns) {
            const long gid = sbase + s0 + tid;
            const int f = trunk_frame(fr, nframes, gid);
            const int k = (int)(gid - fr[f].base);
            s_fr[tid] = f;
            s_px[tid] = (k % fr[f].nbx) * 16;
            s_py[tid] = (k / fr[f].nbx) * 16;
            s_cur[tid] = fr[f].cur;
            s_ref[tid] = fr[f].ref;
            s_pitch[tid] = fr[f].pitch;
            s_w[tid] = fr[f].w;
            s_h[tid] = fr[f].h;
        }
        __syncthreads();
        // the previous iteration's layer-2/3 outputs overwrote padding cells of the planes
        for (int i = tid; i < TC_A23 / 4; i += blockDim.x) reinterpret_cast<uint4*>(A1)[i] = make_uint4(0u, 0u, 0u, 0u);
        // a thread builds 8 consecutive pixels of one of the 32 rows of its
        // sample's planes: one 8-byte load of the reference row (and of the
        // current row inside the central 16x16), or per-byte clamped loads
        // when the 32x32 patch crosses the frame's edge
        static_assert(TC_S * 32 * 4 == 256, "one 8-pixel chunk per thread");
        {
            const int s = tid >> 7, q = tid & 127, yy = q >> 2, c = q & 3;
            uint32_t o[8];
            if (s < ns) {
                const uint8_t* cur = s_cur[s];
                const uint8_t* ref = s_ref[s];
                const int pitch = s_pitch[s], fw = s_w[s], fh = s_h[s];
                const int px = s_px[s], py = s_py[s];
                const int ry = py + yy - 8, rx0 = px - 8 + 8 * c;
                const bool in_cur = yy >= 8 && yy < 24 && (c == 1 || c == 2);
                uint32_t rw[2], cw[2] = {0u, 0u};
                if (px >= 8 && px + 24 <= fw && py >= 8 && py + 24 <= fh) {
                    const uint2 r = *reinterpret_cast<const uint2*>(ref + (size_t)ry * pitch + rx0);
                    rw[0] = r.x; rw[1] = r.y;
                    if (in_cur) {
                        const uint2 u = *reinterpret_cast<const uint2*>(cur + (size_t)ry * pitch + rx0);
                        cw[0] = u.x; cw[1] = u.y;
                    }
                } else {
                    const int ryc = min(max(ry, 0), fh - 1);
                    rw[0] = rw[1] = 0u;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int rxc = min(max(rx0 + k, 0), fw - 1);
                        rw[k >> 2] |= (uint32_t)ref[(size_t)ryc * pitch + rxc] << (8 * (k & 3));
                        if (in_cur) cw[k >> 2] |= (uint32_t)cur[(size_t)ry * pitch + rx0 + k] << (8 * (k & 3));
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float v0 = in_cur ? ((float)((cw[k >> 2] >> (8 * (k & 3))) & 255u) - 128.f) * (1.f / 128.f) : 0.f;
                    const float v1 = ((float)((rw[k >> 2] >> (8 * (k & 3))) & 255u) - 128.f) * (1.f / 128.f);
                    o[k] = bf2_bits(__floats2bfloat162_rn(v0, v1));
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) o[k] = 0u;
            }
            uint4* dst = reinterpret_cast<uint4*>(X + s * 1024 + yy * 32 + 8 * c);
            dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
            dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
        __syncthreads();

        // ---- layers 1 and 2, twice: pass 0 feeds layer 2 the hi parts of the
        // layer-1 output, pass 1 the lo parts, accumulated in the same TMEM tile ----
        for (int pass = 0; pass < 2; ++pass) {
            // layer 1 (mma.sync): output rows of 16 pixels, written to the parity-split planes
            for (int mt = warp; mt < TC_S * 16; mt += 8) {
                const int s = mt >> 4, oy = mt & 15;
                float acc[4][4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
#pragma unroll
                for (int kt = 0; kt < 2; ++kt) {
                    uint32_t a[4];
#pragma unroll
                    for (int qq = 0; qq < 4; ++qq) {
                        const int tap = kt * 8 + t + ((qq & 2) ? 4 : 0);
                        const int ox = g + ((qq & 1) ? 8 : 0);
                        uint32_t v = 0u;
                        if (tap < 9) {
                            const int y = 2 * oy + tap / 3 - 1, xx = 2 * ox + tap % 3 - 1;
                            if (y >= 0 && y < 32 && xx >= 0 && xx < 32) v = X[s * 1024 + y * 32 + xx];
                        }
                        a[qq] = v;
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_bf16(acc[j], a, b1[j][kt]);
                }
                const int py = oy & 1, yl = (oy + py) >> 1;
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int ox = g + 8 * h, c = j * 8 + 2 * t;
                        const int px = ox & 1, xl = (ox + px) >> 1;
                        uint32_t hi, lo;
                        split_relu(acc[j][2 * h] + sb[0][c], acc[j][2 * h + 1] + sb[0][c + 1], hi, lo);
                        *reinterpret_cast<uint32_t*>(A1 + j * TC_CG + (py * 2 + px) * TC_PLANE +
                                                     (yl * TC_S + s) * TC_LINE + xl * 16 + (c & 7) * 2) =
                            pass ? lo : hi;
                    }
            }
            // layer 2 (tcgen05): 18 MMAs from the planes, accumulated in TMEM
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t a_base = tc_smem(A1), b_base = tc_smem(W2c);
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int ky = tap / 3, kx = tap - 3 * ky;
                    const int py = ky == 1 ? 0 : 1, yoff = ky == 2 ? 1 : 0;
                    const int px = kx == 1 ? 0 : 1, xoff = kx == 2 ? 1 : 0;
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t aa = a_base + (2 * ks) * TC_CG + (py * 2 + px) * TC_PLANE +
                                            yoff * TC_S * TC_LINE + xoff * 16;
                        const uint32_t bb = b_base + tap * 2048 + ks * 1024;
                        const uint64_t ad = tc_desc(aa, TC_CG, TC_LINE), bd = tc_desc(bb, 512, 128);
                        const uint32_t accum = (pass | tap | ks) ? 1u : 0u;
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accum) : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(tc_smem(&s_bar)) : "memory");
            }
            // every thread waits for the MMAs (and their reads of the planes) to complete
            uint32_t ok = 0;
            for (uint32_t it = 0; it < TC_WAIT && !ok; ++it) {
                asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                             "selp.u32 %0, 1, 0, p;\n}"
                             : "=r"(ok) : "r"(tc_smem(&s_bar)), "r"(phase) : "memory");
            }
            phase ^= 1u;
            if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&s_fail, 1);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (s_fail) break;
        }
        if (s_fail) break;
        // ---- layer-2 epilogue: warp w reads TMEM lanes 32w .. 32w + 31, row i = (2 * oy + s) * 8 + ox ----
        if (warp < 4) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[32];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                         "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                         "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                           "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                           "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                           "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                           "=r"(v[31])
                         : "r"(tmem + ((uint32_t)(32 * warp) << 16)) : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int i = 32 * warp + lane;
            const int oy = i >> 4, s = (i >> 3) & 1, ox = i & 7;
            const int o = (s * 8 + oy) * TC_R8 + ox * PXW;
#pragma unroll
            for (int c = 0; c < 32; c += 2)
                split_relu(__uint_as_float(v[c]) + sb[1][c], __uint_as_float(v[c + 1]) + sb[1][c + 1],
                           A2h[o + (c >> 1)], A2l[o + (c >> 1)]);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();

        // ---- layer 3 (mma.sync): m-tile = one sample; warp = (sample, n-tile) ----
        {
            Rows<1> rw;
            const int s = warp & 1, nt = warp >> 1;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                rw.s[0][h] = s;
                rw.oy[0][h] = (g >> 2) + 2 * h;
                rw.ox[0][h] = g & 3;
            }
            float acc[1][1][4] = {};
            conv32_hl<8, 1, TC_R8>(A2h, A2l, W3, rw, nt, acc, g, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = nt * 8 + 2 * t;
                const int o = (s * 4 + rw.oy[0][h]) * TC_R4 + rw.ox[0][h] * PXW + nt * 4 + t;
                split_relu(acc[0][0][2 * h] + sb[2][c], acc[0][0][2 * h + 1] + sb[2][c + 1], A3h[o], A3l[o]);
            }
        }
        __syncthreads();

        // ---- layer 4 (mma.sync): rows 4 * sample + pixel (rows 8-15 are padding); fp32 out ----
        if (warp < 4) {
            Rows<1> rw;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                rw.s[0][h] = h ? 0 : (g >> 2);
                rw.oy[0][h] = (g & 3) >> 1;
                rw.ox[0][h] = g & 1;
            }
            float acc[1][1][4] = {};
            conv32_hl<4, 1, TC_R4>(A3h, A3l, W4, rw, warp, acc, g, t);
            const int s = g >> 2, pix = g & 3, c = warp * 8 + 2 * t;
            if (s < ns) {
                const float z0 = acc[0][0][0] + sb[3][c], z1 = acc[0][0][1] + sb[3][c + 1];
                *reinterpret_cast<float2*>(a4 + ((size_t)(s0 + s) * 4 + pix) * CH + c) =
                    make_float2(z0 > 0.f ? z0 : 0.f, z1 > 0.f ? z1 : 0.f);
            }
        }
        // the next iteration clears the planes these layers used only after its first barrier
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (s_fail && tid == 0 && status) atomicOr(status, 1u);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ im2col / col2im
// in: NHWC [n][hin][hin][cin] bf16; cols: [n*ho*ho][kp], ho = hin / 2
__global__ void im2col_kernel(const __nv_bfloat16* __restrict__ in, int n, int hin, int cin, int kp,
                              __nv_bfloat16* __restrict__ cols)
{
    const int ho = hin / 2;
    const long total = (long)n * ho * ho * kp;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int k = (int)(i % kp);
        const long row = i / kp;
        const int ox = (int)(row % ho), oy = (int)((row / ho) % ho);
        const long s = row / ((long)ho * ho);
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (k < 9 * cin) {
            const int tap = k / cin, c = k - tap * cin;
            const int y = 2 * oy + tap / 3 - 1, x = 2 * ox + tap % 3 - 1;
            if (y >= 0 && y < hin && x >= 0 && x < hin) v = in[((s * hin + y) * hin + x) * cin + c];
        }
        cols[i] = v;
    }
}

// dcols: [n*ho*ho][kp] fp32 -> din: NHWC [n][hin][hin][cin] fp32 (gather of the
// at most 4 output pixels and taps that read each input element)
__global__ void col2im_kernel(const float* __restrict__ dcols, int n, int hin, int cin, int kp,
                              float* __restrict__ din)
{
    const int ho = hin / 2;
    const long total = (long)n * hin * hin * cin;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cin);
        const int x = (int)((i / cin) % hin), y = (int)((i / ((long)cin * hin)) % hin);
        const long s = i / ((long)cin * hin * hin);
        float acc = 0.f;
        for (int ky = 0; ky < 3; ++ky) {
            const int t2 = y + 1 - ky;  // = 2 * oy
            if (t2 < 0 || (t2 & 1) || t2 / 2 >= ho) continue;
            for (int kx = 0; kx < 3; ++kx) {
                const int u2 = x + 1 - kx;
                if (u2 < 0 || (u2 & 1) || u2 / 2 >= ho) continue;
                const long row = (s * ho + t2 / 2) * ho + u2 / 2;
                acc += dcols[row * kp + (ky * 3 + kx) * cin + c];
            }
        }
        din[i] = acc;
    }
}

// out[c][r] = in[r][c] for r < rows, c < ncols; zero for rows..rows_pad-1
__global__ void transpose_kernel(const __nv_bfloat16* __restrict__ in, int rows, int ncols, int ld_in,
                                 __nv_bfloat16* __restrict__ out, int rows_pad)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < ncols) ? in[(size_t)r * ld_in + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < ncols && r < rows_pad) out[(size_t)c * rows_pad + r] = tile[threadIdx.x][i];
    }
}

// out[c] = sum over r in order of p[r * ncols + c]: the fixed-order reduction
// of partial sums (split-K products, per-CTA column sums)
__global__ void sum_rows_kernel(const float* __restrict__ p, int nrows, int ncols, float* __restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x) {
        float t = 0.f;
        for (int r = 0; r < nrows; ++r) t += p[(size_t)r * ncols + c];
        out[c] = t;
    }
}

__global__ void sum_doubles_kernel(const double* __restrict__ p, int n, double* __restrict__ out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < n; ++i) t += p[i];
        *out = t;
    }
}

// dz = dA * (A > 0) as bf16 (rows x 32), and this CTA's share of the bias
// gradient (column sums) in part[blockIdx.x][32]
__global__ void relu_back_kernel(const float* __restrict__ da, const __nv_bfloat16* __restrict__ a, long rows,
                                 __nv_bfloat16* __restrict__ dz, float* __restrict__ part_out)
{
    __shared__ float part[32][33];
    const int c = threadIdx.x & 31, rsub = threadIdx.x >> 5;  // blockDim = 256: 8 rows at a time
    float s = 0.f;
    for (long r = blockIdx.x * 8 + rsub; r < rows; r += (long)gridDim.x * 8) {
        const float g = __bfloat162float(a[r * 32 + c]) > 0.f ? da[r * 32 + c] : 0.f;
        dz[r * 32 + c] = __float2bfloat16_rn(g);
        s += g;
    }
    part[rsub][c] = s;
    __syncthreads();
    if (rsub == 0) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += part[i][c];
        part_out[blockIdx.x * 32 + c] = t;
    }
}

// ------------------------------------------------------------------ head
// f[s][i]: the 128 conv-4 features in (c, y, x) order from NHWC [2][2][32],
// then the NSCAL scalars; logits[s][o] = fb[o] + sum_i fw[o][i] f[s][i].  The
// features are bf16 (training forward) or fp32 (inference trunk).
__device__ __forceinline__ float feat(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float feat(float v) { return v; }

template <typename T>
__global__ void head_fwd_kernel(const T* __restrict__ a4, const float* __restrict__ mvf, int n,
                                const float* __restrict__ fw, const float* __restrict__ fb,
                                float* __restrict__ logits)
{
    const long total = (long)n * NLOGIT;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int o = (int)(i % NLOGIT);
        const long s = i / NLOGIT;
        const float* w = fw + (size_t)o * NFEAT;
        float acc = fb[o];
        for (int c = 0; c < 32; ++c)
            for (int p = 0; p < 4; ++p) acc += w[c * 4 + p] * feat(a4[s * 128 + p * 32 + c]);
        for (int q = 0; q < NSCAL; ++q) acc += w[128 + q] * mvf[s * NSCAL + q];
        logits[i] = acc;
    }
}

// per sample: three softmax cross-entropies (dx 0..32, dy 33..65, H/V 66..67)
// against labels; dlogits = (softmax - onehot) * scale; loss partial sums
__global__ void loss_kernel(const float* __restrict__ logits, const int* __restrict__ labels, int n,
                            float scale, float* __restrict__ dlogits, double* __restrict__ loss_part)
{
    double local = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float* z = logits + (size_t)s * NLOGIT;
        float* dz = dlogits + (size_t)s * NLOGIT;
        const int seg0[3] = {0, 33, 66}, segn[3] = {33, 33, 2};
        for (int h = 0; h < 3; ++h) {
            const int b = seg0[h], m = segn[h], tl = labels[s * 3 + h];
            float mx = z[b];
            for (int i = 1; i < m; ++i) mx = fmaxf(mx, z[b + i]);
            float se = 0.f;
            for (int i = 0; i < m; ++i) se += __expf(z[b + i] - mx);
            for (int i = 0; i < m; ++i) dz[b + i] = scale * (__expf(z[b + i] - mx) / se - (i == tl ? 1.f : 0.f));
            local += (double)(__logf(se) + mx - z[b + tl]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0) loss_part[(blockIdx.x * blockDim.x + threadIdx.x) >> 5] = local;
}

// head backward: gfw[o][i] += sum_s dz[s][o] f[s][i]; gfb[o] += sum_s dz[s][o]
__global__ void head_wgrad_kernel(const float* __restrict__ dlogits, const __nv_bfloat16* __restrict__ a4,
                                  const float* __restrict__ mvf, int n, float* __restrict__ gfw,
                                  float* __restrict__ gfb)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;  // over NLOGIT * (NFEAT + 1)
    if (idx >= NLOGIT * (NFEAT + 1)) return;
    const int o = idx / (NFEAT + 1), i = idx - o * (NFEAT + 1);
    float acc = 0.f;
    for (int s = 0; s < n; ++s) {
        const float d = dlogits[(size_t)s * NLOGIT + o];
        float f;
        if (i == NFEAT) f = 1.f;
        else if (i < 128) f = __bfloat162float(a4[(size_t)s * 128 + (i & 3) * 32 + (i >> 2)]);
        else f = mvf[(size_t)s * NSCAL + (i - 128)];
        acc += d * f;
    }
    if (i == NFEAT) gfb[o] += acc;
    else gfw[o * NFEAT + i] += acc;
}

// head backward to the conv-4 outputs: da4 (NHWC fp32 [s][2][2][32])
__global__ void head_dgrad_kernel(const float* __restrict__ dlogits, const float* __restrict__ fw, int n,
                                  float* __restrict__ da4)
{
    const long total = (long)n * 128;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int j = (int)(i % 128);  // NHWC index: p * 32 + c
        const long s = i / 128;
        const int p = j >> 5, c = j & 31;
        const int f = c * 4 + p;  // feature index (c, y, x)
        float acc = 0.f;
        for (int o = 0; o < NLOGIT; ++o) acc += dlogits[s * NLOGIT + o] * fw[o * NFEAT + f];
        da4[i] = acc;
    }
}

// ------------------------------------------------------------------ parameters
// canonical conv weights [32][cin][3][3] -> GEMM layout [32][kp] bf16
__global__ void pack_weights_kernel(const float* __restrict__ p, int cin, int kp, __nv_bfloat16* __restrict__ w)
{
    const int total = 32 * kp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int o = i / kp, k = i - o * kp;
        float v = 0.f;
        if (k < 9 * cin) {
            const int tap = k / cin, c = k - tap * cin;
            v = p[((o * cin + c) * 9) + tap];
        }
        w[i] = __float2bfloat16_rn(v);
    }
}

// GEMM-layout weight gradient [32][kp] -> canonical gradient [32][cin][3][3] (added)
__global__ void unpack_wgrad_kernel(const float* __restrict__ gw, int cin, int kp, float* __restrict__ g)
{
    const int total = 32 * cin * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int o = i / (cin * 9), rem = i - o * cin * 9;
        const int c = rem / 9, tap = rem - c * 9;
        g[i] += gw[o * kp + tap * cin + c];
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

inline int blocks_for(long n, int per = 256, int cap = 4096)
{
    return (int)std::max(1l, std::min((n + per - 1) / per, (long)cap));
}

}  // namespace

// ------------------------------------------------------------------ host launchers
cudaError_t gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, int M,
                 int N, int K, int splits, int mode, const float* bias, __nv_bfloat16* out_bf16, cudaStream_t st)
{
    if (K % GK) return cudaErrorInvalidValue;
    splits = std::max(1, splits);
    int kps = (K + splits - 1) / splits;
    kps = (kps + GK - 1) / GK * GK;
    splits = (K + kps - 1) / kps;
    if (splits > 1) return cudaErrorInvalidValue;  // split K through gemm_splitk
    dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN, splits);
    gemm_kernel<<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, kps, bias, out_bf16, mode);
    return cudaGetLastError();
}

cudaError_t gemm_splitk(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int M, int N,
                        int K, int splits, float* partial, cudaStream_t st)
{
    if (K % GK) return cudaErrorInvalidValue;
    splits = std::min(std::max(1, splits), kMaxSplits);
    int kps = (K + splits - 1) / splits;
    kps = (kps + GK - 1) / GK * GK;
    splits = (K + kps - 1) / kps;
    dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN, splits);
    gemm_kernel<<<grid, 128, 0, st>>>(A, lda, B, ldb, partial, N, M, N, K, kps, nullptr, nullptr, GEMM_PARTIAL);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_rows_kernel<<<(M * N + 255) / 256, 256, 0, st>>>(partial, splits, M * N, C);
    return cudaGetLastError();
}

cudaError_t im2col(const __nv_bfloat16* in, int n, int hin, int cin, int kp, __nv_bfloat16* cols, cudaStream_t st)
{
    const long total = (long)n * (hin / 2) * (hin / 2) * kp;
    im2col_kernel<<<blocks_for(total), 256, 0, st>>>(in, n, hin, cin, kp, cols);
    return cudaGetLastError();
}

cudaError_t col2im(const float* dcols, int n, int hin, int cin, int kp, float* din, cudaStream_t st)
{
    const long total = (long)n * hin * hin * cin;
    col2im_kernel<<<blocks_for(total), 256, 0, st>>>(dcols, n, hin, cin, kp, din);
    return cudaGetLastError();
}

cudaError_t transpose(const __nv_bfloat16* in, int rows, int ncols, int ld_in, __nv_bfloat16* out, int rows_pad,
                      cudaStream_t st)
{
    dim3 grid((rows_pad + 31) / 32, (ncols + 31) / 32);
    transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(in, rows, ncols, ld_in, out, rows_pad);
    return cudaGetLastError();
}

cudaError_t relu_back(const float* da, const __nv_bfloat16* a, long rows, __nv_bfloat16* dz, float* dbias,
                      float* partial, cudaStream_t st)
{
    const int grid = blocks_for(rows, 8, kReluBackCtas);
    relu_back_kernel<<<grid, 256, 0, st>>>(da, a, rows, dz, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_rows_kernel<<<1, 32, 0, st>>>(partial, grid, 32, dbias);
    return cudaGetLastError();
}

size_t trunk_tc_smem_bytes()
{
    return 1024 + (size_t)TC_A1 + TC_W2 + sizeof(uint32_t) * (size_t)TC_S * 1024;
}

cudaError_t trunk_tc(const PropFrame* frames, int nframes, long sbase, int n, const __nv_bfloat16* const* w,
                     const float* params, float* a4, unsigned* status, int num_sms, cudaStream_t st)
{
    TrunkW tw;
    for (int l = 0; l < LAYERS; ++l) {
        tw.w[l] = w[l];
        tw.b[l] = params + PB[l];
    }
    const size_t smem = trunk_tc_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(trunk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int groups = (n + TC_S - 1) / TC_S;
    trunk_tc_kernel<<<std::max(1, std::min(groups, 3 * num_sms)), 256, smem, st>>>(frames, nframes, sbase, n, tw, a4,
                                                                                 status);
    return cudaGetLastError();
}

cudaError_t head_fwd(const __nv_bfloat16* a4, const float* mvf, int n, const float* fw, const float* fb,
                     float* logits, cudaStream_t st)
{
    head_fwd_kernel<<<blocks_for((long)n * NLOGIT), 256, 0, st>>>(a4, mvf, n, fw, fb, logits);
    return cudaGetLastError();
}

cudaError_t head_fwd(const float* a4, const float* mvf, int n, const float* fw, const float* fb, float* logits,
                     cudaStream_t st)
{
    head_fwd_kernel<<<blocks_for((long)n * NLOGIT), 256, 0, st>>>(a4, mvf, n, fw, fb, logits);
    return cudaGetLastError();
}

cudaError_t loss(const float* logits, const int* labels, int n, float scale, float* dlogits, double* loss_sum,
                 double* partial, cudaStream_t st)
{
    const int grid = blocks_for(n, 256, kLossCtas);
    loss_kernel<<<grid, 256, 0, st>>>(logits, labels, n, scale, dlogits, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_doubles_kernel<<<1, 32, 0, st>>>(partial, grid * 8, loss_sum);
    return cudaGetLastError();
}

cudaError_t head_bwd(const float* dlogits, const __nv_bfloat16* a4, const float* mvf, int n, const float* fw,
                     float* gfw, float* gfb, float* da4, cudaStream_t st)
{
    head_wgrad_kernel<<<(NLOGIT * (NFEAT + 1) + 255) / 256, 256, 0, st>>>(dlogits, a4, mvf, n, gfw, gfb);
    head_dgrad_kernel<<<blocks_for((long)n * 128), 256, 0, st>>>(dlogits, fw, n, da4);
    return cudaGetLastError();
}

cudaError_t pack_weights(const float* p, int cin, int kp, __nv_bfloat16* w, cudaStream_t st)
{
    pack_weights_kernel<<<blocks_for(32l * kp), 256, 0, st>>>(p, cin, kp, w);
    return cudaGetLastError();
}

cudaError_t unpack_wgrad(const float* gw, int cin, int kp, float* g, cudaStream_t st)
{
    unpack_wgrad_kernel<<<blocks_for(32l * cin * 9), 256, 0, st>>>(gw, cin, kp, g);
    return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<blocks_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace me
