// cnn.cu -- kernels of the learned start proposal (not in the paper; the
// task adds it): a 4-layer 3x3 stride-2 convolutional trunk over a block's
// 32x32 neighbourhood, and a linear head producing 33 dx, 33 dy and 2 H/V
// logits.  Convolutions run as im2col + a BF16 tensor-core GEMM with FP32
// accumulation (mma.sync m16n8k16); the small head, the loss and the
// optimiser run on the CUDA cores in FP32.
//
// Layouts: activations are NHWC ([sample][y][x][channel]); an im2col row is
// one output pixel, its column k = (ky * 3 + kx) * Cin + c, zero-padded to
// Kp = a multiple of 32.  GEMM weights are [32][Kp] in the same column order.
// The canonical parameter vector (the order the host sees) is
// conv1.w [32][2][3][3], conv1.b, conv2.w [32][32][3][3], conv2.b, conv3.*,
// conv4.*, fc.w [68][134], fc.b; the head's 134 inputs are the 128 conv-4
// outputs in (c, y, x) order followed by 6 neighbour-MV scalars.
#include "me_cnn.cuh"

#include <algorithm>

namespace me {
namespace cnn {
namespace {

// ------------------------------------------------------------------ GEMM
// C[M][N] (fp32) = A[M][K] * B[N][K]^T, A and B bf16 with K contiguous
// (lda, ldb elements), K a multiple of 32 inside each split.  CTA tile 64x32,
// 4 warps of 16x32, k-step 32 through shared memory.  gridDim.z splits K;
// with more than one split the partial sums are added atomically into C.
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
                } else if (mode == GEMM_ATOMIC) {
                    atomicAdd(&Cm[(size_t)r * ldc + col], v);
                } else {  // GEMM_BIAS_RELU: bias + ReLU, stored as bf16
                    const float z = v + bias[col];
                    out_bf16[(size_t)r * ldc + col] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ fused trunk (inference)
// Features and all four convolutions for TS samples at a time, without
// im2col: the two input planes are built from the frames straight into shared
// memory (the features of feat_kernel), each layer is an implicit GEMM whose
// A fragments are gathered from the previous layer's activations in shared
// memory (NHWC, a pixel padded to PXW words so that the 8 output pixels of a
// fragment, two input pixels apart, fall on 8 different bank groups), B
// fragments are read from the GEMM-layout weights (L1-resident), and bias +
// ReLU + bf16 rounding happen in the epilogue.  The arithmetic per output is
// the im2col path's: bf16 operands, fp32 accumulation, one bf16 rounding of
// each activation.  Two CTAs of 8 warps share an SM.
constexpr int TS = 4;     // samples per trunk iteration
constexpr int PXW = 18;   // smem words per pixel of a 32-channel activation (16 + 2 padding)

struct TrunkW {
    const __nv_bfloat16* w[LAYERS];
    const float* b[LAYERS];
};

__device__ __forceinline__ uint32_t pack_relu(float v0, float v1)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Output pixels of a warp's m-tiles: rows g and g + 8 (h = 0, 1) of m-tile i.
template <int NM>
struct Rows {
    int s[NM][2], oy[NM][2], ox[NM][2];
};

// One 3x3 stride-2 layer with 32 input channels (implicit GEMM, K = 9 taps x 32)
// for NM m-tiles and NN n-tiles (from n-tile n0) per warp.
template <int HIN, int NM, int NN>
__device__ __forceinline__ void conv32(const uint32_t* __restrict__ in, const uint32_t* __restrict__ Wl,
                                       const Rows<NM> rw, int n0, float (&acc)[NM][NN][4], int g, int t)
{
#pragma unroll
    for (int i = 0; i < NM; ++i)
#pragma unroll
        for (int j = 0; j < NN; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
        const int ky = tap / 3, kx = tap - 3 * ky;
        int pix[NM][2];  // word offset of the input pixel, -1 outside (zero padding)
#pragma unroll
        for (int i = 0; i < NM; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int y = 2 * rw.oy[i][h] + ky - 1, x = 2 * rw.ox[i][h] + kx - 1;
                pix[i][h] = (y >= 0 && y < HIN && x >= 0 && x < HIN) ? ((rw.s[i][h] * HIN + y) * HIN + x) * PXW : -1;
            }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int w0 = half * 8 + t;  // channel pair 2*w0 (and +8 channels)
            uint32_t bf[NN][2];
#pragma unroll
            for (int j = 0; j < NN; ++j) {
                const uint32_t* wr = Wl + (size_t)((n0 + j) * 8 + g) * 144 + tap * 16 + half * 8 + t;
                bf[j][0] = __ldg(wr);
                bf[j][1] = __ldg(wr + 4);
            }
#pragma unroll
            for (int i = 0; i < NM; ++i) {
                uint32_t a[4];
                a[0] = pix[i][0] >= 0 ? in[pix[i][0] + w0] : 0u;
                a[1] = pix[i][1] >= 0 ? in[pix[i][1] + w0] : 0u;
                a[2] = pix[i][0] >= 0 ? in[pix[i][0] + w0 + 4] : 0u;
                a[3] = pix[i][1] >= 0 ? in[pix[i][1] + w0 + 4] : 0u;
#pragma unroll
                for (int j = 0; j < NN; ++j) mma_bf16(acc[i][j], a, bf[j]);
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

__global__ void __launch_bounds__(256, 2) trunk_kernel(const PropFrame* __restrict__ fr, int nframes, long sbase,
                                                       int n, TrunkW tw, __nv_bfloat16* __restrict__ a4)
{
    extern __shared__ __align__(16) uint32_t tsm[];
    uint32_t* A1 = tsm;                         // [TS][16][16][PXW]
    uint32_t* A2 = A1 + TS * 256 * PXW;         // [TS][8][8][PXW]
    uint32_t* A3 = A2 + TS * 64 * PXW;          // [TS][4][4][PXW]
    uint32_t* X = A2;                           // [TS][32][32] pixels of 2 channels; dead once layer 1 is done
    __shared__ float sb[LAYERS][CH];
    __shared__ int s_fr[TS], s_px[TS], s_py[TS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t* W2 = reinterpret_cast<const uint32_t*>(tw.w[1]);  // [32][144] words each
    const uint32_t* W3 = reinterpret_cast<const uint32_t*>(tw.w[2]);
    const uint32_t* W4 = reinterpret_cast<const uint32_t*>(tw.w[3]);
#pragma unroll
    for (int l = 0; l < LAYERS; ++l)
        if (tid < CH) sb[l][tid] = tw.b[l][tid];
    // layer 1 (K = 18 padded to 32): the B fragments live in registers
    uint32_t b1[4][2][2];
    {
        const uint32_t* w1 = reinterpret_cast<const uint32_t*>(tw.w[0]);  // [32][16] words
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) {
                b1[j][kt][0] = w1[(j * 8 + g) * 16 + kt * 8 + t];
                b1[j][kt][1] = w1[(j * 8 + g) * 16 + kt * 8 + t + 4];
            }
    }
    __syncthreads();

    for (int s0 = blockIdx.x * TS; s0 < n; s0 += gridDim.x * TS) {
        const int ns = min(TS, n - s0);
        if (tid < TS && tid < ns) {
            const long gid = sbase + s0 + tid;
            const int f = trunk_frame(fr, nframes, gid);
            const int k = (int)(gid - fr[f].base);
            s_fr[tid] = f;
            s_px[tid] = (k % fr[f].nbx) * 16;
            s_py[tid] = (k / fr[f].nbx) * 16;
        }
        __syncthreads();  // also: the previous iteration's reads of A2 / A3 are done
        // features (as feat_kernel): channel 0 = the current block centred in a zero 32x32 canvas,
        // channel 1 = the co-located reference patch, coordinates clamped; both (p - 128) / 128
        for (int i = tid; i < TS * 1024; i += blockDim.x) {
            const int s = i >> 10, pix = i & 1023, yy = pix >> 5, xx = pix & 31;
            uint32_t v = 0u;
            if (s < ns) {
                const PropFrame& F = fr[s_fr[s]];
                const int px = s_px[s], py = s_py[s];
                float v0 = 0.f;
                if (yy >= 8 && yy < 24 && xx >= 8 && xx < 24)
                    v0 = ((float)F.cur[(size_t)(py + yy - 8) * F.pitch + (px + xx - 8)] - 128.f) * (1.f / 128.f);
                const int ry = min(max(py + yy - 8, 0), F.h - 1), rxx = min(max(px + xx - 8, 0), F.w - 1);
                const float v1 = ((float)F.ref[(size_t)ry * F.pitch + rxx] - 128.f) * (1.f / 128.f);
                const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
                v = *reinterpret_cast<const uint32_t*>(&h);
            }
            X[i] = v;
        }
        __syncthreads();

        // ---- layer 1: 32x32x2 -> 16x16x32; an m-tile is one output row of 16 pixels ----
        for (int mt = warp; mt < TS * 16; mt += 8) {
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
                    const int tap = kt * 8 + t + ((qq & 2) ? 4 : 0);  // k = 2*tap + c, c = 0, 1 in one word
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
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ox = g + 8 * h, c = j * 8 + 2 * t;
                    A1[((s * 16 + oy) * 16 + ox) * PXW + j * 4 + t] =
                        pack_relu(acc[j][2 * h] + sb[0][c], acc[j][2 * h + 1] + sb[0][c + 1]);
                }
        }
        __syncthreads();

        // ---- layer 2: 16x16x32 -> 8x8x32; m-tile = two output rows; two m-tiles per warp ----
        {
            Rows<2> rw;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int mt = warp + 8 * i;  // 16 m-tiles: sample mt / 4, rows 2*(mt % 4) and +1
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    rw.s[i][h] = mt >> 2;
                    rw.oy[i][h] = 2 * (mt & 3) + h;
                    rw.ox[i][h] = g;
                }
            }
            float acc[2][4][4];
            conv32<16, 2, 4>(A1, W2, rw, 0, acc, g, t);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int c = j * 8 + 2 * t;
                        A2[((rw.s[i][h] * 8 + rw.oy[i][h]) * 8 + rw.ox[i][h]) * PXW + j * 4 + t] =
                            pack_relu(acc[i][j][2 * h] + sb[1][c], acc[i][j][2 * h + 1] + sb[1][c + 1]);
                    }
        }
        __syncthreads();

        // ---- layer 3: 8x8x32 -> 4x4x32; m-tile = one sample (16 pixels); warp = (sample, half of N) ----
        {
            Rows<1> rw;
            const int s = warp & 3, nh = warp >> 2;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                rw.s[0][h] = s;
                rw.oy[0][h] = (g >> 2) + 2 * h;  // rows g and g + 8 of the tile: pixel index r = 4 * oy + ox
                rw.ox[0][h] = g & 3;
            }
            float acc[1][2][4];
            conv32<8, 1, 2>(A2, W3, rw, 2 * nh, acc, g, t);
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = (2 * nh + j) * 8 + 2 * t;
                    A3[((s * 4 + rw.oy[0][h]) * 4 + rw.ox[0][h]) * PXW + (2 * nh + j) * 4 + t] =
                        pack_relu(acc[0][j][2 * h] + sb[2][c], acc[0][j][2 * h + 1] + sb[2][c + 1]);
                }
        }
        __syncthreads();

        // ---- layer 4: 4x4x32 -> 2x2x32; one m-tile = 4 samples x 4 pixels; warp = n-tile ----
        if (warp < 4) {
            Rows<1> rw;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                rw.s[0][h] = (g >> 2) + 2 * h;  // row r = 4 * sample + pixel
                rw.oy[0][h] = (g & 3) >> 1;
                rw.ox[0][h] = g & 1;
            }
            float acc[1][1][4];
            conv32<4, 1, 1>(A3, W4, rw, warp, acc, g, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int s = rw.s[0][h], pix = (g & 3), c = warp * 8 + 2 * t;
                if (s < ns) {
                    const uint32_t v = pack_relu(acc[0][0][2 * h] + sb[3][c], acc[0][0][2 * h + 1] + sb[3][c + 1]);
                    *reinterpret_cast<uint32_t*>(a4 + ((size_t)(s0 + s) * 4 + pix) * CH + c) = v;
                }
            }
        }
    }
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

// dz = dA * (A > 0) as bf16 (rows x 32), and the bias gradient (column sums)
__global__ void relu_back_kernel(const float* __restrict__ da, const __nv_bfloat16* __restrict__ a, long rows,
                                 __nv_bfloat16* __restrict__ dz, float* __restrict__ dbias)
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
        atomicAdd(&dbias[c], t);
    }
}

// ------------------------------------------------------------------ head
// f[s][i]: the 128 conv-4 features in (c, y, x) order from NHWC [2][2][32],
// then the 6 scalars; logits[s][o] = fb[o] + sum_i fw[o][i] f[s][i]
__global__ void head_fwd_kernel(const __nv_bfloat16* __restrict__ a4, const float* __restrict__ mvf, int n,
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
            for (int p = 0; p < 4; ++p) acc += w[c * 4 + p] * __bfloat162float(a4[s * 128 + p * 32 + c]);
        for (int q = 0; q < 6; ++q) acc += w[128 + q] * mvf[s * 6 + q];
        logits[i] = acc;
    }
}

// per sample: three softmax cross-entropies (dx 0..32, dy 33..65, H/V 66..67)
// against labels; dlogits = (softmax - onehot) * scale; loss partial sums
__global__ void loss_kernel(const float* __restrict__ logits, const int* __restrict__ labels, int n,
                            float scale, float* __restrict__ dlogits, double* __restrict__ loss_sum)
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
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, local);
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
        else f = mvf[(size_t)s * 6 + (i - 128)];
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
    if (splits > 1 && mode != GEMM_ATOMIC) return cudaErrorInvalidValue;
    dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN, splits);
    gemm_kernel<<<grid, 128, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, kps, bias, out_bf16, mode);
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
                      cudaStream_t st)
{
    relu_back_kernel<<<blocks_for(rows, 8, 2048), 256, 0, st>>>(da, a, rows, dz, dbias);
    return cudaGetLastError();
}

size_t trunk_smem_bytes()
{
    static_assert(TS * 1024 <= TS * (64 + 16) * PXW, "the feature planes fit in the layer-2/3 buffers");
    return sizeof(uint32_t) * ((size_t)TS * (256 + 64 + 16) * PXW);
}

cudaError_t trunk(const PropFrame* frames, int nframes, long sbase, int n, const __nv_bfloat16* const* w,
                  const float* params, __nv_bfloat16* a4, int num_sms, cudaStream_t st)
{
    TrunkW tw;
    for (int l = 0; l < LAYERS; ++l) {
        tw.w[l] = w[l];
        tw.b[l] = params + PB[l];
    }
    const size_t smem = trunk_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(trunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int groups = (n + TS - 1) / TS;
    trunk_kernel<<<std::max(1, std::min(groups, 2 * num_sms)), 256, smem, st>>>(frames, nframes, sbase, n, tw, a4);
    return cudaGetLastError();
}

cudaError_t head_fwd(const __nv_bfloat16* a4, const float* mvf, int n, const float* fw, const float* fb,
                     float* logits, cudaStream_t st)
{
    head_fwd_kernel<<<blocks_for((long)n * NLOGIT), 256, 0, st>>>(a4, mvf, n, fw, fb, logits);
    return cudaGetLastError();
}

cudaError_t loss(const float* logits, const int* labels, int n, float scale, float* dlogits, double* loss_sum,
                 cudaStream_t st)
{
    loss_kernel<<<blocks_for(n, 256, 1024), 256, 0, st>>>(logits, labels, n, scale, dlogits, loss_sum);
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
