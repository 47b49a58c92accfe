// me_cnn.cuh -- the learned start proposal: sizes, parameter layout and the
// host launchers of cnn.cu.  (Not in the paper: an extension of DCDS.)
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace me {
namespace cnn {

constexpr int NLOGIT = 68;   // 33 dx + 33 dy + 2 H/V
constexpr int NSCAL = 8;     // neighbour scalars: 3 MVs and their component-wise median, each / 16
constexpr int NFEAT = 128 + NSCAL;  // 128 conv-4 outputs + the neighbour scalars
constexpr int CH = 32;       // channels of every conv layer
// canonical parameter offsets
constexpr int P_W1 = 0, P_B1 = P_W1 + CH * 2 * 9;
constexpr int P_W2 = P_B1 + CH, P_B2 = P_W2 + CH * CH * 9;
constexpr int P_W3 = P_B2 + CH, P_B3 = P_W3 + CH * CH * 9;
constexpr int P_W4 = P_B3 + CH, P_B4 = P_W4 + CH * CH * 9;
constexpr int P_FW = P_B4 + CH, P_FB = P_FW + NLOGIT * NFEAT;
constexpr int NPARAMS = P_FB + NLOGIT;  // 37668
// per layer: input side and channels, GEMM K (padded)
constexpr int LAYERS = 4;
constexpr int HIN[LAYERS] = {32, 16, 8, 4};
constexpr int CIN[LAYERS] = {2, CH, CH, CH};
constexpr int KP[LAYERS] = {32, 288, 288, 288};
constexpr int PW[LAYERS] = {P_W1, P_W2, P_W3, P_W4};
constexpr int PB[LAYERS] = {P_B1, P_B2, P_B3, P_B4};

enum { GEMM_STORE = 0, GEMM_PARTIAL = 1, GEMM_BIAS_RELU = 2 };

// Training reductions run in a fixed order (no atomics), so a training step
// gives the same result every time: split-K products and per-CTA partial
// sums go to buffers of these sizes and are summed in order.
constexpr int kMaxSplits = 128;                       // split-K partial products: kMaxSplits * M * N floats
constexpr int kReluBackCtas = 2048;                   // bias-gradient partials: kReluBackCtas * 32 floats
constexpr int kLossCtas = 1024;                       // loss partials: kLossCtas * 8 doubles

cudaError_t gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, int M,
                 int N, int K, int splits, int mode, const float* bias, __nv_bfloat16* out_bf16, cudaStream_t st);
// C[M][N] (written, row stride N) = A B^T with K split into at most `splits`
// parts whose products go to `partial` and are summed in order.
cudaError_t gemm_splitk(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C, int M, int N,
                        int K, int splits, float* partial, cudaStream_t st);
cudaError_t im2col(const __nv_bfloat16* in, int n, int hin, int cin, int kp, __nv_bfloat16* cols, cudaStream_t st);
cudaError_t col2im(const float* dcols, int n, int hin, int cin, int kp, float* din, cudaStream_t st);
cudaError_t transpose(const __nv_bfloat16* in, int rows, int ncols, int ld_in, __nv_bfloat16* out, int rows_pad,
                      cudaStream_t st);
cudaError_t relu_back(const float* da, const __nv_bfloat16* a, long rows, __nv_bfloat16* dz, float* dbias,
                      float* partial, cudaStream_t st);
cudaError_t head_fwd(const __nv_bfloat16* a4, const float* mvf, int n, const float* fw, const float* fb,
                     float* logits, cudaStream_t st);
cudaError_t head_fwd(const float* a4, const float* mvf, int n, const float* fw, const float* fb, float* logits,
                     cudaStream_t st);
cudaError_t loss(const float* logits, const int* labels, int n, float scale, float* dlogits, double* loss_sum,
                 double* partial, cudaStream_t st);
cudaError_t head_bwd(const float* dlogits, const __nv_bfloat16* a4, const float* mvf, int n, const float* fw,
                     float* gfw, float* gfb, float* da4, cudaStream_t st);
cudaError_t pack_weights(const float* p, int cin, int kp, __nv_bfloat16* w, cudaStream_t st);
cudaError_t unpack_wgrad(const float* gw, int cin, int kp, float* g, cudaStream_t st);
cudaError_t adam(float* p, const float* g, float* m, float* v, int n, float lr, int step, cudaStream_t st);

// One frame pair as the proposal kernels see it.  The network works on 16x16
// regions (nbx x nby of them, numbered from base through the frames); the
// search on blocks of `block` pixels (snbx x snby, numbered from sbase): a
// 16x16 block is its own region, four 8x8 blocks share theirs.
struct PropFrame {
    const uint8_t* cur;
    const uint8_t* ref;
    const int16_t* nbr;  // motion field (search grid) for the neighbour scalars and the training labels
    int16_t* mv;         // outputs of the learned search
    uint32_t* sad;
    uint16_t* nsp;
    int32_t w, h, pitch, range;
    int32_t nbx, nby, base;     // region grid
    int32_t block, snbx, snby;  // search grid
    int32_t sbase;
    int32_t pad_;
};

// Inference trunk for the n blocks sbase .. sbase + n - 1 of the frame table
// (blocks numbered through the frames' bases): features from the frames, then
// the four layers (layer 2 on tcgen05 with TMEM accumulators, layers 1, 3 and
// 4 on mma.sync; bf16 weights, each activation carried as two bf16 parts),
// writing conv-4 activations a4 ([n][2][2][32] fp32) in one launch (no
// im2col).  w: the four GEMM-layout weights [32][KP[l]]; params:
// canonical parameters (biases at PB[l]); status (nullable) receives bit 1 if
// the bounded wait for the tensor cores gave up.
cudaError_t trunk_tc(const PropFrame* frames, int nframes, long sbase, int n, const __nv_bfloat16* const* w,
                     const float* params, float* a4, unsigned* status, int num_sms, cudaStream_t st);

}  // namespace cnn
}  // namespace me
