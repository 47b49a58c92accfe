// proposal.cu -- the learned start proposal for DCDS (not in the paper; the
// task adds it): features, training step, inference and the learned-start
// search.
//
// Features of a 16x16 region at (px, py): the current region centred in a
// zero 32x32 canvas, the 32x32 reference patch at the same origin
// (coordinates clamped to the frame), both as (p - 128) / 128; and the final
// MVs of the left, top and top-right blocks of the region's top-left block,
// then their component-wise median, divided by 16 (zero where absent).  With
// 8x8 blocks one proposal serves the region's four blocks.
//
// Training labels come from a motion field (the full-search field computed
// by this library): dx, dy clamped to +-16 (classes 0..32) and H/V = 0 when
// |mvx| >= |mvy|, else 1.  The neighbour scalars use the same field.
//
// Learned-start search: blocks are processed in wavefront order (16x16:
// t = bx + 2 by; 8x8: regions by t = rx + ry, a region's four blocks
// together) so that the left, top and top-right neighbours are final first.  The same kernel
// runs the non-learned control: the start is the component-wise median of the
// three neighbours' MVs (an absent neighbour counts as (0,0)) and the prior is
// vertical when its |dy| > |dx|.  Per block, one
// warp waits for those three (acquire loads, bounded), runs the head on the
// precomputed conv-4 features and the neighbours' MVs, picks the start (argmax
// of the dx and dy heads, ties to the class nearest the centre; the origin
// unless the product of the two heads' softmax maxima is at least 0.6) and the prior
// (V when its logit is larger), and searches: the origin, the neighbours'
// median (learned start only) and the start are evaluated in this order, the
// best one (the earliest on a tie) centres the first pattern (the HCSP, or
// its transpose for a vertical prior), then DCDS steps 2-4.
#include "me.h"
#include "me_cnn.cuh"
#include "me_ctx.h"

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace me::cnn;

struct me_proposal {
    me_ctx* ctx = nullptr;
    float* p = nullptr;  // canonical parameters (device)
    float* g = nullptr;  // gradient
    float* m = nullptr;  // Adam moments
    float* v = nullptr;
    __nv_bfloat16* w[LAYERS] = {nullptr, nullptr, nullptr, nullptr};  // GEMM-layout weights
    int step = 0;
    uint8_t* ws = nullptr;  // workspace
    size_t ws_cap = 0;
    PropFrame* frames = nullptr;  // device frame table
    int frames_cap = 0;
    int* order = nullptr;  // wavefront order
    long order_cap = 0;
    std::vector<int> order_key;  // the (nbx, nby) of every frame the order on the device was built for
};

namespace {

constexpr int kChunk = 8192;  // samples per trunk pass at inference

int fail(me_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(me_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, ME_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int proposal_create(me_ctx* c, me_proposal** out);

// A NULL proposal names the context's own.  Calls that give it weights
// (create = true) make it on first use; the others need it to exist.
int own(me_ctx* c, me_proposal** P, bool create)
{
    if (*P) return ME_OK;
    if (!c->learned) {
        if (!create) return fail(c, ME_ERR_ARG, "the context has no proposal yet (me_proposal_load or _set_params)");
        const int rc = proposal_create(c, &c->learned);
        if (rc != ME_OK) return rc;
    }
    *P = c->learned;
    return ME_OK;
}

// SplitMix64 (Steele, Lea and Flood, 2014): the pair-drawing sequence of me_proposal_train.
uint64_t splitmix64(uint64_t& state)
{
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ int find_frame(const PropFrame* fr, int nframes, long gid)
{
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].base <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int med3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

// The neighbour inputs of block (bx, by) of the search grid: the MVs of its
// left, top and top-right blocks in the frame's neighbour field, then their
// component-wise median, all scaled by 1/16; an absent neighbour (outside the
// frame, or no neighbour field) counts as (0,0).
__device__ __forceinline__ void nbr_scalars(const PropFrame& F, int bx, int by, float* __restrict__ out)
{
    const int nbdx[3] = {-1, 0, 1}, nbdy[3] = {0, -1, -1};
    int mx[3], my[3];
    for (int q = 0; q < 3; ++q) {
        const int ax = bx + nbdx[q], ay = by + nbdy[q];
        mx[q] = my[q] = 0;
        if (F.nbr && ax >= 0 && ax < F.snbx && ay >= 0) {
            const int m = ay * F.snbx + ax;
            mx[q] = F.nbr[2 * m];
            my[q] = F.nbr[2 * m + 1];
        }
        out[2 * q] = mx[q] * (1.f / 16.f);
        out[2 * q + 1] = my[q] * (1.f / 16.f);
    }
    out[6] = med3(mx[0], mx[1], mx[2]) * (1.f / 16.f);
    out[7] = med3(my[0], my[1], my[2]) * (1.f / 16.f);
}

// Inference needs only the neighbour inputs: the fused trunk reads the pixels itself.
__global__ void mvf_kernel(const PropFrame* __restrict__ fr, int nframes, long s0, int n, float* __restrict__ mvf)
{
    for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
        const long gid = s0 + s;
        const PropFrame& F = fr[find_frame(fr, nframes, gid)];
        const int k = (int)(gid - F.base);
        nbr_scalars(F, k % F.nbx, k / F.nbx, mvf + s * NSCAL);
    }
}

// features of samples [s0, s0 + n): x NHWC [n][32][32][2] bf16, mvf [n][NSCAL], labels [n][3]
__global__ void feat_kernel(const PropFrame* __restrict__ fr, int nframes, long s0, int n,
                            __nv_bfloat16* __restrict__ x, float* __restrict__ mvf, int* __restrict__ labels)
{
    const long total = (long)n * 1024;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const long s = idx >> 10;
        const int pix = (int)(idx & 1023), i = pix >> 5, j = pix & 31;
        const long gid = s0 + s;
        const PropFrame& F = fr[find_frame(fr, nframes, gid)];
        const int k = (int)(gid - F.base);
        const int bx = k % F.nbx, by = k / F.nbx;
        const int px = bx * 16, py = by * 16;
        float v0 = 0.f;
        if (i >= 8 && i < 24 && j >= 8 && j < 24)
            v0 = ((float)F.cur[(size_t)(py + i - 8) * F.pitch + (px + j - 8)] - 128.f) * (1.f / 128.f);
        const int yy = min(max(py + i - 8, 0), F.h - 1), xx = min(max(px + j - 8, 0), F.w - 1);
        const float v1 = ((float)F.ref[(size_t)yy * F.pitch + xx] - 128.f) * (1.f / 128.f);
        x[idx * 2] = __float2bfloat16_rn(v0);
        x[idx * 2 + 1] = __float2bfloat16_rn(v1);
        if (pix == 0) {
            nbr_scalars(F, bx, by, mvf + s * NSCAL);
            if (labels) {
                int mx = 0, my = 0;
                if (F.nbr) { mx = F.nbr[2 * k]; my = F.nbr[2 * k + 1]; }
                labels[s * 3] = min(max(mx, -16), 16) + 16;
                labels[s * 3 + 1] = min(max(my, -16), 16) + 16;
                labels[s * 3 + 2] = (abs(mx) >= abs(my)) ? 0 : 1;
            }
        }
    }
}

// ------------------------------------------------------------------ learned-start search

// The wavefront hand-off word of a block: done bit << 32 | its MV.  The waiter
// needs nothing but this word (the MV travels in it, and the blocks' other
// outputs are read only after the kernel), so the flag is written and polled
// with relaxed gpu-scope accesses: no fence on either side of the hand-off.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr uint32_t kSpinLimit = 1u << 22;
constexpr uint32_t kShortSpin = 1u << 12;  // the limit under the failure-detection test hook
// Confidence the learned start needs (product of the dx and dy heads' softmax
// maxima); below it the network proposes the origin.  Chosen among 0.2, 0.4
// and 0.6 on the held-out comparisons with the neighbour-median control.
constexpr float kStartGate = 0.6f;

struct WarpBlock {
    const uint32_t* win;  // the block's reference window, staged in this warp's shared memory
    int ww, rx;           // window words per row; columns left of the block (R rounded up to 4)
    int px, py, dxlo, dxhi, dylo, dyhi, R;
    uint32_t c0, c1;  // this lane's current pixels: 16x16, row lane/2, 8 pixels (half lane%2); 8x8, row
                      // (lane%16)/2, 4 pixels (half lane%2) in c0
};

// Reference-window geometry of a block of B pixels at range R: rows py - R ..
// py + B - 1 + R; words from column px - rx (rx = R rounded up to 4), wide
// enough for the aligned words an unaligned lane segment can touch.
__host__ __device__ inline int win_rx(int R) { return (R + 3) & ~3; }
__host__ __device__ inline int win_words(int R, int B) { return win_rx(R) / 2 + (B == 16 ? 5 : 4); }
__host__ __device__ inline int win_rows(int R, int B) { return B + 2 * R; }

// Stage the window of the block at (px, py) into `win` (the whole warp):
// coalesced word loads, issued together; words outside the frame (never
// read, candidates stay inside the frame) are set to zero.
template <int B>
__device__ __forceinline__ void stage_window(uint32_t* win, const uint8_t* ref, int pitch, int w, int h, int px,
                                             int py, int R, int lane)
{
    const int ww = win_words(R, B), rows = win_rows(R, B), x0 = px - win_rx(R), y0 = py - R;
    for (int i = lane; i < rows * ww; i += 32) {
        const int r = i / ww, c = i - r * ww;
        const int y = y0 + r, x = x0 + 4 * c;
        uint32_t v = 0u;
        if (y >= 0 && y < h && x >= 0 && x + 4 <= w)
            v = __ldg(reinterpret_cast<const uint32_t*>(ref + (size_t)y * pitch + x));
        win[i] = v;
    }
    __syncwarp();
}

// Visit the points (qx[i], qy[i]) of one pattern list: a point outside the
// window/frame or visited before is skipped; the others are marked, counted
// and their SADs computed together (all loads issued before any reduction, so
// the list costs one memory latency).  Returns the mask of evaluated points;
// v[i] holds their SADs in every lane.  16x16: all 32 lanes on each point
// (16 rows x 2 halves of 8 pixels); 8x8: each half-warp on every other point
// (8 rows x 2 halves of 4 pixels).
template <int B, int N>
__device__ __forceinline__ unsigned visit_many(const WarpBlock& b, uint32_t* bm, int& wmin, int& wmax, int& nsp,
                                               const int (&qx)[N], const int (&qy)[N], uint32_t (&v)[N], int lane)
{
    unsigned fresh = 0u;
    if (lane == 0) {
        const int side = 2 * b.R + 1;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (qx[i] < b.dxlo || qx[i] > b.dxhi || qy[i] < b.dylo || qy[i] > b.dyhi) continue;
            const int bit = (qy[i] + b.R) * side + (qx[i] + b.R);
            const uint32_t w = bm[bit >> 5], m = 1u << (bit & 31);
            if (w & m) continue;
            bm[bit >> 5] = w | m;
            wmin = min(wmin, bit >> 5);
            wmax = max(wmax, bit >> 5);
            fresh |= 1u << i;
        }
    }
    fresh = __shfl_sync(0xffffffffu, fresh, 0);
    nsp += __popc(fresh);
    if constexpr (B == 16) {
        const int r = lane >> 1, hh = lane & 1;
        uint32_t w0[N], w1[N], w2[N];
        unsigned sh[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            w0[i] = w1[i] = w2[i] = 0u;
            sh[i] = 0u;
            if ((fresh >> i) & 1u) {
                // byte column of this lane's segment in the window (its alignment equals the frame's)
                const int x = b.rx + qx[i] + 8 * hh;
                const uint32_t* wp = b.win + (qy[i] + b.R + r) * b.ww + (x >> 2);
                sh[i] = (unsigned)(x & 3) * 8u;
                w0[i] = wp[0];
                w1[i] = wp[1];
                if (sh[i]) w2[i] = wp[2];  // inside the staged row whenever the segment is unaligned
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
            uint32_t t = me::sadacc<me::kSadVariant>(__funnelshift_r(w0[i], w1[i], sh[i]), b.c0, 0u);
            v[i] = me::sadacc<me::kSadVariant>(__funnelshift_r(w1[i], w2[i], sh[i]), b.c1, t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    } else {
        constexpr int NS = (N + 1) / 2;  // point slots: half-warp h takes point 2j + h
        const int r = (lane & 15) >> 1, hh = lane & 1, half = lane >> 4;
        uint32_t t[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            const int i = 2 * j + half;
            t[j] = 0u;
            int ox = 0, oy = 0;
            bool use = false;
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k == i) { ox = qx[k]; oy = qy[k]; use = (fresh >> k) & 1u; }
            if (use) {
                const int x = b.rx + ox + 4 * hh;
                const uint32_t* wp = b.win + (oy + b.R + r) * b.ww + (x >> 2);
                const unsigned sh = (unsigned)(x & 3) * 8u;
                const uint32_t lo = wp[0], hi = sh ? wp[1] : 0u;
                t[j] = me::sadacc<me::kSadVariant>(__funnelshift_r(lo, hi, sh), b.c0, 0u);
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < NS; ++j) t[j] += __shfl_xor_sync(0xffffffffu, t[j], o);
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = __shfl_sync(0xffffffffu, t[i / 2], (i & 1) * 16);
    }
    return fresh;
}

// zpart[s][o] = fb[o] + sum over the 128 conv-4 features of fw[o][f] * a4, in
// the head's order (the neighbour terms are added once the neighbours are
// final).  A CTA of 4 x 68 threads stages the weights (transposed) once and
// the features of 32 samples per step; thread (o, q) accumulates output o of
// samples q, q + 4, ..., in the same order as the head kernel.
constexpr int kZS = 32;  // samples per step
__global__ void __launch_bounds__(4 * NLOGIT) zpart_kernel(const float* __restrict__ a4, long total,
                                                           const float* __restrict__ fw,
                                                           const float* __restrict__ fb, float* __restrict__ zpart)
{
    __shared__ float wT[128][NLOGIT];
    __shared__ float af[kZS][129];
    const int tid = threadIdx.x, o = tid % NLOGIT, q = tid / NLOGIT;
    for (int i = tid; i < 128 * NLOGIT; i += blockDim.x) {
        const int oo = i / 128, f = i - oo * 128;
        wT[f][oo] = fw[(size_t)oo * NFEAT + f];
    }
    const float bias = fb[o];
    for (long s0 = (long)blockIdx.x * kZS; s0 < total; s0 += (long)gridDim.x * kZS) {
        __syncthreads();  // wT ready; the previous step's reads of af are done
        for (int i = tid; i < kZS * 128; i += blockDim.x) {
            const int ss = i >> 7, f = i & 127;
            af[ss][f] = (s0 + ss < total) ? a4[(size_t)(s0 + ss) * 128 + (f & 3) * 32 + (f >> 2)] : 0.f;
        }
        __syncthreads();
        float acc[kZS / 4];
#pragma unroll
        for (int k = 0; k < kZS / 4; ++k) acc[k] = bias;
        for (int f = 0; f < 128; ++f) {
            const float w = wT[f][o];
#pragma unroll
            for (int k = 0; k < kZS / 4; ++k) acc[k] += w * af[q + 4 * k][f];
        }
#pragma unroll
        for (int k = 0; k < kZS / 4; ++k) {
            const long ss = s0 + q + 4 * k;
            if (ss < total) zpart[ss * NLOGIT + o] = acc[k];
        }
    }
}

__constant__ int8_t kFirstH[6][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-2, 0}, {2, 0}};  // HCSP
__constant__ int8_t kFirstV[6][2] = {{0, -1}, {0, 1}, {-1, 0}, {1, 0}, {0, -2}, {0, 2}};  // its transpose
__constant__ int8_t kDd[2][4][2] = {{{0, -1}, {0, 1}, {-2, 0}, {2, 0}}, {{-1, 0}, {1, 0}, {0, -2}, {0, 2}}};
__constant__ int8_t kMid[2][2][2] = {{{-1, 0}, {1, 0}}, {{0, -1}, {0, 1}}};

__device__ __forceinline__ int find_search_frame(const PropFrame* fr, int nframes, long gid)
{
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (fr[mid].sbase <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One warp per search block of B pixels, blocks taken in wavefront order.  The
// proposal belongs to the block's 16x16 region (the block itself at 16x16;
// four 8x8 blocks share it): its conv-feature logits (zpart, per region) and
// the final MVs of the left, top and top-right neighbours of the region's
// top-left block.
template <bool LEARNED, int B>
__global__ void __launch_bounds__(256) learned_dcds_kernel(const PropFrame* __restrict__ fr, int nframes,
                                                           const int* __restrict__ order, int total,
                                                           const float* __restrict__ zpart,
                                                           const float* __restrict__ fw,
                                                           unsigned long long* __restrict__ done,
                                                           int* __restrict__ counter,
                                                           int16_t* __restrict__ starts, unsigned* __restrict__ status,
                                                           int max_range, int inject)
{
    // failure-detection test hook: the blocks of the first region in
    // wavefront order never publish their hand-off words, and the waits are
    // shortened
    const uint32_t spin_limit = inject ? kShortSpin : kSpinLimit;
    constexpr int PER = 16 / B;  // blocks per region side
    extern __shared__ uint32_t bm_all[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int side_max = 2 * max_range + 1;
    const int nwb = (side_max * side_max + 31) / 32;
    uint32_t* bm = bm_all + warp * nwb;
    // after the 8 bitmaps: one reference window per warp
    uint32_t* win = bm_all + 8 * nwb + warp * win_rows(max_range, B) * win_words(max_range, B);
    for (int i = lane; i < nwb; i += 32) bm[i] = 0u;
    __syncwarp();
    int wmin = INT_MAX, wmax = -1;
    // learned start: the head's neighbour weights (NSCAL per logit), staged once per CTA
    __shared__ float s_wh[LEARNED ? NLOGIT * NSCAL : 1];
    if (LEARNED) {
        for (int i = threadIdx.x; i < NLOGIT * NSCAL; i += blockDim.x)
            s_wh[i] = __ldg(fw + (size_t)(i / NSCAL) * NFEAT + 128 + i % NSCAL);
        __syncthreads();
    }
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(counter, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        const int gid = order[idx];
        const PropFrame& F = fr[find_search_frame(fr, nframes, gid)];
        const int k = gid - F.sbase;
        const int bx = k % F.snbx, by = k / F.snbx;
        const int rgx = bx / PER, rgy = by / PER;  // the block's region
        const int ax0 = rgx * PER, ay0 = rgy * PER;  // the region's top-left block
        // ---- work that does not depend on the neighbours: the block, the origin's SAD ----
        const int R = F.range, px = bx * B, py = by * B;
        // the window does not depend on the neighbours: its loads overlap the wait below
        stage_window<B>(win, F.ref, F.pitch, F.w, F.h, px, py, R, lane);
        WarpBlock b;
        b.win = win; b.ww = win_words(R, B); b.rx = win_rx(R); b.px = px; b.py = py; b.R = R;
        b.dxlo = max(-R, -px); b.dxhi = min(R, F.w - B - px);
        b.dylo = max(-R, -py); b.dyhi = min(R, F.h - B - py);
        if constexpr (B == 16) {
            const uint32_t* cp = reinterpret_cast<const uint32_t*>(F.cur + (size_t)(py + (lane >> 1)) * F.pitch + px +
                                                                   8 * (lane & 1));
            b.c0 = __ldg(cp);
            b.c1 = __ldg(cp + 1);
        } else {
            b.c0 = __ldg(reinterpret_cast<const uint32_t*>(F.cur + (size_t)(py + ((lane & 15) >> 1)) * F.pitch + px +
                                                           4 * (lane & 1)));
            b.c1 = 0u;
        }
        int nsp = 0;
        uint32_t cval;
        {
            const int qx[1] = {0}, qy[1] = {0};
            uint32_t v[1];
            visit_many<B, 1>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);  // the origin is always a candidate
            cval = v[0];
        }
        float zr[3] = {0.f, 0.f, 0.f};  // this lane's conv-feature logit parts (learned start)
        if (LEARNED) {
            const float* zp = zpart + ((size_t)F.base + (size_t)rgy * F.nbx + rgx) * NLOGIT;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (lane + 32 * j < NLOGIT) zr[j] = __ldg(zp + lane + 32 * j);
        }
        // ---- wait until the region's causal neighbours are final ----
        const int nbdx[3] = {-1, 0, 1}, nbdy[3] = {0, -1, -1};
        int nmx = 0, nmy = 0;  // the neighbour's MV
        bool late = false;
        if (lane < 3) {
            const int ax = ax0 + nbdx[lane], ay = ay0 + nbdy[lane];
            if (ax >= 0 && ax < F.snbx && ay >= 0) {
                const int nk = ay * F.snbx + ax;
                uint32_t it = 0;
                unsigned long long fl;
                // the neighbour publishes its MV with its done bit: one load brings both
                while (((fl = ld_relaxed64(done + F.sbase + nk)) >> 32) == 0ull) {
                    if (++it > spin_limit) { late = true; break; }
                }
                if (!late) {
                    const uint32_t m = (uint32_t)fl;
                    nmx = (int)(int16_t)(m & 0xffffu);
                    nmy = (int)(int16_t)(m >> 16);
                }
            }
        }
        if (__any_sync(0xffffffffu, late) && lane == 0 && status) atomicOr(status, me::STATUS_TIMEOUT);
        int ax3[3], ay3[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ax3[q] = __shfl_sync(0xffffffffu, nmx, q);
            ay3[q] = __shfl_sync(0xffffffffu, nmy, q);
        }
        const int medx = med3(ax3[0], ax3[1], ax3[2]), medy = med3(ay3[0], ay3[1], ay3[2]);
        int sx = 0, sy = 0, pv = 0;
        if constexpr (LEARNED) {
            float mvf[NSCAL];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                mvf[2 * q] = (float)ax3[q] * (1.f / 16.f);
                mvf[2 * q + 1] = (float)ay3[q] * (1.f / 16.f);
            }
            mvf[6] = (float)medx * (1.f / 16.f);
            mvf[7] = (float)medy * (1.f / 16.f);
            // ---- head: the conv-feature part of the logits (zpart, fetched before the
            //      wait) plus the neighbours' terms, in the head's order.  Lane l holds
            //      logits l, l + 32 and l + 64: dx classes 0-31 in its first, dx class 32
            //      (lane 0) and dy classes 0-30 (lanes 1-31) in its second, dy classes 31
            //      and 32 (lanes 0, 1) and the H/V pair (lanes 2, 3) in its third ----
            float z[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float acc = zr[j];
                const int o = min(lane + 32 * j, NLOGIT - 1);  // lanes past the last logit compute a copy, unused
#pragma unroll
                for (int q = 0; q < NSCAL; ++q) acc += s_wh[o * NSCAL + q] * mvf[q];
                z[j] = acc;
            }
            // argmax with ties to the class nearest the centre: 0, -1, +1, -2, +2, ...
            // = the largest logit, then the smallest rank among equal ones
            auto rank = [](int cls) { const int a = cls - 16; return a == 0 ? 0 : (a < 0 ? -2 * a - 1 : 2 * a); };
            auto better = [](float v, int r, float v2, int r2) { return v > v2 || (v == v2 && r < r2); };
            float vx = z[0];
            int cx_ = lane;
            if (lane == 0 && better(z[1], rank(32), vx, rank(cx_))) { vx = z[1]; cx_ = 32; }
            float vy = z[1];  // lanes 1-31: dy class lane - 1; lane 0 replaces it below
            int cy_ = lane - 1;
            if (lane <= 1) {
                const int c2 = 31 + lane;
                if (lane == 0 || better(z[2], rank(c2), vy, rank(cy_))) { vy = z[2]; cy_ = c2; }
            }
            int rx_ = rank(cx_), ry_ = rank(cy_);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float v2 = __shfl_xor_sync(0xffffffffu, vx, o);
                const int c2 = __shfl_xor_sync(0xffffffffu, cx_, o), r2 = __shfl_xor_sync(0xffffffffu, rx_, o);
                if (better(v2, r2, vx, rx_)) { vx = v2; cx_ = c2; rx_ = r2; }
                const float w2 = __shfl_xor_sync(0xffffffffu, vy, o);
                const int d2 = __shfl_xor_sync(0xffffffffu, cy_, o), s2 = __shfl_xor_sync(0xffffffffu, ry_, o);
                if (better(w2, s2, vy, ry_)) { vy = w2; cy_ = d2; ry_ = s2; }
            }
            sx = cx_ - 16;
            sy = cy_ - 16;
            const float zh = __shfl_sync(0xffffffffu, z[2], 2), zv = __shfl_sync(0xffffffffu, z[2], 3);
            pv = zv > zh ? 1 : 0;
            {
                // the network's start only when it is confident: the softmax maxima of
                // the dx and dy heads (1 / sum of exp(z - max)) multiply to kStartGate
                // or more; otherwise the start is the origin (the prior stays)
                float ex = expf(z[0] - vx) + (lane == 0 ? expf(z[1] - vx) : 0.f);
                float ey = (lane >= 1 ? expf(z[1] - vy) : 0.f) + (lane <= 1 ? expf(z[2] - vy) : 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ex += __shfl_xor_sync(0xffffffffu, ex, o);
                    ey += __shfl_xor_sync(0xffffffffu, ey, o);
                }
                if (1.f < kStartGate * ex * ey) { sx = 0; sy = 0; }
            }
        } else {
            // neighbour-median start (absent neighbours count as (0,0))
            sx = medx;
            sy = medy;
            pv = abs(sy) > abs(sx) ? 1 : 0;
        }
        // the region's start, clamped to this block's window and frame
        sx = min(max(sx, b.dxlo), b.dxhi);
        sy = min(max(sy, b.dylo), b.dyhi);
        // ---- search ----
        int cx = 0, cy = 0;
        if (LEARNED) {
            // the neighbours' median (clamped) is evaluated before the network's start
            const int qx[1] = {min(max(medx, b.dxlo), b.dxhi)}, qy[1] = {min(max(medy, b.dylo), b.dyhi)};
            uint32_t v[1];
            const unsigned f = visit_many<B, 1>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);
            if ((f & 1u) && v[0] < cval) { cx = qx[0]; cy = qy[0]; cval = v[0]; }
        }
        {
            // the proposed start (skipped when visited above)
            const int qx[1] = {sx}, qy[1] = {sy};
            uint32_t v[1];
            const unsigned f = visit_many<B, 1>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);
            if ((f & 1u) && v[0] < cval) { cx = sx; cy = sy; cval = v[0]; }
        }
        int bxp = cx, byp = cy;
        uint32_t bsad = cval;
        {
            int qx[6], qy[6];
            uint32_t v[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                qx[i] = cx + (pv ? kFirstV[i][0] : kFirstH[i][0]);
                qy[i] = cy + (pv ? kFirstV[i][1] : kFirstH[i][1]);
            }
            const unsigned f = visit_many<B, 6>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);
#pragma unroll
            for (int i = 0; i < 6; ++i)
                if (((f >> i) & 1u) && v[i] < bsad) { bsad = v[i]; bxp = qx[i]; byp = qy[i]; }
        }
        if (bxp != cx || byp != cy) {
            int pat = (byp == cy) ? 0 : 1;  // switching strategy one
            cx = bxp; cy = byp;
            for (int guard = 0; guard < 4 * side_max * side_max; ++guard) {
                int qx[4], qy[4];
                uint32_t v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) { qx[i] = cx + kDd[pat][i][0]; qy[i] = cy + kDd[pat][i][1]; }
                const unsigned f = visit_many<B, 4>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (((f >> i) & 1u) && v[i] < bsad) { bsad = v[i]; bxp = qx[i]; byp = qy[i]; }
                if (bxp == cx && byp == cy) break;
                if (abs(bxp - cx) + abs(byp - cy) == 1) pat ^= 1;  // switching strategy two
                cx = bxp; cy = byp;
            }
            int qx[2], qy[2];
            uint32_t v[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) { qx[i] = cx + kMid[pat][i][0]; qy[i] = cy + kMid[pat][i][1]; }
            const unsigned f = visit_many<B, 2>(b, bm, wmin, wmax, nsp, qx, qy, v, lane);
#pragma unroll
            for (int i = 0; i < 2; ++i)
                if (((f >> i) & 1u) && v[i] < bsad) { bsad = v[i]; bxp = qx[i]; byp = qy[i]; }
        }
        if (lane == 0) {
            reinterpret_cast<uint32_t*>(F.mv)[k] = (uint32_t)(uint16_t)bxp | ((uint32_t)(uint16_t)byp << 16);
            F.sad[k] = bsad;
            if (F.nsp) F.nsp[k] = (uint16_t)nsp;
            if (starts) {
                starts[(size_t)gid * 3] = (int16_t)sx;
                starts[(size_t)gid * 3 + 1] = (int16_t)sy;
                starts[(size_t)gid * 3 + 2] = (int16_t)pv;
            }
            for (int i = wmin; i <= wmax; ++i) bm[i] = 0u;
            wmin = INT_MAX; wmax = -1;
            if (!(inject && idx < PER * PER))  // the hook withholds the first region's hand-offs
                st_relaxed64(done + gid, (1ull << 32) | ((uint64_t)(uint16_t)byp << 16) | (uint16_t)bxp);
        }
        __syncwarp();
    }
}

inline int nblk(long n, int per = 256, int cap = 4096)
{
    return (int)std::max(1l, std::min((n + per - 1) / per, (long)cap));
}

// ------------------------------------------------------------------ workspace
struct Ws {
    __nv_bfloat16 *x, *cols[LAYERS], *a[LAYERS], *dz, *dzT, *colsT, *wT;
    float *a4f, *mvf, *logits, *dlogits, *da, *dcols, *gw, *part, *bpart;
    int* labels;
    double *loss_sum, *lpart;
};

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

// lay out the workspace for n samples; train adds the backward buffers
size_t ws_layout(uint8_t* base, int n, bool train, Ws* w)
{
    size_t off = 0;
    auto take = [&](size_t bytes) { uint8_t* p = base ? base + off : nullptr; off += al(bytes); return p; };
    const size_t N = (size_t)n;
    const size_t rows_pad0 = (N * 256 + 31) / 32 * 32;
    w->x = (__nv_bfloat16*)take(N * 2048 * 2);
    w->mvf = (float*)take(N * NSCAL * 4);
    w->labels = (int*)take(N * 3 * 4);
    for (int l = 0; l < LAYERS; ++l) {
        // inference runs the fused trunk: no im2col buffers, only the fp32 conv-4 activations
        const size_t ho = HIN[l] / 2;
        w->cols[l] = train ? (__nv_bfloat16*)take(N * ho * ho * KP[l] * 2) : nullptr;
        w->a[l] = train ? (__nv_bfloat16*)take(N * ho * ho * CH * 2) : nullptr;
    }
    w->a4f = train ? nullptr : (float*)take(N * 128 * 4);
    w->logits = (float*)take(N * NLOGIT * 4);
    w->dlogits = (float*)take(N * NLOGIT * 4);
    w->loss_sum = (double*)take(8);
    w->lpart = (double*)take((size_t)kLossCtas * 8 * 8);
    if (train) {
        w->da = (float*)take(N * 8192 * 4);
        w->dz = (__nv_bfloat16*)take(N * 8192 * 2);
        w->dzT = (__nv_bfloat16*)take(CH * rows_pad0 * 2);
        w->colsT = (__nv_bfloat16*)take(std::max(KP[0] * rows_pad0, (size_t)288 * ((N * 64 + 31) / 32 * 32)) * 2);
        w->dcols = (float*)take(N * 64 * 288 * 4);
        w->gw = (float*)take(32 * 288 * 4);
        w->wT = (__nv_bfloat16*)take(288 * 32 * 2);
        w->part = (float*)take((size_t)kMaxSplits * 32 * 288 * 4);
        w->bpart = (float*)take((size_t)kReluBackCtas * 32 * 4);
    }
    return off;
}

int ensure_ws(me_proposal* P, int n, bool train, Ws* w)
{
    const size_t need = ws_layout(nullptr, n, train, w);
    if (P->ws_cap < need) {
        if (P->ws) cudaFree(P->ws);
        P->ws = nullptr;
        P->ws_cap = 0;
        if (cudaMalloc(&P->ws, need) != cudaSuccess) return fail(P->ctx, ME_ERR_NOMEM, "proposal workspace");
        P->ws_cap = need;
    }
    ws_layout(P->ws, n, train, w);
    return ME_OK;
}

// The frame table of a call: the network's 16x16 regions and the search's
// blocks of `block` pixels.  *regions / *blocks receive their totals.
int ensure_frames(me_proposal* P, const me_frame_desc* d, int n, bool labels_from_mv, int block, long* regions,
                  long* blocks)
{
    me_ctx* c = P->ctx;
    if (block != 8 && block != 16) return fail(c, ME_ERR_ARG, "block must be 8 or 16");
    std::vector<PropFrame> t(n);
    long base = 0, sbase = 0;
    for (int i = 0; i < n; ++i) {
        if (!d[i].cur || !d[i].ref || !d[i].mv) return fail(c, ME_ERR_ARG, "cur, ref and mv must not be NULL");
        if (d[i].w <= 0 || d[i].h <= 0 || d[i].w % 16 || d[i].h % 16 || d[i].pitch < d[i].w || d[i].pitch % 16)
            return fail(c, ME_ERR_ARG, "the learned proposal works on 16x16 regions: w, h multiples of 16");
        if (d[i].range < 1 || d[i].range > ME_MAX_RANGE) return fail(c, ME_ERR_ARG, "range must be in 1..32");
        if (((uintptr_t)d[i].cur % 16) || ((uintptr_t)d[i].ref % 16))
            return fail(c, ME_ERR_ARG, "cur/ref must be 16-byte aligned");
        if (((uintptr_t)d[i].mv % 4) || ((uintptr_t)d[i].sad % 4) || ((uintptr_t)d[i].nsp % 2))
            return fail(c, ME_ERR_ARG, "mv/sad must be 4-byte aligned, nsp 2-byte aligned");
        PropFrame f{};
        f.cur = d[i].cur; f.ref = d[i].ref;
        f.nbr = labels_from_mv ? d[i].mv : nullptr;
        f.mv = d[i].mv; f.sad = d[i].sad; f.nsp = d[i].nsp;
        f.w = d[i].w; f.h = d[i].h; f.pitch = d[i].pitch; f.range = d[i].range;
        f.nbx = d[i].w / 16; f.nby = d[i].h / 16;
        f.base = (int)base;
        f.block = block;
        f.snbx = d[i].w / block; f.snby = d[i].h / block;
        f.sbase = (int)sbase;
        base += (long)f.nbx * f.nby;
        sbase += (long)f.snbx * f.snby;
        t[i] = f;
    }
    if (sbase > INT_MAX / 2) return fail(c, ME_ERR_ARG, "too many blocks in one call");
    if (P->frames_cap < n) {
        if (P->frames) cudaFree(P->frames);
        P->frames = nullptr;
        P->frames_cap = 0;
        if (cudaMalloc(&P->frames, sizeof(PropFrame) * n) != cudaSuccess)
            return fail(c, ME_ERR_NOMEM, "proposal frame table");
        P->frames_cap = n;
    }
    cudaError_t e = cudaMemcpy(P->frames, t.data(), sizeof(PropFrame) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "proposal frame table upload");
    *regions = base;
    if (blocks) *blocks = sbase;
    return ME_OK;
}

cudaError_t repack(me_proposal* P, cudaStream_t st)
{
    for (int l = 0; l < LAYERS; ++l) {
        cudaError_t e = pack_weights(P->p + PW[l], CIN[l], KP[l], P->w[l], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// conv trunk + head for n samples whose features are in w->x / w->mvf
cudaError_t forward(me_proposal* P, const Ws& w, int n, bool head, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < LAYERS && e == cudaSuccess; ++l) {
        const __nv_bfloat16* in = l == 0 ? w.x : w.a[l - 1];
        const int ho = HIN[l] / 2;
        e = im2col(in, n, HIN[l], CIN[l], KP[l], w.cols[l], st);
        if (e == cudaSuccess)
            e = gemm(w.cols[l], KP[l], P->w[l], KP[l], nullptr, CH, n * ho * ho, CH, KP[l], 1, GEMM_BIAS_RELU,
                     P->p + PB[l], w.a[l], st);
    }
    if (e == cudaSuccess && head) e = head_fwd(w.a[3], w.mvf, n, P->p + P_FW, P->p + P_FB, w.logits, st);
    return e;
}

// inference: the fused trunk writes the conv-4 activations of blocks
// [s0, s0 + n) to a4 (then the head, whose neighbour scalars are in w.mvf)
cudaError_t forward_infer(me_proposal* P, int nframes, long s0, const Ws& w, int n, float* a4, bool head,
                          cudaStream_t st)
{
    cudaError_t e = trunk_tc(P->frames, nframes, s0, n, P->w, P->p, a4, P->ctx->status, P->ctx->num_sms, st);
    if (e == cudaSuccess && head) e = head_fwd(a4, w.mvf, n, P->p + P_FW, P->p + P_FB, w.logits, st);
    return e;
}

cudaError_t backward(me_proposal* P, const Ws& w, int n, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(P->g, 0, sizeof(float) * NPARAMS, st);
    if (e == cudaSuccess) e = head_bwd(w.dlogits, w.a[3], w.mvf, n, P->p + P_FW, P->g + P_FW, P->g + P_FB, w.da, st);
    for (int l = LAYERS - 1; l >= 0 && e == cudaSuccess; --l) {
        const int ho = HIN[l] / 2;
        const long rows = (long)n * ho * ho;
        const int rows_pad = (int)((rows + 31) / 32 * 32);
        e = relu_back(w.da, w.a[l], rows, w.dz, P->g + PB[l], w.bpart, st);
        if (e == cudaSuccess) e = transpose(w.dz, (int)rows, CH, CH, w.dzT, rows_pad, st);
        if (e == cudaSuccess) e = transpose(w.cols[l], (int)rows, KP[l], KP[l], w.colsT, rows_pad, st);
        if (e == cudaSuccess)
            e = gemm_splitk(w.dzT, rows_pad, w.colsT, rows_pad, w.gw, CH, KP[l], rows_pad,
                            std::max(1, rows_pad / 2048), w.part, st);
        if (e == cudaSuccess) e = unpack_wgrad(w.gw, CIN[l], KP[l], P->g + PW[l], st);
        if (l > 0 && e == cudaSuccess) {
            e = transpose(P->w[l], CH, KP[l], KP[l], w.wT, CH, st);  // W [32][KP] -> [KP][32]
            if (e == cudaSuccess)
                e = gemm(w.dz, CH, w.wT, CH, w.dcols, KP[l], (int)rows, KP[l], CH, 1, GEMM_STORE, nullptr, nullptr, st);
            if (e == cudaSuccess) e = col2im(w.dcols, n, HIN[l], CIN[l], KP[l], w.da, st);
        }
    }
    return e;
}

}  // namespace

extern "C" {

int me_proposal_create(me_ctx* c, me_proposal** out)
{
    if (!c || !out) return ME_ERR_ARG;
    return proposal_create(c, out);
}

}  // extern "C"

namespace {

int proposal_create(me_ctx* c, me_proposal** out)
{
    *out = nullptr;
    me_proposal* P = new me_proposal();
    P->ctx = c;
    bool ok = cudaMalloc(&P->p, sizeof(float) * NPARAMS) == cudaSuccess &&
              cudaMalloc(&P->g, sizeof(float) * NPARAMS) == cudaSuccess &&
              cudaMalloc(&P->m, sizeof(float) * NPARAMS) == cudaSuccess &&
              cudaMalloc(&P->v, sizeof(float) * NPARAMS) == cudaSuccess;
    for (int l = 0; l < LAYERS && ok; ++l) ok = cudaMalloc(&P->w[l], sizeof(__nv_bfloat16) * CH * KP[l]) == cudaSuccess;
    if (ok) ok = cudaMemset(P->p, 0, sizeof(float) * NPARAMS) == cudaSuccess &&
                 cudaMemset(P->m, 0, sizeof(float) * NPARAMS) == cudaSuccess &&
                 cudaMemset(P->v, 0, sizeof(float) * NPARAMS) == cudaSuccess;
    if (ok) ok = repack(P, nullptr) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        me_proposal_free(P);
        return fail(c, ME_ERR_NOMEM, "proposal allocation");
    }
    *out = P;
    return ME_OK;
}

}  // namespace

extern "C" {

void me_proposal_free(me_proposal* P)
{
    if (!P) return;
    cudaFree(P->p); cudaFree(P->g); cudaFree(P->m); cudaFree(P->v);
    for (auto* w : P->w) cudaFree(w);
    cudaFree(P->ws); cudaFree(P->frames); cudaFree(P->order);
    delete P;
}

int me_proposal_set_params(me_ctx* c, me_proposal* P, const float* host)
{
    if (!c || !host) return ME_ERR_ARG;
    const int rc = own(c, &P, true);
    if (rc != ME_OK) return rc;
    cudaError_t e = cudaMemcpy(P->p, host, sizeof(float) * NPARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(P->m, 0, sizeof(float) * NPARAMS);
    if (e == cudaSuccess) e = cudaMemset(P->v, 0, sizeof(float) * NPARAMS);
    if (e == cudaSuccess) e = repack(P, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    P->step = 0;
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "me_proposal_set_params");
}

}  // extern "C"

namespace {

// CRC-32 (the reflected polynomial 0xEDB88320 of IEEE 802.3 / zlib), bitwise.
uint32_t crc32_update(uint32_t crc, const uint8_t* p, size_t n)
{
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

// Checkpoint layout: a 32-byte header, then the parameters and the two Adam
// moment vectors (float32, parameter order, NPARAMS each).
struct CkptHeader {
    char magic[8];       // "MEPROP\0\1"
    uint32_t version;    // 2 (version 1 had 6 neighbour scalars)
    uint32_t nparams;    // ME_PROPOSAL_NPARAMS
    uint32_t nlogits;    // ME_PROPOSAL_NLOGITS
    int32_t step;        // Adam steps taken
    uint32_t crc;        // CRC-32 of the payload
    uint32_t reserved;
};
static_assert(sizeof(CkptHeader) == 32, "checkpoint header layout");
const char kMagic[8] = {'M', 'E', 'P', 'R', 'O', 'P', 0, 1};

}  // namespace

extern "C" {

int me_proposal_save(me_ctx* c, me_proposal* P, const char* path)
{
    if (!c || !path) return ME_ERR_ARG;
    const int rc = own(c, &P, false);
    if (rc != ME_OK) return rc;
    std::vector<float> buf(3 * (size_t)NPARAMS);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(buf.data(), P->p, sizeof(float) * NPARAMS, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + NPARAMS, P->m, sizeof(float) * NPARAMS, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * NPARAMS, P->v, sizeof(float) * NPARAMS, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "me_proposal_save");
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 2;
    h.nparams = NPARAMS;
    h.nlogits = NLOGIT;
    h.step = P->step;
    h.crc = crc32_update(0u, reinterpret_cast<const uint8_t*>(buf.data()), sizeof(float) * buf.size());
    // write a temporary file, then rename it over the target: a crash leaves the old checkpoint whole
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(c, ME_ERR_ARG, "cannot open " + tmp + " for writing");
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(c, ME_ERR_ARG, std::string("cannot write the checkpoint ") + path);
    }
    return ME_OK;
}

int me_proposal_load(me_ctx* c, me_proposal* P, const char* path)
{
    if (!c || !path) return ME_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, ME_ERR_ARG, std::string("cannot open ") + path);
    CkptHeader h{};
    std::vector<float> buf(3 * (size_t)NPARAMS);
    const bool whole = std::fread(&h, sizeof(h), 1, f) == 1 &&
                       std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    const bool trailing = whole && std::fgetc(f) != EOF;
    std::fclose(f);
    if (!whole || trailing) return fail(c, ME_ERR_ARG, "not a proposal checkpoint (wrong size)");
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 2)
        return fail(c, ME_ERR_ARG, "not a proposal checkpoint (magic or version)");
    if (h.nparams != (uint32_t)NPARAMS || h.nlogits != (uint32_t)NLOGIT || h.step < 0)
        return fail(c, ME_ERR_ARG, "checkpoint of a different network shape");
    if (crc32_update(0u, reinterpret_cast<const uint8_t*>(buf.data()), sizeof(float) * buf.size()) != h.crc)
        return fail(c, ME_ERR_ARG, "checkpoint payload damaged (CRC mismatch)");
    const int rc = own(c, &P, true);  // only a valid checkpoint makes the context's proposal
    if (rc != ME_OK) return rc;
    cudaError_t e = cudaMemcpy(P->p, buf.data(), sizeof(float) * NPARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->m, buf.data() + NPARAMS, sizeof(float) * NPARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P->v, buf.data() + 2 * NPARAMS, sizeof(float) * NPARAMS, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = repack(P, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "me_proposal_load");
    P->step = h.step;
    return ME_OK;
}

int me_proposal_get_params(me_ctx* c, me_proposal* P, float* host)
{
    if (!c || !host) return ME_ERR_ARG;
    const int rc = own(c, &P, false);
    if (rc != ME_OK) return rc;
    cudaError_t e = cudaMemcpy(host, P->p, sizeof(float) * NPARAMS, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "me_proposal_get_params");
}

int me_proposal_train_step(me_ctx* c, me_proposal* P, const me_frame_desc* d, int n, float lr, float* loss_out,
                           float* grad_out, void* stream)
{
    if (!c || !d || n <= 0) return ME_ERR_ARG;
    int rc = own(c, &P, true);
    if (rc != ME_OK) return rc;
    long total = 0;
    rc = ensure_frames(P, d, n, true, 16, &total, nullptr);
    if (rc != ME_OK) return rc;
    if (total > 65536) return fail(c, ME_ERR_ARG, "at most 65536 blocks per training step");
    Ws w;
    rc = ensure_ws(P, (int)total, true, &w);
    if (rc != ME_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int ns = (int)total;
    me::Trace trace(c, "me_proposal_train_step", st);
    cudaError_t e = cudaMemsetAsync(w.loss_sum, 0, sizeof(double), st);
    if (e == cudaSuccess) {
        feat_kernel<<<nblk((long)ns * 1024), 256, 0, st>>>(P->frames, n, 0, ns, w.x, w.mvf, w.labels);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = forward(P, w, ns, true, st);
    if (e == cudaSuccess) e = loss(w.logits, w.labels, ns, 1.f / ns, w.dlogits, w.loss_sum, w.lpart, st);
    if (e == cudaSuccess) e = backward(P, w, ns, st);
    if (e == cudaSuccess && lr > 0.f) {
        e = adam(P->p, P->g, P->m, P->v, NPARAMS, lr, ++P->step, st);
        if (e == cudaSuccess) e = repack(P, st);
    }
    double ls = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ls, w.loss_sum, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, P->g, sizeof(float) * NPARAMS, cudaMemcpyDeviceToHost, st);
    trace.close();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "me_proposal_train_step");
    if (loss_out) *loss_out = (float)(ls / ns);
    return ME_OK;
}

int me_proposal_train(me_ctx* c, me_proposal* P, const me_train_cfg* cfg)
{
    if (!c || !cfg) return ME_ERR_ARG;
    if (!cfg->descs || cfg->n <= 0 || cfg->steps < 0 || cfg->pairs_per_step <= 0 || cfg->pairs_per_step > cfg->n ||
        !(cfg->lr > 0.f))
        return fail(c, ME_ERR_ARG, "train config: descs, n > 0, steps >= 0, 1 <= pairs_per_step <= n, lr > 0");
    int rc = own(c, &P, true);
    if (rc != ME_OK) return rc;
    const int n = cfg->n, k = cfg->pairs_per_step;
    std::vector<int> idx(n);
    std::vector<me_frame_desc> sub(k);
    uint64_t state = cfg->seed;
    for (int step = 0; step < cfg->steps; ++step) {
        // k distinct pairs: the first k places of a Fisher-Yates shuffle of 0 .. n-1
        for (int i = 0; i < n; ++i) idx[i] = i;
        for (int j = 0; j < k; ++j) {
            const int r = j + (int)(splitmix64(state) % (uint64_t)(n - j));
            std::swap(idx[j], idx[r]);
            sub[j] = cfg->descs[idx[j]];
        }
        float loss = 0.f;
        rc = me_proposal_train_step(c, P, sub.data(), k, cfg->lr, &loss, nullptr, cfg->stream);
        if (rc != ME_OK) return rc;
        if (cfg->losses) cfg->losses[step] = loss;
    }
    return ME_OK;
}

int me_proposal_logits(me_ctx* c, me_proposal* P, const me_frame_desc* d, float* logits, void* stream)
{
    if (!c || !d || !logits) return ME_ERR_ARG;
    int rc = own(c, &P, false);
    if (rc != ME_OK) return rc;
    long total = 0;
    rc = ensure_frames(P, d, 1, true, 16, &total, nullptr);
    if (rc != ME_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    me::Trace trace(c, "me_proposal_logits", st);
    for (long s0 = 0; s0 < total; s0 += kChunk) {
        const int ns = (int)std::min<long>(kChunk, total - s0);
        Ws w;
        rc = ensure_ws(P, kChunk, false, &w);
        if (rc != ME_OK) return rc;
        mvf_kernel<<<nblk(ns), 256, 0, st>>>(P->frames, 1, s0, ns, w.mvf);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = forward_infer(P, 1, s0, w, ns, w.a4f, true, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(logits + s0 * NLOGIT, w.logits, sizeof(float) * ns * NLOGIT, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "me_proposal_logits");
    }
    // the frame table and workspace are rewritten by the next call on this proposal
    trace.close();
    const cudaError_t e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "me_proposal_logits");
}

}  // extern "C"

namespace {

// The wavefront search over a batch: with a proposal (median = false) the
// CNN proposes the starts; with median = true the neighbour-median does and
// P only lends its buffers.
int wavefront_batch(me_ctx* c, me_proposal* P, const me_frame_desc* d, int n, int block, int16_t* starts,
                    bool median, void* stream)
{
    if (!c || !P || !d || n <= 0) return ME_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!d[i].sad) return fail(c, ME_ERR_ARG, "sad must not be NULL");
    long regions = 0, total = 0;
    int rc = ensure_frames(P, d, n, false, block, &regions, &total);
    if (rc != ME_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    me::Trace trace(c, median ? "me_estimate_median_batch" : "me_estimate_learned_batch", st);
    // buffers after the trunk workspace: conv-4 features and zpart per region,
    // done flags per search block, the counter
    Ws w;
    const size_t trunk = ws_layout(nullptr, kChunk, false, &w);
    const size_t need = al(trunk) + al((size_t)regions * 128 * 4) + al((size_t)total * 8) + 256 +
                        al((size_t)regions * NLOGIT * 4);
    if (P->ws_cap < need) {
        cudaFree(P->ws);
        P->ws = nullptr;
        P->ws_cap = 0;
        if (cudaMalloc(&P->ws, need) != cudaSuccess) return fail(c, ME_ERR_NOMEM, "learned-search workspace");
        P->ws_cap = need;
    }
    ws_layout(P->ws, kChunk, false, &w);
    float* a4all = reinterpret_cast<float*>(P->ws + al(trunk));
    uint8_t* flags = P->ws + al(trunk) + al((size_t)regions * 128 * 4);
    unsigned long long* done = reinterpret_cast<unsigned long long*>(flags);  // per block: done bit << 32 | MV
    int* counter = reinterpret_cast<int*>(flags + al((size_t)total * 8));
    float* zpart = reinterpret_cast<float*>(flags + al((size_t)total * 8) + 256);
    // wavefront order: 16x16 blocks by t = bx + 2 by (left, top and top-right
    // final first); 8x8 blocks by region, t = rx + ry (the neighbours of a
    // region's top-left block lie in its left and top regions), a region's
    // four blocks together; frames interleaved.  It depends only on the
    // frames' grids, so it is kept on the device and rebuilt only when they
    // change.
    std::vector<int> key(2 * (size_t)n + 1);
    key[2 * n] = block;
    for (int i = 0; i < n; ++i) { key[2 * i] = d[i].w / 16; key[2 * i + 1] = d[i].h / 16; }
    cudaError_t e = cudaSuccess;
    if (key != P->order_key || P->order_cap < total) {
        std::vector<int> ord;
        ord.reserve(total);
        std::vector<long> base(n);
        long b0 = 0;
        int tmax = 0;
        const int per = 16 / block;
        for (int i = 0; i < n; ++i) {
            base[i] = b0;
            b0 += (long)key[2 * i] * per * key[2 * i + 1] * per;
            tmax = std::max(tmax, block == 16 ? (key[2 * i] - 1) + 2 * (key[2 * i + 1] - 1)
                                              : (key[2 * i] - 1) + (key[2 * i + 1] - 1));
        }
        for (int tt = 0; tt <= tmax; ++tt)
            for (int i = 0; i < n; ++i) {
                const int rnx = key[2 * i], rny = key[2 * i + 1];
                if (block == 16) {
                    for (int by = 0; by < rny; ++by) {
                        const int bx = tt - 2 * by;
                        if (bx >= 0 && bx < rnx) ord.push_back((int)(base[i] + (long)by * rnx + bx));
                    }
                } else {
                    const int snx = 2 * rnx;
                    for (int ry = 0; ry < rny; ++ry) {
                        const int rx = tt - ry;
                        if (rx < 0 || rx >= rnx) continue;
                        for (int j = 0; j < 2; ++j)
                            for (int ii = 0; ii < 2; ++ii)
                                ord.push_back((int)(base[i] + (long)(2 * ry + j) * snx + 2 * rx + ii));
                    }
                }
            }
        if (P->order_cap < total) {
            cudaFree(P->order);
            P->order = nullptr;
            P->order_cap = 0;
            if (cudaMalloc(&P->order, sizeof(int) * total) != cudaSuccess) return fail(c, ME_ERR_NOMEM, "order table");
            P->order_cap = total;
        }
        P->order_key.clear();  // invalid until the upload below has gone through
        e = cudaMemcpy(P->order, ord.data(), sizeof(int) * total, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) P->order_key = key;
    }
    // the trunk builds the features itself: one launch over every region of the batch
    if (!median && e == cudaSuccess) e = forward_infer(P, n, 0, w, (int)regions, a4all, false, st);
    if (!median && e == cudaSuccess) {
        const int zb = (int)std::max(1l, std::min((regions + kZS - 1) / kZS, (long)c->num_sms * 4));
        zpart_kernel<<<zb, 4 * NLOGIT, 0, st>>>(a4all, regions, P->p + P_FW, P->p + P_FB, zpart);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, al((size_t)total * 8) + 256, st);
    int max_range = 1;
    for (int i = 0; i < n; ++i) max_range = std::max(max_range, d[i].range);
    const int side = 2 * max_range + 1;
    const size_t smem = (size_t)8 * ((side * side + 31) / 32) * 4 +
                        (size_t)8 * win_rows(max_range, block) * win_words(max_range, block) * 4;
    int per_sm = 0;
    auto kern = block == 16 ? (median ? learned_dcds_kernel<false, 16> : learned_dcds_kernel<true, 16>)
                            : (median ? learned_dcds_kernel<false, 8> : learned_dcds_kernel<true, 8>);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (e == cudaSuccess) {
        kern<<<c->num_sms * std::max(1, std::min(per_sm, 4)), 256, smem, st>>>(P->frames, n, P->order, (int)total,
                                                                             median ? nullptr : zpart, P->p + P_FW,
                                                                             done, counter, starts, c->status,
                                                                             max_range, c->inject_wait_timeout);
        e = cudaGetLastError();
    }
    // the host-side tables are reused by the next call: wait for this one
    trace.close();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ME_OK : cuda_fail(c, e, "me_estimate_learned_batch");
}

}  // namespace

extern "C" {

int me_estimate_learned_batch(me_ctx* c, me_proposal* P, const me_frame_desc* d, int n, int block, int16_t* starts,
                              void* stream)
{
    if (!c) return ME_ERR_ARG;
    if (!P) P = c->learned;
    if (!P) return fail(c, ME_ERR_ARG, "learned start: no proposal weights loaded (me_proposal_load)");
    return wavefront_batch(c, P, d, n, block, starts, false, stream);
}

int me_estimate_median_batch(me_ctx* c, const me_frame_desc* d, int n, int block, int16_t* starts, void* stream)
{
    if (!c) return ME_ERR_ARG;
    if (!c->median_ws) {
        int rc = me_proposal_create(c, &c->median_ws);
        if (rc != ME_OK) return rc;
    }
    return wavefront_batch(c, c->median_ws, d, n, block, starts, true, stream);
}

}  // extern "C"
