/*
 * cnn_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain fp64 CPU restatement of the learned start proposal that libme adds
 * to DCDS (it is not in the paper; the paper motivates it through the
 * directional conditional MVP distribution, Sec. II-C-2 and Sec. II-D):
 *
 *   features of the 16x16 region at pixel (px, py) (one 16x16 block, or the
 *   four 8x8 blocks that share one proposal):
 *     channel 0: the current region, zero-padded and centred in 32x32
 *                (pixel (i, j) = cur(py + i - 8, px + j - 8) for 8 <= i, j < 24);
 *     channel 1: the co-located 32x32 reference patch, same origin, with
 *                coordinates clamped to the frame;
 *     both scaled as (p - 128) / 128;
 *     6 scalars: the final MVs of the left, top and top-right neighbours of
 *                the region's top-left block (in the grid of the search's
 *                block size) divided by 16, zero where the neighbour does not
 *                exist;
 *     2 scalars: the component-wise median of those three MVs (an absent
 *                neighbour counts as (0,0)) divided by 16;
 *   network: 4 convolutions 3x3, stride 2, padding 1, 32 output channels, ReLU
 *            (32x32x2 -> 16x16x32 -> 8x8x32 -> 4x4x32 -> 2x2x32), then a linear
 *            layer over the 128 conv features (order c, y, x) followed by the
 *            8 scalars, giving 68 logits: dx in [-16, 16] (33), dy in
 *            [-16, 16] (33), and H/V (2);
 *   loss: the sum of three softmax cross-entropies (dx, dy, H/V).
 *
 * Parameter layout (flat): conv1.w [32][2][3][3], conv1.b [32], conv2.w
 * [32][32][3][3], conv2.b [32], conv3.w, conv3.b, conv4.w, conv4.b,
 * fc.w [68][136], fc.b [68]: 37668 values.
 *
 * Parity: "parity unpinned" with respect to the paper (the paper has no
 * network).  The functions are pinned mathematically by the tests: finite
 * differences of the loss, impulse responses of the convolution, closed forms
 * of the head and the loss.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    C = 32,
    NLOGIT = 68,
    NFEAT = 136,
    NSCAL = 8,
    P_W1 = 0, P_B1 = P_W1 + C * 2 * 9,
    P_W2 = P_B1 + C, P_B2 = P_W2 + C * C * 9,
    P_W3 = P_B2 + C, P_B3 = P_W3 + C * C * 9,
    P_W4 = P_B3 + C, P_B4 = P_W4 + C * C * 9,
    P_FW = P_B4 + C, P_FB = P_FW + NLOGIT * NFEAT,
    P_TOTAL = P_FB + NLOGIT
};

int oracle_cnn_nparams(void) { return P_TOTAL; }

static int med3(int a, int b, int c)
{
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return c < lo ? lo : (c > hi ? hi : c);
}

/* Features of the 16x16 region at pixel (px, py). x: [2][32][32]; mvf: [8];
 * nbr: the motion field of the frame in the grid of `block` (8 or 16) pixels
 * ([nb][2] int16, the final MVs of already decided blocks; NULL = none
 * available). */
void oracle_cnn_features(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                         int px, int py, const int16_t* nbr, int block, double* x, double* mvf)
{
    for (int i = 0; i < 32; ++i) {
        for (int j = 0; j < 32; ++j) {
            double v0 = 0.0;
            if (i >= 8 && i < 24 && j >= 8 && j < 24)
                v0 = (cur[(long)(py + i - 8) * pitch + (px + j - 8)] - 128.0) / 128.0;
            int yy = py + i - 8, xx = px + j - 8;
            yy = yy < 0 ? 0 : (yy > h - 1 ? h - 1 : yy);
            xx = xx < 0 ? 0 : (xx > w - 1 ? w - 1 : xx);
            x[i * 32 + j] = v0;
            x[1024 + i * 32 + j] = (ref[(long)yy * pitch + xx] - 128.0) / 128.0;
        }
    }
    int nbx = w / block, bx = px / block, by = py / block;
    const int nb_dx[3] = {-1, 0, 1}, nb_dy[3] = {0, -1, -1};
    int mx[3], my[3];
    for (int k = 0; k < 3; ++k) {
        int ax = bx + nb_dx[k], ay = by + nb_dy[k];
        mx[k] = my[k] = 0;
        if (nbr && ax >= 0 && ax < nbx && ay >= 0) {
            mx[k] = nbr[2 * ((long)ay * nbx + ax)];
            my[k] = nbr[2 * ((long)ay * nbx + ax) + 1];
        }
        mvf[2 * k] = mx[k] / 16.0;
        mvf[2 * k + 1] = my[k] / 16.0;
    }
    mvf[6] = med3(mx[0], mx[1], mx[2]) / 16.0;
    mvf[7] = med3(my[0], my[1], my[2]) / 16.0;
}

/* 3x3 convolution, stride 2, padding 1: in [cin][hin][hin] -> out [C][hin/2][hin/2]. */
static void conv_fwd(const double* in, int cin, int hin, const double* wt, const double* b, double* out)
{
    int ho = hin / 2;
    for (int o = 0; o < C; ++o)
        for (int i = 0; i < ho; ++i)
            for (int j = 0; j < ho; ++j) {
                double s = b[o];
                for (int c = 0; c < cin; ++c)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int y = 2 * i + ky - 1, x = 2 * j + kx - 1;
                            if (y < 0 || y >= hin || x < 0 || x >= hin) continue;
                            s += wt[((o * cin + c) * 3 + ky) * 3 + kx] * in[(c * hin + y) * hin + x];
                        }
                out[(o * ho + i) * ho + j] = s;
            }
}

static void relu(double* v, int n)
{
    for (int i = 0; i < n; ++i) v[i] = v[i] > 0.0 ? v[i] : 0.0;
}

typedef struct {
    double z1[C * 256], a1[C * 256];
    double z2[C * 64], a2[C * 64];
    double z3[C * 16], a3[C * 16];
    double z4[C * 4], a4[C * 4];
    double f[NFEAT];
    double logits[NLOGIT];
} acts_t;

static void forward(const double* p, const double* x, const double* mvf, acts_t* a)
{
    conv_fwd(x, 2, 32, p + P_W1, p + P_B1, a->z1);
    memcpy(a->a1, a->z1, sizeof a->z1); relu(a->a1, C * 256);
    conv_fwd(a->a1, C, 16, p + P_W2, p + P_B2, a->z2);
    memcpy(a->a2, a->z2, sizeof a->z2); relu(a->a2, C * 64);
    conv_fwd(a->a2, C, 8, p + P_W3, p + P_B3, a->z3);
    memcpy(a->a3, a->z3, sizeof a->z3); relu(a->a3, C * 16);
    conv_fwd(a->a3, C, 4, p + P_W4, p + P_B4, a->z4);
    memcpy(a->a4, a->z4, sizeof a->z4); relu(a->a4, C * 4);
    for (int i = 0; i < 128; ++i) a->f[i] = a->a4[i];
    for (int i = 0; i < NSCAL; ++i) a->f[128 + i] = mvf[i];
    for (int o = 0; o < NLOGIT; ++o) {
        double s = p[P_FB + o];
        for (int i = 0; i < NFEAT; ++i) s += p[P_FW + o * NFEAT + i] * a->f[i];
        a->logits[o] = s;
    }
}

/* Logits of one block. */
void oracle_cnn_forward(const double* params, const double* x, const double* mvf, double* logits)
{
    acts_t* a = (acts_t*)malloc(sizeof(acts_t));
    forward(params, x, mvf, a);
    memcpy(logits, a->logits, sizeof a->logits);
    free(a);
}

/* softmax cross-entropy of logits[0..n) against class t; writes d/dlogit */
static double xent(const double* z, int n, int t, double* dz)
{
    double m = z[0];
    for (int i = 1; i < n; ++i) m = z[i] > m ? z[i] : m;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(z[i] - m);
    for (int i = 0; i < n; ++i) dz[i] = exp(z[i] - m) / s;
    dz[t] -= 1.0;
    return log(s) + m - z[t];
}

/* backward of conv_fwd: accumulates dw, db, and writes din (may be NULL) */
static void conv_bwd(const double* in, int cin, int hin, const double* wt, const double* dout,
                     double* dw, double* db, double* din)
{
    int ho = hin / 2;
    if (din) memset(din, 0, sizeof(double) * cin * hin * hin);
    for (int o = 0; o < C; ++o)
        for (int i = 0; i < ho; ++i)
            for (int j = 0; j < ho; ++j) {
                double g = dout[(o * ho + i) * ho + j];
                db[o] += g;
                for (int c = 0; c < cin; ++c)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int y = 2 * i + ky - 1, x = 2 * j + kx - 1;
                            if (y < 0 || y >= hin || x < 0 || x >= hin) continue;
                            dw[((o * cin + c) * 3 + ky) * 3 + kx] += g * in[(c * hin + y) * hin + x];
                            if (din) din[(c * hin + y) * hin + x] += g * wt[((o * cin + c) * 3 + ky) * 3 + kx];
                        }
            }
}

/* Loss of one block with labels (tdx, tdy in 0..32, thv in 0..1); adds the
 * gradient of the loss with respect to every parameter into grad. */
double oracle_cnn_loss_grad(const double* p, const double* x, const double* mvf, int tdx, int tdy, int thv,
                            double* grad)
{
    acts_t* a = (acts_t*)malloc(sizeof(acts_t));
    forward(p, x, mvf, a);
    double dz[NLOGIT];
    double loss = xent(a->logits, 33, tdx, dz) + xent(a->logits + 33, 33, tdy, dz + 33) +
                  xent(a->logits + 66, 2, thv, dz + 66);
    double df[NFEAT];
    memset(df, 0, sizeof df);
    for (int o = 0; o < NLOGIT; ++o) {
        grad[P_FB + o] += dz[o];
        for (int i = 0; i < NFEAT; ++i) {
            grad[P_FW + o * NFEAT + i] += dz[o] * a->f[i];
            df[i] += dz[o] * p[P_FW + o * NFEAT + i];
        }
    }
    double* d4 = (double*)malloc(sizeof(double) * C * 4);
    double* d3 = (double*)malloc(sizeof(double) * C * 16);
    double* d2 = (double*)malloc(sizeof(double) * C * 64);
    double* d1 = (double*)malloc(sizeof(double) * C * 256);
    for (int i = 0; i < 128; ++i) d4[i] = a->z4[i] > 0.0 ? df[i] : 0.0;
    conv_bwd(a->a3, C, 4, p + P_W4, d4, grad + P_W4, grad + P_B4, d3);
    for (int i = 0; i < C * 16; ++i) d3[i] = a->z3[i] > 0.0 ? d3[i] : 0.0;
    conv_bwd(a->a2, C, 8, p + P_W3, d3, grad + P_W3, grad + P_B3, d2);
    for (int i = 0; i < C * 64; ++i) d2[i] = a->z2[i] > 0.0 ? d2[i] : 0.0;
    conv_bwd(a->a1, C, 16, p + P_W2, d2, grad + P_W2, grad + P_B2, d1);
    for (int i = 0; i < C * 256; ++i) d1[i] = a->z1[i] > 0.0 ? d1[i] : 0.0;
    conv_bwd(x, 2, 32, p + P_W1, d1, grad + P_W1, grad + P_B1, NULL);
    free(d4); free(d3); free(d2); free(d1); free(a);
    return loss;
}
