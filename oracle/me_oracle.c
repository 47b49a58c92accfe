/*
 * me_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of what the motion-estimation
 * path computes: full search (FS), the Directional Cross Diamond Search
 * (DCDS) of Jia & Zhang, its simplified variant DCDS^S, and the six
 * evaluation metrics of Sec. IV.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file; the product library
 * never links, includes or calls it, and it shares no code, header, table or
 * constant with the CUDA path.
 *
 * Conventions (the paper is silent on them; each is a stated reading):
 *   - frames are 8-bit luma, row-major, `pitch` bytes per row;
 *   - the block at pixel (bx,by) of `cur` is compared with the block at
 *     (bx+dx, by+dy) of `ref` (the previous original frame, Sec. I);
 *   - a displacement is a candidate only if |dx|<=R, |dy|<=R and the whole
 *     reference block lies inside the frame (no padding);
 *   - SAD is used as the block distortion measure.  The paper uses MAD
 *     (Sec. II-C, Sec. IV); MAD = SAD / N^2, so every argmin is identical.
 *
 * Parity pins (what fixes each function independently of this file) are
 * listed in the test suite.  DCDS^S, for which the paper prints only
 * sequence averages, is pinned by examples worked by hand from Sec. IV-C on
 * the ideal surface of Sec. III-C-2.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Block distortion: SAD of one block (Sec. I: the matching criterion;  */
/* Sec. II-C: MAD over a 16x16 block, here summed instead of averaged). */
/* ------------------------------------------------------------------ */
uint32_t oracle_sad(const uint8_t* cur, const uint8_t* ref, int pitch,
                    int bx, int by, int block, int dx, int dy)
{
    uint32_t s = 0;
    for (int r = 0; r < block; ++r) {
        for (int c = 0; c < block; ++c) {
            int a = cur[(long)(by + r) * pitch + (bx + c)];
            int b = ref[(long)(by + dy + r) * pitch + (bx + dx + c)];
            s += (uint32_t)(a > b ? a - b : b - a);
        }
    }
    return s;
}

static int iabs_(int v) { return v < 0 ? -v : v; }

/* ------------------------------------------------------------------ */
/* Full search (Sec. I; the "true MV" of Sec. II-C and Table IX).       */
/* Every candidate in the window is evaluated; the result is the       */
/* argmin of the key (SAD, |dx|+|dy|, dy, dx) taken lexicographically. */
/* The paper does not say how FS breaks ties; this centre-biased key is */
/* the stated reading.  nsp = number of candidates evaluated.           */
/* ------------------------------------------------------------------ */
static void fs_one(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                   int block, int range, int bx, int by, int16_t* mv2, uint32_t* sad1, uint16_t* nsp1)
{
    int have = 0, bdx = 0, bdy = 0, count = 0;
    uint32_t bs = 0;
    for (int dy = -range; dy <= range; ++dy) {
        for (int dx = -range; dx <= range; ++dx) {
            if (bx + dx < 0 || bx + dx > w - block) continue;
            if (by + dy < 0 || by + dy > h - block) continue;
            ++count;
            uint32_t s = oracle_sad(cur, ref, pitch, bx, by, block, dx, dy);
            int better;
            if (!have) better = 1;
            else if (s != bs) better = s < bs;
            else if (iabs_(dx) + iabs_(dy) != iabs_(bdx) + iabs_(bdy))
                better = iabs_(dx) + iabs_(dy) < iabs_(bdx) + iabs_(bdy);
            else if (dy != bdy) better = dy < bdy;
            else better = dx < bdx;
            if (better) { have = 1; bs = s; bdx = dx; bdy = dy; }
        }
    }
    mv2[0] = (int16_t)bdx;
    mv2[1] = (int16_t)bdy;
    *sad1 = bs;
    if (nsp1) *nsp1 = (uint16_t)count;
}

int oracle_fs_frame(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                    int block, int range, int16_t* mv, uint32_t* sad, uint16_t* nsp)
{
    if (block <= 0 || w % block || h % block || range < 0) return 1;
    int nbx = w / block, nby = h / block;
    for (int j = 0; j < nby; ++j)
        for (int i = 0; i < nbx; ++i) {
            long k = (long)j * nbx + i;
            fs_one(cur, ref, w, h, pitch, block, range, i * block, j * block,
                   mv + 2 * k, sad + k, nsp ? nsp + k : NULL);
        }
    return 0;
}

/* Full search for the listed blocks only (raster indices idx[0..n)); output
 * entry t belongs to block idx[t].  Used to check large frames by sampling. */
int oracle_fs_blocks(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                     int block, int range, const int32_t* idx, int n,
                     int16_t* mv, uint32_t* sad, uint16_t* nsp)
{
    if (block <= 0 || w % block || h % block || range < 0) return 1;
    int nbx = w / block, nb = nbx * (h / block);
    for (int t = 0; t < n; ++t) {
        if (idx[t] < 0 || idx[t] >= nb) return 1;
        fs_one(cur, ref, w, h, pitch, block, range, (idx[t] % nbx) * block, (idx[t] / nbx) * block,
               mv + 2 * (long)t, sad + t, nsp ? nsp + t : NULL);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* DCDS search patterns (Sec. III-A, Fig. 4; the figure is missing from */
/* the text, the shapes below are the reading fixed by Table VI's       */
/* P = 0.8248 for the HCSP and by all 64 DCDS cells of Table VII).      */
/*                                                                      */
/* HCSP: centre, (+-1,0), (+-2,0), (0,+-1): a 5x3 flat cross, 7 points. */
/* HDSP: centre, distant points (+-2,0), near points (0,+-1).           */
/* VDSP: centre, distant points (0,+-2), near points (+-1,0).           */
/* Middle points (on the long wing, distance 1): HDSP (+-1,0),          */
/* VDSP (0,+-1).  They are not part of the pattern and are only checked */
/* in step 4.                                                           */
/* Offsets are listed in evaluation order; with a strict "<" the       */
/* earlier point keeps a tie.  Table VII does not depend on this order  */
/* among non-centre points; it is a stated, fixed choice.               */
/* ------------------------------------------------------------------ */
static const int HCSP_[7][2] = {{0, 0}, {-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-2, 0}, {2, 0}};
enum { PAT_H = 0, PAT_V = 1 };
/* non-centre points of HDSP / VDSP: near first, then distant */
static const int DDSP_[2][4][2] = {
    {{0, -1}, {0, 1}, {-2, 0}, {2, 0}},
    {{-1, 0}, {1, 0}, {0, -2}, {0, 2}},
};
static const int MIDDLE_[2][2][2] = {
    {{-1, 0}, {1, 0}},
    {{0, -1}, {0, 1}},
};

/* Exported so that a test can check the HCSP shape against Table VI. */
void oracle_hcsp_offsets(int* out14)
{
    for (int i = 0; i < 7; ++i) { out14[2 * i] = HCSP_[i][0]; out14[2 * i + 1] = HCSP_[i][1]; }
}

/* Block distortion callback: returns BDM at displacement (dx,dy). */
typedef int64_t (*oracle_bdm_fn)(void* user, int dx, int dy);

typedef struct {
    int range;
    int dx_min, dx_max, dy_min, dy_max;   /* frame limits on the displacement */
    oracle_bdm_fn bdm;
    void* user;
    int side;                              /* 2*range+1 */
    int64_t* value;                        /* memo of evaluated points */
    unsigned char* seen;
    int nsp;                               /* distinct points evaluated */
} search_t;

static int in_window(const search_t* s, int dx, int dy)
{
    return iabs_(dx) <= s->range && iabs_(dy) <= s->range &&
           dx >= s->dx_min && dx <= s->dx_max && dy >= s->dy_min && dy <= s->dy_max;
}

/* Evaluate the BDM at (dx,dy).  Points outside the window or frame are
 * skipped (return 0).  A point evaluated before is looked up, not
 * recomputed and not counted again; the count of distinct points is the
 * NSP of Sec. III-C.  (Readings forced by Table VII.) */
static int eval_point(search_t* s, int dx, int dy, int64_t* out)
{
    if (!in_window(s, dx, dy)) return 0;
    int idx = (dy + s->range) * s->side + (dx + s->range);
    if (!s->seen[idx]) {
        s->value[idx] = s->bdm(s->user, dx, dy);
        s->seen[idx] = 1;
        s->nsp += 1;
    }
    *out = s->value[idx];
    return 1;
}

/* Evaluate the centre-first list {c, c+off[0..n)} and return the index of
 * the current BMP: the first point with the smallest BDM (strict "<", so
 * the centre keeps a tie).  Index 0 means the centre. */
static int best_of(search_t* s, int cx, int cy, const int (*off)[2], int n,
                   int64_t cval, int* bx, int* by, int64_t* bval)
{
    int best = 0;
    *bx = cx; *by = cy; *bval = cval;
    for (int k = 0; k < n; ++k) {
        int64_t v;
        int px = cx + off[k][0], py = cy + off[k][1];
        if (eval_point(s, px, py, &v) && v < *bval) {
            best = k + 1; *bx = px; *by = py; *bval = v;
        }
    }
    return best;
}

/* VCSP: the HCSP transposed (a project extension used only by the learned
 * start when its direction prior says vertical; not in the paper). */
static const int VCSP_[7][2] = {{0, 0}, {0, -1}, {0, 1}, {-1, 0}, {1, 0}, {0, -2}, {0, 2}};

/*
 * One DCDS search over the window of `range` (Sec. III-B, steps 1-4 and the
 * two switching strategies), started from a proposal: the origin, the
 * candidate (ax, ay) and the start point (sx, sy) are evaluated in this
 * order and the best one (the earliest on a tie) becomes the centre of the
 * first pattern, which is the HCSP, or its transpose when prior_v is set; a
 * candidate that repeats an earlier one is neither evaluated nor counted
 * again.  With both at the origin and prior_v = 0 this is exactly the
 * paper's DCDS.  `simplified` selects DCDS^S (Sec. IV-C): the
 * last step checks only the middle point on the side of the better distant
 * point.  Returns the motion vector, its BDM and the NSP in out[0..3]
 * (out[2] is the BDM truncated to 64 bits, out[3] the NSP).
 *
 * DCDS^S reading (the text gives the idea, not the rule): compare the two
 * distant points of the current pattern around the final centre; a point
 * outside the window/frame counts as +infinity; on equal values the
 * negative side is chosen; when both are outside, both middle points are
 * checked as in DCDS.
 */
int oracle_search_from(oracle_bdm_fn bdm, void* user, int range,
                       int dx_min, int dx_max, int dy_min, int dy_max,
                       int ax, int ay, int sx, int sy, int prior_v, int simplified, int64_t* out)
{
    search_t s;
    s.range = range;
    s.dx_min = dx_min; s.dx_max = dx_max; s.dy_min = dy_min; s.dy_max = dy_max;
    s.bdm = bdm; s.user = user;
    s.side = 2 * range + 1;
    s.value = (int64_t*)calloc((size_t)s.side * s.side, sizeof(int64_t));
    s.seen = (unsigned char*)calloc((size_t)s.side * s.side, 1);
    s.nsp = 0;
    if (!s.value || !s.seen) { free(s.value); free(s.seen); return 1; }

    /* Centre of the first pattern: the origin, or a proposed point when it
     * is strictly better than the ones before it. */
    int64_t cval, sval;
    eval_point(&s, 0, 0, &cval);            /* the origin is always a candidate */
    int cx = 0, cy = 0, bx, by;
    if (eval_point(&s, ax, ay, &sval) && sval < cval) {
        cx = ax; cy = ay; cval = sval;
    }
    if (eval_point(&s, sx, sy, &sval) && sval < cval) {
        cx = sx; cy = sy; cval = sval;
    }
    /* Step 1: HCSP (or VCSP) at that centre. */
    int64_t bval;
    const int (*first)[2] = prior_v ? VCSP_ : HCSP_;
    int k = best_of(&s, cx, cy, &first[1], 6, cval, &bx, &by, &bval);
    int mx = cx, my = cy;
    int64_t mval = cval;
    if (k != 0) {
        /* Switching strategy one: a horizontal BMP selects HDSP, else VDSP. */
        int pat = (by == cy) ? PAT_H : PAT_V;
        cx = bx; cy = by; cval = bval;
        /* Steps 2 and 3: re-centre the directional diamond on the BMP until
         * the centre wins.  Each move strictly lowers the BDM, so this ends. */
        for (;;) {
            k = best_of(&s, cx, cy, DDSP_[pat], 4, cval, &bx, &by, &bval);
            if (k == 0) break;
            /* Switching strategy two: a near point (k = 1, 2) swaps the
             * pattern, a distant point (k = 3, 4) keeps it. */
            if (k <= 2) pat = 1 - pat;
            cx = bx; cy = by; cval = bval;
        }
        /* Step 4: centre and the middle points of the current pattern. */
        if (!simplified) {
            best_of(&s, cx, cy, MIDDLE_[pat], 2, cval, &mx, &my, &mval);
        } else {
            int64_t vm = 0, vp = 0;
            const int (*dist)[2] = &DDSP_[pat][2];
            int hm = eval_point(&s, cx + dist[0][0], cy + dist[0][1], &vm);
            int hp = eval_point(&s, cx + dist[1][0], cy + dist[1][1], &vp);
            if (!hm && !hp) {
                best_of(&s, cx, cy, MIDDLE_[pat], 2, cval, &mx, &my, &mval);
            } else {
                int side = (!hm) ? 1 : (!hp) ? 0 : (vp < vm ? 1 : 0);
                best_of(&s, cx, cy, &MIDDLE_[pat][side], 1, cval, &mx, &my, &mval);
            }
        }
    }
    out[0] = mx; out[1] = my; out[2] = mval; out[3] = s.nsp;
    free(s.value); free(s.seen);
    return 0;
}

/* The paper's DCDS: the search above from the origin with the HCSP. */
int oracle_search(oracle_bdm_fn bdm, void* user, int range,
                  int dx_min, int dx_max, int dy_min, int dy_max,
                  int simplified, int64_t* out)
{
    return oracle_search_from(bdm, user, range, dx_min, dx_max, dy_min, dy_max, 0, 0, 0, 0, 0, simplified, out);
}

typedef struct {
    const uint8_t* cur; const uint8_t* ref; int pitch, bx, by, block;
} sad_user_t;

static int64_t sad_cb(void* u, int dx, int dy)
{
    const sad_user_t* p = (const sad_user_t*)u;
    return (int64_t)oracle_sad(p->cur, p->ref, p->pitch, p->bx, p->by, p->block, dx, dy);
}

static int dcds_one(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                    int block, int range, int simplified, int bx, int by,
                    int16_t* mv2, uint32_t* sad1, uint16_t* nsp1)
{
    sad_user_t u = {cur, ref, pitch, bx, by, block};
    int64_t out[4];
    if (oracle_search(sad_cb, &u, range, -bx, w - block - bx, -by, h - block - by, simplified, out))
        return 1;
    mv2[0] = (int16_t)out[0];
    mv2[1] = (int16_t)out[1];
    *sad1 = (uint32_t)out[2];
    if (nsp1) *nsp1 = (uint16_t)out[3];
    return 0;
}

/* DCDS (or DCDS^S) over every block of a frame, SAD as the BDM. */
int oracle_dcds_frame(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                      int block, int range, int simplified,
                      int16_t* mv, uint32_t* sad, uint16_t* nsp)
{
    if (block <= 0 || w % block || h % block || range < 0) return 1;
    int nbx = w / block, nby = h / block;
    for (int j = 0; j < nby; ++j)
        for (int i = 0; i < nbx; ++i) {
            long k = (long)j * nbx + i;
            if (dcds_one(cur, ref, w, h, pitch, block, range, simplified, i * block, j * block,
                         mv + 2 * k, sad + k, nsp ? nsp + k : NULL)) return 1;
        }
    return 0;
}

/* DCDS for the listed blocks only (see oracle_fs_blocks). */
int oracle_dcds_blocks(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                       int block, int range, int simplified, const int32_t* idx, int n,
                       int16_t* mv, uint32_t* sad, uint16_t* nsp)
{
    if (block <= 0 || w % block || h % block || range < 0) return 1;
    int nbx = w / block, nb = nbx * (h / block);
    for (int t = 0; t < n; ++t) {
        if (idx[t] < 0 || idx[t] >= nb) return 1;
        if (dcds_one(cur, ref, w, h, pitch, block, range, simplified, (idx[t] % nbx) * block,
                     (idx[t] / nbx) * block, mv + 2 * (long)t, sad + t, nsp ? nsp + t : NULL)) return 1;
    }
    return 0;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* DCDS of the block at pixel (bx, by) from the candidate (ax, ay) and the
 * start (sx, sy, prior_v), both clamped to the window and the frame.
 * out = mv x, mv y, SAD, NSP. */
int oracle_dcds_block_from(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch, int block,
                           int range, int bx, int by, int ax, int ay, int sx, int sy, int prior_v, int64_t* out)
{
    int lo_x = -bx > -range ? -bx : -range, hi_x = w - block - bx < range ? w - block - bx : range;
    int lo_y = -by > -range ? -by : -range, hi_y = h - block - by < range ? h - block - by : range;
    sad_user_t u = {cur, ref, pitch, bx, by, block};
    return oracle_search_from(sad_cb, &u, range, -bx, w - block - bx, -by, h - block - by,
                              clampi(ax, lo_x, hi_x), clampi(ay, lo_y, hi_y), clampi(sx, lo_x, hi_x),
                              clampi(sy, lo_y, hi_y), prior_v != 0, 0, out);
}

/* DCDS of every block of a frame from per-block starts: starts[3k..3k+2] =
 * (sx, sy, prior_v), cands[2k..2k+1] (NULL: the origin) the candidate
 * evaluated before the start (16x16 or 8x8 blocks; both clamped to the
 * window and the frame). */
int oracle_dcds_from_starts(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                            int block, int range, const int16_t* starts, const int16_t* cands,
                            int16_t* mv, uint32_t* sad, uint16_t* nsp)
{
    if (block <= 0 || w % block || h % block || range < 0) return 1;
    int nbx = w / block, nby = h / block;
    for (int j = 0; j < nby; ++j)
        for (int i = 0; i < nbx; ++i) {
            long k = (long)j * nbx + i;
            int bx = i * block, by = j * block;
            int lo_x = -bx > -range ? -bx : -range, hi_x = w - block - bx < range ? w - block - bx : range;
            int lo_y = -by > -range ? -by : -range, hi_y = h - block - by < range ? h - block - by : range;
            int sx = clampi(starts[3 * k], lo_x, hi_x), sy = clampi(starts[3 * k + 1], lo_y, hi_y);
            int ax = cands ? clampi(cands[2 * k], lo_x, hi_x) : 0;
            int ay = cands ? clampi(cands[2 * k + 1], lo_y, hi_y) : 0;
            sad_user_t u = {cur, ref, pitch, bx, by, block};
            int64_t out[4];
            if (oracle_search_from(sad_cb, &u, range, -bx, w - block - bx, -by, h - block - by,
                                   ax, ay, sx, sy, starts[3 * k + 2] != 0, 0, out)) return 1;
            mv[2 * k] = (int16_t)out[0];
            mv[2 * k + 1] = (int16_t)out[1];
            sad[k] = (uint32_t)out[2];
            if (nsp) nsp[k] = (uint16_t)out[3];
        }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Evaluation (Sec. II-B and Sec. IV list the six measures; Table IX).  */
/* The motion-compensated frame takes each block from `ref` at its MV;  */
/* e = cur - prediction over the whole frame.                           */
/*   out[0] MAD  = sum|e| / (w*h)                                       */
/*   out[1] MSE  = sum e^2 / (w*h)                                      */
/*   out[2] NSP  = mean search points per block (nsp may be NULL -> 0)  */
/*   out[3] PSNR = 10 log10(255^2 / MSE) dB; MSE = 0 gives 100 dB       */
/*   out[4] distance    = mean Euclidean distance to the FS MV          */
/*   out[5] probability = fraction of blocks whose MV equals the FS MV  */
/* mv_fs may be NULL (out[4] = out[5] = 0).                             */
/* ------------------------------------------------------------------ */
int oracle_eval_frame(const uint8_t* cur, const uint8_t* ref, int w, int h, int pitch,
                      int block, const int16_t* mv, const int16_t* mv_fs,
                      const uint16_t* nsp, double* out)
{
    if (block <= 0 || w % block || h % block) return 1;
    int nbx = w / block, nby = h / block;
    long nb = (long)nbx * nby;
    double sum_abs = 0.0, sum_sq = 0.0, sum_nsp = 0.0, sum_dist = 0.0, n_eq = 0.0;
    for (int j = 0; j < nby; ++j) {
        for (int i = 0; i < nbx; ++i) {
            long k = (long)j * nbx + i;
            int dx = mv[2 * k], dy = mv[2 * k + 1];
            for (int r = 0; r < block; ++r) {
                for (int c = 0; c < block; ++c) {
                    int y = j * block + r, x = i * block + c;
                    double e = (double)cur[(long)y * pitch + x] -
                               (double)ref[(long)(y + dy) * pitch + (x + dx)];
                    sum_abs += fabs(e);
                    sum_sq += e * e;
                }
            }
            if (nsp) sum_nsp += nsp[k];
            if (mv_fs) {
                double ex = dx - mv_fs[2 * k], ey = dy - mv_fs[2 * k + 1];
                sum_dist += sqrt(ex * ex + ey * ey);
                if (ex == 0.0 && ey == 0.0) n_eq += 1.0;
            }
        }
    }
    double npix = (double)w * (double)h;
    out[0] = sum_abs / npix;
    out[1] = sum_sq / npix;
    out[2] = sum_nsp / (double)nb;
    out[3] = out[1] > 0.0 ? 10.0 * log10(255.0 * 255.0 / out[1]) : 100.0;
    out[4] = mv_fs ? sum_dist / (double)nb : 0.0;
    out[5] = mv_fs ? n_eq / (double)nb : 0.0;
    return 0;
}
