"""Pins of the oracle's learned start proposal (not in the paper: parity is
unpinned with respect to the paper; these tests pin the code to mathematics
and to the paper's DCDS it must reduce to)."""
import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import synth

P = 37668
NF = 136  # head inputs: 128 conv features, 6 neighbour MV scalars, their 2 median scalars
# offsets of the parameter tensors in the flat layout
W1, B1 = 0, 576
W2, B2 = 608, 608 + 9216
W3, B3 = B2 + 32, B2 + 32 + 9216
W4, B4 = B3 + 32, B3 + 32 + 9216
FW, FB = B4 + 32, B4 + 32 + 68 * NF


def test_layout():
    assert oracle.cnn_nparams() == P == FB + 68


def _median_h_search(cur, ref, rng, block):
    """The search from the neighbours' median with a horizontal prior: what
    the learned start reduces to when the network proposes the origin."""
    nbx = cur.shape[1] // block

    def propose(m, k0, px, py):
        mx, my = oracle.neighbour_median(m, k0, nbx)
        return 0, 0, 0, mx, my

    return oracle._search_regions(cur, ref, rng, block, propose)


def test_zero_network_reduces_to_the_median_candidate():
    """All logits equal -> the network proposes the origin with a horizontal
    prior, so each block evaluates the origin and the neighbours' median and
    runs DCDS from the better one; on a frame whose neighbours all rest (a
    stationary pair) that is exactly the paper's DCDS."""
    seq = synth.workload_sequence("cif", 2, seed=7, max_motion=16)
    mv, sd, ns, st, _ = oracle.learned_dcds(seq[1], seq[0], 16, np.zeros(P))
    m2, s2, n2, st2 = _median_h_search(seq[1], seq[0], 16, 16)
    assert (st == 0).all() and np.array_equal(st, st2)
    assert np.array_equal(mv, m2) and np.array_equal(sd, s2) and np.array_equal(ns, n2)
    f = seq[0]
    mv, sd, ns, st, _ = oracle.learned_dcds(f, f, 7, np.zeros(P))
    m3, s3, n3 = oracle.dcds(f, f, 16, 7)
    assert np.array_equal(mv, m3) and np.array_equal(sd, s3) and np.array_equal(ns, n3)


def _ideal(mx, my):
    return lambda dx, dy: (dx - mx) ** 2 + (dy - my) ** 2


def test_search_from_closed_forms():
    # start on the true MV: origin + start, then the HCSP around the start: 2 + 6
    assert oracle.search_from(_ideal(5, 3), 7, start=(5, 3)) == (5, 3, 0, 8)
    # a start worse than the origin is evaluated (counted) but not used
    assert oracle.search_from(_ideal(0, 0), 7, start=(4, 4)) == (0, 0, 0, 8)
    # vertical prior: the VCSP contains (0,2); VDSP around it adds 3, middle (0,3) adds 1
    assert oracle.search_from(_ideal(0, 2), 7, prior_v=True) == (0, 2, 0, 11)
    # horizontal MV found by the VCSP's horizontal arm (-1,0)/(1,0) only after moving
    r = oracle.search_from(_ideal(2, 0), 7, prior_v=True)
    assert r[:3] == (2, 0, 0)
    # with the origin start and horizontal prior, the search is the paper's DCDS
    for mx, my in [(3, -2), (-6, 5), (0, 0), (7, 7)]:
        assert oracle.search_from(_ideal(mx, my), 7) == oracle.search(_ideal(mx, my), 7)
    # the extra candidate comes before the start: a right candidate and a
    # wrong start cost one point each, then the HCSP around the candidate
    assert oracle.search_from(_ideal(5, 3), 7, start=(-3, 0), cand=(5, 3)) == (5, 3, 0, 9)
    # equal distortions: the candidate (earlier) keeps the tie
    sym = lambda dx, dy: min((dx - 4) ** 2 + dy ** 2, (dx + 4) ** 2 + dy ** 2)
    assert oracle.search_from(sym, 7, start=(-4, 0), cand=(4, 0))[:2] == (4, 0)
    assert oracle.search_from(sym, 7, start=(4, 0), cand=(-4, 0))[:2] == (-4, 0)
    # a candidate equal to the start is evaluated once
    assert oracle.search_from(_ideal(5, 3), 7, start=(5, 3), cand=(5, 3)) == (5, 3, 0, 8)


def test_start_choice_centre_out():
    # confident heads (one class 30 above the rest): the start is the argmax,
    # clamped to the block's window and frame
    z = np.zeros(68)
    assert oracle.cnn_start(z, 160, 160, 352, 288, 16) == (0, 0, 0)
    z[16 + 3] = 30.0
    z[33 + 16 - 5] = 30.0
    z[67] = 0.5
    assert oracle.cnn_start(z, 160, 160, 352, 288, 16) == (3, -5, 1)
    z3 = np.zeros(68)
    z3[0] = 30.0  # dx = -16 clamped by the frame at the left border
    z3[33 + 16] = 30.0
    assert oracle.cnn_start(z3, 16, 160, 352, 288, 16)[0] == -16
    assert oracle.cnn_start(z3, 0, 160, 352, 288, 16)[0] == 0


def test_start_gate_closed_form():
    """The network's start is kept only when the product of the dx and dy heads'
    softmax maxima reaches 0.6.  One class at logit L and 32 at 0 give a
    maximum of e^L / (e^L + 32); both heads at L = ln 128 give 0.8^2 = 0.64,
    at L = ln 96 0.75^2 = 0.5625.  Ties between two classes split the maximum
    (the tie rule still picks the class nearest the centre)."""
    def heads(L, dx, dy):
        z = np.zeros(68)
        z[16 + dx] = L
        z[33 + 16 + dy] = L
        return z
    z = heads(np.log(128.0), 4, -2)
    assert abs(oracle.start_confidence(z) - 0.64) < 1e-12
    assert oracle.cnn_raw_start(z)[:2] == (4, -2)
    z = heads(np.log(96.0), 4, -2)
    assert abs(oracle.start_confidence(z) - 0.5625) < 1e-12
    assert oracle.cnn_raw_start(z)[:2] == (0, 0)
    # uniform heads: 1/33^2, far below the gate; the prior is still the network's
    z = np.zeros(68)
    z[67] = 1.0
    assert oracle.cnn_raw_start(z) == (0, 0, 1)
    # a two-way tie at a large margin: each maximum 1/2, so 1/4 < 0.6 -> origin
    z = np.zeros(68)
    z[16 - 2] = z[16 + 2] = 40.0
    z[33 + 16] = 40.0
    assert abs(oracle.start_confidence(z) - 0.5) < 1e-12
    assert oracle.cnn_raw_start(z)[:2] == (0, 0)


def test_features_closed_form():
    h, w = 48, 64
    cur = (np.arange(h * w) % 251).astype(np.uint8).reshape(h, w)
    ref = (255 - cur).astype(np.uint8)
    nbr = np.arange(2 * 12, dtype=np.int16).reshape(12, 2)
    x, mvf = oracle.cnn_features(cur, ref, 16, 16, nbr)
    assert x[0, 8, 8] == (int(cur[16, 16]) - 128) / 128 and x[0, 0, 0] == 0.0 and x[0, 23, 23] != 0.0
    assert x[0, 24, 24] == 0.0
    assert x[1, 0, 0] == (int(ref[8, 8]) - 128) / 128
    # left (0,1) -> index 4, top (1,0) -> 1, top-right (2,0) -> 2; then the
    # component-wise medians med(8, 2, 4) = 4 and med(9, 3, 5) = 5; scaled by 1/16
    assert list(mvf) == [8 / 16, 9 / 16, 2 / 16, 3 / 16, 4 / 16, 5 / 16, 4 / 16, 5 / 16]
    x2, mvf2 = oracle.cnn_features(cur, ref, 0, 0, nbr)
    assert x2[1, 0, 0] == (int(ref[0, 0]) - 128) / 128  # clamped corner
    assert list(mvf2) == [0.0] * 8  # no neighbours exist at the top-left block
    # the median counts an absent neighbour as (0,0): the block at (48, 16)
    # has no top-right neighbour; left (2,1) -> index 6, top (3,0) -> 3
    _, mvf3 = oracle.cnn_features(cur, ref, 48, 16, nbr)
    assert list(mvf3) == [12 / 16, 13 / 16, 6 / 16, 7 / 16, 0.0, 0.0, 6 / 16, 7 / 16]


def test_region_features_in_the_8x8_grid():
    """For 8x8 blocks the network sees the 16x16 region, and its neighbour
    scalars are the left, top and top-right 8x8 neighbours of the region's
    top-left block: for the region at (16, 16) in a 64x48 frame (8x8 grid of
    8 x 6 blocks) that is block (2, 2)'s neighbours (1, 2), (2, 1), (3, 1)."""
    h, w = 48, 64
    cur = (np.arange(h * w) % 253).astype(np.uint8).reshape(h, w)
    ref = (cur // 2).astype(np.uint8)
    nbr8 = np.zeros((48, 2), np.int16)
    nbr8[2 * 8 + 1] = (-3, 7)   # left
    nbr8[1 * 8 + 2] = (10, -1)  # top
    nbr8[1 * 8 + 3] = (4, 2)    # top-right
    nbr8[2 * 8 + 3] = (99, 99)  # inside the region: not a neighbour
    x8, mvf = oracle.cnn_features(cur, ref, 16, 16, nbr8, block=8)
    x16, _ = oracle.cnn_features(cur, ref, 16, 16, None, block=16)
    assert np.array_equal(x8, x16)  # the same region pixels
    assert list(mvf) == [-3 / 16, 7 / 16, 10 / 16, -1 / 16, 4 / 16, 2 / 16, 4 / 16, 2 / 16]


def test_uniform_loss():
    x = np.zeros((2, 32, 32))
    loss, g = oracle.cnn_loss_grad(np.zeros(P), x, np.zeros(8), (3, 20, 1))
    assert abs(loss - (2 * np.log(33) + np.log(2))) < 1e-12
    # d loss / d bias of the head = softmax - onehot
    assert abs(g[FB + 3] - (1 / 33 - 1)) < 1e-12 and abs(g[FB + 4] - 1 / 33) < 1e-12
    assert abs(g[FB + 66] - 0.5) < 1e-12 and abs(g[FB + 67] + 0.5) < 1e-12


@pytest.mark.parametrize("tap", [(1, 1), (0, 2), (2, 0)])
def test_conv_impulse_response(tap):
    """Orientation, stride and padding: with one-hot taps the conv chain maps
    an impulse of the current block to a known conv-4 output.

    conv1 uses tap (ky, kx): a1[i][j] = x[2i + ky - 1][2j + kx - 1]; conv2-4
    use the centre tap: a_{l+1}[i][j] = a_l[2i][2j].  So a4[1][1] reads x at
    (16 + ky - 1, 16 + kx - 1)."""
    ky, kx = tap
    p = np.zeros(P)
    p[W1 + (0 * 2 + 0) * 9 + ky * 3 + kx] = 1.0
    for w0 in (W2, W3, W4):
        p[w0 + (0 * 32 + 0) * 9 + 1 * 3 + 1] = 1.0
    feat = 0 * 4 + 1 * 2 + 1  # channel 0, y 1, x 1
    p[FW + 5 * NF + feat] = 1.0
    x = np.zeros((2, 32, 32))
    x[0, 16 + ky - 1, 16 + kx - 1] = 0.75
    lg = oracle.cnn_forward(p, x, np.zeros(8))
    assert lg[5] == 0.75 and np.count_nonzero(lg) == 1
    x2 = np.zeros((2, 32, 32))
    x2[0, 16, 16 + (1 if (ky, kx) != (1, 2) else 2)] = 0.75  # a pixel the tap does not reach
    if (16 + ky - 1, 16 + kx - 1) != (16, 16 + 1):
        assert oracle.cnn_forward(p, x2, np.zeros(8))[5] == 0.0
    # the mv scalars enter after the 128 conv features, the medians last
    p2 = np.zeros(P)
    p2[FW + 7 * NF + 128 + 3] = 2.0
    p2[FW + 9 * NF + 128 + 7] = 3.0
    lg2 = oracle.cnn_forward(p2, x, np.array([0, 0, 0, 0.25, 0, 0, 0, 0.5]))
    assert lg2[7] == 0.5 and lg2[9] == 1.5


def test_gradient_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0.0, 0.1, P)
    for b0 in (B1, B2, B3, B4):
        p[b0:b0 + 32] = np.abs(p[b0:b0 + 32]) + 0.05  # keep units active
    x = rng.uniform(-1, 1, (2, 32, 32))
    mvf = rng.uniform(-1, 1, 8)
    lab = (7, 25, 0)
    loss, g = oracle.cnn_loss_grad(p, x, mvf, lab)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False)
                          for a, b in ((W1, B1), (B1, W2), (W2, B2), (B2, W3), (W3, B3), (W4, B4), (FW, FB), (FB, P))])
    # a small step keeps the perturbation from crossing a ReLU kink (a bias
    # moves every pre-activation of its unit); fp64 rounding of the loss
    # stays near 1e-9 at this step
    h = 1e-7
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.cnn_loss_grad(pp, x, mvf, lab)[0] - oracle.cnn_loss_grad(pm, x, mvf, lab)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


# ---------------------------------------------------------------- neighbour-median start (control)

def test_median_start_closed_forms():
    nbx = 5
    mv = np.zeros((15, 2), np.int16)
    # block 0: no neighbours -> the origin, horizontal prior
    assert oracle.median_start(mv, 0, nbx, 0, 0, 80, 48, 7) == (0, 0, 0)
    # block 6 (bx 1, by 1): left 5, top 1, top-right 2
    mv[5] = (3, 1)
    mv[1] = (5, -2)
    mv[2] = (4, 0)
    assert oracle.median_start(mv, 6, nbx, 16, 16, 80, 48, 7) == (4, 0, 0)
    # vertical prior when |dy| > |dx|
    mv[5], mv[1], mv[2] = (1, 3), (0, 5), (-1, 4)
    assert oracle.median_start(mv, 6, nbx, 16, 16, 80, 48, 7) == (0, 4, 1)
    # clamped by the window and the frame (block at px = 16: dx >= -16)
    mv[5], mv[1], mv[2] = (-20, 0), (-20, 0), (-20, 0)
    assert oracle.median_start(mv, 6, nbx, 16, 16, 80, 48, 32) == (-16, 0, 0)
    assert oracle.median_start(mv, 6, nbx, 16, 16, 80, 48, 7)[0] == -7


def test_median_dcds_on_a_global_shift():
    """White noise shifted by (2, 0), an HCSP point: every block of the first
    row finds it with plain DCDS (its median start is the origin); from the
    second row on the median of the neighbours is the true MV, so an interior
    block evaluates the origin, the start and the 5 HCSP points around the
    start that are new ((0,0) is one of the six), 7 in all, and keeps the start."""
    rng = np.random.default_rng(3)
    cur, ref = synth.shifted_pair(rng, 96, 128, 2, 0)
    mv, sad, nsp, starts = oracle.median_dcds(cur, ref, 7)
    nbx, nby = 8, 6
    m0, s0, n0 = oracle.dcds(cur, ref, 16, 7)
    for bx in range(nbx - 1):
        assert tuple(starts[bx]) == (0, 0, 0)
        assert tuple(mv[bx]) == tuple(m0[bx]) == (2, 0) and nsp[bx] == n0[bx]
    for by in range(1, nby - 1):
        for bx in range(1, nbx - 1):
            k = by * nbx + bx
            assert tuple(starts[k]) == (2, 0, 0)
            assert tuple(mv[k]) == (2, 0) and sad[k] == 0 and nsp[k] == 7


# ---------------------------------------------------------------- 8x8 blocks sharing a region's start

def test_zero_network_reduces_to_the_median_candidate_8x8():
    """All logits equal -> every region proposes (0,0) with a horizontal
    prior, so each of its four 8x8 blocks evaluates the origin and the
    region's neighbour median and runs DCDS from the better one."""
    seq = synth.workload_sequence("cif", 2, seed=17, max_motion=16, scale=(6.0, 3.0))
    mv, sd, ns, st, lg = oracle.learned_dcds(seq[1], seq[0], 16, np.zeros(P), block=8)
    m2, s2, n2, st2 = _median_h_search(seq[1], seq[0], 16, 8)
    assert (st == 0).all() and lg.shape == (396, 68)
    assert np.array_equal(mv, m2) and np.array_equal(sd, s2) and np.array_equal(ns, n2)


def _median_following_head(alpha=4.0):
    """Conv weights zero; the dx logit of class c (displacement d = c - 16) is
    alpha * (16 d * m_x - d^2 / 2) with m_x = median_x / 16 the head's 7th
    scalar, i.e. -alpha / 2 * (d - median_x)^2 up to a per-sample constant:
    its argmax is the median itself for |median| <= 16.  Same for dy; the
    prior logits favour H."""
    p = np.zeros(P)
    for c in range(33):
        d = c - 16
        p[FW + c * NF + 128 + 6] = alpha * 16 * d
        p[FB + c] = -alpha * d * d / 2
        p[FW + (33 + c) * NF + 128 + 7] = alpha * 16 * d
        p[FB + 33 + c] = -alpha * d * d / 2
    p[FB + 66] = 1.0
    return p


@pytest.mark.parametrize("block", [16, 8])
def test_median_following_network_gives_the_median_start(block):
    """A hand-set head that outputs the neighbours' median (and an H prior)
    makes the learned search the search from the median start, computed here
    from the neighbours directly: the median scalars, the argmax and the
    sharing of a region's start by its blocks are wired as stated."""
    seq = synth.workload_sequence("cif", 2, seed=23, max_motion=12, scale=(6.0, 3.0))
    cur, ref = seq[1], seq[0]
    mv, sd, ns, st, _ = oracle.learned_dcds(cur, ref, 16, _median_following_head(), block=block)
    nbx = cur.shape[1] // block

    def propose(m, k0, px, py):
        bx, by = k0 % nbx, k0 // nbx
        cand = [(int(m[ay * nbx + ax][0]), int(m[ay * nbx + ax][1])) if 0 <= ax < nbx and ay >= 0 else (0, 0)
                for ax, ay in ((bx - 1, by), (bx, by - 1), (bx + 1, by - 1))]
        mx, my = sorted(c[0] for c in cand)[1], sorted(c[1] for c in cand)[1]
        return mx, my, 0, mx, my

    m2, s2, n2, st2 = oracle._search_regions(cur, ref, 16, block, propose)
    assert np.array_equal(mv, m2) and np.array_equal(sd, s2) and np.array_equal(ns, n2)
    assert np.array_equal(st, st2)
    assert (st[:, :2] != 0).any()  # the test exercises non-zero starts


def test_median_start_8x8_global_shift_closed_form():
    """White noise shifted by (2, 0): in the first row of regions the median
    of the (partly absent) neighbours is the origin and plain DCDS finds the
    shift; from the second row on the median of the neighbours of every
    region's top-left block is (2, 0), and each of the region's four 8x8
    blocks evaluates the origin, the start and the HCSP around the start
    without the origin (one of its points): 7 points, MV (2, 0), SAD 0 --
    for every block whose HCSP around (2, 0) lies inside the frame (not the
    last block row or column)."""
    rng = np.random.default_rng(5)
    cur, ref = synth.shifted_pair(rng, 96, 128, 2, 0)
    mv, sad, nsp, st = oracle.median_dcds(cur, ref, 7, block=8)
    nbx, nby = 16, 12
    m0, _, n0 = oracle.dcds(cur, ref, 8, 7)
    for bx in range(nbx - 1):
        assert tuple(st[bx]) == (0, 0, 0)  # region row 0, block row 0
        assert tuple(mv[bx]) == (2, 0) and nsp[bx] == n0[bx]
    for by in range(2, nby - 1):
        for bx in range(nbx - 1):
            k = by * nbx + bx
            assert tuple(st[k]) == (2, 0, 0), (bx, by)
            assert tuple(mv[k]) == (2, 0) and sad[k] == 0 and nsp[k] == 7, (bx, by)
