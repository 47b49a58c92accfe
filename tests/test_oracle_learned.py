"""Pins of the oracle's learned start proposal (not in the paper: parity is
unpinned with respect to the paper; these tests pin the code to mathematics
and to the paper's DCDS it must reduce to)."""
import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import synth

P = 37532
# offsets of the parameter tensors in the flat layout
W1, B1 = 0, 576
W2, B2 = 608, 608 + 9216
W3, B3 = B2 + 32, B2 + 32 + 9216
W4, B4 = B3 + 32, B3 + 32 + 9216
FW, FB = B4 + 32, B4 + 32 + 68 * 134


def test_layout():
    assert oracle.cnn_nparams() == P == FB + 68


def test_zero_network_reduces_to_dcds():
    """All logits equal -> start (0,0), horizontal prior -> the paper's DCDS."""
    seq = synth.workload_sequence("cif", 2, seed=7, max_motion=16)
    mv, sd, ns, st, _ = oracle.learned_dcds(seq[1], seq[0], 16, np.zeros(P))
    m2, s2, n2 = oracle.dcds(seq[1], seq[0], 16, 16)
    assert (st == 0).all()
    assert np.array_equal(mv, m2) and np.array_equal(sd, s2) and np.array_equal(ns, n2)


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


def test_start_choice_centre_out():
    z = np.zeros(68)
    assert oracle.cnn_start(z, 160, 160, 352, 288, 16) == (0, 0, 0)
    z[16 + 3] = 1.0
    z[33 + 16 - 5] = 2.0
    z[67] = 0.5
    assert oracle.cnn_start(z, 160, 160, 352, 288, 16) == (3, -5, 1)
    z2 = np.zeros(68)
    z2[16 - 2] = z2[16 + 2] = 1.0  # tie between -2 and +2 -> -2 (checked first)
    assert oracle.cnn_start(z2, 160, 160, 352, 288, 16)[0] == -2
    z3 = np.zeros(68)
    z3[0] = 1.0  # dx = -16 clamped by the frame at the left border
    assert oracle.cnn_start(z3, 16, 160, 352, 288, 16)[0] == -16
    assert oracle.cnn_start(z3, 0, 160, 352, 288, 16)[0] == 0


def test_features_closed_form():
    h, w = 48, 64
    cur = (np.arange(h * w) % 251).astype(np.uint8).reshape(h, w)
    ref = (255 - cur).astype(np.uint8)
    nbr = np.arange(2 * 12, dtype=np.int16).reshape(12, 2)
    x, mvf = oracle.cnn_features(cur, ref, 16, 16, nbr)
    assert x[0, 8, 8] == (int(cur[16, 16]) - 128) / 128 and x[0, 0, 0] == 0.0 and x[0, 23, 23] != 0.0
    assert x[0, 24, 24] == 0.0
    assert x[1, 0, 0] == (int(ref[8, 8]) - 128) / 128
    # left (0,1) -> index 4, top (1,0) -> 1, top-right (2,0) -> 2; scaled by 1/16
    assert list(mvf) == [8 / 16, 9 / 16, 2 / 16, 3 / 16, 4 / 16, 5 / 16]
    x2, mvf2 = oracle.cnn_features(cur, ref, 0, 0, nbr)
    assert x2[1, 0, 0] == (int(ref[0, 0]) - 128) / 128  # clamped corner
    assert list(mvf2) == [0.0] * 6  # no neighbours exist at the top-left block


def test_uniform_loss():
    x = np.zeros((2, 32, 32))
    loss, g = oracle.cnn_loss_grad(np.zeros(P), x, np.zeros(6), (3, 20, 1))
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
    p[FW + 5 * 134 + feat] = 1.0
    x = np.zeros((2, 32, 32))
    x[0, 16 + ky - 1, 16 + kx - 1] = 0.75
    lg = oracle.cnn_forward(p, x, np.zeros(6))
    assert lg[5] == 0.75 and np.count_nonzero(lg) == 1
    x2 = np.zeros((2, 32, 32))
    x2[0, 16, 16 + (1 if (ky, kx) != (1, 2) else 2)] = 0.75  # a pixel the tap does not reach
    if (16 + ky - 1, 16 + kx - 1) != (16, 16 + 1):
        assert oracle.cnn_forward(p, x2, np.zeros(6))[5] == 0.0
    # the mv scalars enter after the 128 conv features
    p2 = np.zeros(P)
    p2[FW + 7 * 134 + 128 + 3] = 2.0
    assert oracle.cnn_forward(p2, x, np.array([0, 0, 0, 0.25, 0, 0]))[7] == 0.5


def test_gradient_finite_differences():
    rng = np.random.default_rng(3)
    p = rng.normal(0.0, 0.1, P)
    for b0 in (B1, B2, B3, B4):
        p[b0:b0 + 32] = np.abs(p[b0:b0 + 32]) + 0.05  # keep units active
    x = rng.uniform(-1, 1, (2, 32, 32))
    mvf = rng.uniform(-1, 1, 6)
    lab = (7, 25, 0)
    loss, g = oracle.cnn_loss_grad(p, x, mvf, lab)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False)
                          for a, b in ((W1, B1), (B1, W2), (W2, B2), (B2, W3), (W3, B3), (W4, B4), (FW, FB), (FB, P))])
    h = 1e-5
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
