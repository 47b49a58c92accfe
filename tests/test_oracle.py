"""Pins of the CPU oracle against the paper and against mathematics (no GPU).

Each test fixes the oracle to something other than itself: numbers printed
in the paper (tests/golden/, each with its citation), closed forms, brute
force on tiny frames, and invariants of the method.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


SCALARS = json.load(open(os.path.join(GOLD, "scalars.json")))


def _ideal(mx, my):
    # Sec. III-C-2: distortion = Euclidean distance to the MV; the squared
    # distance orders points identically and stays an integer.
    return lambda dx, dy: (dx - mx) ** 2 + (dy - my) ** 2


# ---------------------------------------------------------------- DCDS pins

@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_table7_all_cells(sx, sy):
    """Table VII (DCDS): NSP at every MV of the +-7 window, every quadrant,
    and the search ends on the true MV (the ideal surface is uni-modal)."""
    t7 = _table("table7_dcds_nsp.txt").astype(int)
    for y in range(8):
        for x in range(8):
            mx, my = sx * x, sy * y
            rx, ry, val, nsp = oracle.search(_ideal(mx, my), 7)
            assert (rx, ry, val) == (mx, my, 0)
            assert nsp == t7[y, x], (mx, my, nsp, t7[y, x])


# DCDS^S (Sec. IV-C) on the ideal surface, worked by hand from the text: the
# last step checks only the middle point on the side of the distant point
# with the smaller distortion; equal distant points take the negative side, a
# distant point outside the window counts as +infinity, and a distant point
# already evaluated is compared without being counted again.
DCDS_S_WORKED = {
    (0, 0): ((0, 0), 7),     # the centre wins the HCSP: step 4 is never reached
    (1, 0): ((1, 0), 10),    # HDSP at (1,0): 3 new; (-1,0) ties (3,0) -> middle (0,0), seen
    (-1, 0): ((-1, 0), 10),  # (-3,0) ties (1,0) -> middle (-2,0), seen in the HCSP
    (0, 1): ((0, 1), 10),    # VDSP at (0,1): 3 new; (0,-1) ties (0,3) -> middle (0,0), seen (DCDS 11)
    (0, -1): ((0, -1), 11),  # (0,-3) ties (0,1) -> middle (0,-2), new
    (2, 0): ((2, 0), 10),    # (0,0) (from the HCSP) ties (4,0) -> middle (1,0), seen (DCDS 11)
    (-2, 0): ((-2, 0), 11),  # (-4,0) ties (0,0) -> middle (-3,0), new
    (3, 0): ((3, 0), 11),    # (2,0) keeps its tie with (4,0); (4,0) is nearer -> middle (3,0), new
    (0, 2): ((0, 2), 11),    # (0,1) keeps its tie with (0,3); (0,3) is nearer -> middle (0,2), new
    (7, 0): ((6, 0), 16),    # edge: (8,0) is outside, so (4,0)'s side is taken and (7,0) is never
                             # checked (DCDS ends on (7,0) with 17)
}


@pytest.mark.parametrize("mv", sorted(DCDS_S_WORKED))
def test_dcds_s_worked_examples(mv):
    want_mv, want_nsp = DCDS_S_WORKED[mv]
    rx, ry, val, nsp = oracle.search(_ideal(*mv), 7, simplified=True)
    assert (rx, ry) == want_mv and nsp == want_nsp
    assert val == (rx - mv[0]) ** 2 + (ry - mv[1]) ** 2


def test_dcds_s_interior_recovery():
    """Sec. IV-C's premise holds exactly on the ideal surface (the middle point
    on the nearer distant point's side is the nearer middle point), so DCDS^S
    ends on every MV strictly inside the window, as DCDS does (Table VII),
    with at most one point fewer; at the window's edge it may stop one short."""
    R = 7
    for my in range(-R, R + 1):
        for mx in range(-R, R + 1):
            s = oracle.search(_ideal(mx, my), R, simplified=True)
            d = oracle.search(_ideal(mx, my), R)
            assert 0 <= d[3] - s[3] <= 1, (mx, my, d, s)
            if abs(mx) < R and abs(my) < R:
                assert s[:3] == (mx, my, 0), (mx, my, s)
            else:
                assert s[2] <= 1, (mx, my, s)


def test_halfway_stop_counts():
    """Sec. III-C-1: 7 points for a zero MV, 10 for (+-1,0), 11 for (0,+-1)."""
    want = SCALARS["halfway_counts"]["value"]
    for (mx, my) in [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)]:
        key = f"{abs(mx)},{abs(my)}"
        assert oracle.search(_ideal(mx, my), 7)[3] == want[key]


def test_table8_distribution2_ansp():
    """Table VIII: DCDS averages 9.7 points over the window with Table II's
    MVP weights (distribution 2)."""
    p = _table("table2_mvp.txt")
    n = np.zeros((8, 8))
    for y in range(8):
        for x in range(8):
            n[y, x] = oracle.search(_ideal(x, y), 7)[3]
    ansp = float((p * n).sum() / p.sum())
    assert abs(ansp - SCALARS["table8_dcds_distribution2"]["value"]) < 0.05


def test_table6_hcsp_shape():
    """Table VI: the HCSP covers P1 = 0.8248 of Table II with 7 points
    (eta1 = 0.1178); a transposed cross or the 9-point CDS cross would not."""
    p = _table("table2_mvp.txt")
    offs = oracle.hcsp_offsets()
    assert offs[0] == (0, 0) and len(set(offs)) == 7
    quarter = {(abs(dx), abs(dy)) for dx, dy in offs}
    p1 = sum(p[y, x] for x, y in quarter)
    assert abs(p1 - SCALARS["table6_hcsp_p1"]["value"]) < 5e-5
    assert abs(p1 / len(offs) - SCALARS["table6_hcsp_eta1"]["value"]) < 5e-5
    # the same table reproduces two other printed pattern sums (sanity of the fixture)
    cross = {(0, 0), (1, 0), (2, 0), (0, 1), (0, 2)}
    assert abs(sum(p[y, x] for x, y in cross) - SCALARS["table6_cds_cross_p1"]["value"]) < 5e-5
    sq = {(0, 0), (1, 0), (0, 1), (1, 1)}
    assert abs(sum(p[y, x] for x, y in sq) - SCALARS["table6_bbgds_square_p1"]["value"]) < 5e-5


def test_window_clipping_counts():
    """Points outside +-R are skipped and not counted (the reading Table VII
    forces): an MV on the window edge never evaluates beyond it."""
    seen = []

    def bdm(dx, dy):
        seen.append((dx, dy))
        return (dx - 7) ** 2 + dy ** 2

    rx, ry, _, nsp = oracle.search(bdm, 7)
    assert (rx, ry) == (7, 0)
    assert all(abs(dx) <= 7 and abs(dy) <= 7 for dx, dy in seen)
    assert len(set(seen)) == len(seen) == nsp == 17


def test_centre_wins_ties():
    """A flat surface stops at the origin after the HCSP (strict '<')."""
    assert oracle.search(lambda dx, dy: 5, 7)[:2] == (0, 0)
    assert oracle.search(lambda dx, dy: 5, 7)[3] == 7


# ---------------------------------------------------------------- frames

def _brute_fs(cur, ref, B, R):
    """Full search written out with numpy: every candidate, min of the key
    (SAD, |dx|+|dy|, dy, dx)."""
    h, w = cur.shape
    res = []
    for j in range(h // B):
        for i in range(w // B):
            blk = cur[j * B:(j + 1) * B, i * B:(i + 1) * B].astype(np.int64)
            cands = []
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    y, x = j * B + dy, i * B + dx
                    if 0 <= x <= w - B and 0 <= y <= h - B:
                        s = int(np.abs(blk - ref[y:y + B, x:x + B].astype(np.int64)).sum())
                        cands.append((s, abs(dx) + abs(dy), dy, dx))
            b = min(cands)
            res.append((b[3], b[2], b[0], len(cands)))
    return np.array(res)


@pytest.mark.parametrize("B,R,h,w", [(8, 2, 32, 48), (8, 3, 24, 40), (16, 4, 48, 32), (16, 7, 32, 64)])
def test_fs_brute_force(B, R, h, w):
    rng = np.random.default_rng(7 + B + R)
    # low-contrast content so that ties in SAD actually occur
    ref = rng.integers(100, 104, size=(h, w), dtype=np.uint8)
    cur = rng.integers(100, 104, size=(h, w), dtype=np.uint8)
    mv, sd, ns = oracle.fs(cur, ref, B, R)
    want = _brute_fs(cur, ref, B, R)
    np.testing.assert_array_equal(mv[:, 0], want[:, 0])
    np.testing.assert_array_equal(mv[:, 1], want[:, 1])
    np.testing.assert_array_equal(sd, want[:, 2])
    np.testing.assert_array_equal(ns, want[:, 3])


def test_fs_tie_key_order():
    """Equal-SAD candidates: the key (SAD, |dx|+|dy|, dy, dx) decides.

    ref(x, y) = g((x + y) mod 4) with g injective and cur(x, y) = ref(x + 2, y):
    the SAD is zero exactly where dx + dy = 2 (mod 4).  Of those, six points
    have |dx|+|dy| = 2; the smallest dy among them is (0, -2)."""
    h, w, B, R = 48, 48, 16, 4
    g = np.array([10, 90, 170, 250], np.uint8)
    yy, xx = np.mgrid[0:h + 8, 0:w + 8]
    big = g[(xx + yy) % 4]
    ref = big[:h, :w].copy()
    cur = big[:h, 2:w + 2].copy()
    mv, sd, _ = oracle.fs(cur, ref, B, R)
    k = 1 * (w // B) + 1            # the interior block
    assert tuple(mv[k]) == (0, -2) and sd[k] == 0


def test_fs_nsp_full_window():
    """Table IX: FS evaluates 225 points per interior 16x16 block at +-7."""
    rng = np.random.default_rng(3)
    f = synth.textured_frame(rng, 64, 64)
    _, _, ns = oracle.fs(f, f, 16, 7)
    nbx = 4
    interior = [j * nbx + i for j in range(1, 3) for i in range(1, 3)]
    assert all(ns[k] == SCALARS["fs_nsp_r7"]["value"] for k in interior)


@pytest.mark.parametrize("sx,sy", [(3, -2), (-5, 4), (7, 7), (0, -6)])
def test_fs_recovers_global_shift(sx, sy):
    rng = np.random.default_rng(11)
    h, w, B, R = 64, 96, 16, 7
    cur, ref = synth.shifted_pair(rng, h, w, sx, sy)
    mv, sd, _ = oracle.fs(cur, ref, B, R)
    for j in range(h // B):
        for i in range(w // B):
            x, y = i * B + sx, j * B + sy
            if 0 <= x <= w - B and 0 <= y <= h - B:
                k = j * (w // B) + i
                assert tuple(mv[k]) == (sx, sy) and sd[k] == 0


# On white noise the true displacement is the unique zero of the SAD
# surface, so DCDS's path is forced and its count has a closed form:
# the shift lies in the HCSP, the pattern chosen by switching strategy one
# adds 3 new points around it, and step 4 adds the middle points not yet
# visited.
@pytest.mark.parametrize("sx,sy,nsp", [(1, 0, 10), (-1, 0, 10), (0, 1, 11), (0, -1, 11),
                                       (2, 0, 11), (-2, 0, 11), (0, 0, 7)])
def test_dcds_shift_in_hcsp(sx, sy, nsp):
    rng = np.random.default_rng(5)
    h, w, B, R = 64, 80, 16, 7
    cur, ref = synth.shifted_pair(rng, h, w, sx, sy)
    mv, sd, ns = oracle.dcds(cur, ref, B, R)
    nbx = w // B
    for j in range(1, h // B - 1):
        for i in range(1, nbx - 1):
            k = j * nbx + i
            assert tuple(mv[k]) == (sx, sy) and sd[k] == 0 and ns[k] == nsp


def test_dcds_stationary_border_classes():
    """cur == ref: every block stops after the HCSP with MV 0; NSP is the
    number of HCSP points whose block stays inside the frame."""
    rng = np.random.default_rng(9)
    h, w, B = 48, 64, 16
    f = synth.textured_frame(rng, h, w)
    mv, sd, ns = oracle.dcds(f, f, B, 7)
    nbx, nby = w // B, h // B
    hcsp = oracle.hcsp_offsets()
    for j in range(nby):
        for i in range(nbx):
            k = j * nbx + i
            want = sum(1 for dx, dy in hcsp
                       if 0 <= i * B + dx <= w - B and 0 <= j * B + dy <= h - B)
            assert tuple(mv[k]) == (0, 0) and sd[k] == 0 and ns[k] == want
    assert ns[0] == 4 and ns[1] == 6 and ns[nbx] == 5 and ns[nbx + 1] == 7


@pytest.mark.parametrize("B,R", [(16, 7), (8, 7), (16, 15)])
def test_dcds_invariants_on_sequence(B, R):
    frames = synth.sequence(176, 144, 4, seed=0, n_objects=3)
    h, w = frames.shape[1:]
    for t in range(1, len(frames)):
        cur, ref = frames[t], frames[t - 1]
        mf, sf, nf = oracle.fs(cur, ref, B, R)
        md, sd, nd = oracle.dcds(cur, ref, B, R)
        ms, ss, nss = oracle.dcds(cur, ref, B, R, simplified=True)
        nbx = w // B
        for k in range(len(sd)):
            bx, by = (k % nbx) * B, (k // nbx) * B
            for m, s in ((md[k], sd[k]), (ms[k], ss[k]), (mf[k], sf[k])):
                assert abs(m[0]) <= R and abs(m[1]) <= R
                assert 0 <= bx + m[0] <= w - B and 0 <= by + m[1] <= h - B
                assert s == oracle.sad(cur, ref, bx, by, B, int(m[0]), int(m[1]))
        assert np.all(sd >= sf) and np.all(ss >= sd)
        assert np.all(nd <= (2 * R + 1) ** 2) and np.all(nd >= 1)
        # DCDS^S takes DCDS's path and drops at most one middle point
        assert np.all((nd - nss >= 0) & (nd - nss <= 1))
        assert np.all(nf == nf.max()) or nf.min() < (2 * R + 1) ** 2


# ---------------------------------------------------------------- evaluation

def test_eval_closed_forms():
    rng = np.random.default_rng(1)
    h, w, B = 32, 32, 16
    ref = rng.integers(10, 240, size=(h, w), dtype=np.uint8)
    cur = (ref.astype(np.int32) + 3).astype(np.uint8)
    mv = np.zeros((4, 2), np.int16)
    fsmv = mv.copy()
    fsmv[2] = (3, 4)
    nsp = np.array([7, 10, 11, 12], np.uint16)
    e = oracle.evaluate(cur, ref, B, mv, fsmv, nsp)
    assert e["mad"] == 3.0 and e["mse"] == 9.0
    assert abs(e["psnr"] - 10 * np.log10(255.0 ** 2 / 9.0)) < 1e-12
    assert e["nsp"] == 10.0
    assert e["distance"] == 5.0 / 4 and e["probability"] == 3.0 / 4
    # distance is per component: MV (1, 0) against FS (0, 3) is sqrt(10) away
    mv2 = np.zeros((4, 2), np.int16)
    mv2[0] = (1, 0)
    fsmv2 = np.zeros((4, 2), np.int16)
    fsmv2[0] = (0, 3)
    e2 = oracle.evaluate(cur, ref, B, mv2, fsmv2)
    assert abs(e2["distance"] - np.sqrt(10.0) / 4) < 1e-15 and e2["probability"] == 0.75


def test_eval_motion_compensation_direction():
    """A frame built block by block from ref at known MVs compensates to
    zero error: the prediction is ref at (x+dx, y+dy)."""
    rng = np.random.default_rng(2)
    h, w, B = 48, 64, 16
    ref = synth.textured_frame(rng, h, w)
    cur = np.zeros_like(ref)
    nbx, nby = w // B, h // B
    mv = np.zeros((nbx * nby, 2), np.int16)
    for j in range(nby):
        for i in range(nbx):
            dx = int(rng.integers(-i * B, w - B - i * B + 1))
            dy = int(rng.integers(-j * B, h - B - j * B + 1))
            dx, dy = max(-7, min(7, dx)), max(-7, min(7, dy))
            mv[j * nbx + i] = (dx, dy)
            cur[j * B:(j + 1) * B, i * B:(i + 1) * B] = ref[j * B + dy:(j + 1) * B + dy,
                                                            i * B + dx:(i + 1) * B + dx]
    e = oracle.evaluate(cur, ref, B, mv)
    assert e["mse"] == 0.0 and e["mad"] == 0.0 and e["psnr"] == 100.0


def test_sequence_generator_is_seeded():
    a = synth.sequence(176, 144, 3, seed=42)
    b = synth.sequence(176, 144, 3, seed=42)
    c = synth.sequence(176, 144, 3, seed=43)
    assert a.dtype == np.uint8 and a.shape == (3, 144, 176)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
