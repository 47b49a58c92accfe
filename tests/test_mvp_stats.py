"""The motion-vector statistics of Sec. II-C (host arithmetic of
paper_0806_0689_gb300.mvp), pinned to the numbers the paper prints: the
central 5x5 distribution of Fig. 3 reproduces the regional probabilities
printed with it, the corner of Table II and the rows Bx, By of Table III; the
rows Ax, Ay of Table III reproduce eq. (1)-(2)."""
import numpy as np
import pytest

from paper_0806_0689_gb300 import mvp

# Fig. 3: the central 5x5 MVP distribution, rows dy = -2..2, columns dx = -2..2
FIG3 = np.array([
    [0.0008, 0.0013, 0.0031, 0.0014, 0.0008],
    [0.0025, 0.0056, 0.0295, 0.0048, 0.0021],
    [0.0151, 0.0718, 0.5805, 0.0562, 0.0440],
    [0.0024, 0.0068, 0.0277, 0.0070, 0.0021],
    [0.0008, 0.0018, 0.0035, 0.0017, 0.0010],
])
# Table III rows Ax, Ay, Bx, By for d = -7..7
AX = [0.0117, 0.0042, 0.0060, 0.0083, 0.0114, 0.0241, 0.0909, 0.6547, 0.0762, 0.0536, 0.0208, 0.0099, 0.0069, 0.0052, 0.0160]
AY = [0.0065, 0.0049, 0.0035, 0.0048, 0.0070, 0.0122, 0.0549, 0.8074, 0.0548, 0.0137, 0.0082, 0.0058, 0.0048, 0.0039, 0.0078]
BX = [0.0042, 0.0013, 0.0028, 0.0037, 0.0049, 0.0151, 0.0718, 0.5805, 0.0562, 0.0440, 0.0121, 0.0035, 0.0026, 0.0013, 0.0034]
BY = [0.0010, 0.0015, 0.0006, 0.0011, 0.0016, 0.0031, 0.0295, 0.5805, 0.0277, 0.0035, 0.0015, 0.0011, 0.0006, 0.0008, 0.0006]
# Table II, top-left 3x3 (rows |dy|, columns |dx|)
TABLE2 = np.array([[0.5805, 0.1280, 0.0591], [0.0572, 0.0242, 0.0092], [0.0067, 0.0062, 0.0034]])


def _embed(R=7):
    P = np.zeros((2 * R + 1, 2 * R + 1))
    P[R - 2:R + 3, R - 2:R + 3] = FIG3
    return P


def test_regions_reproduce_fig3():
    reg = mvp.regions(_embed())
    printed = {"square5": 0.8745, "diamond5": 0.8557, "cross5": 0.8315, "square3": 0.7899, "hcsp": 0.8248}
    for k, v in printed.items():
        assert abs(reg[k] - v) < 3e-4, (k, reg[k], v)  # the printed cells are rounded to 1e-4


def test_fold_and_axes_reproduce_tables_2_and_3():
    P = _embed()
    T = mvp.quarter_table(P)
    assert np.allclose(T[:3, :3], TABLE2, atol=1.5e-4)
    ax = mvp.axes_1d(P)
    R = 7
    assert np.allclose(ax["Bx"][R - 2:R + 3], BX[5:10], atol=1e-9)
    assert np.allclose(ax["By"][R - 2:R + 3], BY[5:10], atol=1e-9)
    # a one-sided mass lands on the right side of each axis
    Q = np.zeros((15, 15)); Q[R + 0, R + 3] = 1.0  # mv = (3, 0)
    a = mvp.axes_1d(Q)
    assert a["Ax"][R + 3] == 1 and a["Ay"][R] == 1 and a["Bx"][R + 3] == 1 and a["By"].sum() == 0


def test_eq12_statistic_reproduces_the_paper():
    mx, sx = mvp.eq12_statistic(AX)
    my, sy = mvp.eq12_statistic(AY)
    # printed: f_x = N(0.06666, 0.20562), f_y = N(0.06668, 0.16492) -- the two deviations exchanged
    assert round(mx, 5) == 0.06666 and round(my, 5) == 0.06668
    assert round(sy, 5) == 0.20562 and round(sx, 5) == 0.16491
    # the distribution's own moments show the horizontal spread
    assert mvp.moments(AX)[1] > mvp.moments(AY)[1]


def test_conditional_tables_normalise():
    R = 2
    side = 5
    counts = np.zeros(35 * side * side, np.int64)
    hist, d1, d2 = mvp.unpack(counts, R)
    d1[mvp.S1.index((2, 0))][R, R + 2] = 6   # global BMP (2, 0)
    d1[mvp.S1.index((2, 0))][R, R + 2 - 1] = 2
    d2[R, R + 2, 14] = 3                      # Q = (2, 0), current BMP (2, 0)
    d2[R, R + 2, 12] = 1                      # current BMP (0, 0)
    t1 = mvp.d1(d1, (2, 0))
    assert t1.sum() == pytest.approx(1.0) and t1[R, R + 2] == pytest.approx(0.75)
    t2 = mvp.d2(d2, R, (2, 0))
    assert t2[2, 4] == pytest.approx(0.75) and t2[2, 2] == pytest.approx(0.25)


def test_oracle_counts_on_a_global_shift():
    """White noise shifted by (2, 0): every interior block's FS vector, its
    current best-matched point in S1 and in S2 are (2, 0), so all counts fall
    in the three cells of that point."""
    import oracle
    from paper_0806_0689_gb300 import synth
    rng = np.random.default_rng(5)
    cur, ref = synth.shifted_pair(rng, 64, 80, 2, 0)
    R = 7
    mv, _, _ = oracle.fs(cur, ref, 16, R)
    c = oracle.mvp_counts([(cur, ref, mv, R)], R)
    hist, d1, d2 = mvp.unpack(c, R)
    nb = mv.shape[0]
    assert hist.sum() == nb
    n = int((mv == (2, 0)).all(axis=1).sum())
    assert n >= nb - 4  # only the right-border column can miss the shift
    assert hist[R, R + 2] == n
    assert d1[mvp.S1.index((2, 0)), R, R + 2] == n
    assert d2[R, R + 2, 14] == n
