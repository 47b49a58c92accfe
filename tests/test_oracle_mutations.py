"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
in a copy of the oracle's C source -- the step-1 centre losing ties, a switching
rule swapped, a pattern point on the wrong axis, the displacement's sign,
revisited points counted, the search window dropped, the full-search tie
key reordered, the evaluation's distance components swapped, the frame
border off by one, DCDS^S's side reversed or its ties sent the other way --
and the pin suite (tests/test_oracle.py: Table VII, the Sec. III-C-1 counts,
the DCDS^S worked examples, brute force, closed forms) must fail on the copy.
The same is done for the network's oracle and for the host reductions of
the Sec. II-C statistics.  An unmodified copy must pass each suite, so the
failures are the mistakes' own."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, anchor, replacement) in me_oracle.c, checked by tests/test_oracle.py
MUTATIONS = [
    ("step-1 centre loses ties", "int k = best_of(&s, cx, cy, &first[1], 6, cval, &bx, &by, &bval);",
     "int k = best_of(&s, cx, cy, &first[1], 6, cval + 1, &bx, &by, &bval);"),
    ("switching strategy two swapped", "if (k <= 2) pat = 1 - pat;", "if (k > 2) pat = 1 - pat;"),
    ("HDSP near points on the wrong axis", "{{0, -1}, {0, 1}, {-2, 0}, {2, 0}},",
     "{{-1, 0}, {1, 0}, {-2, 0}, {2, 0}},"),
    ("switching strategy one on dx", "int pat = (by == cy) ? PAT_H : PAT_V;",
     "int pat = (bx == cx) ? PAT_H : PAT_V;"),
    ("displacement sign", "int b = ref[(long)(by + dy + r) * pitch + (bx + dx + c)];",
     "int b = ref[(long)(by - dy + r) * pitch + (bx - dx + c)];"),
    ("revisits counted", "s->nsp += 1;", "s->nsp += 1; } else { s->nsp += 1;"),
    ("no search window", "return iabs_(dx) <= s->range && iabs_(dy) <= s->range &&", "return 1 &&"),
    ("full-search tie key reordered", "else if (dy != bdy) better = dy < bdy;",
     "else if (dx != bdx) better = dx < bdx;"),
    ("distance components swapped", "double ex = dx - mv_fs[2 * k], ey = dy - mv_fs[2 * k + 1];",
     "double ex = dx - mv_fs[2 * k + 1], ey = dy - mv_fs[2 * k];"),
    ("frame border off by one", "if (bx + dx < 0 || bx + dx > w - block) continue;",
     "if (bx + dx < 0 || bx + dx > w - block - 1) continue;"),
    ("DCDS^S side reversed", "int side = (!hm) ? 1 : (!hp) ? 0 : (vp < vm ? 1 : 0);",
     "int side = (!hm) ? 1 : (!hp) ? 0 : (vp < vm ? 0 : 1);"),
    ("DCDS^S ties to the positive side", "(vp < vm ? 1 : 0)", "(vp <= vm ? 1 : 0)"),
]


# the same for the proposal network's oracle (cnn_oracle.c), checked by
# tests/test_oracle_learned.py (impulse responses, closed forms of the
# features and the loss, finite-difference gradients)
CNN_MUTATIONS = [
    ("kernel taps transposed", "s += wt[((o * cin + c) * 3 + ky) * 3 + kx] * in[(c * hin + y) * hin + x];",
     "s += wt[((o * cin + c) * 3 + kx) * 3 + ky] * in[(c * hin + y) * hin + x];"),
    ("padding dropped in the forward pass",
     "int y = 2 * i + ky - 1, x = 2 * j + kx - 1;\n"
     "                            if (y < 0 || y >= hin || x < 0 || x >= hin) continue;\n"
     "                            s += wt[",
     "int y = 2 * i + ky, x = 2 * j + kx;\n"
     "                            if (y < 0 || y >= hin || x < 0 || x >= hin) continue;\n"
     "                            s += wt["),
    ("layer-3 ReLU dropped", "memcpy(a->a3, a->z3, sizeof a->z3); relu(a->a3, C * 16);",
     "memcpy(a->a3, a->z3, sizeof a->z3);"),
    ("current block scaled wrongly", "v0 = (cur[(long)(py + i - 8) * pitch + (px + j - 8)] - 128.0) / 128.0;",
     "v0 = (cur[(long)(py + i - 8) * pitch + (px + j - 8)] - 128.0) / 256.0;"),
    ("neighbour MV scale", "mvf[2 * k] = mx[k] / 16.0;", "mvf[2 * k] = mx[k] / 8.0;"),
    ("median axes swapped", "mvf[6] = med3(mx[0], mx[1], mx[2]) / 16.0;", "mvf[6] = med3(my[0], my[1], my[2]) / 16.0;"),
    ("top-right neighbour one block too far", "const int nb_dx[3] = {-1, 0, 1}, nb_dy[3] = {0, -1, -1};",
     "const int nb_dx[3] = {-1, 0, 2}, nb_dy[3] = {0, -1, -1};"),
]


# the host reductions of the Sec. II-C statistics (mvp.py), checked by
# tests/test_mvp_stats.py against the paper's printed Fig. 3 and Tables II-III
MVP_MUTATIONS = [
    ("Table II folded transposed", "T[abs(iy - R), abs(ix - R)] += P[iy, ix]", "T[abs(ix - R), abs(iy - R)] += P[iy, ix]"),
    ("axes swapped", '"Ax": P.sum(axis=0), "Ay": P.sum(axis=1)', '"Ax": P.sum(axis=1), "Ay": P.sum(axis=0)'),
    ("diamond too small", "if abs(x) + abs(y) <= 2", "if abs(x) + abs(y) <= 1"),
    ("population deviation", "v.std(ddof=1)", "v.std(ddof=0)"),
    ("HCSP region missing a point", "(-2, 0), (2, 0))),", "(-2, 0))),"),
]


def _run_pins(tmp_path, src_name="oracle/me_oracle.c", suite="tests/test_oracle.py", old=None, new=None):
    for d in ("oracle", "tests", "paper_0806_0689_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build*", "__pycache__", "*.so", "*.o"))
    if old is not None:
        src = tmp_path / src_name
        text = src.read_text()
        assert text.count(old) == 1, "the mutation's anchor must occur exactly once"
        src.write_text(text.replace(old, new))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", suite],
                          cwd=tmp_path, capture_output=True, text=True, timeout=600)


def _caught(r):
    tail = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    return r.returncode == 1 and "failed" in tail  # a failed pin, not a build or collection error


@pytest.mark.parametrize("suite", ["tests/test_oracle.py", "tests/test_oracle_learned.py", "tests/test_mvp_stats.py"])
def test_unmodified_copy_passes(tmp_path, suite):
    r = _run_pins(tmp_path, suite=suite)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(tmp_path, name, old, new):
    r = _run_pins(tmp_path, old=old, new=new)
    assert _caught(r), (name, r.stdout[-2000:], r.stderr[-1000:])


@pytest.mark.parametrize("name,old,new", CNN_MUTATIONS, ids=[m[0] for m in CNN_MUTATIONS])
def test_network_pins_catch_the_mistake(tmp_path, name, old, new):
    r = _run_pins(tmp_path, "oracle/cnn_oracle.c", "tests/test_oracle_learned.py", old, new)
    assert _caught(r), (name, r.stdout[-2000:], r.stderr[-1000:])


@pytest.mark.parametrize("name,old,new", MVP_MUTATIONS, ids=[m[0] for m in MVP_MUTATIONS])
def test_statistics_pins_catch_the_mistake(tmp_path, name, old, new):
    r = _run_pins(tmp_path, "paper_0806_0689_gb300/mvp.py", "tests/test_mvp_stats.py", old, new)
    assert _caught(r), (name, r.stdout[-2000:], r.stderr[-1000:])
