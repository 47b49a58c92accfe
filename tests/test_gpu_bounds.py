"""The bounds-check build (ME_LIB_VARIANT=check: the DCDS tile kernel checks
every shared-memory read of a staged tile against its window or current-tile
region and every ring and bitmap index, recording a violation instead of
making it).  Run in a child process over frame sizes with partial tiles,
block sizes 8 and 16, ranges 1 to 32, DCDS and DCDS^S, one and two stages,
128 and 256 threads (8x8 blocks at +-32 with 256 threads and one stage run
the visited-box variant), with and without the fused evaluation, and smooth
shifted content whose long search paths reach the window's edges and the
8x8 overflow pass: no check may fire, and every field stays bit-exact with
the oracle (Sec. III-B, IV-C)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys, tempfile
sys.path.insert(0, os.environ["ROOT"])
import numpy as np, torch
import oracle
from paper_0806_0689_gb300 import me, synth, build
assert me.lib_path() == build.paths("check")[1]
cases = []
for name, n, seed in (("qcif", 3, 7001), ("cif", 3, 7002), ("720p", 2, 7003)):
    s = synth.workload_sequence(name, n, seed=seed, max_motion=16)
    cases += [(s[t + 1], s[t]) for t in range(n - 1)]
# smooth content shifted far: long diamond paths, up to the window's edges
# (and, for 8x8 blocks, past the visited box into the overflow pass)
for (h, w, sx, sy) in ((128, 176, 13, -9), (96, 256, -17, 6)):
    yy, xx = np.mgrid[0:h + 96, 0:w + 96].astype(np.float64)
    big = 128 + 60 * np.sin(xx / 17.0) * np.cos(yy / 13.0) + 40 * np.sin((xx + 2 * yy) / 29.0)
    big = np.clip(np.rint(big), 0, 255).astype(np.uint8)
    cases.append((big[48 + sy:48 + sy + h, 48 + sx:48 + sx + w].copy(), big[48:48 + h, 48:48 + w].copy()))
runs = 0
for shape in ("8 8 128 0 1", "8 8 256 0 2", "8 8 256 0 1"):
    for B in ((16, 8) if shape != "8 8 256 0 1" else (8,)):
        for algo in ("dcds", "dcds_s"):
            for R in (1, 7, 16, 32):
                fd, path = tempfile.mkstemp(suffix=".txt")
                lines = "".join(f"{me.ALGOS[algo]} {B} {R} {c.shape[1]}x{c.shape[0]} {shape}\n" for c, _ in cases)
                os.write(fd, lines.encode()); os.close(fd)
                ctx = me.Context(0, tune_cache_path=path)
                items, keep = [], []
                for cur, ref in cases:
                    h, w = cur.shape
                    nb = (w // B) * (h // B)
                    c, r = torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda()
                    mv = torch.empty((nb, 2), dtype=torch.int16, device="cuda")
                    sad = torch.empty(nb, dtype=torch.int32, device="cuda")
                    nsp = torch.empty(nb, dtype=torch.int16, device="cuda")
                    keep.append((c, r, mv, sad, nsp)); items.append((c, r, R, mv, sad, nsp))
                descs = me.Context.frame_descs(items)
                for fused in (False, True):
                    if fused:
                        sums = torch.zeros((len(items), me.ME_NSUMS), dtype=torch.int64, device="cuda")
                        ctx.me_estimate_eval_batch(descs, None, B, algo, sums)
                    else:
                        ctx.me_estimate_batch(descs, B, algo)
                    ctx.me_check_status()   # raises if a check fired
                    for (cur, ref), (_, _, mv, sad, nsp) in zip(cases, keep):
                        want = oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))
                        got = (mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32), nsp.cpu().numpy().view(np.uint16))
                        for g, w_ in zip(got, want):
                            assert np.array_equal(g, w_), (shape, B, algo, R, fused, cur.shape)
                    runs += 1
                ctx.close(); os.unlink(path)
print("bounds ok", runs)
'''


def test_bounds_checked_build_finds_nothing():
    env = dict(os.environ, ME_LIB_VARIANT="check", ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=1500,
                       cwd=ROOT)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "bounds ok 80" in r.stdout
