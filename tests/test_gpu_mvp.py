"""GPU parity of the motion-vector statistics (me_mvp_stats): every count
of the histogram, D1 and D2 equals the oracle's on the same FS fields."""
import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import me, mvp, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("R", [7, 16])
def test_mvp_counts_match_oracle(ctx, R):
    frames, items, keep = [], [], []
    for name, seed in (("qcif", 51), ("cif", 52), ("qcif", 53)):
        s = synth.workload_sequence(name, 3, seed=seed, max_motion=min(R, 16), scale=(4.0, 2.0))
        for t in (1, 2):
            cur, ref = s[t], s[t - 1]
            mv, _, _ = oracle.fs(cur, ref, 16, R)
            frames.append((cur, ref, mv, R))
            c, r, m = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cur, ref, mv))
            sad = torch.zeros(mv.shape[0], dtype=torch.int32, device="cuda")
            keep.append((c, r, m, sad))
            items.append((c, r, R, m, sad, None))
    out = torch.full((35 * (2 * R + 1) ** 2,), -1, dtype=torch.int64, device="cuda")
    ctx.me_mvp_stats(me.Context.frame_descs(items), R, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = oracle.mvp_counts(frames, R)
    assert np.array_equal(got, want), np.argwhere(got != want)[:5]
    hist, d1, d2 = mvp.unpack(got, R)
    nb = sum(f[2].shape[0] for f in frames)
    assert hist.sum() == nb and d1.sum() == nb and d2.sum() == nb
