"""Full-size parity: the stress workload (3840x2160, 60 frame pairs, 8x8
blocks, range +-32, Laplacian motion scales 6/3) and the mixed-stream batch
(8 streams: 2 QCIF, 2 CIF, 2 1280x720, 2 1920x1088, 30 pairs each, 16x16,
+-16), each run as ONE batched launch through a captured graph, as a
production caller would.  Every block of every pair is compared with the
oracle bit for bit, the full search included (the oracle runs one pair per
host core; the full search of a stress pair costs about half a minute of
one core, so its 60 pairs take a couple of minutes on 16 cores);
properties that hold at any size are checked on every block too."""
import numpy as np
import pytest

from _oracle_pool import OraclePool, first_difference
from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


def _alloc(frames, B):
    out = []
    for cur, ref, R in frames:
        h, w = cur.shape
        nb = (w // B) * (h // B)
        out.append((torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), R,
                    torch.full((nb, 2), -999, dtype=torch.int16, device="cuda"),
                    torch.full((nb,), -1, dtype=torch.int32, device="cuda"),
                    torch.full((nb,), -1, dtype=torch.int16, device="cuda")))
    return out


def _graph_run(ctx, items, B, algo):
    descs = me.Context.frame_descs(items)
    g = ctx.me_graph_create(descs, B, algo)
    try:
        ctx.me_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        ctx.me_graph_free(g)
    ctx.me_check_status()
    return [(mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32), nsp.cpu().numpy().view(np.uint16))
            for (_, _, _, mv, sad, nsp) in items]


def _valid_count(w, h, B, R):
    """Closed form of the FS candidate count of every block (window clipped by the frame)."""
    px = np.arange(w // B) * B
    py = np.arange(h // B) * B
    nx = np.minimum(R, w - B - px) - np.maximum(-R, -px) + 1
    ny = np.minimum(R, h - B - py) - np.maximum(-R, -py) + 1
    return (ny[:, None] * nx[None, :]).reshape(-1)


def test_stress_2160p_8x8_range32(ctx):
    B, R, npairs = 8, 32, 60
    seq = synth.workload_sequence("2160p", npairs + 1, seed=4000, max_motion=R, scale=(6.0, 3.0))
    frames = [(seq[t + 1], seq[t], R) for t in range(npairs)]
    d_items = _alloc(frames, B)
    f_items = _alloc(frames, B)
    got_d = _graph_run(ctx, d_items, B, "dcds")
    got_f = _graph_run(ctx, f_items, B, "fs")
    with OraclePool() as pool:
        want_d = pool.fields(frames, B, "dcds")
        want_f = pool.fields(frames, B, "fs")
    h, w = seq[0].shape
    valid = _valid_count(w, h, B, R)
    for t in range(npairs):
        (mv, sad, nsp), (fmv, fsad, fnsp) = got_d[t], got_f[t]
        # every block: FS is the minimum, DCDS never beats it; counts and bounds
        assert (sad >= fsad).all()
        assert np.array_equal(fnsp.astype(np.int64), valid)
        assert (np.abs(mv) <= R).all() and (np.abs(fmv) <= R).all()
        assert (nsp >= 1).all() and (nsp.astype(np.int64) <= valid).all()
        # every block: DCDS and FS bit-exact with the oracle
        d = first_difference(got_d[t], want_d[t])
        assert d is None, f"dcds 2160p pair {t}: {d}"
        d = first_difference(got_f[t], want_f[t])
        assert d is None, f"fs 2160p pair {t}: {d}"


def test_mixed_streams_one_launch(ctx):
    B, R, npairs = 16, 16, 30
    streams = []
    for k, name in enumerate(("qcif", "qcif", "cif", "cif", "720p", "720p", "1080p", "1080p")):
        s = synth.workload_sequence(name, npairs + 1, seed=2000 + k, max_motion=R)
        streams.append(s)
    # interleave the streams frame by frame, as a server batching live streams would
    frames = [(s[t + 1], s[t], R) for t in range(npairs) for s in streams]
    items = _alloc(frames, B)
    got = _graph_run(ctx, items, B, "dcds")
    f_items = _alloc(frames, B)
    got_f = _graph_run(ctx, f_items, B, "fs")
    with OraclePool() as pool:
        want = pool.fields(frames, B, "dcds")
        want_f = pool.fields(frames, B, "fs")
    for t in range(len(frames)):
        d = first_difference(got[t], want[t])
        assert d is None, f"dcds mixed pair {t} ({frames[t][0].shape}): {d}"
        d = first_difference(got_f[t], want_f[t])
        assert d is None, f"fs mixed pair {t} ({frames[t][0].shape}): {d}"
    # the fused evaluation over the same 240-pair batch gives the separate kernel's sums
    descs = me.Context.frame_descs(items)
    sums = torch.zeros((len(items), me.ME_NSUMS), dtype=torch.int64, device="cuda")
    g = ctx.me_graph_create_eval(descs, None, B, "dcds", sums)
    try:
        ctx.me_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        ctx.me_graph_free(g)
    ev = me.Context.eval_descs((c, r, mv, None, nsp) for (c, r, _, mv, sad, nsp) in items)
    ref_sums = torch.zeros_like(sums)
    ctx.me_eval_batch(ev, B, ref_sums)
    torch.cuda.synchronize()
    assert torch.equal(sums, ref_sums)
