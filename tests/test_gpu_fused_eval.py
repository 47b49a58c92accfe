"""GPU parity of the fused search + evaluation path (me_estimate_eval_batch,
me_graph_create_eval): the motion field is bit-identical to the plain
search, the eight sums are bit-identical to me_eval_batch on that field, and
the six measures equal the oracle's evaluation of the oracle's DCDS field
(Sec. IV: MAD, MSE, NSP, PSNR, distance and probability against FS)."""
import math

import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


SUM_DIST_Q24 = 4  # ME_SUM_DIST_Q24 of include/me.h


def _q24(n):
    """round(sqrt(n) * 2^24), exactly: sqrt(N) >= s + 1/2 iff N - s^2 > s."""
    big = n << 48
    s = math.isqrt(big)
    return s + (1 if big - s * s > s else 0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pairs():
    out = []
    for name, seed, R in (("qcif", 3000, 7), ("cif", 3001, 16), ("qcif", 3002, 32), ("cif", 3003, 4)):
        s = synth.workload_sequence(name, 3, seed=seed, max_motion=min(R, 16))
        out += [(s[1], s[0], R), (s[2], s[1], R)]
    return out


def _run(ctx, pairs, B, algo, with_fs, with_nsp, graph=False, reps=1):
    keep, items, fs_fields = [], [], []
    for i, (cur, ref, R) in enumerate(pairs):
        h, w = cur.shape
        nb = (w // B) * (h // B)
        c, r = _dev(cur), _dev(ref)
        mv = torch.full((nb, 2), -999, dtype=torch.int16, device="cuda")
        sad = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
        nsp = torch.full((nb,), -1, dtype=torch.int16, device="cuda") if with_nsp else None
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, R, mv, sad, nsp))
        fs_fields.append(_dev(oracle.fs(cur, ref, B, R)[0]) if (with_fs and i % 3 != 2) else None)
    descs = me.Context.frame_descs(items)
    sums = torch.full((len(pairs), me.ME_NSUMS), 12345, dtype=torch.int64, device="cuda")
    mv_fs = fs_fields if with_fs else None
    if graph:
        g = ctx.me_graph_create_eval(descs, mv_fs, B, algo, sums)
        try:
            got = []
            for _ in range(reps):
                sums.fill_(777)
                ctx.me_graph_launch(g)
                torch.cuda.synchronize()
                got.append(sums.clone())
            for x in got[1:]:
                assert torch.equal(x, got[0])
        finally:
            ctx.me_graph_free(g)
    else:
        ctx.me_estimate_eval_batch(descs, mv_fs, B, algo, sums)
    torch.cuda.synchronize()
    return keep, fs_fields, sums


@pytest.mark.parametrize("B,algo,with_fs,with_nsp,graph", [
    (16, "dcds", True, True, False),
    (8, "dcds", True, True, False),
    (16, "dcds_s", True, False, False),
    (16, "dcds", False, True, True),
    (8, "dcds_s", True, True, True),
])
def test_fused_sums_equal_eval_batch(ctx, B, algo, with_fs, with_nsp, graph):
    pairs = _pairs()
    keep, fs_fields, sums = _run(ctx, pairs, B, algo, with_fs, with_nsp, graph=graph, reps=3)
    # the same field as the plain search
    for (cur, ref, R), (c, r, mv, sad, nsp) in zip(pairs, keep):
        want = oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))
        assert np.array_equal(mv.cpu().numpy(), want[0])
        assert np.array_equal(sad.cpu().numpy().view(np.uint32), want[1])
        if nsp is not None:
            assert np.array_equal(nsp.cpu().numpy().view(np.uint16), want[2])
    # the same sums as the separate evaluation kernel on that field
    ev = me.Context.eval_descs((c, r, mv, f, nsp) for (c, r, mv, sad, nsp), f in zip(keep, fs_fields))
    ref_sums = torch.zeros_like(sums)
    ctx.me_eval_batch(ev, B, ref_sums)
    torch.cuda.synchronize()
    assert torch.equal(sums, ref_sums), (sums - ref_sums).abs().max()
    # and the oracle's measures
    arr = sums.cpu().numpy().view(np.uint64)
    for i, ((cur, ref, R), (c, r, mv, sad, nsp), f) in enumerate(zip(pairs, keep, fs_fields)):
        got = ctx.me_stats_from_sums(arr[i])
        want = oracle.evaluate(cur, ref, B, mv.cpu().numpy(), None if f is None else f.cpu().numpy(),
                               None if nsp is None else nsp.cpu().numpy().view(np.uint16))
        for k in ("mad", "mse", "nsp", "probability"):
            assert got[k] == want[k], (i, k)
        assert abs(got["psnr"] - want["psnr"]) < 1e-9
        assert abs(got["distance"] - want["distance"]) < 1e-7
        if f is not None:  # the distance counter is the exactly rounded Q24 sum
            e = mv.cpu().numpy().astype(np.int64) - f.cpu().numpy().astype(np.int64)
            n = (e * e).sum(axis=1)
            assert int(arr[i][SUM_DIST_Q24]) == sum(_q24(int(v)) for v in n if v), i


def test_fused_rejects_fs_and_bad_sums(ctx):
    cur = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    mv = torch.zeros((16, 2), dtype=torch.int16, device="cuda")
    sad = torch.zeros(16, dtype=torch.int32, device="cuda")
    descs = me.Context.frame_descs([(cur, cur, 4, mv, sad, None)])
    sums = torch.zeros((1, me.ME_NSUMS), dtype=torch.int64, device="cuda")
    with pytest.raises(me.MeError) as e:
        ctx.me_estimate_eval_batch(descs, None, 16, "fs", sums)
    assert e.value.code == me.ME_ERR_UNSUPPORTED
    with pytest.raises(me.MeError) as e:
        ctx.me_estimate_eval_batch(descs, None, 16, "dcds", None)
    assert e.value.code == me.ME_ERR_ARG
