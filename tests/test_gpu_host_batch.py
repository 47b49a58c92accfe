"""GPU parity of me_estimate_host_batch: frames and outputs in host memory,
uploaded and read back by the library in chunks.  Motion fields, SADs and
search-point counts equal the oracle's (Sec. I full search, Sec. III-B DCDS,
Sec. IV-C DCDS^S) for every chunk size, with frames shared between pairs
(a sequence passed as consecutive pairs), with pageable host memory and
across calls that grow the staging; with sums, the Sec. IV sums equal the
device-side fused call on device copies of the same data."""
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


def _host(a, pinned=True):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.pin_memory() if pinned else t.clone()


def _outs(nb, n, pinned=True, with_nsp=True):
    mk = lambda shape, dt: _host(np.full(shape, -7, dtype=dt), pinned)
    mv = mk((n, nb, 2), np.int16)
    sad = mk((n, nb), np.int32)
    nsp = mk((n, nb), np.int16) if with_nsp else None
    return mv, sad, nsp


def _mixed():
    """Pairs of several sizes and ranges, each pair with frames of its own."""
    out = []
    for name, seed, R in (("qcif", 4100, 7), ("cif", 4101, 16), ("qcif", 4102, 32), ("cif", 4103, 4),
                          ("qcif", 4104, 1)):
        s = synth.workload_sequence(name, 3, seed=seed, max_motion=min(R, 16))
        out += [(s[1], s[0], R), (s[2], s[1], R)]
    return out


def _expect(cur, ref, B, R, algo):
    if algo == "fs":
        return oracle.fs(cur, ref, B, R)
    return oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))


def _check(got_mv, got_sad, got_nsp, cur, ref, B, R, algo):
    mv, sad, nsp = _expect(cur, ref, B, R, algo)
    nb = mv.shape[0]
    np.testing.assert_array_equal(got_mv[:nb].numpy(), mv)
    np.testing.assert_array_equal(got_sad[:nb].numpy().view(np.uint32), sad)
    if got_nsp is not None:
        np.testing.assert_array_equal(got_nsp[:nb].numpy().view(np.uint16), nsp)


@pytest.mark.parametrize("B,algo,chunk", [
    (16, "dcds", 0), (16, "dcds", 1), (16, "dcds", 3), (16, "dcds", 10), (8, "dcds", 4),
    (16, "dcds_s", 2), (8, "dcds_s", 0), (16, "fs", 3), (8, "fs", 0),
])
def test_host_batch_equals_oracle(ctx, B, algo, chunk):
    pairs = _mixed()
    keep, items = [], []
    for cur, ref, R in pairs:
        h, w = cur.shape
        nb = (w // B) * (h // B)
        c, r = _host(cur), _host(ref)
        mv, sad, nsp = _outs(nb, 1)
        keep.append((c, r, mv[0], sad[0], nsp[0]))
        items.append((c, r, R, mv[0], sad[0], nsp[0]))
    descs = me.Context.frame_descs(items)
    ctx.me_estimate_host_batch(descs, B, algo, chunk=chunk)
    torch.cuda.synchronize()
    for (cur, ref, R), (_, _, mv, sad, nsp) in zip(pairs, keep):
        _check(mv, sad, nsp, cur, ref, B, R, algo)


def test_sequence_frames_shared(ctx):
    """ref of pair i+1 is the same host buffer as cur of pair i."""
    R, B, n = 16, 16, 9
    seq = synth.workload_sequence("cif", n + 1, seed=4200, max_motion=R)
    frames = _host(np.stack(seq))
    h, w = seq[0].shape
    nb = (w // B) * (h // B)
    mv, sad, nsp = _outs(nb, n)
    descs = me.Context.frame_descs((frames[i + 1], frames[i], R, mv[i], sad[i], nsp[i]) for i in range(n))
    for chunk in (0, 1, 4, n):
        mv.fill_(-7)
        ctx.me_estimate_host_batch(descs, B, "dcds", chunk=chunk)
        torch.cuda.synchronize()
        for i in range(n):
            _check(mv[i], sad[i], nsp[i], seq[i + 1], seq[i], B, R, "dcds")


def test_pageable_host_memory(ctx):
    pairs = _mixed()[:4]
    B = 16
    keep, items = [], []
    for cur, ref, R in pairs:
        h, w = cur.shape
        nb = (w // B) * (h // B)
        c, r = _host(cur, pinned=False), _host(ref, pinned=False)
        mv, sad, nsp = _outs(nb, 1, pinned=False)
        keep.append((c, r, mv[0], sad[0], nsp[0]))
        items.append((c, r, R, mv[0], sad[0], nsp[0]))
    ctx.me_estimate_host_batch(me.Context.frame_descs(items), B, "dcds", chunk=2)
    torch.cuda.synchronize()
    for (cur, ref, R), (_, _, mv, sad, nsp) in zip(pairs, keep):
        _check(mv, sad, nsp, cur, ref, B, R, "dcds")


def test_calls_on_two_streams_and_growing_staging(ctx):
    """A small batch, a larger one on another stream (the staging grows), then
    the small one again: every call's results are its own."""
    B = 16
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    small = _mixed()[:2]
    big = _mixed()
    runs = []
    for pairs, st in ((small, s1), (big, s2), (small, s1), (big, s1)):
        keep, items = [], []
        for cur, ref, R in pairs:
            h, w = cur.shape
            nb = (w // B) * (h // B)
            c, r = _host(cur), _host(ref)
            mv, sad, nsp = _outs(nb, 1)
            keep.append((c, r, mv[0], sad[0], nsp[0]))
            items.append((c, r, R, mv[0], sad[0], nsp[0]))
        ctx.me_estimate_host_batch(me.Context.frame_descs(items), B, "dcds", chunk=3, stream=st)
        runs.append((pairs, keep))
    torch.cuda.synchronize()
    for pairs, keep in runs:
        for (cur, ref, R), (_, _, mv, sad, nsp) in zip(pairs, keep):
            _check(mv, sad, nsp, cur, ref, B, R, "dcds")


@pytest.mark.parametrize("B,algo,chunk", [(16, "dcds", 0), (16, "dcds", 3), (8, "dcds_s", 2)])
def test_host_eval_sums_equal_device_call(ctx, B, algo, chunk):
    pairs = _mixed()
    n = len(pairs)
    h_items, d_items, h_keep, d_keep, h_fs, d_fs = [], [], [], [], [], []
    for i, (cur, ref, R) in enumerate(pairs):
        h, w = cur.shape
        nb = (w // B) * (h // B)
        fsf = oracle.fs(cur, ref, B, R)[0] if i % 3 != 2 else None
        c, r = _host(cur), _host(ref)
        mv, sad, nsp = _outs(nb, 1)
        h_keep.append((mv[0], sad[0], nsp[0]))
        h_items.append((c, r, R, mv[0], sad[0], nsp[0]))
        h_fs.append(None if fsf is None else _host(fsf))
        dc, dr = c.cuda(), r.cuda()
        dmv = torch.empty((nb, 2), dtype=torch.int16, device="cuda")
        dsad = torch.empty((nb,), dtype=torch.int32, device="cuda")
        dnsp = torch.empty((nb,), dtype=torch.int16, device="cuda")
        d_keep.append((dc, dr, dmv, dsad, dnsp))
        d_items.append((dc, dr, R, dmv, dsad, dnsp))
        d_fs.append(None if fsf is None else h_fs[-1].cuda())
    h_sums = _host(np.full((n, me.ME_NSUMS), 99, dtype=np.int64))
    d_sums = torch.zeros((n, me.ME_NSUMS), dtype=torch.int64, device="cuda")
    ctx.me_estimate_host_batch(me.Context.frame_descs(h_items), B, algo, mv_fs=h_fs, sums=h_sums, chunk=chunk)
    ctx.me_estimate_eval_batch(me.Context.frame_descs(d_items), d_fs, B, algo, d_sums)
    torch.cuda.synchronize()
    assert torch.equal(h_sums, d_sums.cpu())
    for (mv, sad, nsp), (_, _, dmv, dsad, dnsp) in zip(h_keep, d_keep):
        assert torch.equal(mv, dmv.cpu()) and torch.equal(sad, dsad.cpu()) and torch.equal(nsp, dnsp.cpu())


def test_argument_errors(ctx):
    cur, ref, R = _mixed()[0]
    B = 16
    nb = (cur.shape[1] // B) * (cur.shape[0] // B)
    c, r = _host(cur), _host(ref)
    mv, sad, nsp = _outs(nb, 1)
    descs = me.Context.frame_descs([(c, r, R, mv[0], sad[0], nsp[0])])
    with pytest.raises(me.MeError) as e:
        ctx.me_estimate_host_batch(descs, B, "dcds", chunk=-1)
    assert e.value.code == 1
    sums = _host(np.zeros((1, me.ME_NSUMS), dtype=np.int64))
    with pytest.raises(me.MeError) as e:
        ctx.me_estimate_host_batch(descs, B, "fs", sums=sums)
    assert e.value.code == 3
