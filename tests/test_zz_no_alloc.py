"""me_estimate_batch_noalloc: the DCDS search for callers that cannot
allocate device memory when they search (real-time paths that must not
synchronise the device through cudaMalloc/cudaFree, hosts whose own pool owns
all device memory, processes at the memory limit).  Its scratch is a fixed
device array inside the library, so these tests check that:

* its fields equal me_estimate_batch's and the CPU oracle's (Sec. III-B DCDS,
  Sec. IV-C DCDS^S), bit for bit, call after call, for both block sizes, for
  batches that take several set-up launches and for the largest batch the
  array holds;
* device memory stays the same across calls once the first call has run;
* a bounded wait that gives up is reported by me_noalloc_check_status, and
  the next call is exact again.

This file is collected last on purpose, and must also pass alone in a fresh
process (the first call on the device performs the one-time set-up).
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(specs, B=16):
    """specs: (workload, seed, range) per pair; outputs pre-filled with junk."""
    items, keep, host = [], [], []
    for name, seed, R in specs:
        s = synth.workload_sequence(name, 2, seed=seed, max_motion=R)
        h, w = s.shape[1:]
        nb = (w // B) * (h // B)
        cur = torch.from_numpy(s[1]).cuda()
        ref = torch.from_numpy(s[0]).cuda()
        outs = (torch.full((nb, 2), -9, dtype=torch.int16, device="cuda"),
                torch.full((nb,), -1, dtype=torch.int32, device="cuda"),
                torch.full((nb,), -1, dtype=torch.int16, device="cuda"))
        keep.append((cur, ref) + outs)
        items.append((cur, ref, R) + outs)
        host.append((s[1], s[0], R))
    return keep, me.Context.frame_descs(items), host


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _noalloc(L, descs, B, algo):
    err = ctypes.create_string_buffer(256)
    rc = L.me_estimate_batch_noalloc(descs, len(descs), B, algo, _stream(), err, len(err))
    assert rc == me.ME_OK, err.value.decode()
    torch.cuda.synchronize()


def _status(L):
    err = ctypes.create_string_buffer(256)
    return L.me_noalloc_check_status(_stream(), err, len(err)), err.value.decode()


def _fields(keep):
    return [(mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32), nsp.cpu().numpy().view(np.uint16))
            for (_, _, mv, sad, nsp) in keep]


def _reset(keep):
    for (_, _, mv, sad, nsp) in keep:
        mv.fill_(-9); sad.fill_(-1); nsp.fill_(-1)


def _check_oracle(got, host, B, algo):
    for g, (cur, ref, R) in zip(got, host):
        want = oracle.dcds(cur, ref, B, R, simplified=(algo == me.ME_ALGO_DCDS_S))
        for a, b in zip(g, want):
            assert np.array_equal(a, b)


def test_noalloc_matches_batch_and_oracle_on_consecutive_calls():
    L = me.load()
    ctx = me.Context(0)
    # two calls in a row, different batches and variants; each compared with
    # the allocating entry point and with the oracle (integer results: exact)
    for spec, algo in (([("qcif", 11, 7), ("cif", 12, 16), ("720p", 13, 16)], me.ME_ALGO_DCDS),
                       ([("cif", 21, 5), ("qcif", 22, 16)], me.ME_ALGO_DCDS_S)):
        keep, descs, host = _batch(spec)
        _noalloc(L, descs, 16, algo)
        got = _fields(keep)
        _check_oracle(got, host, 16, algo)
        _reset(keep)
        ctx.me_estimate_batch(descs, 16, algo)
        torch.cuda.synchronize()
        for g, w in zip(got, _fields(keep)):
            for a, b in zip(g, w):
                assert np.array_equal(a, b)
    assert _status(L)[0] == me.ME_OK
    ctx.close()


@pytest.mark.parametrize("B", [8, 16])
def test_noalloc_chunked_setup_and_full_table(B):
    # 40 descriptors of mixed sizes and ranges take three set-up launches of
    # the descriptor table; 64 fill it exactly
    L = me.load()
    names = ("qcif", "cif", "qcif", "cif", "qcif")
    spec40 = [(names[i % 5], 3000 + i, 1 + (7 * i) % 32) for i in range(40)]
    spec64 = [("qcif", 4000 + i, 1 + (5 * i) % 32) for i in range(me.ME_STATIC_MAX_FRAMES)]
    for spec, algo in ((spec40, me.ME_ALGO_DCDS), (spec64, me.ME_ALGO_DCDS_S)):
        keep, descs, host = _batch(spec, B)
        _noalloc(L, descs, B, algo)
        _check_oracle(_fields(keep), host, B, algo)
    assert _status(L)[0] == me.ME_OK


def test_noalloc_allocates_nothing_after_first_call():
    L = me.load()
    keep16, d16, _ = _batch([("cif", 51, 16), ("qcif", 52, 7)], 16)
    keep8, d8, _ = _batch([("cif", 53, 32), ("qcif", 54, 3)], 8)
    _noalloc(L, d16, 16, me.ME_ALGO_DCDS)  # first call: set-up and kernel loads
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for B, d in ((16, d16), (8, d8), (16, d16), (8, d8)):
        for algo in (me.ME_ALGO_DCDS, me.ME_ALGO_DCDS_S):
            _noalloc(L, d, B, algo)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_timeout_reported_then_exact():
    L = me.load()
    keep, descs, host = _batch([("cif", 61, 7), ("qcif", 62, 16)])
    _noalloc(L, descs, 16, me.ME_ALGO_DCDS)  # set-up done, status clean
    assert _status(L)[0] == me.ME_OK
    _reset(keep)
    assert L.me_inject_wait_timeout(None, 1) == me.ME_OK
    try:
        _noalloc(L, descs, 16, me.ME_ALGO_DCDS)  # returns ME_OK: the failure is on the device
    finally:
        assert L.me_inject_wait_timeout(None, 0) == me.ME_OK
    rc, msg = _status(L)
    assert rc == me.ME_ERR_TIMEOUT and "wait" in msg
    assert _status(L)[0] == me.ME_OK  # reading it cleared it
    for (_, _, mv, sad, nsp) in keep:  # no tile was searched
        assert bool((mv == -9).all()) and bool((sad == -1).all()) and bool((nsp == -1).all())
    _noalloc(L, descs, 16, me.ME_ALGO_DCDS)
    _check_oracle(_fields(keep), host, 16, me.ME_ALGO_DCDS)
    assert _status(L)[0] == me.ME_OK


def test_noalloc_rejects_oversized_batch():
    L = me.load()
    keep, descs1, _ = _batch([("qcif", 31, 7)])
    big = (me.FrameDesc * (me.ME_STATIC_MAX_FRAMES + 1))()
    for i in range(len(big)):
        big[i] = descs1[0]
    err = ctypes.create_string_buffer(256)
    rc = L.me_estimate_batch_noalloc(big, len(big), 16, me.ME_ALGO_DCDS, None, err, len(err))
    assert rc == me.ME_ERR_ARG and b"at most" in err.value
    torch.cuda.synchronize()
    assert (keep[0][3] == -1).all()  # nothing was launched
