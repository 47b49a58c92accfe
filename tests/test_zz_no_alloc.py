"""me_estimate_batch_noalloc: the DCDS search for callers that cannot
allocate device memory (real-time paths that must not synchronise the
device through cudaMalloc/cudaFree, hosts whose own pool owns all device
memory).  Its results must equal me_estimate_batch's, call after call, while
the library allocates nothing for it: its scratch is a fixed device array.

This file is collected last on purpose, and must also pass alone in a fresh
process (the first call on the device performs the one-time set-up).
"""
import ctypes

import numpy as np
import pytest

from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _batch(seeds_sizes):
    items, keep = [], []
    for name, seed, R in seeds_sizes:
        s = synth.workload_sequence(name, 2, seed=seed, max_motion=R)
        h, w = s.shape[1:]
        nb = (w // 16) * (h // 16)
        cur = torch.from_numpy(s[1]).cuda()
        ref = torch.from_numpy(s[0]).cuda()
        outs = (torch.full((nb, 2), -9, dtype=torch.int16, device="cuda"),
                torch.full((nb,), -1, dtype=torch.int32, device="cuda"),
                torch.full((nb,), -1, dtype=torch.int16, device="cuda"))
        keep.append((cur, ref) + outs)
        items.append((cur, ref, R) + outs)
    return keep, me.Context.frame_descs(items)


def _noalloc(L, descs, algo):
    err = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.me_estimate_batch_noalloc(descs, len(descs), 16, algo, stream, err, len(err))
    assert rc == me.ME_OK, err.value.decode()
    torch.cuda.synchronize()


def _host(keep):
    return [(mv.cpu().numpy(), sad.cpu().numpy(), nsp.cpu().numpy()) for (_, _, mv, sad, nsp) in keep]


def test_noalloc_matches_batch_on_consecutive_calls():
    L = me.load()
    ctx = me.Context(0)
    # two calls in a row, different batches and variants; each compared with
    # the allocating entry point on the same inputs (integer results: exact)
    for spec, algo in (([("qcif", 11, 7), ("cif", 12, 16), ("720p", 13, 16)], me.ME_ALGO_DCDS),
                       ([("cif", 21, 5), ("qcif", 22, 16)], me.ME_ALGO_DCDS_S)):
        keep, descs = _batch(spec)
        _noalloc(L, descs, algo)
        got = _host(keep)
        for (_, _, mv, sad, nsp) in keep:
            mv.fill_(-9); sad.fill_(-1); nsp.fill_(-1)
        ctx.me_estimate_batch(descs, 16, algo)
        torch.cuda.synchronize()
        want = _host(keep)
        for g, w in zip(got, want):
            for a, b in zip(g, w):
                assert np.array_equal(a, b)
            assert (g[1] >= 0).all()
    ctx.close()


def test_noalloc_rejects_oversized_batch():
    L = me.load()
    keep, descs1 = _batch([("qcif", 31, 7)])
    big = (me.FrameDesc * (me.ME_STATIC_MAX_FRAMES + 1))()
    for i in range(len(big)):
        big[i] = descs1[0]
    err = ctypes.create_string_buffer(256)
    rc = L.me_estimate_batch_noalloc(big, len(big), 16, me.ME_ALGO_DCDS, None, err, len(err))
    assert rc == me.ME_ERR_ARG and b"at most" in err.value
    torch.cuda.synchronize()
    assert (keep[0][3] == -1).all()  # nothing was launched
