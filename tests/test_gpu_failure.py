"""Failure detection on the GPU without a fault: the DCDS tile kernel's
bounded copy waits are made to run out (me_inject_wait_timeout arms each
CTA's first copy barrier for bytes that never arrive).  The launch must end
within its bound, report ME_ERR_TIMEOUT through me_check_status, write no
output, and leave the context usable: the next search is bit-exact with the
oracle (Sec. III-B DCDS, Sec. IV-C DCDS^S)."""
import time

import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ME_ERR_TIMEOUT = 4


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


def _pairs():
    s = synth.workload_sequence("cif", 4, seed=5100, max_motion=7)
    q = synth.workload_sequence("qcif", 3, seed=5101, max_motion=7)
    return [(s[1], s[0], 7), (s[2], s[1], 16), (s[3], s[2], 7), (q[1], q[0], 4), (q[2], q[1], 7)]


def _items(pairs, B):
    items = []
    for cur, ref, R in pairs:
        h, w = cur.shape
        nb = (w // B) * (h // B)
        items.append((torch.from_numpy(cur).cuda(), torch.from_numpy(ref).cuda(), R,
                      torch.full((nb, 2), -999, dtype=torch.int16, device="cuda"),
                      torch.full((nb,), -1, dtype=torch.int32, device="cuda"),
                      torch.full((nb,), -1, dtype=torch.int16, device="cuda")))
    return items


def _untouched(items):
    return all(bool((mv == -999).all()) and bool((sad == -1).all()) and bool((nsp == -1).all())
               for (_, _, _, mv, sad, nsp) in items)


def _matches_oracle(pairs, items, B, algo):
    for (cur, ref, R), (_, _, _, mv, sad, nsp) in zip(pairs, items):
        want = oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))
        if not (np.array_equal(mv.cpu().numpy(), want[0])
                and np.array_equal(sad.cpu().numpy().view(np.uint32), want[1])
                and np.array_equal(nsp.cpu().numpy().view(np.uint16), want[2])):
            return False
    return True


def _timed_out(ctx, launch):
    ctx.me_inject_wait_timeout(True)
    try:
        t0 = time.perf_counter()
        launch()
        torch.cuda.synchronize()
        elapsed = time.perf_counter() - t0
        with pytest.raises(me.MeError) as e:
            ctx.me_check_status()
        assert e.value.code == ME_ERR_TIMEOUT
    finally:
        ctx.me_inject_wait_timeout(False)
    assert elapsed < 10.0  # the waits are bounded
    ctx.me_check_status()  # the flag was cleared by the report


@pytest.mark.parametrize("B,algo", [(16, "dcds"), (8, "dcds_s")])
def test_timeout_reported_then_context_usable(ctx, B, algo):
    pairs = _pairs()
    items = _items(pairs, B)
    descs = me.Context.frame_descs(items)
    _timed_out(ctx, lambda: ctx.me_estimate_batch(descs, B, algo))
    assert _untouched(items)
    ctx.me_estimate_batch(descs, B, algo)
    torch.cuda.synchronize()
    ctx.me_check_status()
    assert _matches_oracle(pairs, items, B, algo)


def test_timeout_in_fused_evaluation(ctx):
    B = 16
    pairs = _pairs()
    items = _items(pairs, B)
    descs = me.Context.frame_descs(items)
    sums = torch.full((len(pairs), me.ME_NSUMS), 7, dtype=torch.int64, device="cuda")
    _timed_out(ctx, lambda: ctx.me_estimate_eval_batch(descs, None, B, "dcds", sums))
    assert _untouched(items)
    assert bool((sums == 0).all())  # zeroed before the launch, never added to
    ctx.me_estimate_eval_batch(descs, None, B, "dcds", sums)
    torch.cuda.synchronize()
    ctx.me_check_status()
    assert _matches_oracle(pairs, items, B, "dcds")
    assert bool((sums[:, 5] > 0).all())  # the block counts are in


def test_null_context_hook_is_the_noalloc_one(ctx):
    # a NULL context arms the hook of the context-free no-allocation path
    # only: a context's own launches stay normal
    L = me.load()
    assert L.me_inject_wait_timeout(None, 1) == me.ME_OK
    try:
        pairs = _pairs()[:2]
        items = _items(pairs, 16)
        descs = me.Context.frame_descs(items)
        ctx.me_estimate_batch(descs, 16, "dcds")
        torch.cuda.synchronize()
        ctx.me_check_status()
        assert _matches_oracle(pairs, items, 16, "dcds")
    finally:
        assert L.me_inject_wait_timeout(None, 0) == me.ME_OK


@pytest.mark.parametrize("B,kind", [(16, "median"), (8, "median"), (16, "learned"), (8, "learned")])
def test_wavefront_wait_timeout_reported_then_exact(ctx, B, kind):
    """The wavefront searches' neighbour waits: with the hook armed the blocks
    of the first region in wavefront order never publish their hand-off
    words, the blocks that wait for them give up after the shortened wait and
    go on; the call
    ends within its bound, every block is written, me_check_status reports
    ME_ERR_TIMEOUT once, and the next call is bit-exact with the oracle."""
    pairs = _pairs()
    items = _items(pairs, B)
    descs = me.Context.frame_descs(items)
    total = sum(it[3].shape[0] for it in items)
    starts = torch.zeros((total, 3), dtype=torch.int16, device="cuda")
    prop = None
    if kind == "learned":
        prop = ctx.me_proposal_create()
        ctx.me_proposal_set_params(prop, me.proposal_init_params(12))
        run = lambda: ctx.me_estimate_learned_batch(prop, descs, starts, block=B)
    else:
        run = lambda: ctx.me_estimate_median_batch(descs, starts, block=B)
    try:
        _timed_out(ctx, run)
        for (_, _, _, mv, sad, nsp) in items:
            assert bool((mv != -999).any(dim=1).all()) and bool((sad != -1).all())
        run()
        torch.cuda.synchronize()
        ctx.me_check_status()
        st = starts.cpu().numpy()
        base = 0
        for (cur, ref, R), (_, _, _, mv, sad, nsp) in zip(pairs, items):
            nb = mv.shape[0]
            if kind == "median":
                want = oracle.median_dcds(cur, ref, R, block=B)
                assert np.array_equal(st[base:base + nb], want[3])
            else:
                h, w = cur.shape
                want = oracle.dcds_from_starts(cur, ref, B, R, st[base:base + nb],
                                               oracle.region_medians(mv.cpu().numpy(), w, h, B))
            assert np.array_equal(mv.cpu().numpy(), want[0])
            assert np.array_equal(sad.cpu().numpy().view(np.uint32), want[1])
            assert np.array_equal(nsp.cpu().numpy().view(np.uint16), want[2])
            base += nb
    finally:
        if prop is not None:
            ctx.me_proposal_free(prop)
