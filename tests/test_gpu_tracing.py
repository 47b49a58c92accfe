"""Per-call tracing (me_set_tracing / me_last_call_ms): off by default, then
every launching call records CUDA events around its work, whose elapsed time
agrees with events taken around the same call by the caller."""
import pytest

from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tracing_times_calls():
    ctx = me.Context(0)
    try:
        seq = synth.workload_sequence("720p", 3, seed=8100, max_motion=16)
        items = []
        for t in range(2):
            nb = (1280 // 16) * (720 // 16)
            items.append((torch.from_numpy(seq[t + 1]).cuda(), torch.from_numpy(seq[t]).cuda(), 16,
                          torch.empty((nb, 2), dtype=torch.int16, device="cuda"),
                          torch.empty(nb, dtype=torch.int32, device="cuda"), None))
        descs = me.Context.frame_descs(items)
        with pytest.raises(me.MeError) as e:
            ctx.me_last_call_ms()  # nothing traced yet
        assert e.value.code == 3
        ctx.me_estimate_batch(descs, 16, "fs")  # tracing off: still nothing traced
        with pytest.raises(me.MeError):
            ctx.me_last_call_ms()
        ctx.me_set_tracing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.me_estimate_batch(descs, 16, "fs")
        e1.record()
        ms = ctx.me_last_call_ms()
        torch.cuda.synchronize()
        outer = e0.elapsed_time(e1)
        assert 0.0 < ms <= outer * 1.05 + 0.05
        assert ms >= 0.5 * outer  # the call's own work dominates the caller's bracket
        ctx.me_set_tracing(False)
    finally:
        ctx.close()


def test_tracing_ends_before_a_closing_wait():
    """A call that synchronises its stream (here the proposal's logits) records
    its closing event before the wait: the traced time is its device work,
    within the caller's bracket, and grows with the work."""
    ctx = me.Context(0)
    prop = ctx.me_proposal_create()
    try:
        ctx.me_set_tracing(True)
        ctx.me_proposal_set_params(prop, me.proposal_init_params(0))
        times = {}
        for name, (w, h) in (("cif", (352, 288)), ("720p", (1280, 720))):
            seq = synth.workload_sequence(name, 2, seed=8200, max_motion=16)
            nb = (w // 16) * (h // 16)
            mv = torch.zeros((nb, 2), dtype=torch.int16, device="cuda")
            sad = torch.zeros(nb, dtype=torch.int32, device="cuda")
            logits = torch.empty((nb, me.ME_PROPOSAL_NLOGITS), dtype=torch.float32, device="cuda")
            d = me.Context.frame_descs([(torch.from_numpy(seq[1]).cuda(), torch.from_numpy(seq[0]).cuda(), 16,
                                         mv, sad, None)])
            ctx.me_proposal_logits(prop, d, logits)  # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            ctx.me_proposal_logits(prop, d, logits)
            e1.record()
            ms = ctx.me_last_call_ms()
            torch.cuda.synchronize()
            assert 0.0 < ms <= e0.elapsed_time(e1) * 1.05 + 0.05
            assert torch.isfinite(logits).all()
            times[name] = ms
        assert times["720p"] > times["cif"]  # 3,600 blocks against 396
        ctx.me_set_tracing(False)
    finally:
        ctx.me_proposal_free(prop)
        ctx.close()
