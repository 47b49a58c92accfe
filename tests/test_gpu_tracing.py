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
