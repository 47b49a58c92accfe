"""Checkpoint and resume of the learned proposal's training (not in the
paper): a checkpoint holds the parameters, both Adam moment vectors and the
step count, so training resumed from it follows the uninterrupted run bit for
bit (the training kernels reduce in a fixed order); damaged or foreign files
are rejected and leave the network unchanged."""
import numpy as np
import pytest

from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ME_ERR_ARG = 1


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


def _descs(ctx):
    """Two CIF pairs labelled with their full-search fields."""
    seq = synth.workload_sequence("cif", 3, seed=6100, max_motion=16)
    keep, items = [], []
    for t in range(2):
        c = torch.from_numpy(seq[t + 1]).cuda()
        r = torch.from_numpy(seq[t]).cuda()
        nb = (352 // 16) * (288 // 16)
        mv = torch.zeros((nb, 2), dtype=torch.int16, device="cuda")
        sad = torch.zeros(nb, dtype=torch.int32, device="cuda")
        nsp = torch.zeros(nb, dtype=torch.int16, device="cuda")
        ctx.me_estimate(c, r, 16, 16, "fs", mv, sad, nsp)
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, 16, mv, sad, nsp))
    torch.cuda.synchronize()
    return keep, me.Context.frame_descs(items)


def _steps(ctx, prop, descs, k, lr=2e-3):
    return [ctx.me_proposal_train_step(prop, descs, lr) for _ in range(k)]


def test_resume_follows_the_uninterrupted_run(ctx, tmp_path):
    keep, descs = _descs(ctx)
    path = str(tmp_path / "prop.ckpt")
    a = ctx.me_proposal_create()
    b = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(a, me.proposal_init_params(3))
        _steps(ctx, a, descs, 20)
        ctx.me_proposal_save(a, path)
        cont = _steps(ctx, a, descs, 10)
        ctx.me_proposal_load(b, path)
        resumed = _steps(ctx, b, descs, 10)
        # the Adam state came along: a fresh optimiser from the same weights takes other steps
        c = ctx.me_proposal_create()
        try:
            ctx.me_proposal_load(c, path)
            ctx.me_proposal_set_params(c, ctx.me_proposal_get_params(c))  # keeps weights, resets Adam
            fresh = _steps(ctx, c, descs, 10)
        finally:
            ctx.me_proposal_free(c)
        assert resumed == cont  # the same losses, bit for bit
        assert fresh != cont
        pa, pb = ctx.me_proposal_get_params(a), ctx.me_proposal_get_params(b)
        assert np.array_equal(pa, pb)
    finally:
        ctx.me_proposal_free(a)
        ctx.me_proposal_free(b)


def test_save_load_round_trip_is_exact(ctx, tmp_path):
    keep, descs = _descs(ctx)
    p1, p2 = str(tmp_path / "one.ckpt"), str(tmp_path / "two.ckpt")
    a = ctx.me_proposal_create()
    b = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(a, me.proposal_init_params(4))
        _steps(ctx, a, descs, 5)
        ctx.me_proposal_save(a, p1)
        ctx.me_proposal_load(b, p1)
        ctx.me_proposal_save(b, p2)
        assert open(p1, "rb").read() == open(p2, "rb").read()
        assert np.array_equal(ctx.me_proposal_get_params(a), ctx.me_proposal_get_params(b))
        raw = open(p1, "rb").read()
        assert raw[:8] == b"MEPROP\x00\x01" and len(raw) == 32 + 3 * 4 * me.ME_PROPOSAL_NPARAMS
        assert int.from_bytes(raw[20:24], "little") == 5  # Adam steps taken
    finally:
        ctx.me_proposal_free(a)
        ctx.me_proposal_free(b)


@pytest.mark.parametrize("damage", ["payload", "magic", "short", "long", "missing"])
def test_damaged_checkpoints_are_rejected(ctx, tmp_path, damage):
    keep, descs = _descs(ctx)
    good, bad = str(tmp_path / "good.ckpt"), str(tmp_path / "bad.ckpt")
    a = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(a, me.proposal_init_params(5))
        ctx.me_proposal_save(a, good)
        raw = bytearray(open(good, "rb").read())
        if damage == "payload":
            raw[1000] ^= 0x10
        elif damage == "magic":
            raw[0] = ord("X")
        elif damage == "short":
            raw = raw[:-4]
        elif damage == "long":
            raw += b"\0"
        if damage != "missing":
            open(bad, "wb").write(bytes(raw))
        before = ctx.me_proposal_get_params(a)
        with pytest.raises(me.MeError) as e:
            ctx.me_proposal_load(a, bad)
        assert e.value.code == ME_ERR_ARG
        assert np.array_equal(ctx.me_proposal_get_params(a), before)
    finally:
        ctx.me_proposal_free(a)
