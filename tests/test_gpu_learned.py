"""GPU tests of the learned start proposal (not in the paper): logits and
gradients of the BF16 tensor-core network against the fp64 CPU oracle, the
learned-start search bit-exact with the oracle's search from the same
proposals, and what training gains over plain DCDS."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_0806_0689_gb300 import me, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONV = [(0, 576), (608, 608 + 9216), (608 + 9248, 608 + 9248 + 9216), (608 + 2 * 9248, 608 + 2 * 9248 + 9216)]


@pytest.fixture(scope="module")
def ctx():
    c = me.Context(0)
    yield c
    c.close()


def bf16_conv(params):
    """The values the GPU multiplies: conv weights rounded to bf16 (ties to even)."""
    p = params.astype(np.float64).copy()
    t = torch.from_numpy(params.astype(np.float32))
    r = t.to(torch.bfloat16).to(torch.float64).numpy()
    for a, b in CONV:
        p[a:b] = r[a:b]
    return p


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pair(ctx, cur, ref, R, algo="fs"):
    h, w = cur.shape
    nb = (w // 16) * (h // 16)
    c, r = _dev(cur), _dev(ref)
    mv = torch.zeros((nb, 2), dtype=torch.int16, device="cuda")
    sad = torch.zeros(nb, dtype=torch.int32, device="cuda")
    nsp = torch.zeros(nb, dtype=torch.int16, device="cuda")
    if algo:
        ctx.me_estimate(c, r, 16, R, algo, mv, sad, nsp)
    return c, r, mv, sad, nsp


def test_logits_match_oracle(ctx):
    seq = synth.workload_sequence("cif", 3, seed=11, max_motion=16)
    cur, ref = seq[2], seq[1]
    params = me.proposal_init_params(1)
    prop = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(prop, params)
        c, r, mv, sad, nsp = _pair(ctx, cur, ref, 16)
        desc = me.Context.frame_descs([(c, r, 16, mv, sad, nsp)])
        nb = mv.shape[0]
        lg = torch.zeros((nb, 68), dtype=torch.float32, device="cuda")
        ctx.me_proposal_logits(prop, desc, lg)
        torch.cuda.synchronize()
        got = lg.cpu().numpy()
        field = mv.cpu().numpy()
        pref = bf16_conv(params)
        nbx = cur.shape[1] // 16
        worst = 0.0
        for k in range(0, nb, 3):
            x, mvf = oracle.cnn_features(cur, ref, (k % nbx) * 16, (k // nbx) * 16, field)
            want = oracle.cnn_forward(pref, x, mvf)
            worst = max(worst, float(np.abs(got[k] - want).max()))
        assert worst < 1e-2, worst
    finally:
        ctx.me_proposal_free(prop)


def test_gradients_match_oracle(ctx):
    seq = synth.workload_sequence("qcif", 2, seed=12, max_motion=16)
    cur, ref = seq[1], seq[0]
    params = me.proposal_init_params(2)
    prop = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(prop, params)
        c, r, mv, sad, nsp = _pair(ctx, cur, ref, 16)
        desc = me.Context.frame_descs([(c, r, 16, mv, sad, nsp)])
        loss, g = ctx.me_proposal_train_step(prop, desc, 0.0, want_grad=True)
        field = mv.cpu().numpy()
        pref = bf16_conv(params)
        nbx, nb = cur.shape[1] // 16, field.shape[0]
        gref = np.zeros(me.ME_PROPOSAL_NPARAMS)
        lref = 0.0
        for k in range(nb):
            x, mvf = oracle.cnn_features(cur, ref, (k % nbx) * 16, (k // nbx) * 16, field)
            dx, dy = int(field[k, 0]), int(field[k, 1])
            lab = (min(max(dx, -16), 16) + 16, min(max(dy, -16), 16) + 16, 0 if abs(dx) >= abs(dy) else 1)
            lref += oracle.cnn_loss_grad(pref, x, mvf, lab, gref)[0]
        gref /= nb
        lref /= nb
        assert abs(loss - lref) < 1e-2 * max(1.0, lref)
        bounds = CONV + [(576, 608), (608 + 9216, 608 + 9248), (37532 - 68 - 68 * 134, 37532 - 68), (37532 - 68, 37532)]
        for a, b in bounds:
            num = np.linalg.norm(g[a:b] - gref[a:b])
            den = np.linalg.norm(gref[a:b]) + 1e-12
            assert num / den < 5e-2, (a, b, num / den)
        # unchanged parameters with lr = 0
        assert np.array_equal(ctx.me_proposal_get_params(prop), params)
    finally:
        ctx.me_proposal_free(prop)


def _learned(ctx, prop, pairs, R):
    keep, items = [], []
    for cur, ref in pairs:
        c, r, mv, sad, nsp = _pair(ctx, cur, ref, R, algo=None)
        keep.append((mv, sad, nsp))
        items.append((c, r, R, mv, sad, nsp))
    descs = me.Context.frame_descs(items)
    total = sum(k[0].shape[0] for k in keep)
    starts = torch.zeros((total, 3), dtype=torch.int16, device="cuda")
    ctx.me_estimate_learned_batch(prop, descs, starts)
    torch.cuda.synchronize()
    ctx.me_check_status()
    outs = [(mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32), nsp.cpu().numpy().view(np.uint16))
            for mv, sad, nsp in keep]
    return outs, starts.cpu().numpy()


def test_learned_search_matches_oracle(ctx):
    pairs = []
    for name, seed in (("cif", 21), ("qcif", 22), ("cif", 23)):
        s = synth.workload_sequence(name, 2, seed=seed, scale=(6.0, 3.0), max_motion=16)
        pairs.append((s[1], s[0]))
    params = me.proposal_init_params(3)
    prop = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(prop, params)
        outs, starts = _learned(ctx, prop, pairs, 16)
        base = 0
        pref = bf16_conv(params)
        checked = agree = 0
        for (cur, ref), (mv, sad, nsp) in zip(pairs, outs):
            nb = mv.shape[0]
            st = starts[base:base + nb]
            base += nb
            # the search from the GPU's proposals is bit-exact with the oracle's
            m2, s2, n2 = oracle.dcds_from_starts(cur, ref, 16, 16, st)
            assert np.array_equal(mv, m2) and np.array_equal(sad, s2) and np.array_equal(nsp, n2)
            # the proposals equal the oracle network's, except at near-ties
            h, w = cur.shape
            nbx = w // 16
            for k in range(0, nb, 2):
                px, py = (k % nbx) * 16, (k // nbx) * 16
                x, mvf = oracle.cnn_features(cur, ref, px, py, mv)
                lg = oracle.cnn_forward(pref, x, mvf)
                want = oracle.cnn_start(lg, px, py, w, h, 16)
                gaps = []
                for seg in (lg[:33], lg[33:66], lg[66:]):
                    top = np.sort(seg)[-2:]
                    gaps.append(top[1] - top[0])
                checked += 1
                if min(gaps) < 1e-2:
                    continue
                agree += tuple(int(v) for v in st[k]) == want
                assert tuple(int(v) for v in st[k]) == want, (k, st[k], want)
        assert checked > 100
    finally:
        ctx.me_proposal_free(prop)


def test_zero_network_is_plain_dcds(ctx):
    s = synth.workload_sequence("cif", 2, seed=31, max_motion=16)
    prop = ctx.me_proposal_create()
    try:
        outs, starts = _learned(ctx, prop, [(s[1], s[0])], 16)
        _, _, mv, sad, nsp = _pair(ctx, s[1], s[0], 16, algo="dcds")
        assert (starts == 0).all()
        assert np.array_equal(outs[0][0], mv.cpu().numpy())
        assert np.array_equal(outs[0][2], nsp.cpu().numpy().view(np.uint16))
    finally:
        ctx.me_proposal_free(prop)


def test_median_start_matches_oracle(ctx):
    """The non-learned control: DCDS from the neighbour-median start, bit-exact
    with the oracle (MVs, SADs, search-point counts and the starts), on frames
    with large motion and on a 1080p pair."""
    pairs = []
    for name, seed in (("cif", 41), ("qcif", 42), ("720p", 43)):
        s = synth.workload_sequence(name, 2, seed=seed, scale=(6.0, 3.0), max_motion=16)
        pairs.append((s[1], s[0]))
    keep, items = [], []
    for cur, ref in pairs:
        c, r, mv, sad, nsp = _pair(ctx, cur, ref, 16, algo=None)
        keep.append((mv, sad, nsp))
        items.append((c, r, 16, mv, sad, nsp))
    total = sum(k[0].shape[0] for k in keep)
    starts = torch.zeros((total, 3), dtype=torch.int16, device="cuda")
    ctx.me_estimate_median_batch(me.Context.frame_descs(items), starts)
    torch.cuda.synchronize()
    ctx.me_check_status()
    st = starts.cpu().numpy()
    base = 0
    for (cur, ref), (mv, sad, nsp) in zip(pairs, keep):
        nb = mv.shape[0]
        m2, s2, n2, st2 = oracle.median_dcds(cur, ref, 16)
        assert np.array_equal(mv.cpu().numpy(), m2)
        assert np.array_equal(sad.cpu().numpy().view(np.uint32), s2)
        assert np.array_equal(nsp.cpu().numpy().view(np.uint16), n2)
        assert np.array_equal(st[base:base + nb], st2)
        base += nb


def test_training_gain(ctx):
    """Trained on full-search fields of synthetic CIF video with large motion,
    the proposal lowers the search points per block against plain DCDS at a
    PSNR within 0.05 dB (held-out pairs)."""
    kw = dict(scale=(6.0, 3.0), max_motion=16)
    train = []
    for sd in range(20):
        s = synth.workload_sequence("cif", 6, seed=100000 + sd, **kw)
        train += [(s[t], s[t - 1]) for t in range(1, 6)]
    items, keep = [], []
    for cur, ref in train:
        c, r, mv, sad, nsp = _pair(ctx, cur, ref, 16, algo="fs")
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, 16, mv, sad, nsp))
    torch.cuda.synchronize()
    descs = me.Context.frame_descs(items)
    prop = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(prop, me.proposal_init_params(4))
        losses = me.train_proposal(ctx, prop, descs, steps=3000, lr=3e-3, pairs_per_step=4)
        assert np.mean(losses[-30:]) < 0.8 * np.mean(losses[:10])
        test = []
        for sd in range(3):
            s = synth.workload_sequence("cif", 4, seed=5000 + sd, **kw)
            test += [(s[t], s[t - 1]) for t in range(1, 4)]
        outs, _ = _learned(ctx, prop, test, 16)
        nsp_l, nsp_d, ps_l, ps_d = [], [], [], []
        for (cur, ref), (mv, sad, nsp) in zip(test, outs):
            mvd, sdd, nsd = oracle.dcds(cur, ref, 16, 16)
            nsp_l.append(nsp.mean()); nsp_d.append(nsd.mean())
            ps_l.append(oracle.evaluate(cur, ref, 16, mv)["psnr"])
            ps_d.append(oracle.evaluate(cur, ref, 16, mvd)["psnr"])
        print("learned NSP %.2f plain %.2f | PSNR %.3f vs %.3f" % (np.mean(nsp_l), np.mean(nsp_d), np.mean(ps_l),
                                                                   np.mean(ps_d)))
        assert np.mean(nsp_l) < np.mean(nsp_d)
        assert np.mean(ps_l) > np.mean(ps_d) - 0.05
    finally:
        ctx.me_proposal_free(prop)


def test_wavefront_search_mixed_ranges(ctx):
    """Both start-predicted searches over one batch whose pairs have different
    ranges (1, 7, 16, 32: the staged windows are sized by the largest): the
    median-start search against the oracle, the learned-start search against
    the oracle's search from the same starts; MVs, SADs and counts bit-exact."""
    pairs = []
    for (name, seed), R in zip((("cif", 51), ("qcif", 52), ("cif", 53), ("qcif", 54)), (1, 7, 16, 32)):
        s = synth.workload_sequence(name, 2, seed=seed, scale=(6.0, 3.0), max_motion=min(R, 16))
        pairs.append((s[1], s[0], R))

    def run(fn):
        keep, items = [], []
        for cur, ref, R in pairs:
            c, r, mv, sad, nsp = _pair(ctx, cur, ref, R, algo=None)
            keep.append((mv, sad, nsp))
            items.append((c, r, R, mv, sad, nsp))
        total = sum(k[0].shape[0] for k in keep)
        starts = torch.zeros((total, 3), dtype=torch.int16, device="cuda")
        fn(me.Context.frame_descs(items), starts)
        torch.cuda.synchronize()
        ctx.me_check_status()
        outs = [(mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32), nsp.cpu().numpy().view(np.uint16))
                for mv, sad, nsp in keep]
        return outs, starts.cpu().numpy()

    outs, st = run(lambda d, s: ctx.me_estimate_median_batch(d, s))
    base = 0
    for (cur, ref, R), (mv, sad, nsp) in zip(pairs, outs):
        nb = mv.shape[0]
        m2, s2, n2, st2 = oracle.median_dcds(cur, ref, R)
        assert np.array_equal(mv, m2) and np.array_equal(sad, s2) and np.array_equal(nsp, n2), R
        assert np.array_equal(st[base:base + nb], st2), R
        base += nb
    prop = ctx.me_proposal_create()
    try:
        ctx.me_proposal_set_params(prop, me.proposal_init_params(7))
        outs, st = run(lambda d, s: ctx.me_estimate_learned_batch(prop, d, s))
    finally:
        ctx.me_proposal_free(prop)
    base = 0
    for (cur, ref, R), (mv, sad, nsp) in zip(pairs, outs):
        nb = mv.shape[0]
        m2, s2, n2 = oracle.dcds_from_starts(cur, ref, 16, R, st[base:base + nb])
        assert np.array_equal(mv, m2) and np.array_equal(sad, s2) and np.array_equal(nsp, n2), R
        assert (np.abs(mv) <= R).all()
        base += nb
