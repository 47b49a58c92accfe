"""GPU parity: every motion vector, SAD and search-point count produced by
the CUDA path through the C-ABI equals the CPU oracle's, bit for bit.

Inputs are the seeded synthetic luma sequences (paper_0806_0689_gb300.synth)
shaped like the paper's QCIF/CIF workloads, plus edge cases: ranges 1..32,
single-block frames, stationary content, ragged tiles, mixed-size batches
and the full 1080p benchmark batch (every block).
"""
import ctypes

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _outs(h, w, B):
    nb = (w // B) * (h // B)
    return (torch.full((nb, 2), -999, dtype=torch.int16, device="cuda"),
            torch.full((nb,), -1, dtype=torch.int32, device="cuda"),
            torch.full((nb,), -1, dtype=torch.int16, device="cuda"))


def _host(mv, sad, nsp):
    torch.cuda.synchronize()
    return (mv.cpu().numpy(), sad.cpu().numpy().view(np.uint32),
            None if nsp is None else nsp.cpu().numpy().view(np.uint16))


def gpu_search(ctx, cur, ref, B, R, algo):
    h, w = cur.shape
    c, r = _dev(cur), _dev(ref)
    mv, sad, nsp = _outs(h, w, B)
    ctx.me_estimate(c, r, B, R, algo, mv, sad, nsp)
    return _host(mv, sad, nsp)


def oracle_search(cur, ref, B, R, algo):
    if algo == "fs":
        return oracle.fs(cur, ref, B, R)
    return oracle.dcds(cur, ref, B, R, simplified=(algo == "dcds_s"))


def assert_same(got, want, what=""):
    for name, g, o in zip(("mv", "sad", "nsp"), got, want):
        if not np.array_equal(g, o):
            bad = np.argwhere(np.asarray(g).reshape(len(g), -1) != np.asarray(o).reshape(len(o), -1))[:5]
            raise AssertionError(f"{what}: {name} differs at {bad.tolist()}: gpu {g[bad[:, 0]]} oracle {o[bad[:, 0]]}")


ALGOS = ["dcds", "dcds_s", "fs"]


@pytest.fixture(scope="module")
def qcif():
    # 10 frame pairs, 3 moving objects, +-7 motion (the QCIF workload)
    return synth.workload_sequence("qcif", 11, seed=0)


@pytest.fixture(scope="module")
def cif():
    return synth.workload_sequence("cif", 5, seed=1000)


@pytest.mark.parametrize("algo", ALGOS)
def test_qcif_sequence_bit_exact(ctx, qcif, algo):
    for t in range(1, len(qcif)):
        got = gpu_search(ctx, qcif[t], qcif[t - 1], 16, 7, algo)
        assert_same(got, oracle_search(qcif[t], qcif[t - 1], 16, 7, algo), f"pair {t}")


@pytest.mark.parametrize("B", [16, 8])
@pytest.mark.parametrize("R", [7, 15])
@pytest.mark.parametrize("algo", ALGOS)
def test_cif_bit_exact(ctx, cif, B, R, algo):
    for t in (1, 3):
        got = gpu_search(ctx, cif[t], cif[t - 1], B, R, algo)
        assert_same(got, oracle_search(cif[t], cif[t - 1], B, R, algo), f"pair {t} B{B} R{R}")


@pytest.fixture(scope="module")
def cif100():
    """The CIF workload: a 100-frame sequence, 8 moving objects."""
    return synth.workload_sequence("cif", 100, seed=1000)


@pytest.mark.parametrize("B", [16, 8])
@pytest.mark.parametrize("R", [7, 15])
def test_cif_workload_every_field(ctx, cif100, B, R):
    """Every block of all 99 pairs of the CIF workload, one batched launch
    per search: DCDS (Sec. III-B), DCDS^S (Sec. IV-C) and FS bit-exact with
    the oracle."""
    from _oracle_pool import OraclePool, first_difference
    pairs = [(cif100[t], cif100[t - 1]) for t in range(1, len(cif100))]
    with OraclePool() as pool:
        for algo in ALGOS:
            keep, descs = _batch(ctx, pairs, B, algo, [R] * len(pairs))
            ctx.me_estimate_batch(descs, B, algo)
            torch.cuda.synchronize()
            ctx.me_check_status()
            want = pool.fields([(c, r, R) for c, r in pairs], B, algo)
            for t, ((c, r, mv, sad, nsp), w) in enumerate(zip(keep, want)):
                d = first_difference(_host(mv, sad, nsp), w)
                assert d is None, f"{algo} B{B} R{R} pair {t}: {d}"


@pytest.mark.parametrize("R", [1, 2, 3, 16, 31, 32])
@pytest.mark.parametrize("B", [16, 8])
@pytest.mark.parametrize("algo", ALGOS)
def test_range_edges(ctx, R, B, algo):
    # large motion so that searches reach the window edge
    seq = synth.sequence(112, 80, 3, seed=77 + R, n_objects=4, scale=(6.0, 3.0), max_motion=R)
    got = gpu_search(ctx, seq[2], seq[1], B, R, algo)
    assert_same(got, oracle_search(seq[2], seq[1], B, R, algo), f"R{R} B{B}")


@pytest.mark.parametrize("w,h,B", [(16, 16, 16), (16, 8, 8), (32, 8, 8), (16, 48, 16), (48, 16, 16)])
@pytest.mark.parametrize("algo", ALGOS)
def test_tiny_frames(ctx, w, h, B, algo):
    rng = np.random.default_rng(w * 100 + h)
    cur, ref = synth.shifted_pair(rng, h, w, 1, 0)
    ref = (ref // 4 + 100).astype(np.uint8)  # low contrast: SAD ties occur
    got = gpu_search(ctx, cur, ref, B, 7, algo)
    assert_same(got, oracle_search(cur, ref, B, 7, algo), f"{w}x{h}")


@pytest.mark.parametrize("algo", ["dcds", "dcds_s"])
def test_stationary_closed_form(ctx, algo):
    rng = np.random.default_rng(4)
    f = synth.textured_frame(rng, 48, 64)
    mv, sad, nsp = gpu_search(ctx, f, f, 16, 7, algo)
    assert (mv == 0).all() and (sad == 0).all()
    # HCSP points whose block stays inside the frame
    hcsp = oracle.hcsp_offsets()
    for k in range(len(nsp)):
        i, j = k % 4, k // 4
        want = sum(1 for dx, dy in hcsp if 0 <= i * 16 + dx <= 48 and 0 <= j * 16 + dy <= 32)
        assert nsp[k] == want


@pytest.mark.parametrize("sx,sy", [(1, 0), (0, 1), (2, 0), (-2, 0), (0, -1), (5, -3)])
def test_global_shift(ctx, sx, sy):
    rng = np.random.default_rng(12)
    cur, ref = synth.shifted_pair(rng, 96, 128, sx, sy)
    for algo in ALGOS:
        assert_same(gpu_search(ctx, cur, ref, 16, 7, algo), oracle_search(cur, ref, 16, 7, algo), algo)


def smooth_pair(h, w, sx, sy, margin=48):
    """(cur, ref) of smooth, slowly varying content shifted by (sx, sy): the
    diamond search walks towards the shift in many small steps, so paths run
    far from the block's HCSP winner (NSP up to about 110 at +-32)."""
    yy, xx = np.mgrid[0:h + 2 * margin, 0:w + 2 * margin].astype(np.float64)
    big = 128 + 60 * np.sin(xx / 17.0) * np.cos(yy / 13.0) + 40 * np.sin((xx + 2 * yy) / 29.0)
    big = np.clip(np.rint(big), 0, 255).astype(np.uint8)
    ref = big[margin:margin + h, margin:margin + w].copy()
    cur = big[margin + sy:margin + sy + h, margin + sx:margin + sx + w].copy()
    return cur, ref


@pytest.mark.parametrize("B", [8, 16])
@pytest.mark.parametrize("algo", ["dcds", "dcds_s"])
def test_long_diamond_paths(ctx, B, algo):
    """Long search paths, bit-exact: 8x8 blocks at +-32 (256 threads, where
    the launcher takes the visited-box variant) keep their visited points in
    a box of displacements -16 .. 15 and send a block whose path leaves it to
    the overflow pass, which searches it again with +-R bitmaps; a block
    whose final MV lies outside the box has been through it (149 of the 736
    here, with many more that left the box and came back).  Two pairs in
    one batch (the overflow list is per tile), and the same search with the
    Sec. IV sums fused."""
    pairs = [smooth_pair(128, 176, 13, -9), smooth_pair(96, 256, -17, 6)]
    keep, descs = _batch(ctx, pairs, B, algo, [32, 32])
    ctx.me_estimate_batch(descs, B, algo)
    torch.cuda.synchronize()
    far = outside = 0
    for (cur, ref), (c, r, mv, sad, nsp) in zip(pairs, keep):
        got = _host(mv, sad, nsp)
        want = oracle_search(cur, ref, B, 32, algo)
        assert_same(got, want, f"{algo} B{B}")
        far += int((np.abs(got[0]).max(1) >= 12).sum())
        outside += int(((got[0] < -16) | (got[0] > 15)).any(1).sum())
    assert far > 20, far
    assert outside > 20, outside
    # fused: the same fields, and sums equal to the oracle's measures of them
    keep2, descs2 = _batch(ctx, pairs, B, algo, [32, 32])
    fs = [_dev(oracle.fs(cur, ref, B, 32)[0]) for cur, ref in pairs]
    sums = torch.zeros((len(pairs), me.ME_NSUMS), dtype=torch.int64, device="cuda")
    ctx.me_estimate_eval_batch(descs2, fs, B, algo, sums)
    torch.cuda.synchronize()
    for i, ((cur, ref), (c, r, mv, sad, nsp)) in enumerate(zip(pairs, keep2)):
        got = _host(mv, sad, nsp)
        want = oracle_search(cur, ref, B, 32, algo)
        assert_same(got, want, f"fused {algo} B{B}")
        ev = oracle.evaluate(cur, ref, B, want[0], fs[i].cpu().numpy(), want[2])
        st = ctx.me_stats_from_sums(sums[i].cpu().numpy().view(np.uint64))
        for k in ("mad", "mse", "nsp", "probability"):
            assert st[k] == ev[k], k


def _batch(ctx, frames_list, B, algo, rngs):
    """frames_list: list of (cur, ref) numpy pairs.  Returns list of outputs."""
    keep, items = [], []
    for (cur, ref), R in zip(frames_list, rngs):
        h, w = cur.shape
        c, r = _dev(cur), _dev(ref)
        mv, sad, nsp = _outs(h, w, B)
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, R, mv, sad, nsp))
    descs = me.Context.frame_descs(items)
    return keep, descs


def test_batch_mixed_sizes_matches_oracle(ctx):
    pairs, rngs = [], []
    for name, seed, R in (("qcif", 2000, 16), ("cif", 2002, 16), ("qcif", 2001, 7), ("720p", 2004, 16),
                          ("cif", 2003, 5)):
        s = synth.workload_sequence(name, 3, seed=seed, max_motion=R)
        pairs += [(s[1], s[0]), (s[2], s[1])]
        rngs += [R, R]
    for algo in ALGOS:
        keep, descs = _batch(ctx, pairs, 16, algo, rngs)
        ctx.me_estimate_batch(descs, 16, algo)
        torch.cuda.synchronize()
        for (cur, ref), R, (c, r, mv, sad, nsp) in zip(pairs, rngs, keep):
            got = _host(mv, sad, nsp)
            if algo == "fs" and cur.shape[1] > 400:
                idx = np.random.default_rng(0).choice(len(got[1]), 200, replace=False)
                want = oracle.fs_blocks(cur, ref, 16, R, idx)
                got = tuple(g[idx] for g in got)
            else:
                want = oracle_search(cur, ref, 16, R, algo)
            assert_same(got, want, f"{algo} {cur.shape} R{R}")


def test_graph_replay_and_determinism(ctx, cif):
    pairs = [(cif[t], cif[t - 1]) for t in range(1, 5)]
    keep, descs = _batch(ctx, pairs, 16, "dcds", [16] * 4)
    g = ctx.me_graph_create(descs, 16, "dcds")
    try:
        results = []
        for rep in range(3):
            for (_, _, mv, sad, nsp) in keep:
                mv.fill_(-7); sad.fill_(-1); nsp.fill_(-1)
            ctx.me_graph_launch(g)
            torch.cuda.synchronize()
            results.append([_host(mv, sad, nsp) for (_, _, mv, sad, nsp) in keep])
        for rep in (1, 2):
            for a, b in zip(results[0], results[rep]):
                assert_same(a, b, "replay")
        for (cur, ref), got in zip(pairs, results[0]):
            assert_same(got, oracle.dcds(cur, ref, 16, 16), "graph vs oracle")
    finally:
        ctx.me_graph_free(g)


@pytest.mark.parametrize("algo", ["dcds", "fs"])
def test_queue_order_does_not_change_results(ctx, qcif, cif, algo):
    """The same frames in shuffled batch orders (so different CTAs take
    different tiles in a different order from the work queue): every frame's
    outputs, and for DCDS its fused evaluation sums, are byte-identical."""
    pairs = [(qcif[t], qcif[t - 1], 7) for t in range(1, 6)] + [(cif[t], cif[t - 1], 16) for t in range(1, 5)]
    keep, _ = _batch(ctx, [(c, r) for c, r, _ in pairs], 16, algo, [R for _, _, R in pairs])
    ref_out, ref_sums = None, None
    for seed in range(4):
        order = np.random.default_rng(seed).permutation(len(pairs)) if seed else np.arange(len(pairs))
        for (_, _, mv, sad, nsp) in keep:
            mv.fill_(-7); sad.fill_(-1); nsp.fill_(-1)
        items = [(keep[i][0], keep[i][1], pairs[i][2], keep[i][2], keep[i][3], keep[i][4]) for i in order]
        descs = me.Context.frame_descs(items)
        sums = None
        if algo == "dcds":
            sums = torch.zeros((len(pairs), me.ME_NSUMS), dtype=torch.int64, device="cuda")
            ctx.me_estimate_eval_batch(descs, None, 16, algo, sums)
        else:
            ctx.me_estimate_batch(descs, 16, algo)
        out = [_host(mv, sad, nsp) for (_, _, mv, sad, nsp) in keep]
        if sums is not None:
            s = sums.cpu().numpy()
            sums_by_frame = np.empty_like(s)
            sums_by_frame[order] = s
        if ref_out is None:
            ref_out = out
            ref_sums = sums_by_frame if sums is not None else None
        else:
            for a, b2 in zip(ref_out, out):
                assert_same(b2, a, f"order {seed}")
            if sums is not None:
                assert np.array_equal(sums_by_frame, ref_sums)


@pytest.fixture(scope="module")
def bench_batch():
    """The benchmark's own batch: 48 pairs of the seeded 1080p sequence
    (seed 2000), 16x16 blocks, +-16."""
    seq = synth.workload_sequence("1080p", 49, seed=2000, max_motion=16)
    return [(seq[t], seq[t - 1]) for t in range(1, len(seq))]


@pytest.fixture(scope="module")
def bench_oracle(bench_batch):
    """The oracle's DCDS and FS fields of every block of the benchmark batch."""
    from _oracle_pool import OraclePool
    pairs = [(c, r, 16) for c, r in bench_batch]
    with OraclePool() as pool:
        return {"dcds": pool.fields(pairs, 16, "dcds"), "fs": pool.fields(pairs, 16, "fs")}


def test_full_1080p_batch_every_block(ctx, bench_batch, bench_oracle):
    """The benchmark's workload through a captured batch (48 1080p pairs,
    16x16, +-16): every block of every pair bit-exact with the oracle, for
    DCDS and FS."""
    from _oracle_pool import first_difference
    pairs = bench_batch
    for algo in ("dcds", "fs"):
        keep, descs = _batch(ctx, pairs, 16, algo, [16] * len(pairs))
        g = ctx.me_graph_create(descs, 16, algo)
        ctx.me_graph_launch(g)
        torch.cuda.synchronize()
        ctx.me_graph_free(g)
        ctx.me_check_status()
        for t, ((c, r, mv, sad, nsp), want) in enumerate(zip(keep, bench_oracle[algo])):
            d = first_difference(_host(mv, sad, nsp), want)
            assert d is None, f"{algo} 1080p pair {t}: {d}"


def test_full_1080p_fused_step_every_block(ctx, bench_batch, bench_oracle):
    """The benchmark's timed step itself: the captured fused search +
    evaluation over the benchmark batch (16x16, +-16, the FS field as mv_fs).
    Every block bit-exact with the oracle's DCDS; the sums equal the separate
    evaluation kernel's on the same field, and every frame's six measures
    (Sec. IV) equal the oracle's evaluation of the oracle's fields."""
    from _oracle_pool import first_difference
    pairs = bench_batch
    n = len(pairs)
    fs_keep, fs_descs = _batch(ctx, pairs, 16, "fs", [16] * n)
    ctx.me_estimate_batch(fs_descs, 16, "fs")
    keep, descs = _batch(ctx, pairs, 16, "dcds", [16] * n)
    sums = torch.zeros((n, me.ME_NSUMS), dtype=torch.int64, device="cuda")
    fs_fields = [k[2] for k in fs_keep]
    g = ctx.me_graph_create_eval(descs, fs_fields, 16, "dcds", sums)
    try:
        for _ in range(2):  # replays refill the sums from zero
            ctx.me_graph_launch(g)
        torch.cuda.synchronize()
    finally:
        ctx.me_graph_free(g)
    ctx.me_check_status()
    for t, ((c, r, mv, sad, nsp), want) in enumerate(zip(keep, bench_oracle["dcds"])):
        d = first_difference(_host(mv, sad, nsp), want)
        assert d is None, f"fused 1080p pair {t}: {d}"
    e = me.Context.eval_descs((k[0], k[1], k[2], f, k[4]) for k, f in zip(keep, fs_fields))
    sep = torch.zeros_like(sums)
    ctx.me_eval_batch(e, 16, sep)
    torch.cuda.synchronize()
    assert torch.equal(sums, sep)
    host_sums = sums.cpu().numpy().view(np.uint64)
    for t, (cur, ref) in enumerate(pairs):
        dmv, _, dnsp = bench_oracle["dcds"][t]
        want = oracle.evaluate(cur, ref, 16, dmv, bench_oracle["fs"][t][0], dnsp)
        got = ctx.me_stats_from_sums(host_sums[t])
        for k in ("mad", "mse", "nsp", "probability"):
            assert got[k] == want[k], (t, k)
        assert abs(got["psnr"] - want["psnr"]) < 1e-9
        assert abs(got["distance"] - want["distance"]) < 1e-7  # per-block distances summed in 2^-24 units


def test_eval_matches_oracle(ctx, cif):
    B, R = 16, 7
    for t in (1, 2):
        cur, ref = cif[t], cif[t - 1]
        fs_out = oracle.fs(cur, ref, B, R)
        dc_out = oracle.dcds(cur, ref, B, R)
        want = oracle.evaluate(cur, ref, B, dc_out[0], fs_out[0], dc_out[2])
        sums = torch.zeros(me.ME_NSUMS, dtype=torch.int64, device="cuda")
        ctx.me_eval(_dev(cur), _dev(ref), B, _dev(dc_out[0]), sums, mv_fs=_dev(fs_out[0]),
                    nsp=_dev(dc_out[2].view(np.int16)))
        torch.cuda.synchronize()
        got = ctx.me_stats_from_sums(sums.cpu().numpy().view(np.uint64))
        for k in ("mad", "mse", "nsp", "probability"):
            assert got[k] == want[k], k
        assert abs(got["psnr"] - want["psnr"]) < 1e-9
        assert abs(got["distance"] - want["distance"]) < 1e-7


def test_eval_batch_per_frame(ctx, qcif):
    B, R = 16, 7
    items, wants, keep = [], [], []
    for t in range(1, 5):
        cur, ref = qcif[t], qcif[t - 1]
        mv, _, nsp = oracle.dcds(cur, ref, B, R)
        wants.append(oracle.evaluate(cur, ref, B, mv, None, nsp))
        k = (_dev(cur), _dev(ref), _dev(mv), None, _dev(nsp.view(np.int16)))
        keep.append(k)
        items.append(k)
    sums = torch.zeros((len(items), me.ME_NSUMS), dtype=torch.int64, device="cuda")
    ctx.me_eval_batch(me.Context.eval_descs(items), B, sums)
    torch.cuda.synchronize()
    arr = sums.cpu().numpy().view(np.uint64)
    for i, want in enumerate(wants):
        got = ctx.me_stats_from_sums(arr[i])
        assert got["mse"] == want["mse"] and got["nsp"] == want["nsp"] and got["mad"] == want["mad"]


def test_invalid_arguments_rejected(ctx):
    L, h = ctx.L, ctx.h
    f = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    mv, sad, nsp = _outs(64, 64, 16)
    P = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
    s = ctypes.c_void_p(0)
    ok = L.me_estimate(h, P(f), P(f), 64, 64, 16, 7, 1, P(mv), P(sad), P(nsp), s)
    assert ok == me.ME_OK
    cases = [
        (P(f), P(f), 60, 64, 16, 7, 1),   # width not a multiple of 16
        (P(f), P(f), 64, 60, 16, 7, 1),   # height not a multiple of the block
        (P(f), P(f), 64, 64, 4, 7, 1),    # block size
        (P(f), P(f), 64, 64, 16, 0, 1),   # range 0
        (P(f), P(f), 64, 64, 16, 33, 1),  # range above 32
        (P(f, 1), P(f), 32, 32, 16, 7, 1),  # misaligned frame
        (None, P(f), 64, 64, 16, 7, 1),   # null frame
        (P(f), P(f), 64, 64, 16, 7, 9),   # unknown algo
    ]
    for a in cases:
        assert L.me_estimate(h, *a, P(mv), P(sad), P(nsp), s) == me.ME_ERR_ARG, a
        assert len(L.me_last_error(h)) > 0
    assert L.me_estimate(h, P(f), P(f), 64, 64, 16, 7, 1, None, P(sad), P(nsp), s) == me.ME_ERR_ARG
    # the learned start without weights loaded into the context is an argument error
    assert L.me_estimate(h, P(f), P(f), 64, 64, 16, 7, 3, P(mv), P(sad), P(nsp), s) == me.ME_ERR_ARG
    assert b"no proposal" in L.me_last_error(h)
    assert L.me_estimate_batch(h, None, 0, 16, 1, s) == me.ME_ERR_ARG
    ctx.me_check_status()


def test_absdiff_peak(ctx):
    rates, used = ctx.me_absdiff_peak(iters=256)
    assert len(rates) == 4 and all(r > 1e12 for r in rates)
    assert 0 <= used < 4


def test_tune_keeps_parity(ctx, cif):
    cur, ref = cif[2], cif[1]
    for algo in ("dcds", "fs"):
        c, r = _dev(cur), _dev(ref)
        mv, sad, nsp = _outs(*cur.shape, 16)
        chosen = ctx.me_tune(c, r, 16, 7, algo, mv, sad, nsp)
        assert chosen >= 0
        assert_same(_host(mv, sad, nsp), oracle_search(cur, ref, 16, 7, algo), f"tuned {algo}")
        # the tuned shape is used by later calls too
        assert_same(gpu_search(ctx, cur, ref, 16, 7, algo), oracle_search(cur, ref, 16, 7, algo), algo)


# launch shapes as the tune cache stores them: tx ty threads k stages
DCDS_SHAPES = {
    "tile128_s1": "8 8 128 0 1",
    "tile128_s2": "8 8 128 0 2",
    "tile256_s1": "8 8 256 0 1",
    "tile256_s2": "8 8 256 0 2",
}


@pytest.mark.parametrize("shape", sorted(DCDS_SHAPES))
def test_every_dcds_kernel_shape(tmp_path, cif, shape):
    """The DCDS kernel in every CTA size and tile staging the tuner may
    choose gives the oracle's results; a shape is forced through the tune
    cache file of a fresh context."""
    cur, ref = cif[3], cif[2]
    h, w = cur.shape
    cases = [(16, 7, "dcds"), (8, 15, "dcds"), (16, 32, "dcds_s"), (8, 3, "dcds_s")]
    path = tmp_path / "tune.txt"
    path.write_text("".join(f"{me.ALGOS[a]} {B} {R} {w}x{h} {DCDS_SHAPES[shape]}\n" for B, R, a in cases))
    c2 = me.Context(0, tune_cache_path=str(path))
    try:
        for B, R, algo in cases:
            want = oracle_search(cur, ref, B, R, algo)
            for rep in range(3):  # repeated launches reuse the slot's queue
                assert_same(gpu_search(c2, cur, ref, B, R, algo), want, f"{shape} {algo} B{B} R{R} rep{rep}")
        c2.me_check_status()
    finally:
        c2.close()


@pytest.mark.parametrize("shape", ["tile128_s2", "tile256_s1"])
def test_dcds_shape_graph_replays(tmp_path, qcif, shape):
    """Graph replays of a forced shape: a mixed-size batch, replayed with
    the outputs cleared in between, matches the oracle every time."""
    pairs = [(qcif[t], qcif[t - 1]) for t in range(1, 4)]
    path = tmp_path / "tune.txt"
    path.write_text(f"{me.ALGOS['dcds']} 16 16 176x144 {DCDS_SHAPES[shape]}\n")
    c2 = me.Context(0, tune_cache_path=str(path))
    try:
        keep, descs = _batch(c2, pairs, 16, "dcds", [16] * len(pairs))
        g = c2.me_graph_create(descs, 16, "dcds")
        try:
            for rep in range(4):
                for (_, _, mv, sad, nsp) in keep:
                    mv.fill_(-7); sad.fill_(-1); nsp.fill_(-1)
                c2.me_graph_launch(g)
                for (cur, ref), (_, _, mv, sad, nsp) in zip(pairs, keep):
                    assert_same(_host(mv, sad, nsp), oracle.dcds(cur, ref, 16, 16), f"{shape} replay {rep}")
        finally:
            c2.me_graph_free(g)
        c2.me_check_status()
    finally:
        c2.close()


@pytest.mark.parametrize("R", [1, 7, 15, 32])
def test_fs_dual_sizes_match_oracle(ctx, cif, qcif, R):
    """One sweep gives the 16x16 and the 8x8 full searches, each bit-exact."""
    pairs = [(cif[2], cif[1]), (qcif[4], qcif[3]), (cif[4], cif[3])]
    items16, items8, keep = [], [], []
    for cur, ref in pairs:
        h, w = cur.shape
        c, r = _dev(cur), _dev(ref)
        o16 = _outs(h, w, 16)
        o8 = _outs(h, w, 8)
        keep.append((cur, ref, o16, o8))
        items16.append((c, r, R) + o16)
        items8.append((c, r, R) + o8)
    ctx.me_fs_dual_batch(me.Context.frame_descs(items16), me.Context.frame_descs(items8))
    torch.cuda.synchronize()
    ctx.me_check_status()
    for cur, ref, o16, o8 in keep:
        assert_same(_host(*o16), oracle.fs(cur, ref, 16, R), f"dual 16x16 R{R}")
        assert_same(_host(*o8), oracle.fs(cur, ref, 8, R), f"dual 8x8 R{R}")


@pytest.mark.parametrize("B,pad", [(16, 16), (8, 48)])
def test_padded_pitch(ctx, qcif, cif, B, pad):
    """Frames whose rows are wider than the image (pitch = w + pad): every
    search, the fused evaluation and the host-memory batch read only the
    image, with results bit-exact with the oracle on the unpadded frames."""
    pairs = [(qcif[2], qcif[1], 7), (cif[2], cif[1], 16), (cif[3], cif[2], 32)]

    def padded(a, device):
        h, w = a.shape
        t = torch.full((h, w + pad), 255, dtype=torch.uint8)
        t[:, :w] = torch.from_numpy(a)
        t = t.to(device) if device == "cuda" else t.pin_memory()
        return t[:, :w]

    for algo in ("dcds", "dcds_s", "fs"):
        items, keep = [], []
        for cur, ref, R in pairs:
            h, w = cur.shape
            c, r = padded(cur, "cuda"), padded(ref, "cuda")
            assert c.stride(0) == w + pad
            mv, sad, nsp = _outs(h, w, B)
            keep.append((mv, sad, nsp))
            items.append((c, r, R, mv, sad, nsp))
        ctx.me_estimate_batch(me.Context.frame_descs(items), B, algo)
        for (cur, ref, R), (mv, sad, nsp) in zip(pairs, keep):
            assert_same(_host(mv, sad, nsp), oracle_search(cur, ref, B, R, algo), f"{algo} pitch {pad}")
    # fused evaluation against the separate kernel on the same padded frames
    items, keep = [], []
    for cur, ref, R in pairs:
        h, w = cur.shape
        c, r = padded(cur, "cuda"), padded(ref, "cuda")
        mv, sad, nsp = _outs(h, w, B)
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, R, mv, sad, nsp))
    sums = torch.zeros((len(pairs), me.ME_NSUMS), dtype=torch.int64, device="cuda")
    ctx.me_estimate_eval_batch(me.Context.frame_descs(items), None, B, "dcds", sums)
    sep = torch.zeros_like(sums)
    ctx.me_eval_batch(me.Context.eval_descs((c, r, mv, None, nsp) for c, r, mv, sad, nsp in keep), B, sep)
    torch.cuda.synchronize()
    assert torch.equal(sums, sep)
    # host-memory batch from padded pinned frames
    items, keep = [], []
    for cur, ref, R in pairs:
        h, w = cur.shape
        c, r = padded(cur, "cpu"), padded(ref, "cpu")
        nb = (w // B) * (h // B)
        mv = torch.empty((nb, 2), dtype=torch.int16).pin_memory()
        sad = torch.empty((nb,), dtype=torch.int32).pin_memory()
        nsp = torch.empty((nb,), dtype=torch.int16).pin_memory()
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, R, mv, sad, nsp))
    ctx.me_estimate_host_batch(me.Context.frame_descs(items), B, "dcds", chunk=2)
    torch.cuda.synchronize()
    for (cur, ref, R), (_, _, mv, sad, nsp) in zip(pairs, keep):
        got = (mv.numpy(), sad.numpy().view(np.uint32), nsp.numpy().view(np.uint16))
        assert_same(got, oracle_search(cur, ref, B, R, "dcds"), f"host pitch {pad}")
