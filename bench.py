"""Benchmark: DCDS macroblocks/s at 1080p on GB300 (plus FS beside it).

One step = one pass of the motion-estimation hot path over one batch:
DCDS over NPAIRS independent 1920x1088 frame pairs (16x16 blocks, +-16) with
motion compensation and the sums of the six measures of Sec. IV fused into
the same persistent launch over the global tile queue, replayed from a
captured CUDA graph (the search alone and the separate evaluation kernel are
timed outside the timed region for context; their sums are checked equal).
Inputs are resident in HBM and larger than L2 (each pair has its own two
frames).  The FS field of the same batch (the "true MV" of Sec. II-C) is
computed before timing for the PSNR/distance comparison, and FS itself is
timed separately and reported under "fs".

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_, H_, B_, R_ = 1920, 1088, 16, 16
NPAIRS = 48
WORKLOAD = f"1080p {W_}x{H_} luma, 16x16 blocks, range +-16, {NPAIRS} independent frame pairs per step"
METRIC = "DCDS macroblocks/s at 1080p on 1 GB300; search pts/MB and PSNR vs FS & plain"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--pairs", type=int, default=NPAIRS)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-learned", action="store_true")
    p.add_argument("--no-workloads", action="store_true", help="skip the mixed-stream and stress context lines")
    p.add_argument("--no-tune", action="store_true", help="use the library's default launch shapes")
    return p.parse_args()


def rank_seed(rank):
    """Each rank generates its own sequence: the shards share no frame."""
    return 2000 + 7 * rank


def _frames(rank, npairs):
    """Seeded synthetic 1080p sequence; pair i = (frame i+1, frame i)."""
    from paper_0806_0689_gb300 import synth
    seq = synth.workload_sequence("1080p", npairs + 1, seed=rank_seed(rank), max_motion=R_)
    return seq


def max_over_ranks(x, dist=None, device="cpu"):
    """The slowest rank's time (all ranks receive it); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank_step, world, ms_total, steps):
    """Whole-job throughput: the units all ranks processed per step over the
    (slowest rank's) time per step.  Returns (units/s, ms per step)."""
    ms_step = ms_total / steps
    return units_per_rank_step * world / (ms_step * 1e-3), ms_step


# ---------------------------------------------------------------- CPU oracle

def _oracle_worker(args):
    seq_seed, t, reps = args
    import oracle
    from paper_0806_0689_gb300 import synth
    seq = synth.workload_sequence("1080p", t + 2, seed=seq_seed, max_motion=R_)
    cur, ref = seq[t + 1], seq[t]
    n = 0
    t0 = time.perf_counter()
    for _ in range(reps):
        mv, sad, nsp = oracle.dcds(cur, ref, B_, R_)
        oracle.evaluate(cur, ref, B_, mv, None, nsp)
        n += len(sad)
    return n, time.perf_counter() - t0


def cpu_baseline(seconds_hint=20.0):
    """Time the CPU oracle (as it stands) on a bounded sample of the same
    workload: whole 1080p pairs, DCDS + evaluation, one process per core."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    # one calibration pair to size the sample
    n, dt = _oracle_worker((2000, 0, 1))
    reps = max(1, int(seconds_hint / max(dt, 1e-3) / 4))
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(2000, i % 4, reps) for i in range(cores)])
    wall = time.perf_counter() - t0
    mbs = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return {"value": mbs / busy, "unit": "macroblocks/s", "cores": cores, "kind": "oracle",
            "one_core_value": n / dt,
            "sample": f"{cores} processes x {reps} whole 1080p pairs each (DCDS + evaluation), "
                      f"{mbs} macroblocks in {busy:.1f} s (wall {wall:.1f} s)"}


# ---------------------------------------------------------------- ncu traffic

def _kernel_rev():
    """Hash of the sources the DCDS tile kernel is built from."""
    import hashlib
    h = hashlib.sha1()
    for f in ("dcds.cu", "dcds_common.cuh", "me_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_0806_0689_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


def _profiled_traffic(npairs):
    """dram bytes (read + write) of one DCDS launch from the committed ncu
    summary, scaled to this batch; None once dcds.cu has changed since the
    counters were taken."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", "dcds_kernel_1080p.md")).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*(\d+)\s+pairs:\s*(\d+)\s+dcds_src_sha1:\s*([0-9a-f]+)", txt)
    if not m or m.group(3) != _kernel_rev():
        return None
    return int(m.group(1)) * npairs / int(m.group(2))


# ---------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.p = None
        self.dev = dev
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocked(torch, fn, seconds=1.2):
    """Run fn repeatedly for at least `seconds` (synchronising every few
    calls) while nvidia-smi samples the clocks; returns the clock record."""
    clk = Clocks(torch.cuda.current_device())
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(8):
            fn()
        torch.cuda.synchronize()
    rec = clk.stop()
    rec["window_s"] = time.perf_counter() - t0
    return rec


# ---------------------------------------------------------------- learned proposal

def other_workloads(ctx, me, torch, dev, hbm_peak, sad_peak):
    """Context beside the headline: plain DCDS and FS on the mixed-stream
    batch (8 streams: 2 QCIF, 2 CIF, 2 1280x720, 2 1920x1088, 30 pairs each,
    16x16, +-16; one launch each) and on a 12-pair sample of the stress
    workload (3840x2160, 8x8, +-32, motion scales 6/3), each with the
    library's tuner run first, as a caller would."""
    from paper_0806_0689_gb300 import synth
    out = {}
    cases = {
        "mixed_streams_8x30_pairs_16x16_r16": (16, 16, [
            (name, 2000 + k, 30, (2.0, 1.0)) for k, name in
            enumerate(("qcif", "qcif", "cif", "cif", "720p", "720p", "1080p", "1080p"))]),
        "stress_2160p_8x8_r32_12_pairs": (8, 32, [("2160p", 4000, 12, (6.0, 3.0))]),
    }
    for key, (B, R, streams) in cases.items():
        seqs = [synth.workload_sequence(n, np_ + 1, seed=sd, max_motion=min(R, 16) if B == 16 else R, scale=sc)
                for n, sd, np_, sc in streams]
        frames = [(sq[t + 1], sq[t]) for t in range(max(x[2] for x in streams)) for sq in seqs if t + 1 < len(sq)]
        items, keep = [], []
        nblocks, fbytes, absdiff_fs = 0, 0, 0.0
        for cur, ref in frames:
            h, w = cur.shape
            nb = (w // B) * (h // B)
            c, r = torch.from_numpy(cur).to(dev), torch.from_numpy(ref).to(dev)
            mv = torch.empty((nb, 2), dtype=torch.int16, device=dev)
            sad = torch.empty((nb,), dtype=torch.int32, device=dev)
            nsp = torch.empty((nb,), dtype=torch.int16, device=dev)
            keep.append((c, r, mv, sad, nsp))
            items.append((c, r, R, mv, sad, nsp))
            nblocks += nb
            fbytes += 2 * w * h
        d = me.Context.frame_descs(items)
        res = {"pairs": len(frames), "blocks_per_launch": nblocks, "input_bytes": fbytes}
        for algo in ("dcds", "fs"):
            ctx.me_tune_batch(d, B, algo)
            g = ctx.me_graph_create(d, B, algo)
            for _ in range(3):
                ctx.me_graph_launch(g)
            torch.cuda.synchronize()
            reps = 20 if algo == "dcds" else 3
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ctx.me_graph_launch(g)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            ctx.me_graph_free(g)
            nsp_sum = float(sum(int(x[4].cpu().numpy().view(np.uint16).astype(np.int64).sum()) for x in keep))
            r_ = {"launch_ms": ms, "blocks_per_s": nblocks / (ms * 1e-3), "nsp_per_block": nsp_sum / nblocks,
                  "absdiff_frac_of_sad_rate": nsp_sum * B * B / (ms * 1e-3) / sad_peak}
            if algo == "dcds":
                alg = fbytes + nblocks * 10
                r_["hbm_frac"] = alg / (ms * 1e-3) / 1e9 / hbm_peak
            res[algo] = r_
        out[key] = res
        del items, keep
    return out


def cnn_flop_per_block():
    """Forward FLOPs of the start proposal per 16x16 region (2 per
    multiply-add): four 3x3 stride-2 convolutions (2 -> 32 channels at 16x16
    outputs, then 32 -> 32 at 8x8, 4x4 and 2x2) and the linear head (128
    conv features + 8 neighbour scalars -> 68 logits)."""
    conv = sum(2 * o * o * 32 * cin * 9 for o, cin in ((16, 2), (8, 32), (4, 32), (2, 32)))
    return conv + 2 * (128 + 8) * 68


def _descs_for(me, torch, dev, pairs, R, B):
    keep, items = [], []
    for cur, ref in pairs:
        h, w = cur.shape
        nb = (w // B) * (h // B)
        c, r = torch.from_numpy(cur).to(dev), torch.from_numpy(ref).to(dev)
        m = torch.zeros((nb, 2), dtype=torch.int16, device=dev)
        sd_ = torch.zeros(nb, dtype=torch.int32, device=dev)
        ns = torch.zeros(nb, dtype=torch.int16, device=dev)
        keep.append((c, r, m, sd_, ns))
        items.append((c, r, R, m, sd_, ns))
    return keep, me.Context.frame_descs(items)


def _quality(ctx, me, torch, keep, B, mv_fs=None):
    """Mean NSP, PSNR and FS-equal probability of the fields in `keep` (the
    Sec. IV measures from this library's evaluation kernel)."""
    sums = torch.zeros((len(keep), me.ME_NSUMS), dtype=torch.int64, device=keep[0][0].device)
    ev = me.Context.eval_descs((c, r, m, None if mv_fs is None else mv_fs[i], ns)
                               for i, (c, r, m, sd_, ns) in enumerate(keep))
    ctx.me_eval_batch(ev, B, sums)
    torch.cuda.synchronize()
    st = [ctx.me_stats_from_sums(x) for x in sums.cpu().numpy().view(np.uint64)]
    out = {"nsp_per_block": float(np.mean([x["nsp"] for x in st])), "psnr_db": float(np.mean([x["psnr"] for x in st]))}
    if mv_fs is not None:
        out["probability_fs"] = float(np.mean([x["probability"] for x in st]))
    return out


def _timed_call(torch, fn, reps=3):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _compare(ctx, me, torch, dev, prop, pairs, R, B, with_fs=False):
    """Plain DCDS, the neighbour-median control and the learned start on the
    same pairs: blocks/s of one batched call each, NSP and PSNR."""
    nblocks = sum((c.shape[0] // B) * (c.shape[1] // B) for c, _ in pairs)
    out = {"pairs": len(pairs), "blocks": nblocks}
    mv_fs = None
    if with_fs:
        kf, df = _descs_for(me, torch, dev, pairs, R, B)
        ms = _timed_call(torch, lambda: ctx.me_estimate_batch(df, B, "fs"), reps=1)
        mv_fs = [k[2] for k in kf]
        out["fs"] = dict(_quality(ctx, me, torch, kf, B), blocks_per_s=nblocks / (ms * 1e-3), ms=ms)
    for kind in ("plain", "median", "learned"):
        keep, d = _descs_for(me, torch, dev, pairs, R, B)
        if kind == "plain":
            call = lambda: ctx.me_estimate_batch(d, B, "dcds")
        elif kind == "median":
            call = lambda: ctx.me_estimate_median_batch(d, block=B)
        else:
            call = lambda: ctx.me_estimate_learned_batch(prop, d, block=B)
        ms = _timed_call(torch, call)
        out[kind] = dict(_quality(ctx, me, torch, keep, B, mv_fs), blocks_per_s=nblocks / (ms * 1e-3), ms=ms)
    out["learned_minus_median"] = {"nsp": out["learned"]["nsp_per_block"] - out["median"]["nsp_per_block"],
                                   "psnr_db": out["learned"]["psnr_db"] - out["median"]["psnr_db"]}
    return out


def learned_leg(ctx, me, torch, dev, curs, refs, mv_plain, mv_fs, st_plain, nb, npairs,
                tensor_peak=None, train_seqs=400, steps=6000):
    """The learned start proposal (not in the paper), per the task's
    learned-proposal workload: trained on full-search fields this library
    computes on 2,000 synthetic CIF pairs (seeds from 100000, disjoint from
    every evaluation seed; half with the motion scales 2/1, half 6/3), then
    compared with plain DCDS and the neighbour-median control on held-out
    CIF and 720p pairs, on the benchmark batch, and on the stress workload
    (3840x2160, 8x8 blocks sharing their 16x16 region's proposal, +-32)."""
    from paper_0806_0689_gb300 import synth
    t0 = time.perf_counter()
    train = []
    for sd in range(train_seqs):
        scale = (6.0, 3.0) if sd % 2 else (2.0, 1.0)
        s = synth.workload_sequence("cif", 6, seed=100000 + sd, max_motion=R_, scale=scale)
        train += [(s[t], s[t - 1]) for t in range(1, 6)]
    keep_t, descs = _descs_for(me, torch, dev, train, R_, B_)
    ctx.me_estimate_batch(descs, B_, "fs")  # labels: this library's full search
    torch.cuda.synchronize()
    t_labels = time.perf_counter() - t0
    prop = ctx.me_proposal_create()
    ctx.me_proposal_set_params(prop, me.proposal_init_params(0))
    t1 = time.perf_counter()
    losses = me.train_proposal(ctx, prop, descs, steps=steps, lr=2e-3, pairs_per_step=4, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del keep_t, descs
    # the CNN forward alone (features, trunk, head) on one 1080p pair, timed by
    # the library's own per-call events, against the sustained bf16 tensor peak
    logits = torch.empty((nb, me.ME_PROPOSAL_NLOGITS), dtype=torch.float32, device=dev)
    sad_t = torch.empty((nb,), dtype=torch.int32, device=dev)
    d_one = me.Context.frame_descs([(curs[0], refs[0], R_, mv_plain[0], sad_t, None)])
    ctx.me_set_tracing(True)
    tf = []
    for rep in range(11):
        ctx.me_proposal_logits(prop, d_one, logits)
        if rep > 0:
            tf.append(ctx.me_last_call_ms())
    ctx.me_set_tracing(False)
    fwd_ms = float(np.median(tf))
    fwd_tflops = cnn_flop_per_block() * nb / (fwd_ms * 1e-3) / 1e12
    cnn_forward = {"blocks": nb, "ms": fwd_ms, "flop_per_block": cnn_flop_per_block(),
                   "bound": "tensor", "achieved": fwd_tflops, "unit": "TFLOP/s",
                   "peak": tensor_peak, "frac": fwd_tflops / tensor_peak if tensor_peak else None,
                   "peak_source": "bf16 sustained of measured" if tensor_peak else None,
                   "call": "me_proposal_logits on one 1080p pair (median of 10, me_last_call_ms)"}
    # the benchmark batch: learned and median against plain DCDS, beside the FS field
    mv_l = torch.empty_like(mv_plain)
    sad_l = torch.empty((npairs, nb), dtype=torch.int32, device=dev)
    nsp_l = torch.empty((npairs, nb), dtype=torch.int16, device=dev)
    d_l = me.Context.frame_descs((curs[i], refs[i], R_, mv_l[i], sad_l[i], nsp_l[i]) for i in range(npairs))
    keep_l = [(curs[i], refs[i], mv_l[i], sad_l[i], nsp_l[i]) for i in range(npairs)]
    fs_list = [mv_fs[i] for i in range(npairs)]
    ms = _timed_call(torch, lambda: ctx.me_estimate_learned_batch(prop, d_l))
    q_l = _quality(ctx, me, torch, keep_l, B_, fs_list)
    ms_m = _timed_call(torch, lambda: ctx.me_estimate_median_batch(d_l))
    q_m = _quality(ctx, me, torch, keep_l, B_, fs_list)
    mean = lambda rows, k: float(np.mean([r[k] for r in rows]))
    bench_batch = {"macroblocks_per_s": npairs * nb / (ms * 1e-3), "ms_per_batch": ms,
                   "nsp_per_mb": q_l["nsp_per_block"], "psnr_db": q_l["psnr_db"],
                   "probability_fs": q_l["probability_fs"],
                   "plain_nsp_per_mb": mean(st_plain, "nsp"), "plain_psnr_db": mean(st_plain, "psnr"),
                   "psnr_minus_plain_db": q_l["psnr_db"] - mean(st_plain, "psnr"),
                   "median_start_control": {"macroblocks_per_s": npairs * nb / (ms_m * 1e-3), "ms_per_batch": ms_m,
                                            "nsp_per_mb": q_m["nsp_per_block"], "psnr_db": q_m["psnr_db"],
                                            "probability_fs": q_m["probability_fs"]}}
    # held-out CIF and 720p pairs (the learned-proposal workload's evaluation)
    held = {}
    for name, nfr, seeds, scale in (("cif", 4, range(5000, 5010), (6.0, 3.0)), ("cif", 4, range(5000, 5010), (2.0, 1.0)),
                                    ("720p", 3, range(5100, 5104), (6.0, 3.0)), ("720p", 3, range(5100, 5104), (2.0, 1.0))):
        pairs = []
        for sd in seeds:
            s = synth.workload_sequence(name, nfr, seed=sd, max_motion=R_, scale=scale)
            pairs += [(s[t], s[t - 1]) for t in range(1, nfr)]
        held[f"{name}_scales_{scale[0]:g}_{scale[1]:g}"] = _compare(ctx, me, torch, dev, prop, pairs, R_, B_)
    # the stress workload: 12 pairs of 3840x2160, 8x8 blocks, +-32, scales 6/3
    s = synth.workload_sequence("2160p", 13, seed=4000, max_motion=32, scale=(6.0, 3.0))
    stress = _compare(ctx, me, torch, dev, prop, [(s[t + 1], s[t]) for t in range(12)], 32, 8, with_fs=True)
    ctx.me_proposal_free(prop)
    return dict(bench_batch,
                training={"pairs": len(train), "steps": steps, "pairs_per_step": 4, "lr": 2e-3,
                          "first_loss": float(np.mean(losses[:20])), "final_loss": float(np.mean(losses[-50:])),
                          "label_seconds": t_labels, "train_seconds": t_train,
                          "labels": "full-search fields from this library (CIF, seeds >= 100000, scales 2/1 and 6/3)",
                          "call": "me_proposal_train (the loop in the library)"},
                cnn_forward=cnn_forward, held_out=held, stress_2160p_8x8_r32_12_pairs=stress)


# ---------------------------------------------------------------- reference arm

_REF_PAIR = None


def _ref_init(seed, t):
    """Pool initialiser of the reference arm: each process holds one pair."""
    global _REF_PAIR
    from paper_0806_0689_gb300 import synth
    seq = synth.workload_sequence("1080p", t + 2, seed=seed, max_motion=R_)
    _REF_PAIR = (seq[t + 1], seq[t])


def _ref_step(_):
    """One pair of the workload through the oracle: DCDS, then the Sec. IV measures."""
    import oracle
    cur, ref = _REF_PAIR
    mv, sad, nsp = oracle.dcds(cur, ref, B_, R_)
    oracle.evaluate(cur, ref, B_, mv, None, nsp)
    return len(sad)


def run_reference(a, rank, world):
    """The reference arm: the CPU oracle, as it stands, on the host cores.
    Rank 0 alone runs and prints.  Each step is a bounded sample of the
    workload: one whole 1080p pair per core, searched and evaluated."""
    if rank != 0:
        return None
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    # one single-process pool per core, each holding its own pair (pairs 0-3 of the sequence, in turn)
    pools = [ctx.Pool(1, initializer=_ref_init, initargs=(2000, i % 4)) for i in range(cores)]

    def one_step():
        return sum(r.get() for r in [p.apply_async(_ref_step, (0,)) for p in pools])
    blocks, t_total = 0, 0.0
    try:
        for _ in range(max(0, a.warmup)):
            one_step()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            blocks += one_step()
        t_total = time.perf_counter() - t0
    finally:
        for p in pools:
            p.terminate()
    value = blocks / t_total
    ms_step = t_total / max(a.steps, 1) * 1e3
    cb = {"value": value, "unit": "macroblocks/s", "cores": cores, "kind": "oracle",
          "sample": f"each step: {cores} whole 1080p pairs (one per core), DCDS + evaluation; "
                    f"{a.steps} steps, {blocks} macroblocks in {t_total:.1f} s"}
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "macroblocks/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic (seeded luma video generator; the paper's sequences are not available)",
            "config": {"workload": WORKLOAD, "block": B_, "range": R_},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "macroblocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# ---------------------------------------------------------------- our arm

def main():
    a = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)

    # the oracle's process pool is started before the first CUDA call
    cb = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline()

    import torch
    from paper_0806_0689_gb300 import me

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    npairs = a.pairs
    seq = _frames(rank, npairs)
    ctx = me.Context(local)
    nbx, nby = W_ // B_, H_ // B_
    nb = nbx * nby
    dev = torch.device("cuda", local)
    # each pair owns its two frames: no input is shared between pairs
    curs = [torch.from_numpy(seq[i + 1]).to(dev) for i in range(npairs)]
    refs = [torch.from_numpy(seq[i]).to(dev) for i in range(npairs)]
    mv = torch.empty((npairs, nb, 2), dtype=torch.int16, device=dev)
    sad = torch.empty((npairs, nb), dtype=torch.int32, device=dev)
    nsp = torch.empty((npairs, nb), dtype=torch.int16, device=dev)
    mv_fs = torch.empty_like(mv)
    sad_fs = torch.empty_like(sad)
    nsp_fs = torch.empty_like(nsp)
    sums = torch.zeros((npairs, me.ME_NSUMS), dtype=torch.int64, device=dev)
    sums_fs = torch.zeros_like(sums)

    d_dcds = me.Context.frame_descs((curs[i], refs[i], R_, mv[i], sad[i], nsp[i]) for i in range(npairs))
    d_fs = me.Context.frame_descs((curs[i], refs[i], R_, mv_fs[i], sad_fs[i], nsp_fs[i]) for i in range(npairs))
    e_dcds = me.Context.eval_descs((curs[i], refs[i], mv[i], mv_fs[i], nsp[i]) for i in range(npairs))
    e_fs = me.Context.eval_descs((curs[i], refs[i], mv_fs[i], None, nsp_fs[i]) for i in range(npairs))
    # launch shapes picked by the library's tuner on this batch (outputs are recomputed below)
    tuned = None
    if not a.no_tune:
        tuned = {"dcds": ctx.me_tune_batch(d_dcds, B_, "dcds"), "fs": ctx.me_tune_batch(d_fs, B_, "fs")}
    # one step = DCDS over the batch with the Sec. IV measures fused in (one kernel)
    fs_list = [mv_fs[i] for i in range(npairs)]
    g_step = ctx.me_graph_create_eval(d_dcds, fs_list, B_, "dcds", sums)
    g_dcds = ctx.me_graph_create(d_dcds, B_, "dcds")
    g_fs = ctx.me_graph_create(d_fs, B_, "fs")
    stream = torch.cuda.current_stream()

    # FS reference field (the "true MV"), then its quality
    ctx.me_graph_launch(g_fs)
    ctx.me_eval_batch(e_fs, B_, sums_fs)
    torch.cuda.synchronize()

    def step():
        ctx.me_graph_launch(g_step)

    for _ in range(max(3, a.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, events on the launching stream ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # the clock sampler runs across the timed steps: started a little before
    # them (the same step runs meanwhile, untimed) and kept on afterwards, so
    # that its window covers at least 1.2 s of this load
    clk = Clocks(local)
    w0 = time.perf_counter()
    while time.perf_counter() - w0 < 0.3:
        for _ in range(20):
            ctx.me_graph_launch(g_step)
        torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(a.steps):
        e0, e1 = ev[i]
        e0.record(stream)
        ctx.me_graph_launch(g_step)
        e1.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    while time.perf_counter() - w0 < 1.2:
        for _ in range(20):
            ctx.me_graph_launch(g_step)
        torch.cuda.synchronize()
    clocks = clk.stop()
    clocks["window_s"] = time.perf_counter() - w0
    clocks["window"] = "the timed steps plus untimed repeats of the same step before and after them"
    if dist:
        dist.barrier()
    ms_total = t_start.elapsed_time(t_end)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]

    # context, outside the timed region: the search alone and the separate evaluation pass
    def _time(fn, reps=20):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    search_only_ms = _time(lambda: ctx.me_graph_launch(g_dcds))
    # L2 check: the same step over three copies of the inputs in turn (three
    # times the bytes between reuses of any address), against one set
    rot_sets, rot_graphs = [], [g_step]
    for _ in range(2):
        c2, r2 = [x.clone() for x in curs], [x.clone() for x in refs]
        d2 = me.Context.frame_descs((c2[i], r2[i], R_, mv[i], sad[i], nsp[i]) for i in range(npairs))
        rot_sets.append((c2, r2))
        rot_graphs.append(ctx.me_graph_create_eval(d2, fs_list, B_, "dcds", sums))
    rot_i = [0]

    def _rot():
        ctx.me_graph_launch(rot_graphs[rot_i[0] % 3])
        rot_i[0] += 1
    rot_ms = _time(_rot, reps=60)
    single_ms = _time(lambda: ctx.me_graph_launch(g_step), reps=60)
    for g in rot_graphs[1:]:
        ctx.me_graph_free(g)
    del rot_sets
    l2_check = {"sets": 3, "bytes_between_reuses": 3 * 2 * npairs * W_ * H_, "ms_per_step": rot_ms,
                "one_set_ms_per_step": single_ms}
    sums_sep = torch.zeros_like(sums)
    unfused_eval_ms = _time(lambda: ctx.me_eval_batch(e_dcds, B_, sums_sep))
    ctx.me_graph_launch(g_step)
    torch.cuda.synchronize()
    assert torch.equal(sums_sep, sums), "fused and separate evaluation sums differ"
    ms_total = max_over_ranks(ms_total, dist, dev)
    mbs_step = npairs * nb
    value, ms_step = job_value(mbs_step, world, ms_total, a.steps)

    # ---- quality of the last step (identical every step) ----
    s_d = sums.cpu().numpy().view(np.uint64)
    s_f = sums_fs.cpu().numpy().view(np.uint64)
    st_d = [ctx.me_stats_from_sums(s_d[i]) for i in range(npairs)]
    st_f = [ctx.me_stats_from_sums(s_f[i]) for i in range(npairs)]
    mean = lambda rows, k: float(np.mean([r[k] for r in rows]))

    # ---- DCDS^S (Sec. IV-C) on the same batch, fused the same way: Table X's comparison ----
    mv_s, sad_s, nsp_s = torch.empty_like(mv), torch.empty_like(sad), torch.empty_like(nsp)
    sums_s = torch.zeros_like(sums)
    d_s = me.Context.frame_descs((curs[i], refs[i], R_, mv_s[i], sad_s[i], nsp_s[i]) for i in range(npairs))
    g_s = ctx.me_graph_create_eval(d_s, fs_list, B_, "dcds_s", sums_s)
    simpl_ms = _time(lambda: ctx.me_graph_launch(g_s))
    ctx.me_graph_free(g_s)
    s_s = sums_s.cpu().numpy().view(np.uint64)
    st_s = [ctx.me_stats_from_sums(s_s[i]) for i in range(npairs)]
    simpl_line = {"launch_ms": simpl_ms, "macroblocks_per_s": mbs_step / (simpl_ms * 1e-3),
                  "nsp_per_mb": mean(st_s, "nsp"), "psnr_db": mean(st_s, "psnr"),
                  "nsp_minus_dcds": mean(st_s, "nsp") - mean(st_d, "nsp"),
                  "psnr_minus_dcds_db": mean(st_s, "psnr") - mean(st_d, "psnr"),
                  "paper_table_x": "NSP -0.16 to -0.36, PSNR -0.014 to -0.364 dB on its sequences"}

    # ---- Sec. II-C statistics of the FS field (the directional model's inputs) ----
    from paper_0806_0689_gb300 import mvp
    mvp_counts = torch.zeros(35 * (2 * R_ + 1) ** 2, dtype=torch.int64, device=dev)
    ctx.me_mvp_stats(d_fs, R_, mvp_counts)
    torch.cuda.synchronize()
    hist, _, _ = mvp.unpack(mvp_counts.cpu().numpy(), R_)
    P = mvp.probabilities(hist)
    ax = mvp.axes_1d(P)
    mvp_line = {"regions": mvp.regions(P),
                "horizontal_axis_share": float(ax["Bx"].sum() - P[R_, R_]),
                "vertical_axis_share": float(ax["By"].sum() - P[R_, R_]),
                "var_x": mvp.moments(ax["Ax"])[1], "var_y": mvp.moments(ax["Ay"])[1],
                "paper_regions": {"square5": 0.8745, "diamond5": 0.8557, "cross5": 0.8315, "square3": 0.7899,
                                  "hcsp": 0.8248}}

    # ---- FS timed on its own (same batch) ----
    fs_ms = []
    for _ in range(3):
        ctx.me_graph_launch(g_fs)
    torch.cuda.synchronize()
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.me_graph_launch(g_fs)
        e1.record(stream)
        torch.cuda.synchronize()
        fs_ms.append(e0.elapsed_time(e1))

    # ---- both block sizes in one full-search sweep (8x8 outputs of the same batch) ----
    nb8 = 4 * nb
    mv8 = torch.empty((npairs, nb8, 2), dtype=torch.int16, device=dev)
    sad8 = torch.empty((npairs, nb8), dtype=torch.int32, device=dev)
    nsp8 = torch.empty((npairs, nb8), dtype=torch.int16, device=dev)
    d8 = me.Context.frame_descs((curs[i], refs[i], R_, mv8[i], sad8[i], nsp8[i]) for i in range(npairs))

    def _time2(fn, reps=3):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    dual_ms = _time2(lambda: ctx.me_fs_dual_batch(d_fs, d8))
    fs8_ms = _time2(lambda: ctx.me_estimate_batch(d8, 8, "fs"))
    fs_dual = {"launch_ms": dual_ms, "fs16_ms": float(np.median(fs_ms)), "fs8_ms": fs8_ms,
               "speedup_vs_two_searches": (float(np.median(fs_ms)) + fs8_ms) / dual_ms}

    # ---- end to end through the C-ABI with host buffers ----
    # me_estimate_host_batch uploads the frames (and the FS fields the sums
    # need) from pinned host memory chunk by chunk, searches each chunk while
    # the next uploads, and copies MV, SAD, NSP and the sums back.
    h_cur = torch.from_numpy(np.stack(seq[1:npairs + 1])).pin_memory()
    h_ref = torch.from_numpy(np.stack(seq[0:npairs])).pin_memory()
    h_fs = mv_fs.cpu().pin_memory()
    h_fs_list = [h_fs[i] for i in range(npairs)]
    h_mv = torch.empty((npairs, nb, 2), dtype=torch.int16).pin_memory()
    h_sad = torch.empty((npairs, nb), dtype=torch.int32).pin_memory()
    h_nsp = torch.empty((npairs, nb), dtype=torch.int16).pin_memory()
    h_sums = torch.empty((npairs, me.ME_NSUMS), dtype=torch.int64).pin_memory()
    hd = me.Context.frame_descs((h_cur[i], h_ref[i], R_, h_mv[i], h_sad[i], h_nsp[i]) for i in range(npairs))

    stream_b = torch.cuda.Stream(device=dev)

    def _e2e_ms(descs, chunk, k, two_streams=True):
        """Steps issued on two streams in turn (the library alternates two
        staging sets, so one step's uploads run while the previous step's
        last chunk is searched), or all on one stream."""
        streams = (stream, stream_b) if two_streams else (stream,)
        step = lambda i: ctx.me_estimate_host_batch(descs, B_, "dcds", mv_fs=h_fs_list, sums=h_sums, chunk=chunk,
                                                    stream=streams[i % len(streams)])
        for i in range(4):
            step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stream_b.wait_event(e0)
        for i in range(k):
            step(i)
        eb = torch.cuda.Event()
        eb.record(stream_b)
        stream.wait_event(eb)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    # the host link's own rate: one pinned 100 MB upload, timed alone
    d_tmp = torch.empty(h_cur.shape, dtype=torch.uint8, device=dev)
    d_tmp.copy_(h_cur, non_blocking=True)
    torch.cuda.synchronize()
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    for _ in range(3):
        d_tmp.copy_(h_cur, non_blocking=True)
    l1.record(stream)
    torch.cuda.synchronize()
    link_gbs = 3 * h_cur.numel() / (l0.elapsed_time(l1) * 1e-3) / 1e9
    del d_tmp

    k2 = max(6, min(50, a.steps // 4))
    chunk_sweep = {str(ch): _e2e_ms(hd, ch, 6) for ch in (npairs, npairs // 2, npairs // 4, npairs // 8)
                   if ch >= 1}
    e2e_ms = _e2e_ms(hd, 0, k2)
    e2e_one_stream_ms = _e2e_ms(hd, 0, k2, two_streams=False)
    h2d = 2 * npairs * H_ * W_ + npairs * nb * 4
    d2h = npairs * nb * (4 + 4 + 2) + npairs * me.ME_NSUMS * 8
    assert np.array_equal(h_mv.numpy(), mv.cpu().numpy()), "host-batch field differs from the device call"
    assert np.array_equal(h_sums.numpy(), sums.cpu().numpy()), "host-batch sums differ from the device call"
    # the same pairs passed as one sequence: each frame is uploaded once
    h_seq = torch.from_numpy(np.stack(seq[:npairs + 1])).pin_memory()
    hs = me.Context.frame_descs((h_seq[i + 1], h_seq[i], R_, h_mv[i], h_sad[i], h_nsp[i]) for i in range(npairs))
    seq_ms = _e2e_ms(hs, 0, k2)
    assert np.array_equal(h_mv.numpy(), mv.cpu().numpy()), "sequence host-batch field differs"
    e2e_seq = {"value": mbs_step * world / (seq_ms * 1e-3), "unit": "macroblocks/s",
               "h2d_bytes_per_step": (npairs + 1) * H_ * W_ + npairs * nb * 4, "d2h_bytes_per_step": d2h,
               "ms_per_step": seq_ms,
               "input": f"the same {npairs} pairs passed as one {npairs + 1}-frame host sequence "
                        "(ref of pair i+1 = cur of pair i, uploaded once)"}

    # ---- roofline of the dominant kernel (DCDS) ----
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dcds_launch_ms = float(np.mean(step_ms))  # average launch duration over the timed steps
    # frames once, MV/SAD/NSP out, the FS field in, eight sums out
    alg_bytes = npairs * (2 * W_ * H_ + nb * 10 + nb * 4 + me.ME_NSUMS * 8)
    achieved = alg_bytes / (dcds_launch_ms * 1e-3) / 1e9
    rates, used = ctx.me_absdiff_peak(iters=4096)
    sad_peak = max(rates)
    clk_absdiff = clocked(torch, lambda: ctx.me_absdiff_peak(iters=4096))
    clk_fs = clocked(torch, lambda: ctx.me_graph_launch(g_fs))
    nsp_mean = mean(st_d, "nsp")
    fs_launch_ms = float(np.median(fs_ms))
    fs_absdiff = float(np.sum(nsp_fs.cpu().numpy().view(np.uint16).astype(np.float64))) * B_ * B_
    dcds_absdiff = nsp_mean * nb * npairs * B_ * B_
    traffic = _profiled_traffic(npairs)

    line = {
        "metric": METRIC,
        "value": value, "unit": "macroblocks/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8", "data": "synthetic (seeded luma video generator; the paper's sequences are not available)",
        "config": {"workload": WORKLOAD, "block": B_, "range": R_, "pairs_per_step": npairs,
                   "macroblocks_per_step": mbs_step, "parallelism": f"replicas x{world} (no collective)",
                   "l2": f"inputs {2 * npairs * W_ * H_ / 1e6:.0f} MB per step > 129 MB L2; no flush"},
        "quality": {"dcds_nsp_per_mb": nsp_mean, "dcds_psnr_db": mean(st_d, "psnr"),
                    "fs_psnr_db": mean(st_f, "psnr"), "fs_nsp_per_mb": mean(st_f, "nsp"),
                    "dcds_mad": mean(st_d, "mad"), "fs_mad": mean(st_f, "mad"),
                    "dcds_mse": mean(st_d, "mse"), "fs_mse": mean(st_f, "mse"),
                    "dcds_distance_to_fs": mean(st_d, "distance"),
                    "dcds_probability_fs": mean(st_d, "probability")},
        "roofline": {"kernel": "dcds_kernel", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                     "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_source": peak_src, "launch_ms": dcds_launch_ms,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "sad_bound_frac": (dcds_absdiff / (dcds_launch_ms * 1e-3)) / sad_peak},
        "fs": {"macroblocks_per_s": mbs_step / (fs_launch_ms * 1e-3), "launch_ms": fs_launch_ms,
               "roofline": {"bound": "alu", "achieved": fs_absdiff / (fs_launch_ms * 1e-3) / 1e12,
                            "peak": sad_peak / 1e12, "unit": "Tabsdiff/s",
                            "frac": fs_absdiff / (fs_launch_ms * 1e-3) / sad_peak,
                            "peak_source": "measured byte-absdiff microbenchmark (me_absdiff_peak)"}},
        "fs_two_sizes_one_sweep": fs_dual,
        "absdiff_peak_per_s": {"variants": rates, "used": used},
        "mvp_statistics_fs_field": mvp_line,
        "dcds_s": simpl_line,
        "tuned_shape_index": tuned,
        "step_kernels": "dcds_kernel with the Sec. IV sums fused (one launch per step)",
        "search_only_ms": search_only_ms, "unfused_eval_ms": unfused_eval_ms,
        "l2_rotation_check": l2_check,
        "e2e": {"value": mbs_step * world / (e2e_ms * 1e-3), "unit": "macroblocks/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": "me_estimate_host_batch (pinned host frames, FS fields and outputs; fused sums; "
                        "default chunk; steps on two streams in turn)",
                "one_stream_ms_per_step": e2e_one_stream_ms, "chunk_sweep_ms": chunk_sweep,
                "host_link_gbs": link_gbs, "host_link_floor_ms": h2d / (link_gbs * 1e9) * 1e3},
        "e2e_sequence": e2e_seq,
        "gpu_launches": a.steps,
        "clocks": clocks,
        "clock_normalised": {
            "note": "time x the median SM clock sampled while that work ran (kilocycles), and rates per cycle",
            "dcds_step_kcycles": dcds_launch_ms * clocks["sm_mhz"] if clocks.get("sm_mhz") else None,
            "fs_launch_kcycles": fs_launch_ms * clk_fs["sm_mhz"] if clk_fs.get("sm_mhz") else None,
            "absdiff_peak_per_cycle_per_sm": (sad_peak / (clk_absdiff["sm_mhz"] * 1e6) /
                                              torch.cuda.get_device_properties(dev).multi_processor_count
                                              if clk_absdiff.get("sm_mhz") else None),
            "clocks_fs": clk_fs, "clocks_absdiff": clk_absdiff},
    }
    if cb is not None:
        line["cpu_baseline"] = cb
    if not a.no_learned:
        line["learned"] = learned_leg(ctx, me, torch, dev, curs, refs, mv, mv_fs, st_d, nb, npairs,
                                      tensor_peak=peaks.get("bf16_tflops_sustained"))
    if not a.no_workloads:
        line["other_workloads"] = other_workloads(ctx, me, torch, dev, hbm_peak, sad_peak)
    ctx.me_graph_free(g_step)
    ctx.me_graph_free(g_dcds)
    ctx.me_graph_free(g_fs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
