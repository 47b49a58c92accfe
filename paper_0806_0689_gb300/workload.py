"""Run one search of the library over one of the seeded synthetic workloads,
a few times in a row -- the command the profiles' ncu captures run.

    python -m paper_0806_0689_gb300.workload --workload cif --block 16 --range 7 --algo dcds --pairs 99
    python -m paper_0806_0689_gb300.workload --workload 2160p --block 8 --range 32 --algo dcds --pairs 12
    python -m paper_0806_0689_gb300.workload --workload 2160p --block 8 --range 32 --algo learned --pairs 4

Workloads are those of synth.WORKLOADS (seed 1000 for CIF as in the CIF
workload, 4000 with motion scales 6/3 for 2160p as in the stress workload,
2000 otherwise).  --algo: fs, dcds, dcds_s, eval (DCDS with the Sec. IV
measures fused, against the FS field), median or learned (an untrained
network: the cost of the learned start does not depend on its weights).
Every call runs --reps times on the current stream; the line printed at the
end gives the median time of one call (CUDA events around it, host work
included).
"""
from __future__ import annotations

import argparse

from . import me, synth

SEEDS = {"cif": 1000, "2160p": 4000}


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="cif", choices=sorted(synth.WORKLOADS))
    p.add_argument("--block", type=int, default=16, choices=(8, 16))
    p.add_argument("--range", type=int, default=7)
    p.add_argument("--algo", default="dcds", choices=("fs", "dcds", "dcds_s", "eval", "median", "learned"))
    p.add_argument("--pairs", type=int, default=8)
    p.add_argument("--reps", type=int, default=4)
    a = p.parse_args(argv)
    import torch

    scale = (6.0, 3.0) if a.workload == "2160p" else (2.0, 1.0)
    seq = synth.workload_sequence(a.workload, a.pairs + 1, seed=SEEDS.get(a.workload, 2000), max_motion=a.range,
                                  scale=scale)
    ctx = me.Context(0)
    items, keep = [], []
    for t in range(a.pairs):
        c, r = torch.from_numpy(seq[t + 1]).cuda(), torch.from_numpy(seq[t]).cuda()
        h, w = seq[0].shape
        nb = (w // a.block) * (h // a.block)
        mv = torch.zeros((nb, 2), dtype=torch.int16, device="cuda")
        sad = torch.zeros(nb, dtype=torch.int32, device="cuda")
        nsp = torch.zeros(nb, dtype=torch.int16, device="cuda")
        keep.append((c, r, mv, sad, nsp))
        items.append((c, r, a.range, mv, sad, nsp))
    d = me.Context.frame_descs(items)
    if a.algo == "eval":
        fs_items = [(c, r, a.range, torch.zeros_like(mv), torch.zeros_like(sad), torch.zeros_like(nsp))
                    for c, r, mv, sad, nsp in keep]
        ctx.me_estimate_batch(me.Context.frame_descs(fs_items), a.block, "fs")
        sums = torch.zeros((a.pairs, me.ME_NSUMS), dtype=torch.int64, device="cuda")
        run = lambda: ctx.me_estimate_eval_batch(d, [x[3] for x in fs_items], a.block, "dcds", sums)
    elif a.algo == "median":
        run = lambda: ctx.me_estimate_median_batch(d, block=a.block)
    elif a.algo == "learned":
        prop = ctx.me_proposal_create()
        ctx.me_proposal_set_params(prop, me.proposal_init_params(0))
        run = lambda: ctx.me_estimate_learned_batch(prop, d, block=a.block)
    else:
        run = lambda: ctx.me_estimate_batch(d, a.block, a.algo)
    ms = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.me_check_status()
    blocks = sum(x[2].shape[0] for x in keep)
    ms.sort()
    print(f"{a.workload} block {a.block} range {a.range} {a.algo}: {a.pairs} pairs, {blocks} blocks, "
          f"{a.reps} calls, median {ms[len(ms) // 2]:.3f} ms per call")


if __name__ == "__main__":
    main()
