"""Learned warm start of the coarse solve: data from the solver, training on the
GPU with the library's own tensor-core kernels, and evaluation against the plain
start.

The network (``Net``) maps an instance's coarse grid (speed, target, obstacles,
sigma, lambda) to its coarse value and feedback control; its value channel
replaces the large constant the coarse solve of Section 4.3 starts from.  The
coarse solve has the last word: it runs to the same tolerance from the predicted
start (falling back to the plain start when the prediction is far off), so the
fixed point is the same and only the sweep count changes.

    python -m paper_1502_01629_gb300.warmstart --train 20000 --eval 1000 --epochs 10 --lr 2e-3 \
        --save-weights paper_1502_01629_gb300/warmstart_weights.npy --large --out result.json

Instances follow ``hjb_inputs.warmstart_instance`` (257^2 fine, 129^2 coarse,
0-4 obstacles); training seeds start at 100000, evaluation seeds at 900000, so
the two sets are disjoint.  Orchestration only: every computation runs in the
library (batched coarse solves and pre-computation, network forward, loss,
backward and Adam on the GPU).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

TRAIN_SEED0 = 100000
EVAL_SEED0 = 900000
NC = 129


def _make(seed):
    import hjb_inputs
    return hjb_inputs.warmstart_instance(seed)


def generate(seeds, procs: int = 0):
    """Instances for the seeds (a spawn pool of processes when procs > 1)."""
    procs = procs or min(16, os.cpu_count() or 1)
    if procs <= 1 or len(seeds) < 8:
        return [_make(s) for s in seeds]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_make, list(seeds), chunksize=8)


class Dataset:
    """Network inputs and targets of many instances, resident on the GPU."""

    def __init__(self, count: int, device):
        import torch
        self.count = count
        self.x = torch.empty((count, NC, NC, 16), dtype=torch.int16, device=device)
        self.tval = torch.empty((count, NC, NC), dtype=torch.float32, device=device)
        self.tctrl = torch.empty((count, NC, NC), dtype=torch.uint8, device=device)
        self.free = torch.empty((count, NC, NC), dtype=torch.uint8, device=device)


def build_dataset(seeds, device, chunk: int = 1000, procs: int = 0, tol_c: float = 1e-6, log=None) -> Dataset:
    """Solve the coarse problems and pre-computation of every instance (batched)
    and keep the network inputs and targets on the device."""
    from . import Batch
    seeds = list(seeds)
    ds = Dataset(len(seeds), device)
    for c0 in range(0, len(seeds), chunk):
        t0 = time.time()
        insts = generate(seeds[c0:c0 + chunk], procs)
        t1 = time.time()
        with Batch.from_instances(insts) as B:
            B.precompute(tol_c=tol_c)
            n = len(insts)
            B.net_inputs(ds.x[c0:c0 + n])
            B.net_targets(ds.tval[c0:c0 + n], ds.tctrl[c0:c0 + n], ds.free[c0:c0 + n])
        if log:
            log(f"dataset {c0 + len(insts)}/{len(seeds)}: generate {t1 - t0:.1f}s, solve {time.time() - t1:.1f}s")
    return ds


def train(net, ds: Dataset, epochs: int = 3, batch: int = 32, lr: float = 1e-3, w_value: float = 1.0,
          w_ctrl: float = 0.05, seed: int = 0, log=None) -> list:
    """Adam over shuffled mini-batches (learning rate on a cosine schedule down to
    lr / 20); returns the per-epoch mean losses (value, control)."""
    import torch
    rng = np.random.default_rng(np.random.PCG64(seed))
    hist = []
    steps_total = max(1, epochs * (ds.count // batch))
    step = 0
    for ep in range(epochs):
        order = rng.permutation(ds.count)
        lv = lc = 0.0
        nb = 0
        t0 = time.time()
        for b0 in range(0, ds.count - batch + 1, batch):
            idx = torch.from_numpy(np.sort(order[b0:b0 + batch])).to(ds.x.device)
            x = ds.x.index_select(0, idx).contiguous()
            tv = ds.tval.index_select(0, idx).contiguous()
            tc = ds.tctrl.index_select(0, idx).contiguous()
            fr = ds.free.index_select(0, idx).contiguous()
            n_free = int(fr.sum().item())
            if n_free == 0:
                continue
            frac = step / steps_total
            lr_t = lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * frac)))
            step += 1
            l = net.train_step(x, tv, tc, fr, n_free, lr=lr_t, w_value=w_value, w_ctrl=w_ctrl)
            lv += l[0]
            lc += l[1]
            nb += 1
        hist.append((lv / max(1, nb), lc / max(1, nb)))
        if log:
            log(f"epoch {ep}: value loss {hist[-1][0]:.3e} control loss {hist[-1][1]:.3f} ({time.time() - t0:.1f}s)")
    return hist


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_weights.npy")


def load_trained(path: str = WEIGHTS, max_batch: int = 32):
    """The network with the parameters a training run saved (``--save-weights``),
    or None when the file is absent."""
    if not os.path.exists(path):
        return None
    from . import Net
    net = Net(max_batch=max_batch, height=NC, width=NC)
    net.set_params(np.load(path).astype(np.float64))
    return net


def evaluate(net, insts, tol_c: float = 1e-6, k_sweeps: int = 4, accept_tol: float = 1e-3,
             tol32: float = 1.25e-7, tol64: float = 1e-6, accept_tols=(1e-3, 1e-2, 5e-2, 0.2),
             batch_kw=None) -> dict:
    """The instances solved twice as one batch: from the plain coarse start and
    from the network's prediction (accepted after k_sweeps refinement sweeps when
    the last sweep moves no node by more than accept_tol, else the plain coarse
    solve).  Reports the coarse stage (sweeps, time with inference) and the whole
    patchy solve to FP64 residual tol64 (time, largest difference of the two
    fine solutions, which share the fixed point)."""
    import torch
    from . import Batch
    dev = torch.device("cuda")

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, (time.perf_counter() - t0) * 1e3

    with Batch.from_instances(insts, **(batch_kw or {})) as B:
        n = len(insts)
        x = torch.empty((n, NC, NC, 16), dtype=torch.int16, device=dev)
        B.net_inputs(x)

        def predict():
            for b0 in range(0, n, net.max_batch):
                b1 = min(n, b0 + net.max_batch)
                net.forward(x[b0:b1], b1 - b0)
                B.coarse_warm(net.output_ptr(), first=b0, count=b1 - b0, k_sweeps=k_sweeps,
                              fallback_tol=accept_tol)

        # coarse stage alone (each path once untimed to load the kernels)
        B.coarse_warm(None)
        B.coarse_solve(tol_c=tol_c)
        (st_p, sw_p, _), ms_c_plain = timed(lambda: B.coarse_solve(tol_c=tol_c))
        predict()
        B.coarse_solve(tol_c=tol_c)
        _, ms_inf = timed(predict)
        (st_w, sw_w, fb), ms_c_warm = timed(lambda: B.coarse_solve(tol_c=tol_c))
        # whole patchy solve to the FP64 residual, plain and from the prediction
        B.coarse_warm(None)
        (sp, rp), ms_plain = timed(lambda: B.solve(tol_c=tol_c, tol32=tol32, tol64=tol64))
        u_plain = [B.get_value(i) for i in range(n)]
        scale = max(1.0, max(float(np.abs(u).max()) for u in u_plain))
        sweep = []
        for at in accept_tols:
            def warm_solve():
                for b0 in range(0, n, net.max_batch):
                    b1 = min(n, b0 + net.max_batch)
                    net.forward(x[b0:b1], b1 - b0)
                    B.coarse_warm(net.output_ptr(), first=b0, count=b1 - b0, k_sweeps=k_sweeps, fallback_tol=at)
                return B.solve(tol_c=tol_c, tol32=tol32, tol64=tol64)
            warm_solve()
            (sw2, rw), ms_warm = timed(warm_solve)
            _, _, fb2 = B.coarse_solve(tol_c=tol_c)
            diff = max(float(np.abs(B.get_value(i) - u_plain[i]).max()) for i in range(n))
            sweep.append(dict(accept_tol=at, accepted=int(n - fb2.sum()), solve_ms_warm_incl_inference=ms_warm,
                              solve_time_saved_fraction=float(1.0 - ms_warm / ms_plain),
                              fp32_steps=sw2["fp32_passes"], residual_max=float(rw.max()),
                              max_abs_diff_of_solutions=diff))
        B.coarse_warm(None)
    return dict(instances=n, tol_c=tol_c, k_sweeps=k_sweeps, accept_tol=accept_tol,
                coarse_sweeps_plain_mean=float(sw_p.mean()), coarse_sweeps_warm_mean=float(sw_w.mean()),
                coarse_sweeps_saved_fraction=float(1.0 - sw_w.sum() / sw_p.sum()),
                accepted=int(n - fb.sum()), fallbacks=int(fb.sum()),
                coarse_ms_plain=ms_c_plain, coarse_ms_warm=ms_c_warm, inference_ms=ms_inf,
                coarse_time_saved_fraction=float(1.0 - (ms_c_warm + ms_inf) / ms_c_plain),
                solve_ms_plain=ms_plain, fp32_steps_plain=sp["fp32_passes"],
                residual_max_plain=float(rp.max()), value_scale=scale, whole_solve=sweep)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--eval", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--procs", type=int, default=0)
    ap.add_argument("--out", default="")
    ap.add_argument("--save-weights", default="", help="write the trained parameters (float32 .npy)")
    ap.add_argument("--load-weights", default="", help="skip the training: parameters from this file")
    ap.add_argument("--large", action="store_true",
                    help="also the 4097^2 workload (coarse 129^2) as a batch of one on the worklist")
    args = ap.parse_args(argv)
    log = lambda m: print(m, file=sys.stderr, flush=True)
    # instances are generated in spawn processes; the first CUDA call comes after
    import torch
    from . import Net
    dev = torch.device("cuda")
    if args.load_weights:
        net = load_trained(args.load_weights, args.batch)
        hist, t_data, t_train = [], 0.0, 0.0
    else:
        t0 = time.time()
        ds = build_dataset(range(TRAIN_SEED0, TRAIN_SEED0 + args.train), dev, procs=args.procs, log=log)
        t_data = time.time() - t0
        net = Net(max_batch=args.batch, height=NC, width=NC)
        net.set_params(net.init_params(seed=1))
        t0 = time.time()
        hist = train(net, ds, epochs=args.epochs, batch=args.batch, lr=args.lr, log=log)
        t_train = time.time() - t0
        del ds
        torch.cuda.empty_cache()
        if args.save_weights:
            np.save(args.save_weights, net.get_params().astype(np.float32))
    res = {}
    if args.eval > 0:
        ev_insts = generate(range(EVAL_SEED0, EVAL_SEED0 + args.eval), args.procs)
        res = evaluate(net, ev_insts)
    if args.large:
        import hjb_inputs
        res["large4097"] = evaluate(net, [hjb_inputs.large_instance()], accept_tols=(1e-3, 0.05, 0.2),
                                    batch_kw=dict(schedule=3))
    res.update(train_instances=0 if args.load_weights else args.train, epochs=args.epochs,
               batch=args.batch, lr=args.lr, loss_history=hist, seconds_dataset=t_data,
               seconds_training=t_train)
    line = json.dumps(res)
    print(line)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")
    net.close()


if __name__ == "__main__":
    main()
