"""Benchmark: GP log-likelihood evaluations per second at n = 2^20 on one GB300.

Workload (the paper's 1-D covariance experiments, Sec. 5, in the n = 2^20 form): 2^20
points uniform on [-1, 1] (seed 1002), y ~ N(0, 1) (seed 1003), sigma^2 = 1e-2, leaf 128,
eps = 1e-12, nrhs = 1, two kernels: Matern-3/2 with ell = 0.1 and exponential with
ell = 0.2. One step = one log-likelihood evaluation of each kernel for its hyperparameters
on the fixed points: recompression (ACA) + factorization with the solve fused + log det +
y^T C^-1 y. Two forms are timed: FP64 throughout, and mixed (the leaf stage, the ACA
columns and the panels in double-float arithmetic on the FP32 pipe; right-hand sides, sums,
node matrices and log dets FP64); the headline is the faster form among those whose
results meet the 1e-10 accuracy bar. The ordering of the points depends on x only and is done once, outside the
timed region (as in a hyperparameter sweep). Every result is checked after timing against
the exact O(n) oracles (Kalman filter, Ornstein-Uhlenbeck closed form) and exact residual
rows; the accuracy is reported in the JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 20  # the benchmark size; --n changes it only for profiling captures
LEAF = 128
EPS = 1e-12
SIGMA2 = 1e-2
KERNELS = [("matern32", 0.1), ("exp", 0.2)]
SEED = 1002
COMPRESSION = "aca"  # cross approximation; --compression chebyshev for profiling captures
METRIC = "GP log-likelihood evals/sec (solve+logdet) at n=2^20, 1 GB300, at 1e-10 rel err"
FP64_PEAK = 152 * 2 * 2 * 2.07e9  # SMs x FP64 FMA/clk/SM x 2 flop x max SM clock

# DRAM bytes (read + write) of one launch of each form's leaf kernel at n = 2^20 (the
# bench's own launch: 8192 leaves, 26 panel columns + 1 right-hand side), measured by ncu
# (profiles/leaf_kernel_dram_n2p20.md); None when the kernel has changed since.
DENSE_SAMPLE_N = 1200  # the dense-limit case timed on both the oracle and the GPU
LEAF_TRAFFIC_BYTES = {0: 259840768 + 723815680, 1: 258910976 + 735765504}


def config():
    return {"workload": "1-D GP, n=2^20 U[-1,1], Matern-3/2 ell=0.1 + exponential ell=0.2, "
                        "sigma^2=1e-2, leaf 128, eps=1e-12, nrhs=1",
            "n": N, "leaf": LEAF, "eps": EPS, "sigma2": SIGMA2,
            "kernels": [f"{k}:ell={e}" for k, e in KERNELS],
            "evals_per_step": len(KERNELS), "compression": COMPRESSION,
            "l2": "inputs larger than L2 (1 GB leaf factors + 0.2 GB panels per eval)"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def combine_ranks(ms: float, units_local: int, world: int, device=None):
    """Whole-job throughput of N replicas (one independent problem per rank, no data-path
    collective): the slowest rank's time (max over ranks) and the units all ranks processed.
    Returns (ms_max, units per second)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_local * world / (ms / 1e3)


def reference_runs_here(rank: int) -> bool:
    """The reference arm (the CPU oracle) runs and prints on rank 0 only."""
    return rank == 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def leaf_flops(ctx_info):
    """Algorithmic FP64 flops of one leaf-kernel launch: per leaf of p points, Cholesky
    p^3/3, two triangular solves 2 p^2 W on W = R + nrhs columns, and the level-(kappa-1)
    partial products 2 p r W. Kernel-function evaluations are not counted."""
    p = N >> ctx_info["kappa"]
    W = ctx_info["R"] + 1
    nleaf = 1 << ctx_info["kappa"]
    return nleaf * (p ** 3 / 3.0 + 2.0 * p * p * W + 2.0 * p * ctx_info["r_last"] * W)


def accuracy(x, y, perm, kern, ell, ll, logdet, sol):
    """Relative errors against exact O(n) oracles (no HODLR involved)."""
    import oracle as O
    xs, ys = x[perm, 0], y[perm]
    if kern == "exp":
        sol_c, ld_c = O.ou_closed_form(xs, ell, 1.0, SIGMA2, ys)
        q_c = float(ys @ sol_c)
    else:
        ld_c, q_c = O.matern_kalman(xs, 3, ell, 1.0, SIGMA2, ys)
    ll_c = -0.5 * q_c - 0.5 * ld_c - 0.5 * N * np.log(2 * np.pi)
    rows = np.unique(np.linspace(0, N - 1, 32).astype(np.int64))
    Cx = O.dense_matvec_rows(x, kern, [ell, 1.0], SIGMA2, sol, rows)
    return {"logdet": abs(logdet - ld_c) / abs(ld_c), "loglik": abs(ll - ll_c) / abs(ll_c),
            "residual_rows": float(np.abs(Cx - y[rows]).max() / np.abs(y).max())}


# Double-float (mixed form) leaf kernel: FP64-equivalent peak of the FP32 pipe. The
# cheapest double-float multiply-add the kernel executes, a term of a compensated dot
# product (TwoProd by FMA with the cross terms, TwoSum, error accumulation), is 12 FP32
# instructions; the sequential updates (TwoProd, TwoSum, FastTwoSum) take 15.
FF_PEAK = 152 * 128 * 2.07e9 / 12 * 2
FORMS = {1: ("mixed", "f64/f32x2", "k_leaf_ff<512,true> (double-float leaf block build + "
                                   "L D L^T + panel solves)", FF_PEAK,
             "FP32 pipe in double-float multiply-adds: 152 SMs x 128 lanes x 2.07 GHz / 12 "
             "instructions x 2 flop"),
         0: ("fp64", "f64", "k_leaf<true,512> (leaf block build + L D L^T + panel solves)",
             FP64_PEAK, "FP64 derived: 152 SMs x 2 FMA/clk x 2.07 GHz x 2 flop")}


def measure_form(args, precision, x, y, xd, yd, stream, world, rank, local, dev):
    """Time one form: K steps of (recompress + fused factor/solve + log det) per kernel."""
    import torch
    import torch.distributed as dist

    from paper_1403_6015_gb300 import hodlr as H
    ctxs = [H.Hodlr(xd, kern, [ell, 1.0], SIGMA2, LEAF, EPS, max_rank=16, max_nrhs=1,
                    stream=stream.cuda_stream, precision=precision, compression=args.compression)
            for kern, ell in KERNELS]
    outs = torch.zeros(len(KERNELS), dtype=torch.float64, device=dev)
    # launch configuration per context, chosen by the library's autotuner (untimed)
    tuning = {}
    for h, (kern, ell) in zip(ctxs, KERNELS):
        if not args.no_autotune:
            h.autotune(yd, reps=3)
        tuning[kern] = h.tuning()

    def step(leaf_ms=None):
        for i, (h, (kern, ell)) in enumerate(zip(ctxs, KERNELS)):
            h.rebuild([ell, 1.0], SIGMA2)
            h.loglik(yd, out=outs[i:i + 1])
            if leaf_ms is not None:
                leaf_ms.append(h.phase_ms()["leaf_kernel"])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = sum(h.counters()["launches"] for h in ctxs)
    leaf_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step(leaf_ms)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = sum(h.counters()["launches"] for h in ctxs) - launches0
    ms, value = combine_ranks(ms, args.steps * len(KERNELS), world, dev)
    res = {"value": value, "ms_per_step": ms / args.steps, "gpu_launches": launches,
           "clocks": clk.summary(), "phase_ms": ctxs[0].phase_ms(), "tuning": tuning}

    # end to end through the C ABI with host buffers: pinned y in, host scalar out
    y_host = torch.from_numpy(y).pin_memory().numpy()
    host_out = np.zeros(len(KERNELS))
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for i, (h, (kern, ell)) in enumerate(zip(ctxs, KERNELS)):
                h.rebuild([ell, 1.0], SIGMA2)
                host_out[i] = h.loglik(y_host)
        torch.cuda.synchronize()
        res["e2e"] = args.steps * len(KERNELS) * world / (time.perf_counter() - t0)

    # roofline of the dominant kernel (the leaf kernel of the first covariance)
    h0 = ctxs[0]
    ranks = h0.ranks()
    kappa = h0.tree()[0]
    R = sum(int(ranks[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(kappa))
    info = {"kappa": kappa, "R": R, "r_last": int(ranks[(1 << (kappa - 1)) - 1:].max())}
    lm = float(np.mean(leaf_ms[0::len(KERNELS)]))
    name, dtype, kname, peak, note = FORMS[precision]
    achieved = leaf_flops(info) / (lm / 1e3)
    res["dtype"] = dtype
    res["roofline"] = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                       "unit": "TFLOP/s", "frac": achieved / peak,
                       "traffic": LEAF_TRAFFIC_BYTES.get(precision), "kernel": kname,
                       "kernel_ms": lm, "peak_note": note}

    # accuracy (outside the timed region)
    acc = {}
    if rank == 0 and not args.no_accuracy:
        for i, (h, (kern, ell)) in enumerate(zip(ctxs, KERNELS)):
            h.rebuild([ell, 1.0], SIGMA2)
            sol = h.factor_solve(y)
            _, perm = h.tree()
            acc[kern] = accuracy(x, y, perm, kern, ell, float(outs[i].item()), h.logdet(), sol)
        if not args.no_e2e:
            acc["host_vs_device_loglik"] = float(np.max(np.abs(host_out - outs.cpu().numpy())))
    res["accuracy"] = acc
    res["accepted"] = bool(acc) and all(
        max(v["logdet"], v["loglik"], v["residual_rows"]) <= 1e-10
        for k, v in acc.items() if isinstance(v, dict))
    for h in ctxs:
        h.close()
    return res


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1403_6015_gb300 import build_lib
    from paper_1403_6015_gb300 import inputs as I

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build_lib.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # replicas: every rank evaluates its own copy of the workload (independent problems)
    x, y = I.workload_1d(N, SEED + 1000 * rank)
    xd = torch.from_numpy(x).to(dev)
    yd = torch.from_numpy(y).to(dev)
    forms = [args.precision] if args.precision >= 0 else [1, 0]
    results = {p: measure_form(args, p, x, y, xd, yd, stream, world, rank, local, dev)
               for p in forms}
    # headline: the fastest form that met the 1e-10 accuracy bar
    ok = [p for p in forms if results[p]["accepted"] or args.no_accuracy]
    head = max(ok, key=lambda p: results[p]["value"]) if ok else forms[-1]
    r = results[head]
    cpu = cpu_baseline(x, y) if (rank == 0 and world == 1 and not args.no_cpu) else None
    sweeps = run_sweeps(args) if (rank == 0 and not args.no_sweeps) else None
    supp = run_supplementary(args) if (rank == 0 and not args.no_sweeps) else None
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": "evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": r["dtype"], "form": FORMS[head][0],
            "data": "synthetic (seeded splitmix64 points and N(0,1) right-hand side)",
            "config": config(),
            "e2e": {"value": r.get("e2e"), "unit": "evals/s",
                    "h2d_bytes_per_step": len(KERNELS) * N * 8,
                    "d2h_bytes_per_step": len(KERNELS) * 8},
            "roofline": r["roofline"],
            "phase_ms": r["phase_ms"],
            "tuning": r["tuning"],
            "gpu_launches": r["gpu_launches"],
            "clocks": r["clocks"],
            "accuracy": r["accuracy"],
            "accepted": r["accepted"],
            "cpu_baseline": cpu,
            "sweeps": sweeps,
            "supplementary": supp,
        }
        if r.get("phase_ms"):
            # the headline including the point ordering in every evaluation
            per_eval = r["ms_per_step"] / len(KERNELS) + r["phase_ms"]["ordering"]
            line["evals_per_s_including_ordering"] = 1e3 / per_eval
        for p in forms:
            if p != head:
                o = results[p]
                line[FORMS[p][0] + "_form"] = {
                    "value": o["value"], "ms_per_step": o["ms_per_step"], "dtype": o["dtype"],
                    "e2e": o.get("e2e"), "roofline": o["roofline"], "phase_ms": o["phase_ms"],
                    "tuning": o["tuning"], "accuracy": o["accuracy"], "accepted": o["accepted"]}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def sweep_settings(nset, seed):
    """ell log-uniform in [0.05, 2], sigma^2 log-uniform in [1e-4, 1] (the hyperparameter
    sweep workload)."""
    from paper_1403_6015_gb300 import inputs as I
    u = I.uniform01(seed, 2 * nset)
    ell = np.exp(np.log(0.05) + u[:nset] * (np.log(2.0) - np.log(0.05)))
    s2 = np.exp(np.log(1e-4) + u[nset:] * (np.log(1.0) - np.log(1e-4)))
    return ell, s2


def run_sweeps(args):
    """Batched evaluation (outside the headline's timed region): 256 Matern-5/2 settings on
    n = 65536 points, graph-replayed on one context and forked over 8 lanes, against the
    adaptive per-setting loop; 64 independent problems of uneven size, one lane each; the
    learned rank predictor's gain on a squared-exponential sweep whose ranks vary with ell;
    and the predictor at scale on 2-D n = 2^20 points."""
    import torch

    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    from paper_1403_6015_gb300 import rank_model as RM
    n = 1 << 16
    x, y = I.workload_1d(n, 1004)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        yd = torch.from_numpy(y).cuda()
    stream.synchronize()
    out = {}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    # (1) 256 Matern-5/2 settings: one captured evaluation replayed per setting
    nset = 256
    ell, s2 = sweep_settings(nset, 2004)
    res = {"n": n, "settings": nset, "kernel": "matern52", "leaf": 128, "eps": 1e-12}
    for prec, name in [(0, "fp64"), (1, "mixed")]:
        h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=prec,
                    stream=stream.cuda_stream)

        def adaptive():
            v = np.zeros(nset)
            for b in range(nset):
                h.rebuild([ell[b], 1.0], s2[b])
                v[b] = h.loglik(yd)
            return v
        adaptive()  # warm-up
        ref, ta = timed(adaptive)
        h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
        theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
        sig = torch.from_numpy(s2.copy()).cuda()
        status = torch.zeros(nset, dtype=torch.int32, device="cuda")
        h.loglik_sweep(theta, sig, yd, status=status)  # capture
        got, tg = timed(lambda: h.loglik_sweep(theta, sig, yd, status=status).cpu().numpy())
        res[name] = {"graph_evals_per_s": nset / tg, "adaptive_evals_per_s": nset / ta,
                     "speedup": ta / tg, "max_rel_diff": float(np.max(np.abs(got - ref) / np.abs(ref))),
                     "status_ok": bool((status.cpu().numpy() == 0).all())}
        h.close()
        # the same settings on L presized contexts (lanes), each on its own stream: one
        # graph forks every round into all lanes, which run concurrently
        L = 8
        lane_streams = [torch.cuda.Stream() for _ in range(L)]
        ctxs = []
        for ls in lane_streams:
            hl = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=prec,
                         stream=ls.cuda_stream)
            hl.presize(np.full(hl.tree()[0], 4, dtype=np.int32))
            ctxs.append(hl)
        outl = torch.zeros(nset, dtype=torch.float64, device="cuda")
        status.fill_(-1)
        H.loglik_batched(ctxs, theta, sig, yd, outl, status, stream=stream.cuda_stream)
        gotl, tl = timed(lambda: H.loglik_batched(ctxs, theta, sig, yd, outl, status,
                                                  stream=stream.cuda_stream).cpu().numpy())
        res[name].update({"lanes": L, "lanes_evals_per_s": nset / tl, "lanes_speedup": ta / tl,
                          "lanes_max_rel_diff": float(np.max(np.abs(gotl - ref) / np.abs(ref))),
                          "lanes_status_ok": bool((status.cpu().numpy() == 0).all())})
        for hl in ctxs:
            hl.close()
    out["batched_matern52"] = res

    # (1b) 64 independent problems of uneven size (n log-uniform in [2^12, 2^18]), four
    # settings each: one lane per problem against the per-problem adaptive loop
    ninst, per = 64, 4
    un = I.uniform01(3003, ninst)
    sizes = np.round(np.exp(np.log(4096.0) + un * (np.log(262144.0) - np.log(4096.0)))).astype(int)
    res = {"instances": ninst, "settings_per_instance": per, "n_min": int(sizes.min()),
           "n_max": int(sizes.max()), "n_total": int(sizes.sum()), "kernel": "matern52",
           "leaf": 128, "eps": 1e-12}
    # torch hands out streams round-robin from a pool of 32: a fresh origin and 16 lane
    # streams created back to back are distinct; instances share lane streams round-robin
    origin = torch.cuda.Stream()
    pool = [torch.cuda.Stream() for _ in range(16)]
    for prec, name in [(0, "fp64"), (1, "mixed")]:
        inst = []
        for i, ni in enumerate(sizes):
            xi, yi = I.workload_1d(int(ni), 3100 + i)
            e_i, s_i = sweep_settings(per, 3300 + i)
            si = pool[i % len(pool)]
            hi = H.Hodlr(xi, "matern52", [e_i[0], 1.0], s_i[0], 128, 1e-12, precision=prec,
                         stream=si.cuda_stream)
            th = torch.from_numpy(np.stack([e_i, np.ones(per)], 1).copy()).cuda()
            sg = torch.from_numpy(s_i.copy()).cuda()
            yi_d = torch.from_numpy(yi).cuda()
            inst.append((hi, si, e_i, s_i, th, sg, yi_d,
                         torch.zeros(per, dtype=torch.float64, device="cuda"),
                         torch.full((per,), -1, dtype=torch.int32, device="cuda")))
        torch.cuda.synchronize()

        def adaptive_inst():
            v = np.zeros((ninst, per))
            for i, (hi, si, e_i, s_i, th, sg, yi_d, _, _) in enumerate(inst):
                for b in range(per):
                    hi.rebuild([e_i[b], 1.0], s_i[b])
                    v[i, b] = hi.loglik(yi_d)
            return v
        adaptive_inst()
        ref, ta = timed(adaptive_inst)
        for hi, *_ in inst:
            hi.presize(np.full(hi.tree()[0], 4, dtype=np.int32))
        lanes = [H.hodlr_batch_lane(hi._ctx, th.data_ptr(), sg.data_ptr(), yi_d.data_ptr(),
                                    o.data_ptr(), st.data_ptr(), 0, 1, per)
                 for hi, si, e_i, s_i, th, sg, yi_d, o, st in inst]

        def lanes_inst():
            st = H.hodlr_loglik_batched(lanes, origin.cuda_stream)
            if st != H.HODLR_OK:
                raise H.HodlrError(st, "; ".join(sorted({H.hodlr_last_error(t[0]._ctx)
                                                         for t in inst})))
            return np.stack([o.cpu().numpy() for *_, o, st in inst])
        lanes_inst()
        got, tl = timed(lanes_inst)
        ok = all(bool((st.cpu().numpy() == 0).all()) for *_, st in inst)
        res[name] = {"lane_streams": len(pool),
                     "adaptive_evals_per_s": ninst * per / ta, "lanes_evals_per_s": ninst * per / tl,
                     "speedup": ta / tl, "max_rel_diff": float(np.max(np.abs(got - ref) / np.abs(ref))),
                     "status_ok": ok,
                     "points_per_s": float(sizes.sum()) * per / tl}
        for hi, *_ in inst:
            hi.close()
    out["uneven_instances"] = res

    # (2) learned rank predictor: trained on the GPU on the FP64 compressor's blocks
    t0 = time.perf_counter()
    probs = []
    ells_tr = np.exp(np.linspace(np.log(0.03), np.log(2.0), 9))
    for i, nn in enumerate([1 << 12, 1 << 13]):
        xt, _ = I.workload_1d(nn, 900 + i)
        for kern in ["exp", "se", "matern32", "matern52"]:
            for e in ells_tr:
                for eps in [1e-8, 1e-12]:
                    probs.append((xt, kern, float(e), 0.01, 64, eps))
    X, T, R = RM.collect_pairs(probs)
    net = RM.RankMLP(seed=7)
    loss = net.train(X, T, steps=1500, lr=3e-3)
    t_train = time.perf_counter() - t0
    nset = 64
    ell, s2 = sweep_settings(nset, 2005)
    h = H.Hodlr(x, "se", [ell[0], 1.0], s2[0], 128, 1e-10, stream=stream.cuda_stream)

    def adaptive_se():
        v = np.zeros(nset)
        for b in range(nset):
            h.rebuild([ell[b], 1.0], s2[b])
            v[b] = h.loglik(yd)
        return v
    adaptive_se()
    ref, ta = timed(adaptive_se)
    RM.sweep_with_predictor(h, net, ell, s2, yd, margin=1)  # captures the groups' graphs
    (got, st), tp = timed(lambda: RM.sweep_with_predictor(h, net, ell, s2, yd, margin=1))
    # the same presizes on 8 lanes (batched rounds over the settings of each group)
    origin = torch.cuda.Stream()
    lane_streams = [torch.cuda.Stream() for _ in range(8)]
    lanes = [H.Hodlr(x, "se", [ell[0], 1.0], s2[0], 128, 1e-10, stream=ls.cuda_stream)
             for ls in lane_streams]
    RM.sweep_with_predictor(h, net, ell, s2, yd, margin=1, lanes=lanes, stream=origin.cuda_stream)
    (gotl, stl), tl = timed(lambda: RM.sweep_with_predictor(h, net, ell, s2, yd, margin=1, lanes=lanes,
                                                            stream=origin.cuda_stream))
    # the baseline at equal batching: the same 8 lanes and settings, presized from one
    # adaptive probe at the smallest ell (no network; margin 0: the probe's ranks bound
    # every setting's here, and it measured fastest)
    RM.sweep_with_probe(h, ell, s2, yd, margin=0, lanes=lanes, stream=origin.cuda_stream)
    (gotb, stb), tb = timed(lambda: RM.sweep_with_probe(h, ell, s2, yd, margin=0, lanes=lanes,
                                                        stream=origin.cuda_stream))
    for c in lanes:
        c.close()
    out["predictor_se"] = {
        "n": n, "settings": nset, "kernel": "se", "eps": 1e-10,
        "adaptive_evals_per_s": nset / ta, "predicted_evals_per_s": nset / tp, "gain": ta / tp,
        "predicted_lanes": 8, "predicted_lanes_evals_per_s": nset / tl, "lanes_gain": ta / tl,
        "lanes_fallbacks": stl["fallbacks"],
        "lanes_max_rel_diff": float(np.max(np.abs(gotl - ref) / np.abs(ref))),
        "probe_lanes_evals_per_s": nset / tb, "gain_equal_batching": tb / tl,
        "probe_fallbacks": stb["fallbacks"], "probe_level_ranks": stb["probe_level_ranks"],
        "probe_max_rel_diff": float(np.max(np.abs(gotb - ref) / np.abs(ref))),
        "presized_rank_sum": {"predictor": stl["presized_rank_sum"],
                              "probe": stb["presized_rank_sum"]},
        "groups": st["groups"], "fallbacks": st["fallbacks"],
        "max_rel_diff": float(np.max(np.abs(got - ref) / np.abs(ref))),
        "train": {"pairs": int(X.shape[0]), "final_mse": loss, "seconds": t_train,
                  "steps": 1500}}
    h.close()

    # (2b) where the network replaces a probe per problem: 64 independent problems of uneven
    # size (n log-uniform in [2^12, 2^16]), squared-exponential, eps 1e-10, two settings
    # each, all in one batched launch. Baseline at equal batching: each problem presized
    # from one adaptive compression at its smallest ell (an adaptive evaluation with host
    # synchronisations per problem); predictor: each problem presized by the network.
    ninst, per = 64, 2
    un = I.uniform01(3013, ninst)
    sizes = np.round(np.exp(np.log(4096.0) + un * (np.log(65536.0) - np.log(4096.0)))).astype(int)
    pool = [torch.cuda.Stream() for _ in range(16)]
    origin = torch.cuda.Stream()
    ictx, iset, iys = [], [], []
    for i, ni in enumerate(sizes):
        xi, yi = I.workload_1d(int(ni), 3200 + i)
        e_i, s_i = sweep_settings(per, 3400 + i)
        ictx.append(H.Hodlr(xi, "se", [e_i[0], 1.0], s_i[0], 128, 1e-10,
                            stream=pool[i % len(pool)].cuda_stream))
        iset.append((e_i, s_i))
        iys.append(torch.from_numpy(yi).cuda())
    torch.cuda.synchronize()

    def adaptive_inst():
        res = []
        for hi, (e_i, s_i), yi in zip(ictx, iset, iys):
            hi.presize(None)
            v = np.zeros(per)
            for b in range(per):
                hi.rebuild([float(e_i[b]), 1.0], float(s_i[b]))
                v[b] = hi.loglik(yi)
            res.append(v)
        return res
    adaptive_inst()
    ref_i, ta_i = timed(adaptive_inst)
    RM.instances_with_probe(ictx, iset, iys, origin.cuda_stream, margin=0)
    (got_b, st_b), tb_i = timed(lambda: RM.instances_with_probe(ictx, iset, iys, origin.cuda_stream,
                                                                margin=0))
    RM.instances_with_predictor(ictx, net, iset, iys, origin.cuda_stream, margin=1)
    (got_p, st_p), tp_i = timed(lambda: RM.instances_with_predictor(ictx, net, iset, iys,
                                                                    origin.cuda_stream, margin=1))
    relmax = lambda got: max(float(np.max(np.abs(a - b) / np.abs(b))) for a, b in zip(got, ref_i))
    out["predictor_instances"] = {
        "instances": ninst, "settings_per_instance": per, "n_min": int(sizes.min()),
        "n_max": int(sizes.max()), "kernel": "se", "eps": 1e-10, "leaf": 128, "form": "fp64",
        "adaptive_evals_per_s": ninst * per / ta_i,
        "probe_evals_per_s": ninst * per / tb_i, "predicted_evals_per_s": ninst * per / tp_i,
        "gain_equal_batching": tb_i / tp_i, "probe_fallbacks": st_b["fallbacks"],
        "predictor_fallbacks": st_p["fallbacks"],
        "presized_rank_sum": {"predictor": st_p["presized_rank_sum"], "probe": st_b["presized_rank_sum"]},
        "max_rel_diff": {"probe": relmax(got_b), "predictor": relmax(got_p)}}
    for hi in ictx:
        hi.close()
    net.close()

    # (3) the predictor at scale: 2-D n = 2^20 U[0,1]^2, squared-exponential ell = 0.1,
    # eps = 1e-10 (top-level ranks ~225), mixed form; adaptive against predictor-presized
    # at equal accuracy. The network is retrained with 2-D problems up to n = 2^16.
    t0 = time.perf_counter()
    probs = []
    for i, nn in enumerate([1 << 12, 1 << 13, 1 << 14, 1 << 15, 1 << 16]):
        lo = 0.04 if nn <= (1 << 14) else 0.06
        x2s, _ = I.workload_2d(nn, 950 + i)
        x1s, _ = I.workload_1d(nn, 900 + i)
        for e in np.exp(np.linspace(np.log(lo), np.log(1.0), 11)):
            for eps in [1e-8, 1e-10]:
                probs.append((x2s, "se", float(e), 0.01, 128, eps))
                if nn <= (1 << 14):
                    probs.append((x1s, "se", float(e), 0.01, 128, eps))
    X, T, R = RM.collect_pairs(probs, max_rank=512)
    net = RM.RankMLP(seed=7)
    loss = net.train(X, T, steps=3000, lr=3e-3)
    t_train = time.perf_counter() - t0
    n2 = 1 << 20
    x2, y2 = I.workload_2d(n2, 1400)
    x2d = torch.from_numpy(x2).cuda()
    y2d = torch.from_numpy(np.ascontiguousarray(y2).reshape(-1)).cuda()
    h = H.Hodlr(x2d, "se", [0.1, 1.0], 1e-2, 128, 1e-10, max_rank=320, precision=1)
    k2 = h.tree()[0]
    r2 = h.ranks()
    lv = [int(r2[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(k2)]

    def one_eval():
        h.rebuild([0.1, 1.0], 1e-2)
        return h.loglik(y2d)
    one_eval()
    ll_a, ta = timed(one_eval)
    pre = RM.presize_profile(h, net, 0.1, margin=1, scale=1.08)
    h.presize(pre)
    one_eval()
    ll_p, tp = timed(one_eval)
    flags = h.status_flags()
    if flags:  # the fallback: the adaptive path
        h.presize(None)
        ll_p, tf = timed(one_eval)
        tp += tf
    out["predictor_2d"] = {
        "n": n2, "d": 2, "kernel": "se", "ell": 0.1, "sigma2": 1e-2, "eps": 1e-10, "form": "mixed",
        "adaptive_level_ranks": lv, "presized_level_ranks": [int(v) for v in pre],
        "adaptive_s_per_eval": ta, "predicted_s_per_eval": tp, "gain": ta / tp,
        "fallback": bool(flags), "rel_diff": abs(ll_p - ll_a) / abs(ll_a),
        "train": {"pairs": int(X.shape[0]), "final_mse": loss, "seconds": t_train, "steps": 3000},
        "ell_0.02": "not run: top-level ranks above 850 at n = 65536 and growing with n, "
                    "beyond the 512 cap"}
    h.close()
    net.close()
    return out


def run_supplementary(args):
    """Measurements beside the headline (untimed by it): the paper's phase split at n = 2^20
    (solve-only with 1 and 16 right-hand sides and log det given a factor, ordering), the
    mixed form with refinement on n = 2^22 (1-D squared-exponential ell = 0.05,
    sigma^2 = 1e-3), and rows shaped like the paper's tables (points on [-3, 3]^d, unit
    length scale: the Gaussian, exponential, inverse multiquadric, biharmonic and
    multiquadric at n = 1e6 in 1-D, the multiquadric at n = 1e5 in 2-D, the Gaussian at
    n = 5000 in 32 and 64 dimensions) next to the paper's single-core timings (context
    only)."""
    import torch

    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    out = {}

    def ms_of(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    # (1) phases at n = 2^20, mixed form, per covariance
    x, y = I.workload_1d(N, SEED)
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y).cuda()
    Y16 = torch.from_numpy(I.normal(N, SEED + 7, 16)).cuda().t().contiguous().t()  # column-major
    ph = {}
    for kern, ell in KERNELS:
        h = H.Hodlr(xd, kern, [ell, 1.0], SIGMA2, LEAF, EPS, max_rank=16, max_nrhs=16, precision=1)
        order_ms = h.phase_ms()["ordering"]
        comp_ms = ms_of(lambda: h.rebuild([ell, 1.0], SIGMA2))
        h.rebuild([ell, 1.0], SIGMA2)

        def factor_once():
            h.rebuild([ell, 1.0], SIGMA2)
            h.factor()
        fac_ms = ms_of(factor_once) - comp_ms
        s1 = ms_of(lambda: h.solve(yd))
        s16 = ms_of(lambda: h.solve(Y16))
        det_ms = ms_of(lambda: h.logdet())
        xt = torch.from_numpy(I.uniform_points(256, 1, -1.0, 1.0, SEED + 9)).cuda()
        pm = ms_of(lambda: h.predict(xt, yd, var=False))
        pv = ms_of(lambda: h.predict(xt, yd, var=True))
        ph[kern] = {"ordering_ms": order_ms, "compression_ms": comp_ms, "factor_ms": fac_ms,
                    "solve_nrhs1_ms": s1, "solve_nrhs16_ms": s16, "logdet_given_factor_ms": det_ms,
                    "predict_256_mean_ms": pm, "predict_256_mean_var_ms": pv}
        h.close()
    out["phases_n2p20_mixed"] = ph

    # (1a) the headline workload in the batched form: the two covariances as two lanes of
    # hodlr_loglik_batched, presized to their exact ranks (2 for Matern-3/2, 1 for the
    # exponential: semiseparable in 1-D), 20 rounds, against the sequential
    # single-context evaluations of the headline (same inputs, same results expected)
    rounds = 20
    lanes, keep = [], []
    for kern, ell in KERNELS:
        s = torch.cuda.Stream()
        h = H.Hodlr(xd, kern, [ell, 1.0], SIGMA2, LEAF, EPS, max_rank=16, max_nrhs=1, precision=1,
                    stream=s.cuda_stream)
        h.presize(np.full(h.tree()[0], {"matern32": 2, "exp": 1}[kern], dtype=np.int32))
        th = torch.tensor([[ell, 1.0]] * rounds, dtype=torch.float64, device="cuda")
        sg = torch.full((rounds,), SIGMA2, dtype=torch.float64, device="cuda")
        o = torch.zeros(rounds, dtype=torch.float64, device="cuda")
        st = torch.full((rounds,), -1, dtype=torch.int32, device="cuda")
        lanes.append(H.hodlr_batch_lane(h._ctx, th.data_ptr(), sg.data_ptr(), yd.data_ptr(),
                                        o.data_ptr(), st.data_ptr(), 0, 1, rounds))
        keep.append((h, s, th, sg, o, st))
    origin = torch.cuda.Stream()
    torch.cuda.synchronize()
    H.hodlr_loglik_batched(lanes, origin.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.hodlr_loglik_batched(lanes, origin.cuda_stream)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    seqc = [H.Hodlr(xd, kern, [ell, 1.0], SIGMA2, LEAF, EPS, max_rank=16, max_nrhs=1, precision=1)
            for kern, ell in KERNELS]

    def seq_round():
        vals = []
        for h, (_, e) in zip(seqc, KERNELS):
            h.rebuild([e, 1.0], SIGMA2)
            vals.append(h.loglik(yd))
        return vals
    ref = seq_round()
    ts = ms_of(seq_round, reps=rounds) / 1e3 * rounds
    got = [float(k[4][-1].item()) for k in keep]
    out["batched_form_headline_workload"] = {
        "lanes": len(KERNELS), "rounds": rounds, "presize": "exact ranks (Matern-3/2: 2, exponential: 1)",
        "form": "mixed", "batched_evals_per_s": len(KERNELS) * rounds / tb,
        "sequential_evals_per_s": len(KERNELS) * rounds / ts,
        "status_ok": all(bool((k[5].cpu().numpy() == 0).all()) for k in keep),
        "max_rel_diff": max(abs(g - r) / abs(r) for g, r in zip(got, ref))}
    for k in keep:
        k[0].close()
    for h in seqc:
        h.close()

    # (1b) the analytic compression (Chebyshev interpolation) against the cross
    # approximation on the same evaluation: compression time, ranks, log-likelihood
    cheb = {}
    for kern, ell in KERNELS + [("se", 0.3)]:
        row = {}
        for comp in ("aca", "chebyshev"):
            h = H.Hodlr(xd, kern, [ell, 1.0], SIGMA2, LEAF, EPS, precision=1, compression=comp)
            comp_ms = ms_of(lambda: h.rebuild([ell, 1.0], SIGMA2))

            def ev():
                h.rebuild([ell, 1.0], SIGMA2)
                return h.loglik(yd)
            ev_ms = ms_of(ev)
            k2 = h.tree()[0]
            rk = h.ranks()
            row[comp] = {"compression_ms": comp_ms, "eval_ms": ev_ms, "loglik": ev(),
                         "level_ranks": [int(rk[(1 << j) - 1:(1 << (j + 1)) - 1].max())
                                         for j in range(k2)]}
            h.close()
        row["loglik_rel_diff"] = abs(row["aca"]["loglik"] - row["chebyshev"]["loglik"]) / abs(
            row["aca"]["loglik"])
        cheb[f"{kern}_ell{ell}"] = row
    out["chebyshev_vs_aca_n2p20_mixed"] = cheb

    # (2) mixed precision + refinement at n = 2^22 (1-D squared-exponential)
    n3 = 1 << 22
    x3, y3 = I.workload_1d(n3, 1003)
    x3d = torch.from_numpy(x3).cuda()
    y3d = torch.from_numpy(y3).cuda()
    res3 = {"n": n3, "kernel": "se", "ell": 0.05, "sigma2": 1e-3, "leaf": 128, "eps": 1e-12}
    lls = {}
    for prec, name, rmax in [(1, "mixed_refined", 2), (0, "fp64", 0)]:
        h = H.Hodlr(x3d, "se", [0.05, 1.0], 1e-3, 128, 1e-12, max_rank=64, precision=prec,
                    refine_maxit=rmax, refine_tol=1e-13)

        def ev():
            h.rebuild([0.05, 1.0], 1e-3)
            return h.loglik(y3d)
        ev()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            lls[name] = ev()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        k3 = h.tree()[0]
        r3 = h.ranks()
        entry = {"evals_per_s": 1.0 / dt, "s_per_eval": dt,
                 "level_ranks": [int(r3[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(k3)]}
        if prec == 1:
            entry["refine_corrections"], entry["refine_residual"] = h.refine_info()
            h.rebuild([0.05, 1.0], 1e-3)
            sol = h.factor_solve(y3)
            import oracle as O
            rows = np.unique(np.linspace(0, n3 - 1, 16).astype(np.int64))
            Cx = O.dense_matvec_rows(x3, "se", [0.05, 1.0], 1e-3, sol, rows)
            entry["residual_rows"] = float(np.abs(Cx - y3[rows]).max() / np.abs(y3).max())
        res3[name] = entry
        h.close()
    res3["loglik_rel_diff_mixed_vs_fp64"] = abs(lls["mixed_refined"] - lls["fp64"]) / abs(lls["fp64"])
    out["mixed_refined_n2p22"] = res3

    # (3) paper-shaped rows: n = 1e6 on [-3, 3]; the paper's phases (Assembly = ordering +
    # compression, Factor, Solve, Det.) and the relative error of the solution of C x = b
    # with b made from a known x (b = C~ x through the library's own product)
    # (name: kernel, ell, sigma^2, d, n, the paper's seconds for assembly/factor/solve/det)
    paper = {"gaussian_2I+exp(-r^2)": ("se", 0.5 ** 0.5, 2.0, 1, 1000000, [14.1, 23.2, 0.834, 1.52]),
             "exponential_I+exp(-r)": ("exp", 1.0, 1.0, 1, 1000000, [18.8, 8.05, 0.636, 1.35]),
             "inverse_multiquadric_I+1/sqrt(1+r^2)": ("imq", 1.0, 1.0, 1, 1000000,
                                                      [14.2, 26.8, 1.02, 1.49]),
             "biharmonic_2I+r^2log(r)": ("biharmonic", 1.0, 2.0, 1, 1000000, [51.3, 81.9, 1.28, 3.40]),
             "multiquadric_I+sqrt(1+r^2)": ("mq", 1.0, 1.0, 1, 1000000, [10.9, 17.1, 0.814, 1.94]),
             "multiquadric_I+sqrt(1+r^2)_2d": ("mq", 1.0, 1.0, 2, 100000, [6.54, 6.95, 0.177, 0.31]),
             "gaussian_2I+exp(-r^2)_d32_n5000": ("se", 0.5 ** 0.5, 2.0, 32, 5000, [0.15, 0.061, 0.004, 0.001]),
             "gaussian_2I+exp(-r^2)_d64_n5000": ("se", 0.5 ** 0.5, 2.0, 64, 5000, [0.21, 0.059, 0.001, 0.001])}
    rows4 = {}
    for name, (kern, ell, s2, d4, n4, ptimes) in paper.items():
        x4 = I.uniform_points(n4, d4, -3.0, 3.0, 1005 + d4)
        xt = I.normal(n4, 1006)
        r = {"n": n4, "d": d4, "kernel": kern, "ell": ell, "sigma2": s2, "leaf": LEAF, "eps": EPS,
             "paper_s (one CPU core)": dict(zip(["assembly", "factor", "solve", "det"], ptimes))}
        forms = [(0, "fp64")] if kern in H.INDEFINITE else [(0, "fp64"), (1, "mixed")]
        for prec, fname in forms:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                h = H.Hodlr(x4, kern, [ell, 1.0], s2, LEAF, EPS, precision=prec, max_rank=512)
            except H.HodlrError as e:
                r[fname] = {"error": str(e)}
                continue
            torch.cuda.synchronize()
            asm_s = time.perf_counter() - t0
            b = h.matvec(xt)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.factor()
            torch.cuda.synchronize()
            fac_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            xs = h.solve(b)
            torch.cuda.synchronize()
            sol_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            _, sign = h.logdet_signed()
            det_s = time.perf_counter() - t0
            kap = h.tree()[0]
            rk = h.ranks()
            r[fname] = {"assembly_s": asm_s, "factor_s": fac_s, "solve_s": sol_s, "det_s": det_s,
                        "note": "assembly includes the host-to-device copy of x; solve "
                                "includes host copies of b and x",
                        "error": float(np.linalg.norm(xs - xt) / np.linalg.norm(xt)),
                        "det_sign": sign,
                        "top_ranks": [int(rk[(1 << j) - 1:(1 << (j + 1)) - 1].max())
                                      for j in range(min(kap, 4))]}
            h.close()
        rows4[name] = r
    out["paper_shaped"] = rows4
    out["dense_limit_rows"] = dense_limit_rows(H, I, torch)
    return out


def factor_flops(lr, n, nleaf_sizes, nrhs=1):
    """Algorithmic FP64 flops of one factorization with padded level ranks lr (Sec. 3.2):
    per level j the node LUs 2^j (2/3)(2 r_j)^3 and substitutions 2^j 2 (2 r_j)^2 (c_j + nrhs),
    the sweep's update 2 n r_j (c_j + nrhs) and half-node sums 2 n r_{j-1} (c_j + nrhs), and
    per leaf of p points the L D L^T p^3 / 3, the solves 2 p^2 (R + nrhs) and the finest
    level's partials 2 p r_{K-1} (R + nrhs)."""
    K = len(lr)
    c = np.concatenate([[0], np.cumsum(lr)])
    f = 0.0
    for j in range(K):
        r, w = lr[j], c[j] + nrhs
        f += (1 << j) * (2.0 / 3.0 * (2 * r) ** 3 + 2.0 * (2 * r) ** 2 * w)
        f += 2.0 * n * r * w
        if j > 0:
            f += 2.0 * n * lr[j - 1] * w
    p = np.asarray(nleaf_sizes, dtype=np.float64)
    f += (p ** 3 / 3.0 + 2.0 * p ** 2 * (c[K] + nrhs) + 2.0 * p * (lr[K - 1] if K else 0) * (c[K] + nrhs)).sum()
    return f


def dense_limit_rows(H, I, torch):
    """The paper's Gaussian rows whose off-diagonal blocks are close to full rank (Sec. 5:
    the three-dimensional column at n = 10 000, the unscaled d = 4 and scaled d = 8 rows of
    the d-dimensional tables at n = 5000; C = 2I + exp(-r^2)), leaf 128, eps 1e-12,
    max_rank n/2. Assembly (ordering + compression), factor, solve and det timed per call
    (the second of two builds, so that one-time set-up is excluded), log det against the
    oracle's stored value (tests/golden, written by its own script) or dense Cholesky, and
    the factorization's algorithmic FP64 rate against the derived FP64 peak."""
    rows = {
        "gaussian_d4_n1200_oracle_sample": (None, DENSE_SAMPLE_N, 4, 3.0, 2100, None),
        "gaussian_3d_n10000": ("d3", 10000, 3, 3.0, 2003, [15.4, 17.3, 0.113, 0.91]),
        "gaussian_d4_n5000": ("d4", 5000, 4, 3.0, 2004, [9.67, 21.25, 0.073, 0.088]),
        "gaussian_scaled_d8_n5000": (None, 5000, 8, 3.0 / np.sqrt(8.0), 2008, [40.8, 138.4, 0.186, 0.359]),
    }
    out = {}
    for name, (gname, n, d, half, seed, ptimes) in rows.items():
        x = I.uniform_points(n, d, -half, half, seed)
        y = I.normal(n, seed + 1)
        r = {"n": n, "d": d, "cube_half_width": half, "leaf": LEAF, "eps": EPS, "max_rank": n // 2}
        if ptimes:
            r["paper_s (laptop, one core)"] = dict(zip(["assembly", "factor", "solve", "det"], ptimes))
        else:
            r["note"] = "the case cpu_baseline.dense_limit_sample times on the oracle"
        if gname:
            with open(os.path.join(ROOT, "tests", "golden", f"fullrank_{gname}.json")) as f:
                g = json.load(f)
            ref_ld, r["reference"] = g["logdet"], "oracle (stored value)"
            r["oracle_s_when_stored"] = g["oracle_seconds"]
        else:
            import scipy.linalg as sl
            from scipy.spatial.distance import cdist
            C = np.exp(-cdist(x, x, "sqeuclidean"))
            C[np.diag_indices_from(C)] += 2.0
            ref_ld, r["reference"] = 2.0 * np.log(np.diag(sl.cho_factor(C, lower=True)[0])).sum(), "dense Cholesky (LAPACK)"
        for prec, fname in [(0, "fp64"), (1, "mixed")]:
            for rep in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = H.Hodlr(x, "se", [0.5 ** 0.5, 1.0], 2.0, LEAF, EPS, precision=prec, max_rank=n // 2)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                h.factor()
                t2 = time.perf_counter()
                sol = h.solve(y)
                t3 = time.perf_counter()
                ld = h.logdet()
                t4 = time.perf_counter()
                ph = h.phase_ms()
                lr = [int(v) for v in h.level_ranks()]
                kap, _ = h.tree()
                h.close()
            # leaf sizes of the balanced tree: n split in halves kappa times
            sizes = [n]
            for _ in range(kap):
                sizes = [q for m in sizes for q in (m // 2, m - m // 2)]
            fl = factor_flops(lr, n, sizes)
            r[fname] = {"assembly_ms": 1e3 * (t1 - t0), "compression_ms": ph["compression"],
                        "factor_ms": 1e3 * (t2 - t1), "solve_ms": 1e3 * (t3 - t2),
                        "det_ms": 1e3 * (t4 - t3), "total_ms": 1e3 * (t4 - t0),
                        "logdet": ld, "logdet_rel_err": abs(ld - ref_ld) / abs(ref_ld),
                        "level_ranks": lr,
                        "factor_gflop": fl / 1e9,
                        "factor_fp64_tflops": fl / (ph["factor"] * 1e-3) / 1e12,
                        "factor_frac_of_fp64_peak": fl / (ph["factor"] * 1e-3) / FP64_PEAK,
                        "note": "assembly includes the host-to-device copy of x and the ordering; "
                                "solve includes the host copies of y and x"}
        out[name] = r
    return out


def cpu_model() -> str:
    """The host CPU's model name (/proc/cpuinfo on x86, lscpu on Arm, else the machine)."""
    import platform
    import subprocess
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def cpu_baseline(x, y):
    """The oracle (plain FP64 CPU HODLR, OpenMP over the nodes of a level) on one full step
    of the same workload: one log-likelihood evaluation of each kernel at n = 2^20, on all
    host cores (the reported value) and on one core; then, on all cores, the paper's
    per-phase split (Assembly = ordering + compression, Factor, Solve, Det.)."""
    import os
    import oracle as O
    from paper_1403_6015_gb300 import inputs as I
    cores = os.cpu_count() or 1
    O.set_num_threads(0)
    threads = O.num_threads()
    t0 = time.perf_counter()
    for kern, ell in KERNELS:
        O.Hodlr(x, kern, [ell, 1.0], SIGMA2, LEAF, EPS).loglik(y)
    dt = time.perf_counter() - t0
    phases = {}
    for kern, ell in KERNELS:
        t = [time.perf_counter()]
        h = O.Hodlr(x, kern, [ell, 1.0], SIGMA2, LEAF, EPS)
        t.append(time.perf_counter())
        h.factor()
        t.append(time.perf_counter())
        h.solve(y)
        t.append(time.perf_counter())
        h.logdet()
        t.append(time.perf_counter())
        phases[kern] = {k: t[i + 1] - t[i] for i, k in enumerate(["assembly_s", "factor_s",
                                                                  "solve_s", "det_s"])}
    O.set_num_threads(1)
    t0 = time.perf_counter()
    for kern, ell in KERNELS:
        O.Hodlr(x, kern, [ell, 1.0], SIGMA2, LEAF, EPS).loglik(y)
    d1 = time.perf_counter() - t0
    O.set_num_threads(0)
    # a dense-limit sample: the d = 4 Gaussian row's cube at n = 1200 (every level of full or
    # nearly full rank), one build + factor + solve + log det; the GPU's time on the same
    # case is in the supplementary dense_limit_rows
    xd = I.uniform_points(DENSE_SAMPLE_N, 4, -3.0, 3.0, 2100)
    yd = I.normal(DENSE_SAMPLE_N, 2101)
    t0 = time.perf_counter()
    hd = O.Hodlr(xd, "se", [0.5 ** 0.5, 1.0], 2.0, LEAF, EPS, max_rank=DENSE_SAMPLE_N // 2)
    hd.factor_solve(yd)
    hd.logdet()
    dd = time.perf_counter() - t0
    return {"value": len(KERNELS) / dt, "unit": "evals/s", "cores": threads,
            "kind": "oracle", "sample": "one full step: one loglik per kernel at n=2^20 "
                                        f"({dt:.1f} s on {threads} threads)",
            "cpu_model": cpu_model(), "host_cores": cores,
            "single_thread": {"value": len(KERNELS) / d1, "unit": "evals/s", "cores": 1,
                              "sample": f"the same step on one thread ({d1:.1f} s)"},
            "phases_all_cores": phases,
            "dense_limit_sample": {"seconds": dd, "cores": threads,
                                   "sample": f"C = 2I + exp(-r^2), n = {DENSE_SAMPLE_N} points uniform in "
                                             "[-3, 3]^4, leaf 128, eps 1e-12: build, factor, solve, log det"}}


def run_reference(args):
    """The oracle as the reference arm, on rank 0 only; each step is one full-size step."""
    rank, world, _ = dist_env()
    if not reference_runs_here(rank):
        return
    import oracle as O
    from paper_1403_6015_gb300 import inputs as I
    x, y = I.workload_1d(N, SEED)
    O.build()

    def step():
        for kern, ell in KERNELS:
            O.Hodlr(x, kern, [ell, 1.0], SIGMA2, LEAF, EPS).loglik(y)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * len(KERNELS) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(),
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": "full workload, every step",
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_batched():
    """One batched call for launch-list captures: 4 presized lanes of one n = 65536 point set
    (Matern-5/2, leaf 128, eps 1e-12, mixed form), 16 settings, so 4 rounds."""
    import torch

    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    n, nset, L = 65536, 16, 4
    x, y = I.workload_1d(n, 1003)
    ell, s2 = sweep_settings(nset, 2004)
    ctxs = []
    for s in [torch.cuda.Stream() for _ in range(L)]:
        h = H.Hodlr(x, "matern52", [ell[0], 1.0], s2[0], 128, 1e-12, precision=1, stream=s.cuda_stream)
        h.presize(np.full(h.tree()[0], 4, dtype=np.int32))
        ctxs.append(h)
    theta = torch.from_numpy(np.stack([ell, np.ones(nset)], 1).copy()).cuda()
    sig = torch.from_numpy(s2.copy()).cuda()
    yd = torch.from_numpy(y).cuda()
    out = torch.zeros(nset, dtype=torch.float64, device="cuda")
    status = torch.zeros(nset, dtype=torch.int32, device="cuda")
    origin = torch.cuda.Stream()
    torch.cuda.synchronize()
    H.loglik_batched(ctxs, theta, sig, yd, out, status, stream=origin.cuda_stream)
    torch.cuda.synchronize()
    print(json.dumps({"profile_batched": {"lanes": L, "settings": nset,
                                          "status_ok": bool((status.cpu().numpy() == 0).all())}}))


def profile_dense_row(name):
    """One factorization of a dense-limit row for launch-list and kernel captures: the
    3-D n = 10 000 or the d = 4 n = 5000 Gaussian row of Sec. 5 (the stored oracle inputs,
    FP64 form, leaf 128, eps 1e-12, max_rank n/2): build, factor with the right-hand side,
    log det against the oracle's stored value."""
    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    with open(os.path.join(ROOT, "tests", "golden", f"fullrank_{name}.json")) as f:
        g = json.load(f)
    n = g["n"]
    x = I.uniform_points(n, g["d"], g["box"][0], g["box"][1], g["seed_points"])
    y = I.normal(n, g["seed_y"])
    h = H.Hodlr(x, "se", [g["ell"], g["amp"]], g["sigma2"], g["leaf"], g["eps"], max_rank=n // 2)
    h.factor_solve(y)
    ld = h.logdet()
    print(json.dumps({"profile_dense_row": name, "logdet_rel_err": abs(ld - g["logdet"]) / abs(g["logdet"]),
                      "phase_ms": h.phase_ms()}))


def dense_3d_column(sizes=(20000, 50000, 100000)):
    """The three-dimensional column of the paper's Gaussian table (Sec. 5: C = 2I + exp(-r^2),
    points uniform in [-3, 3]^3) at its larger n, FP64 form, leaf 128, eps 1e-12, max_rank
    min(n/2, 8192): assembly, factor and solve timed per call, and the exact residual
    |C x - y| on 24 rows, each row's product summed in numpy from the covariance's
    definition (no HODLR involved)."""
    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    paper = {20000: [30.9, 33.1, 0.224, 1.06], 50000: [75.5, 76.3, 0.434, 1.68],
             100000: [149.0, 166.0, 0.923, 3.11]}
    out = {}
    for n in sizes:
        x = I.uniform_points(n, 3, -3.0, 3.0, 2300 + n % 97)
        y = I.normal(n, 2301)
        t0 = time.perf_counter()
        h = H.Hodlr(x, "se", [0.5 ** 0.5, 1.0], 2.0, LEAF, EPS, max_rank=min(n // 2, 8192))
        t1 = time.perf_counter()
        h.factor()
        t2 = time.perf_counter()
        sol = h.solve(y)
        t3 = time.perf_counter()
        ld = h.logdet()
        t4 = time.perf_counter()
        kap, _ = h.tree()
        rk = h.ranks()
        h.close()
        rows = np.unique(np.linspace(0, n - 1, 24).astype(np.int64))
        res = 0.0
        for i in rows:
            cx = np.exp(-((x - x[i]) ** 2).sum(1)) @ sol + 2.0 * sol[i]
            res = max(res, abs(cx - y[i]))
        out[str(n)] = {"assembly_s": t1 - t0, "factor_s": t2 - t1, "solve_s": t3 - t2,
                       "det_s": t4 - t3, "total_s": t4 - t0, "logdet": ld,
                       "level_max_rank": [int(rk[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(kap)],
                       "residual_rows_rel": res / np.abs(y).max(),
                       "paper_s (laptop, one core)": dict(zip(["assembly", "factor", "solve", "det"], paper.get(n, [])))}
    print(json.dumps({"dense_3d_column": out}))


def dimension_tables(n=5000, dims=(1, 2, 4, 8, 16, 32, 64)):
    """The paper's two d-dimensional Gaussian tables (Sec. 5: C = 2I + exp(-r^2), n = 5000,
    points uniform in the unscaled cube [-3, 3]^d and in the scaled cube
    [-3/sqrt(d), 3/sqrt(d)]^d), FP64 form, leaf 128, eps 1e-12, max_rank n/2: assembly,
    factor, solve and det timed per call, log det against dense Cholesky (LAPACK)."""
    import scipy.linalg as sl
    from scipy.spatial.distance import cdist
    from paper_1403_6015_gb300 import hodlr as H
    from paper_1403_6015_gb300 import inputs as I
    paper = {"unscaled": {1: [0.02, 0.087, 0.002, 0.001], 2: [1.17, 2.043, 0.027, 0.014],
                          4: [9.67, 21.25, 0.073, 0.088], 8: [10.4, 7.773, 0.041, 0.039],
                          16: [0.09, 0.168, 0.002, 0.002], 32: [0.15, 0.061, 0.004, 0.001],
                          64: [0.21, 0.059, 0.001, 0.001]},
             "scaled": {1: [0.02, 0.087, 0.002, 0.001], 2: [0.70, 1.157, 0.017, 0.005],
                        4: [33.6, 108.2, 0.165, 0.360], 8: [40.8, 138.4, 0.186, 0.359],
                        16: [41.9, 138.7, 0.182, 0.358], 32: [43.4, 174.1, 0.174, 0.354],
                        64: [42.2, 142.2, 0.181, 0.346]}}
    out = {}
    # one build first, so that no row carries the process's first-use set-up
    H.Hodlr(I.uniform_points(n, 1, -3.0, 3.0, 2400), "se", [0.5 ** 0.5, 1.0], 2.0, LEAF, EPS).close()
    for table in ["unscaled", "scaled"]:
        out[table] = {}
        for d in dims:
            half = 3.0 if table == "unscaled" else 3.0 / np.sqrt(d)
            x = I.uniform_points(n, d, -half, half, 2400 + d)
            y = I.normal(n, 2401)
            t0 = time.perf_counter()
            h = H.Hodlr(x, "se", [0.5 ** 0.5, 1.0], 2.0, LEAF, EPS, max_rank=n // 2)
            t1 = time.perf_counter()
            h.factor()
            t2 = time.perf_counter()
            h.solve(y)
            t3 = time.perf_counter()
            ld = h.logdet()
            t4 = time.perf_counter()
            kap, _ = h.tree()
            rk = h.ranks()
            h.close()
            C = np.exp(-cdist(x, x, "sqeuclidean"))
            C[np.diag_indices_from(C)] += 2.0
            ldd = 2.0 * np.log(np.diag(sl.cho_factor(C, lower=True)[0])).sum()
            out[table][str(d)] = {
                "assembly_s": t1 - t0, "factor_s": t2 - t1, "solve_s": t3 - t2, "det_s": t4 - t3,
                "total_s": t4 - t0, "logdet_rel_err_vs_dense": abs(ld - ldd) / abs(ldd),
                "level_max_rank": [int(rk[(1 << j) - 1:(1 << (j + 1)) - 1].max()) for j in range(kap)],
                "paper_s (laptop, one core)": dict(zip(["assembly", "factor", "solve", "det"], paper[table][d]))}
    print(json.dumps({"dimension_tables": out}))


def main():
    global N, COMPRESSION
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the accuracy checks")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the hyperparameter sweeps")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch configuration")
    ap.add_argument("--n", type=int, default=N, help="points (profiling captures only)")
    ap.add_argument("--precision", type=int, default=-1,
                    help="-1: both forms (default), 0: FP64 only, 1: mixed only")
    ap.add_argument("--compression", default="aca", choices=["aca", "chebyshev"],
                    help="compression of the timed evaluations (profiling captures)")
    ap.add_argument("--dimension-tables", action="store_true",
                    help="the d-dimensional Gaussian tables at n = 5000, d = 1 ... 64 (about a minute)")
    ap.add_argument("--dense-3d-column", action="store_true",
                    help="the 3-D Gaussian column at n = 20 000, 50 000, 100 000 (about a minute)")
    ap.add_argument("--profile-dense-row", choices=["d3", "d4"], default=None,
                    help="one factorization of a dense-limit Gaussian row (for captures)")
    ap.add_argument("--profile-batched", action="store_true",
                    help="run one small batched call (4 lanes, 16 Matern-5/2 settings, "
                         "n=65536, mixed form) and exit: the case of the batched launch list")
    args = ap.parse_args()
    N = args.n
    COMPRESSION = args.compression
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.dimension_tables:
        from paper_1403_6015_gb300 import build_lib
        build_lib.build()
        dimension_tables()
        return
    if args.dense_3d_column:
        from paper_1403_6015_gb300 import build_lib
        build_lib.build()
        dense_3d_column()
        return
    if args.profile_dense_row:
        from paper_1403_6015_gb300 import build_lib
        build_lib.build()
        profile_dense_row(args.profile_dense_row)
        return
    if args.profile_batched:
        profile_batched()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
