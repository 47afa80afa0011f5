"""Throughput of the boundary-MPS PEPS search on synthetic Chimera instances.

One step = one batch of 32 independent 16x16 Chimera-like instances solved
concurrently (each a full solve: boundary MPSs bottom-up, then the
branch-and-bound search over every site), every instance 2048 spins in
K_{4,4} cells (256-state clusters), J ~ N(0,1), h ~ N(0, 0.1) on the 2^-24
grid, beta 1, chi 32, one variational sweep per boundary row (the value of
the paper's example), beam 1024.  Metric: beam states per second (sum over
sites of live beam x cluster states, divided by the solve time) and the
time to solution of the mixed-precision path next to the plain FP64 GPU
path, whose best energy must be equal.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: independent instances per rank (replicas, weak scaling); rank 0
prints the JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# batch: instances per step, one lockstep group per 152 (one instance per SM
# for the groups' one-CTA kernels)
WORKLOAD = dict(L=16, couplings="gauss", h_sigma=0.1, beta=1.0, chi=32, beam=1024, sweeps=1, batch=152)
METRIC = "beam states/sec & time-to-solution vs plain FP64 GPU at equal best energy"


# DRAM bytes (read + write) per instance and launch of a dominant kernel,
# from an ncu capture of mid-solve launches (dram__bytes_read.sum +
# dram__bytes_write.sum divided by the instances one launch covers), for the
# kernel as it is now; a kernel not listed here reports null.
NCU_TRAFFIC_BYTES = {
    # the 8-warp kernel in a group of 8 instances: 17.4 MB read + 248.3 MB
    # written per launch (almost all of it the environments it writes)
    "k_renv_tc": (17.4e6 + 248.3e6) / 8,
}

# kernels whose products run on the tensor cores (split TF32: three TF32
# passes per FP32-accurate multiply-add)
TENSOR_KERNELS = ("k_renv_tc", "k_umma_tf32x3")


def make_instance(seed):
    import instances
    return instances.chimera(WORKLOAD["L"], seed, couplings=WORKLOAD["couplings"], h_sigma=WORKLOAD["h_sigma"])


def config_dict(extra=None):
    L = WORKLOAD["L"]
    c = {"workload": f"{WORKLOAD['batch']} x chimera{L}x{L}_gauss_K44 ({8 * L * L} spins, d=256), "
                     f"beta={WORKLOAD['beta']:g}, chi={WORKLOAD['chi']}, {WORKLOAD['sweeps']} sweep, "
                     f"beam={WORKLOAD['beam']}",
         "L": WORKLOAD["L"], "spins": 8 * WORKLOAD["L"] ** 2, "cluster_states": 256, "beta": WORKLOAD["beta"],
         "chi": WORKLOAD["chi"], "num_sweeps": WORKLOAD["sweeps"], "beam": WORKLOAD["beam"], "couplings": "J~N(0,1), h~N(0,0.1) on 2^-24 grid",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


class Clocks:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_oracle_sample(seed, max_sites=6):
    """Oracle on a bounded sample of one 16x16 solve: the full boundary phase
    (all 15 boundary MPSs) and the first max_sites sites of the search.  From
    the third site on the beam is full (1024 x 256 candidates per site), so
    the per-site cost of sites 2 .. max_sites-1 projects the search over all
    256 sites; the value is the projected full solve's beam states per
    second."""
    import numpy as np

    from oracle import boundary, peps, search, tables
    inst = make_instance(seed)
    t0 = time.perf_counter()
    fg = tables.from_ising(inst)
    p = peps.build(fg, WORKLOAD["beta"])
    bd = boundary.boundary_mpses(p, WORKLOAD["chi"], WORKLOAD["sweeps"])
    t_boundary = time.perf_counter() - t0
    beam = [search._Partial((), 0, 0.0, np.ones(1))]
    cols = fg.cols
    cand = 0
    B = bd[1]
    for b in beam:
        b.R = search.right_envs(p, B, 0, None)
    site_t, site_c = [], []
    for s in range(max_sites):
        ts = time.perf_counter()
        c0 = cand
        i, j = divmod(s, cols)
        ks = search.key_sites(fg, s)
        children = {}
        for b in beam:
            lc = search.log_conditional(p, B, i, j, b.lenv, b.R, b.states)
            dEs = search.delta_energies(fg, s, b.states)
            for x in range(fg.d[s]):
                st = b.states + (x,)
                E = b.E + int(dEs[x])
                key = tuple(st[t] for t in ks)
                cand += 1
                cur = children.get(key)
                if cur is None or (E, st) < (cur[1], cur[0]):
                    children[key] = (st, E, b.logp + float(lc[x]), b)
        cands = sorted(children.values(), key=lambda c: (-c[2], c[1], c[0]))[:WORKLOAD["beam"]]
        new = []
        for st, E, lp, parent in sorted(cands, key=lambda c: c[0]):
            v = parent.lenv @ B.sites[j][:, p.site(i, j).PD[st[-1]], :]
            new.append(search._Partial(st, E, lp, v / np.max(np.abs(v)), parent.R))
        beam = new
        site_t.append(time.perf_counter() - ts)
        site_c.append(cand - c0)
    dt = time.perf_counter() - t0
    n_sites = fg.n_sites
    full = 2  # sites 0 and 1 fill the beam
    per_site_t = statistics.mean(site_t[full:]) if len(site_t) > full else site_t[-1]
    per_site_c = statistics.mean(site_c[full:]) if len(site_c) > full else site_c[-1]
    proj_t = t_boundary + sum(site_t[:full]) + per_site_t * (n_sites - full)
    proj_c = sum(site_c[:full]) + per_site_c * (n_sites - full)
    cores = len(os.sched_getaffinity(0))
    return {"value": proj_c / proj_t, "unit": "beam states/s", "cores": cores, "kind": "oracle",
            "sample": f"1 instance (chimera16x16 gauss, chi=32, 1 sweep, beam=1024): all 15 boundary MPSs "
                      f"({t_boundary:.1f} s) + the first {max_sites} search sites ({cand} beam states, "
                      f"{sum(site_t):.1f} s); value = projected full solve ({proj_c:.3g} beam states in "
                      f"{proj_t:.0f} s, sites {full}.. at the measured per-site cost {per_site_t:.2f} s)",
            "sampled_rate": cand / dt, "boundary_s": t_boundary, "projected_solve_s": proj_t}


def cpu_oracle_chimera3x3(seeds=(0, 1)):
    """Full oracle solves of the plain FP64 workload (3x3 Chimera, +-1, beta
    1, chi 16, beam 256): beam states per second, no sampling."""
    import instances as I
    from oracle import search, tables
    cand, t = 0.0, 0.0
    for sd in seeds:
        fg = tables.from_ising(I.chimera(3, sd))
        t0 = time.perf_counter()
        res = search.solve(fg, search.Params(beta=1.0, chi=16, beam=256))
        t += time.perf_counter() - t0
        cand += sum(c for c, _ in res.steps)
    return {"value": cand / t, "unit": "beam states/s", "seeds": len(seeds), "s": t}


def cpu_oracle_chimera3x3_one_thread():
    """cpu_oracle_chimera3x3 in a child process with every BLAS pool at 1
    thread (the variables are read when NumPy loads)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = "import bench, json; print(json.dumps(bench.cpu_oracle_chimera3x3()))"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def sweeps_to_fidelity(trace, best, tol=1e-6):
    """Sweeps until F_k / F_best = exp(2 (log_overlap_k - best)) >= 1 - tol
    (len(trace) + 1 when never reached)."""
    import numpy as np
    ok = np.nonzero(2.0 * (np.asarray(trace) - best) >= np.log1p(-tol))[0]
    return int(ok[0]) + 1 if ok.size else len(trace) + 1


def warm_start_leg(spg, ctx, torch, n_train=16, n_eval=2, eval_rows=(2, 9), n_sweeps=12, steps=1500, chi=64,
                   hidden=256):
    """The learned warm start (trained on 12x12 +-1 Chimera instances,
    judged on unseen 16x16 ones at chi 64, scaled down to bench minutes): an
    MLP from the couplings near a boundary row to that row's MPS
    sites, trained by the library's own kernels on every row the method
    builds for n_train 12x12 +-1 Chimera instances at chi 64, then judged on
    unseen 16x16 instances by the plain contraction: sweeps until the
    fidelity with W psi reaches 1 - 1e-6 of the best compression, from the
    network's start and from the SVD zipper's."""
    import numpy as np

    import instances as I
    prm = spg.params(beta=1.0, chi=chi, num_sweeps=1, precision=spg.SPG_MIXED)
    t0 = time.perf_counter()
    X, T = [], []
    for k in range(n_train):
        inst = I.chimera(12, 10000 + k)
        prob = spg.spg_problem_ising(ctx, inst)
        out, _ = spg.spg_boundary_export(ctx, prob, prm, 0)
        T.append(out.reshape((inst.grid_rows - 1) * inst.grid_cols, -1))
        X.append(np.concatenate([spg.spg_warm_features(prob, r) for r in range(1, inst.grid_rows)]))
        prob.close()
    Xd = torch.tensor(np.concatenate(X), device="cuda")
    Td = torch.cat(T).contiguous()
    del T
    t_gen = time.perf_counter() - t0
    net = spg.Mlp(ctx, spg.SPG_WS_FEATURES, hidden, 16 * chi * chi, seed=0)
    l0, _ = net.loss_grad(Xd[:256], Td[:256])
    t1 = time.perf_counter()
    loss = net.train(Xd, Td, batch=64, steps=steps, lr=1e-3, seed=1)
    t_train = time.perf_counter() - t1
    spg.spg_set_warm_start(ctx, net)
    counts = {"zipper": [], "network": []}
    first = []
    t2 = time.perf_counter()
    for k in range(n_eval):
        inst = I.chimera(16, 20000 + k)
        prob = spg.spg_problem_ising(ctx, inst)
        for row in eval_rows:
            tz, tn = spg.spg_sweep_trace(ctx, prob, prm, row, 2, n_sweeps)
            best = max(tz.max(), tn.max())
            counts["zipper"].append(sweeps_to_fidelity(tz, best))
            counts["network"].append(sweeps_to_fidelity(tn, best))
            first.append({"zipper": float(tz[0] - best), "network": float(tn[0] - best)})
        prob.close()
    t_eval = time.perf_counter() - t2
    spg.spg_set_warm_start(ctx, None)
    samples = int(Xd.shape[0])
    del Xd, Td
    return {"workload": f"train: every boundary row of {n_train} chimera12x12 +-1 instances at chi={chi} "
                        f"({samples} sites, 1 sweep per row); evaluate: rows {list(eval_rows)} of {n_eval} unseen "
                        f"chimera16x16 +-1 at chi={chi}, {n_sweeps} sweeps from each start",
            "network": f"{spg.SPG_WS_FEATURES}-{hidden}-{hidden}-{16 * chi * chi} tanh MLP, FP32 training "
                       f"(Adam, lr 1e-3, batch 64, {steps} steps), BF16 inference",
            "loss_initial": l0, "loss_final": loss,
            "sweeps_to_1e-6": counts, "mean_sweeps": {k: float(np.mean(v)) for k, v in counts.items()},
            "log_overlap_deficit_after_1_sweep": first,
            "seconds": {"generate": t_gen, "train": t_train, "evaluate": t_eval}}


def rank_instance_seed(rank: int) -> int:
    """Replicas: every rank solves its own independent instance."""
    return 1000 + rank


def aggregate_over_ranks(tot_ms: float, tot_cand: float, device="cpu"):
    """Whole-job figures of independent replicas: the slowest rank's time and
    the beam states of all ranks (no data-path collective; this reduction of
    two scalars happens once, after the timed region)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tot_ms, tot_cand
    t = torch.tensor([tot_ms], dtype=torch.float64, device=device)
    c = torch.tensor([tot_cand], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def kernel_profile(spg, ctx, prob, prm):
    """{kernel: [launches, device ms, flops]} of one solve, timed by event
    nodes captured into the solve's graph (device times, no host gaps)."""
    spg.spg_profile(ctx, True)
    spg.spg_solve(ctx, prob, prm).get()
    kern = spg.spg_profile_report(ctx)
    spg.spg_profile(ctx, False)
    return kern


def group_kernel_profile(spg, ctx, probs, prm):
    """The same for one lockstep group of the given problems (every launch
    covers all of them; its flops are the group's)."""
    spg.spg_profile(ctx, True)
    for r in spg.spg_solve_group(ctx, probs, prm):
        r.get()
    kern = spg.spg_profile_report(ctx)
    spg.spg_profile(ctx, False)
    return kern


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        cpu_oracle_sample(0, max_sites=2)
    for k in range(args.steps):
        vals.append(cpu_oracle_sample(0, max_sites=4))
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "beam states/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(), "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "beam states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--batch", type=int, default=WORKLOAD["batch"], help="instances solved concurrently per step")
    ap.add_argument("--ncu-solve", action="store_true",
                    help="solve the batch once (its first, uncaptured occurrence) and exit: the command of an ncu "
                         "launch list of one step's kernels; prints no bench line")
    ap.add_argument("--group-max", type=int, default=0,
                    help="most instances per lockstep group (0: automatic, 1: every instance on its own stream)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-king", action="store_true", help="skip the king's-graph Potts solves")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm-start leg")
    ap.add_argument("--L", type=int, default=None,
                    help="grid side override (profiling of a smaller case of the same kernels)")
    ap.add_argument("--beam", type=int, default=None,
                    help="beam override (batches of small-beam solves; not the benchmark workload)")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="tile shapes timed at each shape's first uncaptured launch (on) or the built-in ones (off)")
    ap.add_argument("--only-main", action="store_true",
                    help="timed steps only (no end-to-end, FP64, uneven-batch or profile runs): the ncu "
                         "launch list")
    args = ap.parse_args()
    if args.L:
        WORKLOAD["L"] = args.L
    if args.beam:
        WORKLOAD["beam"] = args.beam
    WORKLOAD["batch"] = args.batch
    if args.impl == "reference":
        return run_reference(args)

    # the package first: it asks for 32 hardware work queues, which only
    # applies before the process creates its CUDA context
    import paper_2502_02317_gb300 as spg
    import torch

    spg.spg_autotune_set(spg.SPG_TUNE_ON if args.autotune == "on" else spg.SPG_TUNE_OFF)
    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    NB = args.batch
    stream = torch.cuda.Stream()
    ctx = spg.Context(local, stream=stream.cuda_stream)
    insts = [make_instance(rank_instance_seed(rank) * 100 + k) for k in range(NB)]
    probs = [spg.spg_problem_ising(ctx, i) for i in insts]
    prec = spg.SPG_MIXED if args.precision == "mixed" else spg.SPG_FP64

    def params(p):
        return spg.params(beta=WORKLOAD["beta"], chi=WORKLOAD["chi"], beam=WORKLOAD["beam"], precision=p,
                          num_sweeps=WORKLOAD["sweeps"], group_max=args.group_max)

    prm = params(prec)
    prms = [prm] * NB
    if args.ncu_solve:
        rs = spg.spg_solve_batch(ctx, probs, prms)
        n = sum(r.info()["kernel_launches"] / max(1, r.info()["group_size"]) for r in rs)
        for r in rs:
            r.get()
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"ncu_solve": {"instances": NB, "kernel_launches": int(round(n))}}))
        return 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    # warm-up: the first solve of a (problem, params) runs uncaptured, the
    # second is captured into CUDA graphs, later ones replay them
    for _ in range(max(args.warmup, 3)):
        for r in spg.spg_solve_batch(ctx, probs, prms):
            r.get()
    barrier()
    times, cands, launches, infos, bests, group_sizes = [], [], [], [], [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            rs, ms_step = timed(lambda: spg.spg_solve_batch(ctx, probs, prms))
            times.append(ms_step)
            inf = [r.info() for r in rs]
            infos.append(inf[0])
            cands.append(sum(i["candidates"] for i in inf))
            # a lockstep group's results each report the group's launches
            launches.append(sum(i["kernel_launches"] / max(1, i["group_size"]) for i in inf))
            group_sizes.append(max(i["group_size"] for i in inf))
            bests = [int(r.get()[1][0]) for r in rs]
    barrier()
    ms = statistics.mean(times)
    tot_ms, tot_cand = aggregate_over_ranks(sum(times), sum(cands), device="cuda")
    value = tot_cand / (tot_ms / 1e3)

    line = {"metric": METRIC, "value": value, "unit": "beam states/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == spg.SPG_MIXED else "f64", "data": "synthetic",
            "config": config_dict({"precision": args.precision,
                                   "parallelism": f"replicas x{world}, {NB} instances per GPU in lockstep groups "
                                                  f"of up to {max(group_sizes) if group_sizes else 1} "
                                                  f"(one launch sequence per group)"}),
            "gpu_launches": int(sum(launches)), "clocks": clk.summary()}
    # the autotuner's choices for the shapes of the timed step (timed during
    # the warm-up's uncaptured solves; the timed steps replay graphs
    # captured with them)
    choices = {}
    timed_shapes = spg.spg_autotune_report()
    for kern, _dev, _grp, _shape, choice, _us in timed_shapes:
        choices.setdefault(kern, {}).setdefault(str(choice), 0)
        choices[kern][str(choice)] += 1
    line["autotune"] = {"mode": args.autotune, "shapes_timed": len(timed_shapes), "variant_counts": choices}
    if args.only_main:
        # per-kernel device times of one more solve (after the timed steps),
        # to set beside an ncu launch list of the timed step
        kern = kernel_profile(spg, ctx, probs[0], prm)
        ktot = sum(v[1] for v in kern.values())
        line["kernels"] = {k: {"launches": int(v[0]), "ms": round(v[1], 3), "share": round(v[1] / ktot, 4)}
                           for k, v in sorted(kern.items(), key=lambda kv: -kv[1][1])}
        if rank == 0:
            print(json.dumps(line))
        return 0

    # time to solution of one instance (graph replay), its phases
    for _ in range(3):
        spg.spg_solve(ctx, probs[0], prm).get()
    r1, tts_ms = timed(lambda: spg.spg_solve(ctx, probs[0], prm))
    inf1 = r1.info()
    line["tts_s"] = tts_ms / 1e3
    line["best_energies"] = [b * 2.0 ** -insts[0].energy_shift for b in bests]
    line["phase_ms"] = {"boundary": inf1["ms_boundary"], "search": inf1["ms_search"]}
    line["diagnostics"] = {"near_ties": inf1["near_ties"], "degenerate_cuts": inf1["degenerate_cuts"],
                           "jacobi_sweeps_max": inf1["jacobi_sweeps_max"], "error_flags": inf1["error_flags"]}

    # end to end through the C ABI from host arrays: every step a new batch
    # of instances (drawn before the timed region) enters through the public
    # API -- new couplings written into the existing problems (tables built
    # on the host, uploaded in place, 32 host threads), the batch solved by
    # replaying the captured solves, results read back to the host
    from concurrent.futures import ThreadPoolExecutor
    steps_insts = [[make_instance(rank_instance_seed(rank) * 100 + 50000 + st_ * NB + k) for k in range(NB)]
                   for st_ in range(args.steps)]
    pool = ThreadPoolExecutor(max_workers=NB)
    e2e_times, e2e_build, e2e_cands = [], [], []
    for st_ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        list(pool.map(lambda pi: spg.spg_problem_update_ising(pi[0], pi[1].J, pi[1].h),
                      zip(probs, steps_insts[st_])))
        t1 = time.perf_counter()
        rs = spg.spg_solve_batch(ctx, probs, prms)
        outs = [r.get() for r in rs]
        e2e_times.append(time.perf_counter() - t0)
        e2e_build.append(t1 - t0)
        e2e_cands.append(sum(r.info()["candidates"] for r in rs))
    pool.shutdown()
    n_sites = insts[0].grid_rows * insts[0].grid_cols
    # per problem and step: the value tables written in place (local E and
    # the left, up and anti-diagonal reduced tables, int64)
    h2d = NB * 8 * n_sites * (256 + 3 * 256)
    d2h = sum(len(o[1]) * (2 * n_sites + 8 + 8) + 16 for o in outs)
    line["e2e"] = {"value": sum(e2e_cands) / sum(e2e_times), "unit": "beam states/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   # per step: the tables of the new instances (host build +
                   # upload), then the batch solved from its captured graphs
                   "build_s": statistics.mean(e2e_build),
                   "solve_s": statistics.mean(e2e_times) - statistics.mean(e2e_build),
                   "path": "spg_problem_update_ising + spg_solve_batch (graph replay) + spg_result_get"}
    # the problems hold the last step's instances now: restore the timed batch
    for pr, inst in zip(probs, insts):
        spg.spg_problem_update_ising(pr, inst.J, inst.h)

    # plain FP64 GPU path: the same instance's time to solution, timed like
    # the mixed one (graph replay after warm-up runs), and the best energies
    # of 8 instances of the batch against the mixed path's
    if prec != spg.SPG_FP64:
        p64 = params(spg.SPG_FP64)
        for _ in range(2):  # uncaptured first solve, then the graph capture
            spg.spg_solve(ctx, probs[0], p64).get()
        t64 = []
        for _ in range(min(args.steps, 2)):
            r641, ms641 = timed(lambda: spg.spg_solve(ctx, probs[0], p64))
            r641.get()
            t64.append(ms641)
        nb8 = min(8, NB)
        rs64, ms64 = timed(lambda: spg.spg_solve_batch(ctx, probs[:nb8], [p64] * nb8))
        b64 = [int(r.get()[1][0]) for r in rs64]
        tts64 = statistics.mean(t64) / 1e3
        line["fp64_gpu"] = {"tts_s": tts64, "tts_runs": len(t64), "batch8_first_run_ms": ms64,
                            "equal_best_energy": all(a == b for a, b in zip(b64, bests[:nb8])),
                            "instances_compared": nb8,
                            "speedup_mixed_vs_fp64": {"single_instance": tts64 / line["tts_s"]}}
        # the mixed result's own log-marginal error against plain FP64 (every
        # returned state's conditionals along its path)
        rc_ = spg.spg_solve(ctx, probs[0], spg.params(beta=WORKLOAD["beta"], chi=WORKLOAD["chi"],
                                                      beam=WORKLOAD["beam"], precision=prec,
                                                      num_sweeps=WORKLOAD["sweeps"], check_fp64=1))
        line["max_logmarg_err"] = rc_.max_logmarg_err()
        line["fp64_rows"] = rc_.info()["fp64_rows"]

    # beta = 4 (the precision config's second temperature): one instance,
    # mixed against plain FP64, times after warm-up, best energies, and the
    # mixed result's log-marginal error against FP64
    if WORKLOAD["L"] == 16 and prec != spg.SPG_FP64:
        b4 = {}
        for bprec in (prec, spg.SPG_FP64):
            bprm = spg.params(beta=4.0, chi=WORKLOAD["chi"], beam=WORKLOAD["beam"], precision=bprec,
                              num_sweeps=WORKLOAD["sweeps"])
            for _ in range(2):
                spg.spg_solve(ctx, probs[0], bprm).get()
            rb, msb = timed(lambda: spg.spg_solve(ctx, probs[0], bprm))
            _, Eb, _ = rb.get()
            b4[bprec] = {"tts_s": msb / 1e3, "best_energy_fixed": int(Eb[0]),
                         "beam_states_per_s": rb.info()["candidates"] / (msb / 1e3),
                         "precision_used": "fp64" if rb.info()["precision_used"] == spg.SPG_FP64 else "mixed"}
        rcb = spg.spg_solve(ctx, probs[0], spg.params(beta=4.0, chi=WORKLOAD["chi"], beam=WORKLOAD["beam"],
                                                      precision=prec, num_sweeps=WORKLOAD["sweeps"], check_fp64=1))
        line["beta4"] = {"workload": "chimera16x16 gauss (first instance), beta=4, chi=32, 1 sweep, beam=1024",
                         "mixed": b4[prec], "fp64": b4[spg.SPG_FP64],
                         "equal_best_energy": b4[prec]["best_energy_fixed"] == b4[spg.SPG_FP64]["best_energy_fixed"],
                         "speedup_mixed_vs_fp64": b4[spg.SPG_FP64]["tts_s"] / b4[prec]["tts_s"],
                         "max_logmarg_err": rcb.max_logmarg_err()}

    # batching pattern on uneven instances: 64 Chimera L ~ U{6..12}, +-1,
    # chi in {16, 32} per instance, beam 512, all in flight together
    import instances as I
    if WORKLOAD["L"] == 16:
        un = I.batch_chimera(64, 6, 12, 5000 + rank)
        up = [spg.spg_problem_ising(ctx, inst) for inst, _ in un]
        upr = [spg.params(beta=1.0, chi=c, beam=512, precision=prec) for _, c in un]
        for _ in range(2):
            for r in spg.spg_solve_batch(ctx, up, upr):
                r.get()
        rsu, msu = timed(lambda: spg.spg_solve_batch(ctx, up, upr))
        cu = sum(r.info()["candidates"] for r in rsu)
        line["batch_uneven"] = {"instances": 64, "L": "U{6..12}", "chi": "{16,32}", "beam": 512, "ms": msu,
                                "beam_states_per_s": cu / (msu / 1e3)}

    # king's graph: 16x16 Potts sites with 16 states, N(0,1) local and
    # pairwise tables on all 8-neighbour edges, chi 64, beam 2048 (left bonds
    # of 16 x 16); time to solution of the mixed path next to the plain FP64
    # path, same instance, best energies compared
    if WORKLOAD["L"] == 16 and not args.no_king:
        kinst = I.king_potts(16, 16, 7)
        kp = spg.spg_problem_potts(ctx, kinst)
        kres = {}
        for kprec, reps in ((prec, 3), (spg.SPG_FP64, 1)):
            kprm = spg.params(beta=1.0, chi=64, beam=2048, precision=kprec)
            for _ in range(reps - 1):
                spg.spg_solve(ctx, kp, kprm).get()
            rk, msk = timed(lambda: spg.spg_solve(ctx, kp, kprm))
            stk, Ek, _ = rk.get()
            ik = rk.info()
            kres[kprec] = {"tts_s": msk / 1e3, "best_energy_fixed": int(Ek[0]),
                           "beam_states_per_s": ik["candidates"] / (msk / 1e3),
                           "phase_ms": {"boundary": ik["ms_boundary"], "search": ik["ms_search"]},
                           "error_flags": ik["error_flags"]}
        line["king_potts16x16_d16"] = {
            "workload": "king's graph 16x16, Potts d=16, E~N(0,1) on 2^-24 grid, 930 edges, beta=1, chi=64, beam=2048",
            "mixed": kres[prec], "fp64": kres[spg.SPG_FP64],
            "equal_best_energy": kres[prec]["best_energy_fixed"] == kres[spg.SPG_FP64]["best_energy_fixed"],
            "speedup_mixed_vs_fp64": kres[spg.SPG_FP64]["tts_s"] / kres[prec]["tts_s"]}

    # the learned warm start of the variational compression
    if WORKLOAD["L"] == 16 and not args.no_warm:
        line["warm_start"] = warm_start_leg(spg, ctx, torch)

    # one extra solve with per-kernel device times (graph-captured event
    # nodes; not part of the timed steps): the roofline of the top kernel
    # the timed step's own launch shape: one of its lockstep groups (as
    # large as the step's largest), or one solve when the step ran ungrouped
    gsize = max(1, int(group_sizes[-1])) if group_sizes else 1
    kern = (group_kernel_profile(spg, ctx, probs[:gsize], prm) if gsize > 1
            else kernel_profile(spg, ctx, probs[0], prm))
    ktot = sum(v[1] for v in kern.values())
    top = sorted(kern.items(), key=lambda kv: -kv[1][1])
    line["kernels"] = {k: {"launches": int(v[0]), "ms": round(v[1], 3), "share": round(v[1] / ktot, 4),
                           "avg_us": round(1e3 * v[1] / v[0], 2)} for k, v in top[:10]}
    # ALU peaks measured on this device (FMA throughput of all SMs), next to
    # the unit-count figure at the clock seen during the timed region
    props = torch.cuda.get_device_properties(local)
    clk_mhz = line["clocks"].get("sm_max_mhz") or 2070.0
    peak32 = spg.spg_peak_probe("fp32", stream=stream)
    peak64 = spg.spg_peak_probe("fp64", stream=stream)
    line["alu_peaks"] = {"fp32_tflops": peak32, "fp64_tflops": peak64, "sms": props.multi_processor_count,
                         "fp32_units_tflops": props.multi_processor_count * 128 * 2 * clk_mhz * 1e6 / 1e12,
                         "source": "measured: k_fma_probe (8 independent FMA chains per thread, 8 blocks of 256 "
                                   "threads per SM), CUDA events"}
    alu_peak = peak32 if prec == spg.SPG_MIXED else peak64
    peaks, src = measured_peaks()
    # TF32 dense: the measured BF16 peak (sustained: kernels inside a long
    # step) x the nominal TF32/BF16 ratio 1.1/2.25; FP32-accurate split-TF32
    # products deliver a third of it
    tf32x3_peak = peaks["bf16_tflops_sustained"] * 1.1 / 2.25 / 3.0

    def kernel_roofline(name, nl, ms_k, fl_k):
        tensor = name in TENSOR_KERNELS and prec == spg.SPG_MIXED
        achieved = fl_k / (ms_k / 1e3) / 1e12 if ms_k > 0 else 0.0
        peak = tf32x3_peak if tensor else alu_peak
        traffic = NCU_TRAFFIC_BYTES.get(name)
        return {"kernel": name, "bound": "tensor" if tensor else "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic * gsize if traffic is not None else None,
                "peak_source": (f"measured BF16 sustained {peaks['bf16_tflops_sustained']} TF/s x 1.1/2.25 (TF32) / 3 "
                                "(split-TF32 passes), " + src if tensor else
                                f"measured {'FP32' if prec == spg.SPG_MIXED else 'FP64'} FMA throughput "
                                f"(k_fma_probe, {props.multi_processor_count} SMs)"),
                "share_of_step": round(ms_k / ktot, 4), "flops_per_launch": fl_k / nl,
                "avg_launch_us": 1e3 * ms_k / nl, "instances_per_launch": gsize}
    # the dominant kernel of the step (largest device time) with its
    # algorithmic flops, and the other counted kernels beside it
    counted = [kv for kv in top if kv[1][2] > 0]
    name, (nl, ms_k, fl_k) = counted[0] if counted else top[0]
    line["roofline"] = {**kernel_roofline(name, nl, ms_k, fl_k), "hbm_peak_gbs": peaks.get("hbm_gbs"),
                        "peaks_source": src,
                        "dominant_uncounted": [k for k, _ in top[:3] if k not in dict(counted)]}
    line["kernel_rooflines"] = [kernel_roofline(k, *v) for k, v in counted[:6]]
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample(0)
        line["cpu_baseline_chimera3x3"] = {"all_cores": {**cpu_oracle_chimera3x3(),
                                                         "cores": len(os.sched_getaffinity(0))},
                                           "one_thread": {**cpu_oracle_chimera3x3_one_thread(), "cores": 1},
                                           "workload": "full oracle solves of 3x3 Chimera +-1, beta 1, chi 16, "
                                                       "beam 256 (seeds 0, 1)"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
