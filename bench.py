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

WORKLOAD = dict(L=16, couplings="gauss", h_sigma=0.1, beta=1.0, chi=32, beam=1024, sweeps=1, batch=32)
METRIC = "beam states/sec & time-to-solution vs plain FP64 GPU at equal best energy"


# DRAM bytes (read + write) per launch of a dominant kernel, from an ncu
# capture of two mid-solve launches of the 16x16 solve (dram__bytes_read.sum
# + dram__bytes_write.sum, mean of the two), for the kernel as it is now; a
# kernel not listed here reports null.  (k_cgs2_rows: 118,400 B was measured
# on the per-vector panel version, before the Cholesky-QR panels; not listed
# until its counters are taken again.)
NCU_TRAFFIC_BYTES = {}


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
    """Oracle on a bounded sample: full boundary MPSs + the first sites of the
    search (beam states counted on those sites)."""
    import numpy as np

    from oracle import boundary, peps, search, tables
    inst = make_instance(seed)
    t0 = time.perf_counter()
    fg = tables.from_ising(inst)
    p = peps.build(fg, WORKLOAD["beta"])
    bd = boundary.boundary_mpses(p, WORKLOAD["chi"], WORKLOAD["sweeps"])
    # search restricted to the first max_sites sites of row 0
    beam = [search._Partial((), 0, 0.0, np.ones(1))]
    cols = fg.cols
    cand = 0
    B = bd[1]
    for b in beam:
        b.R = search.right_envs(p, B, 0, None)
    for s in range(max_sites):
        i, j = divmod(s, cols)
        ks = search.key_sites(fg, s)
        children = {}
        for b in beam:
            lc = search.log_conditional(p, B, i, j, b.lenv, b.R, b.states)
            for x in range(fg.d[s]):
                st = b.states + (x,)
                E = b.E + search.delta_energy(fg, s, x, b.states)
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
    dt = time.perf_counter() - t0
    cores = len(os.sched_getaffinity(0))
    return {"value": cand / dt, "unit": "beam states/s", "cores": cores, "kind": "oracle",
            "sample": f"1 instance: tables + all 15 boundary MPSs (chi=32, full SVD, 1 sweep) + the first {max_sites} "
                      f"search sites ({cand} beam states) in {dt:.1f} s"}


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
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-king", action="store_true", help="skip the king's-graph Potts solves")
    ap.add_argument("--L", type=int, default=None,
                    help="grid side override (profiling of a smaller case of the same kernels)")
    ap.add_argument("--beam", type=int, default=None,
                    help="beam override (batches of small-beam solves; not the benchmark workload)")
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
                          num_sweeps=WORKLOAD["sweeps"])

    prm = params(prec)
    prms = [prm] * NB
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
    times, cands, launches, infos, bests = [], [], [], [], []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            rs, ms_step = timed(lambda: spg.spg_solve_batch(ctx, probs, prms))
            times.append(ms_step)
            inf = [r.info() for r in rs]
            infos.append(inf[0])
            cands.append(sum(i["candidates"] for i in inf))
            launches.append(sum(i["kernel_launches"] for i in inf))
            bests = [int(r.get()[1][0]) for r in rs]
    barrier()
    ms = statistics.mean(times)
    tot_ms, tot_cand = aggregate_over_ranks(sum(times), sum(cands), device="cuda")
    value = tot_cand / (tot_ms / 1e3)

    line = {"metric": METRIC, "value": value, "unit": "beam states/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == spg.SPG_MIXED else "f64", "data": "synthetic",
            "config": config_dict({"precision": args.precision,
                                   "parallelism": f"replicas x{world}, {NB} instances in flight per GPU"}),
            "gpu_launches": int(sum(launches)), "clocks": clk.summary()}
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

    # end to end through the C ABI from host arrays: problems built and
    # copied, the batch solved, results copied back
    e2e_times, e2e_build = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ps = [spg.spg_problem_ising(ctx, i) for i in insts]
        t1 = time.perf_counter()
        rs = spg.spg_solve_batch(ctx, ps, prms)
        outs = [r.get() for r in rs]
        e2e_times.append(time.perf_counter() - t0)
        e2e_build.append(t1 - t0)
        for r in rs:
            r.close()
        for p_ in ps:
            p_.close()
    n_sites = insts[0].grid_rows * insts[0].grid_cols
    # device tables per problem: E (int64) + 4 projectors (uint8) per state,
    # 2 reduced 16x16 int64 tables, dims, state lists, merge keys per site
    h2d = NB * (n_sites * (8 * 256 + 4 * 256 + 2 * 256 + 8 * 256 * 2 + 4 * 8 + 4 * 17 + 4 * 41 + 4) + 4)
    d2h = sum(len(o[1]) * (2 * n_sites + 8 + 8) + 16 for o in outs)
    line["e2e"] = {"value": statistics.mean(cands) / statistics.mean(e2e_times), "unit": "beam states/s",
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   # per step: problem construction (host tables + upload), and
                   # the first (uncaptured) solve of the new problems + results
                   "build_s": statistics.mean(e2e_build),
                   "solve_s": statistics.mean(e2e_times) - statistics.mean(e2e_build)}

    # plain FP64 GPU path on the same batch: time, equal best energies
    if prec != spg.SPG_FP64:
        p64 = [params(spg.SPG_FP64)] * NB
        rs64, ms64 = timed(lambda: spg.spg_solve_batch(ctx, probs, p64))
        b64 = [int(r.get()[1][0]) for r in rs64]
        r641, ms641 = timed(lambda: spg.spg_solve(ctx, probs[0], p64[0]))
        r641.get()
        line["fp64_gpu"] = {"batch_ms": ms64, "tts_s": ms641 / 1e3,
                            "equal_best_energy": all(a == b for a, b in zip(b64, bests)),
                            "speedup_mixed_vs_fp64": {"batch": ms64 / ms, "single_instance": ms641 / tts_ms}}

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

    # one extra solve with per-kernel device times (graph-captured event
    # nodes; not part of the timed steps): the roofline of the top kernel
    kern = kernel_profile(spg, ctx, probs[0], prm)
    ktot = sum(v[1] for v in kern.values())
    top = sorted(kern.items(), key=lambda kv: -kv[1][1])
    line["kernels"] = {k: {"launches": int(v[0]), "ms": round(v[1], 3), "share": round(v[1] / ktot, 4),
                           "avg_us": round(1e3 * v[1] / v[0], 2)} for k, v in top[:10]}
    clk_mhz = 2070.0
    # ALU peaks from unit counts: 152 SMs x (128 FP32 | 2 FP64) FMA/clk x 2 flop x clock
    alu_peak = 152 * (128 if prec == spg.SPG_MIXED else 2) * 2 * clk_mhz * 1e6 / 1e12
    name, (nl, ms_k, fl_k) = next((kv for kv in top if kv[1][2] > 0), top[0])
    achieved = fl_k / (ms_k / 1e3) / 1e12 if ms_k > 0 else 0.0
    peaks, src = measured_peaks()
    line["roofline"] = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                        "frac": achieved / alu_peak, "traffic": NCU_TRAFFIC_BYTES.get(name),
                        "peak_source": f"derived: 152 SMs x {'128 FP32' if prec == spg.SPG_MIXED else '2 FP64'} "
                                       f"FMA/clk x 2 x {clk_mhz:.0f} MHz",
                        "share_of_solve": round(ms_k / ktot, 4), "flops_per_launch": fl_k / nl,
                        "avg_launch_us": 1e3 * ms_k / nl, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                        "peaks_source": src}
    if rank == 0 and not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample(0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
