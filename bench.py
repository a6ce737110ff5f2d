#!/usr/bin/env python
"""Benchmark: periodic LR-CCSD Jacobian products on GB300.

One step = one pass of the response solver's hot path over a batch of right-hand
sides: the full Jacobian product A.X (particle-particle ladder with W built from the
dressed DF factors, hole-hole, ring, singles-coupling and Fock-like terms) on every
vector of the batch.  The default workload is the Nk=5, nocc=8, nvir=40, naux=160
chain with the 15 (component, +-omega) systems of the 3x3 alpha tensor at
omega in {0, 0.05, 0.1} Ha.  Inputs are seeded synthetic data (synth.make_problem);
ground-state amplitudes are random with the magnitude of converged ones (the cost of
a product does not depend on their values).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_NOMINAL_GFLOPS = 1250.0  # GB300 FP64 pipe, nominal (profiling recipe table)
# DRAM bytes (read + write) of one FP64 ladder-contraction launch of this workload (15 vectors),
# from a one-pass ncu capture of this build's kernel (profiles/ladder_c2_fp64.md)
LADDER_TRAFFIC_BYTES = 23.36e9 + 1.00e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("LRCC_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _max_over_ranks(dist, x):
    """Slowest rank's time (the job's time); a CPU tensor on the gloo backend."""
    if dist is None:
        return x
    import torch
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Seed of a rank's right-hand sides: replicas work on disjoint synthetic vectors."""
    return 2000 + 97 * rank


class ClockSampler:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return fallback


# dipole components and frequencies (Ha) of each workload; a product step covers one vector
# per (component, +-omega) system (omega = 0 counted once)
WORKLOADS = {
    "c1": ([2], [0.0, 0.1]),
    "c2": ([0, 1, 2], [0.0, 0.05, 0.1]),
    "c3": ([0, 1, 2], [0.0, 0.03, 0.06, 0.09, 0.12, 0.15]),
    "c4": ([0, 2], [0.0, 0.05, 0.1, 0.15]),
    "c5": ([0, 1, 2], [0.0, 0.05, 0.1]),
}


def workload(cfg_name):
    from synth import CONFIGS
    c = dict(CONFIGS[cfg_name])
    comps, omegas = WORKLOADS[cfg_name]
    nsys = sum(len(comps) * (1 if w == 0 else 2) for w in omegas)
    return c, comps, omegas, nsys


def cpu_oracle_rate(cfg, nblocks, seed=1266):
    """Oracle Jacobian product on `nblocks` sampled doubles blocks; returns
    (products per second scaled to a full product, seconds, threads, sample text)."""
    import numpy as np
    import torch
    from synth import make_problem, random_amplitudes
    from oracle import rcc
    nk, o, v, Q = cfg["nk"], cfg["nocc"], cfg["nvir"], cfg["naux"]
    p = make_problem(nk, o, v, Q, seed=seed)
    R = rcc.RCC(p)
    t1, t2 = random_amplitudes(nk, o, v, seed=seed + 1, scale1=0.01, scale2=0.01)
    x1, x2 = random_amplitudes(nk, o, v, seed=seed + 2, scale1=1.0, scale2=1.0)
    rng = np.random.default_rng(seed)
    allb = [(a, b, c) for a in range(nk) for b in range(nk) for c in range(nk)]
    pick = [allb[i] for i in rng.choice(len(allb), size=nblocks, replace=False)]
    T = torch.as_tensor
    t0 = time.perf_counter()
    R.jacobian(T(t1), T(t2), T(x1), T(x2), blocks=pick)
    dt = time.perf_counter() - t0
    frac = nblocks / len(allb)
    sample = (f"oracle A.X (exact 5-point stencil of the residual) on {nblocks} of {len(allb)} doubles "
              f"blocks of one vector, scaled by the block fraction")
    return frac / dt, dt, torch.get_num_threads(), sample


def run_reference(args):
    dist, rank, ws = _dist()
    if rank != 0:
        return
    cfg, comps, omegas, nsys = workload(args.config)
    nb = args.ref_blocks
    for _ in range(args.warmup):
        cpu_oracle_rate(cfg, nb)
    rates, secs = [], 0.0
    threads, sample = None, ""
    for _ in range(args.steps):
        r, dt, threads, sample = cpu_oracle_rate(cfg, nb)
        rates.append(r)
        secs += dt
    value = args.steps / sum(1.0 / r for r in rates)
    line = {"impl": "reference", "metric": "LR-CCSD Jacobian products/s", "value": value,
            "unit": "products/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {"workload": f"{args.config}: Nk={cfg['nk']} nocc={cfg['nocc']} nvir={cfg['nvir']} "
                                   f"naux={cfg['naux']}", "rhs_per_step": 1},
            "cpu_baseline": {"kind": "oracle", "cores": threads, "sample": sample, "value": value,
                             "unit": "products/s"},
            "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _fixed_elems(lr, nk, o, v, Q):
    """Fixed-arena size (complex elements) from the plan introspection call."""
    import ctypes as C
    from paper_2508_01266_gb300._lib import lib, lrcc_dims
    d = lrcc_dims(nk, o, v, Q, 0)
    h = C.c_void_p()
    if lib.lrcc_plan_create(C.byref(d), 1 << 26, C.byref(h)) != 0:
        return 0
    ar = (C.c_int64 * 5)()
    off = (C.c_int64 * 11)()
    fl = (C.c_double * 3)()
    lib.lrcc_plan_info(h, ar, off, fl)
    lib.lrcc_plan_destroy(h)
    return int(ar[0])


def alpha_wall_time(lr):
    """alpha(w) wall time on the C1 workload (Nk=3, nocc=4, nvir=16, naux=48; alpha_zz at
    w = 0 and 0.1 Ha), everything on the GPU: integrals in, CCSD T and Lambda solved
    (lrcc_solve_ground_state), alpha to host (lrcc_polarizability); FP64 and BF16x3 with
    FP64 refinement.  Times are host wall clock from the first ABI call to alpha on host."""
    from synth import make_problem, CONFIGS
    c = CONFIGS["c1"]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    out = {"workload": f"c1: Nk={nk} nocc={o} nvir={v} naux={Q}, alpha_zz at omega in {{0, 0.1}} Ha"}
    for name, prec in (("fp64", 0), ("bf16x3", 2)):
        t0 = time.perf_counter()
        prob = lr.Problem(nk, o, v, Q)
        prob.set_integrals(p.L, p.eps, p.dip)
        *_, e, ginfo = prob.solve_ground_state(lr.default_options(conv_tol=1e-10, max_iter=300))
        t1 = time.perf_counter()
        a, info = prob.polarizability([2], [0.0, 0.1], lr.default_options(precision=prec, conv_tol=1e-10,
                                                                         refine_tol=1e-8, max_iter=300))
        t2 = time.perf_counter()
        prob.close()
        out[name] = {"seconds": t2 - t0, "ground_state_seconds": t1 - t0, "response_seconds": t2 - t1,
                     "alpha_zz": [float(x.real) for x in a[:, 0, 0]], "ccsd_energy_per_cell": e,
                     "iterations": {"ccsd": int(ginfo[0]), "lambda": int(ginfo[2]), "response": int(info[0])}}
    out["max_abs_diff_bf16x3_vs_fp64"] = max(abs(x - y) for x, y in zip(out["fp64"]["alpha_zz"],
                                                                           out["bf16x3"]["alpha_zz"]))
    return out


def time_mixed(lr, prob, X1, X2, Y1, Y2, args, st, dist, products):
    """Time the tensor-core products (BF16x3 and TF32) on the same vectors; Y1/Y2 are the
    FP64 results (None: no error column)."""
    import torch
    mixed = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    BF16_PEAK = _measured_peak("bf16_tflops", 1900.0)
    for prec, name, peak, passes in ((2, "bf16x3", BF16_PEAK, 3), (1, "tf32", BF16_PEAK * 1.1 / 2.25, 1)):
        # the tensor-core products run with the autotuner (per-op kernel choice measured once
        # during warm-up) and as CUDA graphs
        opts = lr.default_options(precision=prec, autotune=1, use_graphs=1)
        M1, M2 = torch.empty_like(X1), torch.empty_like(X2)
        for _ in range(args.warmup):
            prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        torch.cuda.synchronize()
        m0 = prob.kernel_launches
        e0.record(st)
        for _ in range(args.steps):
            prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        e1.record(st)
        torch.cuda.synchronize()
        mms = _max_over_ranks(dist, e0.elapsed_time(e1))
        launches = int(prob.kernel_launches - m0)
        # one more product with per-op events (eager, same tuned kernels) for the ladder rate
        prob.profile(True)
        prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        lms, ln, lfl = prob.profile_query("ladder")
        ams, an, afl = prob.profile_query("")
        prob.profile(False)
        err = None
        if Y1 is not None:
            err = max(float((M1 - Y1).abs().max() / Y1.abs().max()), float((M2 - Y2).abs().max() / Y2.abs().max()))
        lach = (lfl / max(ln, 1)) / ((lms / max(ln, 1)) * 1e-3) / 1e12 if ln else None
        mixed[name] = {"value": products / (mms / 1000.0), "unit": "products/s", "ms_per_step": mms / args.steps,
                       "autotune": True, "cuda_graphs": True,
                       "gpu_launches": launches,
                       "max_rel_err_vs_fp64": err,
                       "ladder": {"achieved_tflops_algorithmic": lach,
                                  "tensor_pipe_tflops": lach * passes if lach else None,
                                  "peak_tflops": peak, "frac": (lach * passes / peak) if lach else None,
                                  "peak_source": "measured bf16 dense (MEASURED_PEAKS.json)" if prec == 2 else
                                  "measured bf16 x nominal tf32/bf16 ratio 1.1/2.25"},
                       "step_tflops_algorithmic": afl / (ams * 1e-3) / 1e12 if ams else None}
    return mixed


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--nrhs", type=int, default=0, help="vectors per step (default: all systems of the workload)")
    ap.add_argument("--ref-blocks", type=int, default=8, help="doubles blocks of one vector in the oracle sample (about 1.6 s each on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-alpha", action="store_true", help="skip the alpha wall-time measurement")
    ap.add_argument("--mixed-only", action="store_true",
                    help="time only the tensor-core (mixed precision) products (profiling runs)")
    ap.add_argument("--shape", default="",
                    help="Nk,nocc,nvir,naux overriding the workload's sizes (small cases for ncu captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    import paper_2508_01266_gb300 as lr
    from synth import make_problem, random_amplitudes, random_probe

    cfg, comps, omegas, nsys = workload(args.config)
    if args.shape:
        cfg = dict(zip(("nk", "nocc", "nvir", "naux"), (int(x) for x in args.shape.split(","))))
    nk, o, v, Q = cfg["nk"], cfg["nocc"], cfg["nvir"], cfg["naux"]
    nrhs = args.nrhs or nsys
    p = make_problem(nk, o, v, Q, seed=1266)
    t1, t2 = random_amplitudes(nk, o, v, seed=1267, scale1=0.01, scale2=0.01)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    prob_fixed_gb = 16.0 * _fixed_elems(lr, nk, o, v, Q) / 1e9
    x1, x2 = random_probe(nk, o, v, seed=replica_seed(rank), nrhs=nrhs)
    dev = torch.device("cuda", local)
    X1 = torch.as_tensor(x1, device=dev).contiguous()
    X2 = torch.as_tensor(x2 * nk, device=dev).contiguous()
    Y1 = torch.empty_like(X1)
    Y2 = torch.empty_like(X2)
    st = torch.cuda.current_stream()
    if args.mixed_only:  # profiling runs: tensor-core products only, one informational line
        mixed = time_mixed(lr, prob, X1, X2, None, None, args, st, dist, nrhs * args.steps * ws)
        if rank == 0:
            print(json.dumps({"profiling": True, "workload": cfg, "rhs_per_step": nrhs, "mixed_precision": mixed}),
                  flush=True)
        prob.close()
        return

    def step():
        prob.jacobian_apply(X1, X2, y1=Y1, y2=Y2)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    prob.profile(True)
    n0 = prob.kernel_launches
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = prob.kernel_launches - n0
    lad_ms, lad_n, lad_fl = prob.profile_query("ladder")
    wb_ms, wb_n, wb_fl = prob.profile_query("W build")
    all_ms, all_n, all_fl = prob.profile_query("")
    prob.profile(False)
    clk = clocks.stop()
    ms = _max_over_ranks(dist, ms)
    products = nrhs * args.steps * ws
    value = products / (ms / 1000.0)

    # end to end through the Python/C-ABI call with pinned host buffers
    h1 = torch.as_tensor(x1).pin_memory()
    h2 = torch.as_tensor(x2 * nk).pin_memory()
    o1 = torch.empty_like(h1).pin_memory()
    o2 = torch.empty_like(h2).pin_memory()

    def e2e_step():
        d1 = h1.to(dev, non_blocking=True)
        d2 = h2.to(dev, non_blocking=True)
        r1, r2 = prob.jacobian_apply(d1, d2)
        o1.copy_(r1, non_blocking=True)
        o2.copy_(r2, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e = {"value": products / e2e_s, "unit": "products/s",
           "h2d_bytes_per_step": int(h1.numel() * 16 + h2.numel() * 16),
           "d2h_bytes_per_step": int(o1.numel() * 16 + o2.numel() * 16)}

    lad_per_launch_fl = lad_fl / max(lad_n, 1)
    lad_avg_ms = lad_ms / max(lad_n, 1)
    achieved = lad_per_launch_fl / (lad_avg_ms * 1e-3) / 1e9 if lad_n else None
    default_workload = args.config == "c2" and not args.shape and nrhs == 15
    roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
            "frac": (achieved / FP64_NOMINAL_GFLOPS) if achieved else None,
            "traffic": LADDER_TRAFFIC_BYTES if default_workload else None,
            "kernel": "zgemm_seg_kernel (ladder contraction)",
            "peak_source": "FP64 nominal 1.25 TFLOP/s of the profiling recipe (DFMA probe measured 1.195)",
            "ladder_share_of_step": lad_ms / max(all_ms, 1e-9), "wbuild_share_of_step": wb_ms / max(all_ms, 1e-9),
            "step_gflops_algorithmic": all_fl / (all_ms * 1e-3) / 1e9 if all_ms else None}

    # mixed precision: the same product with the GEMMs on tcgen05 (BF16x3 and TF32, FP32 accumulate)
    mixed = {} if args.no_mixed else time_mixed(lr, prob, X1, X2, Y1, Y2, args, st, dist, products)

    alpha = None
    if rank == 0 and not args.no_alpha:
        alpha = alpha_wall_time(lr)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, dt, threads, sample = cpu_oracle_rate(cfg, args.ref_blocks)
        cpu = {"value": r, "unit": "products/s", "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": dt}
    if rank == 0:
        line = {"metric": "LR-CCSD Jacobian products/s", "value": value, "unit": "products/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic",
                "config": {"workload": (f"{args.config}: Nk={nk} nocc={o} nvir={v} naux={Q}, {nrhs} vectors per "
                                        f"step ({len(comps)} dipole components x omega in {omegas} Ha, +-omega)"),
                           "precision": "fp64", "rhs_per_step": nrhs, "parallelism": f"replicas x{ws}",
                           "l2": (f"working set larger than L2 (vector {16 * nk**3 * o * o * v * v / 1e6:.0f} MB, "
                                  f"fixed intermediates {prob_fixed_gb:.1f} GB); no flush")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "mixed_precision": mixed, "alpha_wall_time": alpha,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    prob.close()
    if dist is not None:
        dist.destroy_process_group()

if __name__ == "__main__":
    main()
