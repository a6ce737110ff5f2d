#!/usr/bin/env python
"""Benchmark: periodic LR-CCSD Jacobian products on GB300.

One step = one pass of the response solver's hot path over a batch of right-hand
sides: the full Jacobian product A.X (particle-particle ladder with W built from the
dressed DF factors, hole-hole, ring, singles-coupling and Fock-like terms) on every
vector of the batch.  The default workload is the Nk=5, nocc=8, nvir=40, naux=160
chain of the 3x3 alpha tensor at omega in {0, 0.05, 0.1} Ha; a step is the batch of
the three dipole components at one frequency (one right-hand-side batch of that alpha
solve; 15 such vectors make the whole tensor).  Inputs are seeded synthetic data
(synth.make_problem); ground-state amplitudes are random with the magnitude of
converged ones (the cost of a product does not depend on their values).

--gpus N without a launcher starts N replica ranks itself (one process per GPU, gloo
for the max-over-ranks timing); under torchrun the ranks come from the environment.

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
# DRAM bytes (read + write) per launch of the dominant kernel, from an ncu capture (profiles/):
# (kernel source file, the marker that ends the kernel's part of it, sha256 prefix of the text
# before the marker when the counters were taken, bytes per launch at the default workload).
# The part hashed is the GEMM kernel and its launchers; the bench reports null once it has
# changed since.
TRAFFIC_RECORD = ("paper_2508_01266_gb300/csrc/kernels_f64.cu", "// layout permutation", "8bb6474981a87c0d",
                  3.2225e9)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("LRCC_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _free_port():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _replica(rank, argv, world, port, backend):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world), LRCC_BENCH_BACKEND=backend)
    sys.argv = [sys.argv[0]] + list(argv)
    main()


def spawn_replicas(n, argv):
    """--gpus N without a launcher: N replica ranks, one process per GPU (RANK, LOCAL_RANK,
    WORLD_SIZE set as torchrun would), gloo for the barrier and the max-over-ranks time (the
    replicas exchange nothing else)."""
    import torch.multiprocessing as mp
    mp.start_processes(_replica, args=(argv, n, _free_port(), os.environ.get("LRCC_BENCH_BACKEND", "gloo")),
                       nprocs=n, join=True, start_method="spawn")


def _source_sha(rel, marker):
    """sha256 prefix of a source file's text before the first occurrence of marker."""
    import hashlib
    try:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            text = f.read()
    except OSError:
        return None
    i = text.find(marker)
    return hashlib.sha256(text[:i].encode()).hexdigest()[:16] if i >= 0 else None


def host_cpu():
    """CPU model and logical core count of the host (for the oracle baseline)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware") and ":" in ln:
                    model = ln.split(":", 1)[1].strip()
                    break
                if k == "cpu part" and model is None:
                    model = "arm cpu part " + ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return {"cpu_model": model, "host_logical_cores": os.cpu_count()}


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
    """The oracle as it stands, on the host cores, on a bounded sample of the same workload:
    each step runs the oracle's product on a sample of doubles blocks of one vector; value =
    products/s scaled by the block fraction (the oracle's cost is the same for every block)."""
    dist, rank, ws = _dist()
    if rank != 0:
        return
    cfg, comps, omegas, nsys = workload(args.config)
    nb = args.ref_blocks
    for _ in range(args.warmup):
        cpu_oracle_rate(cfg, nb)
    rates, secs = [], []
    threads, sample = None, ""
    for _ in range(args.steps):
        r, dt, threads, sample = cpu_oracle_rate(cfg, nb)
        rates.append(r)
        secs.append(dt)
    value = args.steps / sum(1.0 / r for r in rates)
    cpu = {"kind": "oracle", "cores": threads, "sample": sample, "value": value, "unit": "products/s",
           **host_cpu()}
    line = {"impl": "reference", "metric": "LR-CCSD Jacobian products/s", "value": value,
            "unit": "products/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(secs) / len(secs),
            "ms_per_step_note": "wall time of one sampled step (a fraction of one product); value is scaled "
                                "to whole products",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128", "data": "synthetic",
            "config": {"workload": f"{args.config}: Nk={cfg['nk']} nocc={cfg['nocc']} nvir={cfg['nvir']} "
                                   f"naux={cfg['naux']}", "rhs_per_step": 1},
            "cpu_baseline": cpu,
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


def time_mixed(lr, prob, X1, X2, Y1, Y2, steps, warmup, st, dist, products, autotune=True, precs=(2, 1)):
    """Time the tensor-core products (BF16x3 and TF32) on the same vectors; Y1/Y2 are the
    FP64 results (None: no error column).  The timed loop runs without per-op events; one
    more product with per-op events (same tuned kernels, eager) gives the ladder rate."""
    import torch
    mixed = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    BF16_PEAK = _measured_peak("bf16_tflops", 1900.0)
    for prec, name, peak, passes in ((2, "bf16x3", BF16_PEAK, 3), (1, "tf32", BF16_PEAK * 1.1 / 2.25, 1)):
        if prec not in precs:
            continue
        # the tensor-core products run as CUDA graphs, with the autotuner (per-op kernel choice
        # measured once during warm-up) unless autotune is off
        opts = lr.default_options(precision=prec, autotune=int(autotune), use_graphs=1)
        M1, M2 = torch.empty_like(X1), torch.empty_like(X2)
        for _ in range(max(warmup, 2)):
            prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        torch.cuda.synchronize()
        m0 = prob.kernel_launches
        e0.record(st)
        for _ in range(steps):
            prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        e1.record(st)
        torch.cuda.synchronize()
        mms = _max_over_ranks(dist, e0.elapsed_time(e1))
        launches = int(prob.kernel_launches - m0)
        prob.profile(True)
        prob.jacobian_apply(X1, X2, y1=M1, y2=M2, options=opts)
        lms, ln, lfl = prob.profile_query("ladder")
        ams, an, afl = prob.profile_query("")
        prob.profile(False)
        err = None
        if Y1 is not None:
            err = max(float((M1 - Y1).abs().max() / Y1.abs().max()), float((M2 - Y2).abs().max() / Y2.abs().max()))
        lach = (lfl / max(ln, 1)) / ((lms / max(ln, 1)) * 1e-3) / 1e12 if ln else None
        mixed[name] = {"value": products / (mms / 1000.0), "unit": "products/s", "ms_per_step": mms / steps,
                       "steps": steps, "autotune": bool(autotune), "cuda_graphs": True,
                       "gpu_launches": launches,
                       "max_rel_err_vs_fp64": err,
                       "ladder": {"achieved_tflops_algorithmic": lach,
                                  "tensor_pipe_tflops": lach * passes if lach else None,
                                  "peak_tflops": peak, "frac": (lach * passes / peak) if lach else None,
                                  "peak_source": "measured bf16 dense (MEASURED_PEAKS.json)" if prec == 2 else
                                  "measured bf16 x nominal tf32/bf16 ratio 1.1/2.25"},
                       "step_tflops_algorithmic": afl / (ams * 1e-3) / 1e12 if ams else None}
    return mixed


def extra_workload(lr, name, steps, dist, rank):
    """BF16x3 products/s (autotuned, CUDA graphs) at a larger workload: all (component, +-omega)
    vectors of the workload in one batch, as many as fit."""
    import torch
    from synth import make_problem, random_amplitudes, random_probe
    cfg, comps, omegas, nsys = workload(name)
    nk, o, v, Q = cfg["nk"], cfg["nocc"], cfg["nvir"], cfg["naux"]
    nrhs = {"c3": 18, "c4": 1, "c5": 4}.get(name, nsys)  # c3: 3 components x 6 frequencies
    t0 = time.perf_counter()
    p = make_problem(nk, o, v, Q, seed=1266)
    t1, t2 = random_amplitudes(nk, o, v, seed=1267, scale1=0.01, scale2=0.01)
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    prob.set_ground_state(t1, t2 * nk)
    del p, t1, t2
    x1, x2 = random_probe(nk, o, v, seed=replica_seed(rank), nrhs=nrhs)
    X1 = torch.as_tensor(x1).cuda()
    X2 = torch.as_tensor(x2 * nk).cuda()
    del x1, x2
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    st = torch.cuda.current_stream()
    # default kernel choices: the autotuner's per-op timing would take minutes at these sizes
    m = time_mixed(lr, prob, X1, X2, None, None, steps, 1, st, dist, nrhs * steps, autotune=False,
                   precs=(2,))["bf16x3"]
    prob.close()
    del X1, X2
    torch.cuda.empty_cache()
    return {"workload": f"{name}: Nk={nk} nocc={o} nvir={v} naux={Q}", "rhs_per_step": nrhs, "bf16x3": m,
            "setup_seconds": setup}


# alpha(w) runs at full size (one JSON line each): components, frequencies (Ha), whether both
# forms of the response function are computed (the left-response workload)
ALPHA_RUNS = {
    "c2": ([0, 1, 2], [0.0, 0.05, 0.1], False),
    "c3": ([0, 1, 2], [0.0, 0.03, 0.06, 0.09, 0.12, 0.15], False),
    "c5": ([0, 2], [0.0, 0.05, 0.1], True),
    "c4": ([0, 2], [0.0, 0.05, 0.1, 0.15], False),
}


def alpha_run(lr, name, prec, refine_tol=1e-7):
    """Integrals in, ground state (T, Lambda) and alpha out, everything on the GPU: the
    ground state in the same precision mode (FP64 residuals decide its convergence), the
    perturbed-amplitude systems of all components and +-w solved as one batch."""
    import numpy as np
    from synth import make_problem, CONFIGS
    comps, omegas, forms = ALPHA_RUNS[name]
    c = CONFIGS[name]
    nk, o, v, Q = c["nk"], c["nocc"], c["nvir"], c["naux"]
    p = make_problem(nk, o, v, Q, seed=1266)
    t0 = time.perf_counter()
    prob = lr.Problem(nk, o, v, Q)
    prob.set_integrals(p.L, p.eps, p.dip)
    del p
    gopt = lr.default_options(precision=prec, conv_tol=1e-9, refine_tol=1e-9, max_iter=300)
    *_, e, ginfo = prob.solve_ground_state(gopt)
    t1 = time.perf_counter()
    depth = 6 if name in ("c5", "c4") else 8  # a shorter DIIS history keeps the left-response groups on the GPU
    aopt = lr.default_options(precision=prec, conv_tol=1e-10, refine_tol=refine_tol, max_iter=300,
                              diis_depth=depth)
    # alpha at one frequency needs only that frequency's (component, +-w) systems; each system
    # holds about 22 vectors in the solver (8-deep DIIS history of iterates and errors, right-hand
    # side, solution, F vector, residual, product input and output; 25 with the left solves), so
    # the frequencies are solved in as few groups as device memory allows
    import torch
    vec_gb = 16.0 * (nk * o * v + nk ** 3 * o * o * v * v) / 1e9
    per_sys = (2 * depth + (9 if forms else 6)) * vec_gb
    budget = 0.4 * torch.cuda.get_device_properties(torch.cuda.current_device()).total_memory / 1e9
    groups, cur, cur_n = [], [], 0
    for w in omegas:
        ns = len(comps) * (1 if w == 0 else 2)
        if cur and (cur_n + ns) * per_sys > budget:
            groups.append(cur)
            cur, cur_n = [], 0
        cur.append(w)
        cur_n += ns
    groups.append(cur)
    a_parts, s_parts, iters, status = [], [], 0, 0
    for grp in groups:
        if forms:
            ag, sg, info = prob.polarizability_forms(comps, grp, aopt)
            s_parts.append(sg)
        else:
            ag, info = prob.polarizability(comps, grp, aopt)
        a_parts.append(ag)
        iters += int(info[0])
        status = status or int(info[1])
    a = np.concatenate(a_parts)
    asym = np.concatenate(s_parts) if forms else None
    t2 = time.perf_counter()
    launches = prob.kernel_launches
    prob.close()
    out = {"alpha_run": name, "workload": f"{name}: Nk={nk} nocc={o} nvir={v} naux={Q}", "precision":
           {0: "fp64", 1: "tf32", 2: "bf16x3"}[prec], "comps": comps, "omegas": omegas,
           "systems": sum(len(comps) * (1 if w == 0 else 2) for w in omegas),
           "ground_state": {"seconds": t1 - t0, "energy_per_cell": e, "newton_or_jacobi_steps": int(ginfo[0]),
                            "lambda_iterations": int(ginfo[2]), "conv_tol": 1e-9},
           "alpha_seconds": t2 - t1, "iterations": iters, "status": status,
           "frequency_groups": groups,
           "refine_tol": refine_tol if prec else None,
           "alpha_real": np.round(a.real, 9).tolist(),
           "max_abs_imag": float(np.abs(a.imag).max()),
           "max_abs_asymmetry": float(np.abs(a - a.transpose(0, 2, 1)).max()),
           "gpu_launches": int(launches)}
    if asym is not None:
        sym_asym = 0.5 * (asym + asym.transpose(0, 2, 1))
        out["left_response"] = {"alpha_symmetrised_real": np.round(sym_asym.real, 9).tolist(),
                                "max_abs_diff_symmetrised_vs_symmetric_form": float(np.abs(sym_asym - a).max()),
                                "max_rel_diff": float(np.abs(sym_asym - a).max() / np.abs(a).max())}
    return out


def alpha_batch_run(lr, prec):
    """The mixed-size batch at its real shapes, (Nk, nocc, nvir) = (3,4,24), (5,6,32), (7,8,48)
    with naux = 4 nvir: ground states, then alpha_zz at w = 0 and 0.1 Ha for the three chains in
    one lrcc_batch_polarizability call, then each chain alone; the batch must equal the solo runs
    bitwise (its kernels are deterministic whatever runs beside them)."""
    import numpy as np
    from synth import make_problem
    shapes = [(3, 4, 24), (5, 6, 32), (7, 8, 48)]
    comps, omegas = [2], [0.0, 0.1]
    probs, out = [], {"alpha_run": "mixed-size batch", "shapes": shapes, "comps": comps, "omegas": omegas,
                      "precision": {0: "fp64", 1: "tf32", 2: "bf16x3"}[prec], "ground_state_seconds": []}
    opts = lr.default_options(precision=prec, conv_tol=1e-9, refine_tol=1e-9, max_iter=300)
    for nk, o, v in shapes:
        p = make_problem(nk, o, v, 4 * v, seed=1266)
        pr = lr.Problem(nk, o, v, 4 * v)
        pr.set_integrals(p.L, p.eps, p.dip)
        t0 = time.perf_counter()
        pr.solve_ground_state(opts)
        out["ground_state_seconds"].append(time.perf_counter() - t0)
        probs.append(pr)
    aopts = lr.default_options(precision=prec, conv_tol=1e-10, refine_tol=1e-7, max_iter=300)
    t0 = time.perf_counter()
    batch = lr.batch_polarizability(probs, comps, omegas, aopts)
    out["batch_seconds"] = time.perf_counter() - t0
    solo, t_solo = [], 0.0
    for pr in probs:
        t0 = time.perf_counter()
        solo.append(pr.polarizability(comps, omegas, aopts))
        t_solo += time.perf_counter() - t0
        pr.close()
    out["solo_seconds_total"] = t_solo
    out["alpha_zz"] = [[float(x) for x in a[:, 0, 0].real] for a, _ in batch]
    out["bitwise_equal_to_solo"] = [bool(np.array_equal(a, b)) for (a, _), (b, _) in zip(batch, solo)]
    out["status"] = [int(i[1]) for _, i in batch]
    return out


def dry_run(args):
    """Rank setup only (no GPU, no library): every rank reports its rank and replica seed; rank 0
    prints one line.  Used by the CPU tests of the replica launch."""
    dist, rank, ws = _dist()
    t = _max_over_ranks(dist, 1.0 + rank)
    seeds = [replica_seed(r) for r in range(ws)]
    if dist is not None:
        import torch
        got = [None] * ws
        dist.all_gather_object(got, (rank, int(os.environ.get("LOCAL_RANK", "0")), replica_seed(rank)))
        seeds = got
        dist.barrier()
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": ws, "ranks": seeds, "max_over_ranks": t}), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--nrhs", type=int, default=0,
                    help="vectors per step (default: the dipole components of the workload, one frequency)")
    ap.add_argument("--ref-blocks", type=int, default=8, help="doubles blocks of one vector in the oracle sample (about 1.6 s each on 16 cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-alpha", action="store_true", help="skip the alpha wall-time measurement")
    ap.add_argument("--extra", default="c3,c5,c4",
                    help="comma-separated larger workloads whose BF16x3 products/s are added (empty: none)")
    ap.add_argument("--extra-steps", type=int, default=3)
    ap.add_argument("--mixed-only", action="store_true",
                    help="time only the tensor-core (mixed precision) products (profiling runs)")
    ap.add_argument("--fp64-only", action="store_true", help="time only the FP64 product (profiling runs)")
    ap.add_argument("--shape", default="",
                    help="Nk,nocc,nvir,naux overriding the workload's sizes (small cases for ncu captures)")
    ap.add_argument("--dry-run", action="store_true", help="rank setup only, no GPU (CPU tests)")
    ap.add_argument("--alpha", default="", help="run alpha(w) end to end at a workload (c2, c3, c5, c4) and print "
                                                 "one JSON line instead of the product benchmark")
    ap.add_argument("--alpha-precision", type=int, default=2, help="0 FP64, 1 TF32, 2 BF16x3")
    ap.add_argument("--alpha-comps", default="", help="override the alpha run's components (e.g. 2)")
    ap.add_argument("--alpha-omegas", default="", help="override the alpha run's frequencies (e.g. 0.0)")
    ap.add_argument("--report", type=int, default=-1,
                    help="print the per-op CUDA-event report of one product in this precision (0, 1, 2) "
                         "over the step's vectors and exit (profiling runs)")
    ap.add_argument("--transpose", action="store_true", help="--report: the transposed product")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        spawn_replicas(args.gpus, sys.argv[1:])
        return
    if args.dry_run:
        dry_run(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return

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

    if args.alpha:
        if args.alpha != "batch" and (args.alpha_comps or args.alpha_omegas):
            comps0, omegas0, forms0 = ALPHA_RUNS[args.alpha]
            ALPHA_RUNS[args.alpha] = ([int(x) for x in args.alpha_comps.split(",")] if args.alpha_comps else comps0,
                                      [float(x) for x in args.alpha_omegas.split(",")] if args.alpha_omegas
                                      else omegas0, forms0)
        if rank == 0:
            res = alpha_batch_run(lr, args.alpha_precision) if args.alpha == "batch" else \
                alpha_run(lr, args.alpha, args.alpha_precision)
            print(json.dumps(res), flush=True)
        return

    cfg, comps, omegas, nsys = workload(args.config)
    if args.shape:
        cfg = dict(zip(("nk", "nocc", "nvir", "naux"), (int(x) for x in args.shape.split(","))))
    nk, o, v, Q = cfg["nk"], cfg["nocc"], cfg["nvir"], cfg["naux"]
    nrhs = args.nrhs or len(comps)
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
        mixed = time_mixed(lr, prob, X1, X2, None, None, args.steps, args.warmup, st, dist, nrhs * args.steps * ws)
        if rank == 0:
            print(json.dumps({"profiling": True, "workload": cfg, "rhs_per_step": nrhs, "mixed_precision": mixed}),
                  flush=True)
        prob.close()
        return

    if args.report >= 0:  # per-op table of one product (after warm-up launches with the same options)
        ropts = lr.default_options(precision=args.report, autotune=1 if args.report else 0)
        for _ in range(max(args.warmup, 1)):
            prob.jacobian_apply(X1, X2, transpose=args.transpose, y1=Y1, y2=Y2, options=ropts)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        prob.jacobian_apply(X1, X2, transpose=args.transpose, y1=Y1, y2=Y2, options=ropts)
        e1.record(st)
        torch.cuda.synchronize()
        prob.profile(True)
        prob.jacobian_apply(X1, X2, transpose=args.transpose, y1=Y1, y2=Y2, options=ropts)
        rows = prob.profile_report()
        prob.profile(False)
        tot = sum(r[1] for r in rows)
        if rank == 0:
            print(f"# {args.config}{' ' + args.shape if args.shape else ''}: {nrhs} vectors, precision {args.report}, "
                  f"{'transposed' if args.transpose else 'forward'} product: {e0.elapsed_time(e1):.2f} ms "
                  f"(CUDA events, no per-op events); per-op events below sum to {tot:.2f} ms")
            print("# op\tms\tlaunches\talgorithmic flops\tshare\tTFLOP/s")
            for tag, ms_, n_, fl in rows:
                print(f"{tag}\t{ms_:.3f}\t{n_}\t{fl:.4g}\t{100 * ms_ / tot:.1f}%\t"
                      f"{(fl / (ms_ * 1e-3) / 1e12 if ms_ > 0 else 0):.3f}")
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
    clk = clocks.stop()
    ms = _max_over_ranks(dist, ms)
    products = nrhs * args.steps * ws
    value = products / (ms / 1000.0)

    # per-op CUDA events on one more (untimed) product: the GEMM kernel's rate and the ladder
    prob.profile(True)
    step()
    rep = prob.profile_report()
    lad_ms, lad_n, lad_fl = prob.profile_query("ladder")
    all_ms, all_n, all_fl = prob.profile_query("")
    prob.profile(False)
    gemm_ms = sum(r[1] for r in rep if r[3] > 0)
    gemm_fl = sum(r[3] for r in rep if r[3] > 0)
    gemm_n = sum(r[2] for r in rep if r[3] > 0)
    if rank == 0 and args.fp64_only:
        print(json.dumps({"profiling": True, "workload": cfg, "rhs_per_step": nrhs, "ms_per_step": ms / args.steps,
                          "value": value, "report": rep[:20]}), flush=True)
        prob.close()
        return

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

    # roofline of the dominant kernel's dominant op: the ladder contraction launches of the FP64
    # tiled GEMM (SURVEY's unit: 8 flops per complex multiply-add of the ladder, here the
    # pair-swap-halved count the kernel launches).  The kernel executes 6 flops per complex
    # multiply-add (Gauss's three-product form): `executed_frac` is the FP64 pipe's utilisation.
    lad_rate = lad_fl / (lad_ms * 1e-3) / 1e9 if lad_ms else None
    gemm_rate = gemm_fl / (gemm_ms * 1e-3) / 1e9 if gemm_ms else None
    default_workload = args.config == "c2" and not args.shape and nrhs == len(comps)
    traffic = None
    if TRAFFIC_RECORD and default_workload and _source_sha(TRAFFIC_RECORD[0], TRAFFIC_RECORD[1]) == TRAFFIC_RECORD[2]:
        traffic = TRAFFIC_RECORD[3]
    roof = {"bound": "alu", "achieved": lad_rate, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
            "frac": (lad_rate / FP64_NOMINAL_GFLOPS) if lad_rate else None,
            "executed_frac": (0.75 * lad_rate / FP64_NOMINAL_GFLOPS) if lad_rate else None,
            "traffic": traffic,
            "kernel": "zgemm_seg_kernel<double,64,64,8,4,4>, ladder contraction launches",
            "launches_per_step": lad_n,
            "flops_per_launch": lad_fl / max(lad_n, 1),
            "peak_source": "FP64 nominal 1.25 TFLOP/s of the profiling recipe (152 SMs x 2 DFMA/clk x 2.07 GHz)",
            "all_fp64_gemm_gflops": gemm_rate, "all_fp64_gemm_executed_frac":
                (0.75 * gemm_rate / FP64_NOMINAL_GFLOPS) if gemm_rate else None,
            "gemm_launches_per_step": gemm_n,
            "ladder_share_of_step": lad_ms / max(all_ms, 1e-9),
            "gemm_share_of_step": gemm_ms / max(all_ms, 1e-9),
            "step_gflops_algorithmic": all_fl / (all_ms * 1e-3) / 1e9 if all_ms else None,
            "profile": "per-op CUDA events on one untimed product after the timed region"}

    # mixed precision: the same product with the GEMMs on tcgen05 (BF16x3 and TF32, FP32 accumulate)
    mixed = {} if args.no_mixed else time_mixed(lr, prob, X1, X2, Y1, Y2, args.steps, args.warmup, st, dist,
                                                 products)
    if mixed and default_workload:
        # the whole alpha batch of the workload (15 vectors: 3 components x {0, +-0.05, +-0.1})
        z1, z2 = random_probe(nk, o, v, seed=replica_seed(rank) + 1, nrhs=nsys)
        Z1 = torch.as_tensor(z1, device=dev)
        Z2 = torch.as_tensor(z2 * nk, device=dev)
        del z1, z2
        m15 = time_mixed(lr, prob, Z1, Z2, None, None, args.steps, args.warmup, st, dist, nsys * args.steps * ws,
                         precs=(2,))
        mixed["bf16x3_whole_alpha_batch"] = dict(m15["bf16x3"], rhs_per_step=nsys)
        del Z1, Z2
    prob.close()
    del X1, X2, Y1, Y2, h1, h2, o1, o2
    torch.cuda.empty_cache()
    extras = {}
    for name in [x for x in args.extra.split(",") if x] if not args.no_mixed and not args.shape else []:
        extras[name] = extra_workload(lr, name, args.extra_steps, dist, rank)

    alpha = None
    if rank == 0 and not args.no_alpha:
        alpha = alpha_wall_time(lr)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, dt, threads, sample = cpu_oracle_rate(cfg, args.ref_blocks)
        cpu = {"value": r, "unit": "products/s", "cores": threads, "kind": "oracle", "sample": sample,
               "seconds": dt, **host_cpu()}
    if rank == 0:
        line = {"metric": "LR-CCSD Jacobian products/s", "value": value, "unit": "products/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic",
                "config": {"workload": (f"{args.config}: Nk={nk} nocc={o} nvir={v} naux={Q}, {nrhs} vectors per "
                                        f"step (the {len(comps)} dipole components at one frequency of the "
                                        f"alpha tensor at omega in {omegas} Ha)"),
                           "precision": "fp64", "rhs_per_step": nrhs, "parallelism": f"replicas x{ws}",
                           "l2": (f"working set larger than L2 (vector {16 * nk**3 * o * o * v * v / 1e6:.0f} MB, "
                                  f"fixed intermediates {prob_fixed_gb:.1f} GB); no flush")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "mixed_precision": mixed, "larger_workloads": extras, "alpha_wall_time": alpha,
                "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
