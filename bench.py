#!/usr/bin/env python3
"""Throughput benchmark of the Pauli-coefficient propagation path.

Workload (default): the paper-scale plain-method case -- n = 4 qubits, a
60,200-gate layered ansatz (RX, RY, RZ on every qubit then a CNOT ring, 10% of
rotation slots replaced by H or S, theta ~ U[0, 2 pi), seed 1002); each step
propagates the 4 generators Z_k of |0^4> forward and the observable Z_0 Z_1
backward to <Z_0 Z_1>.

Metric: Pauli-coefficient updates per second = sum over propagated vectors of
gates x 4^n, per second (5 vectors x 60,200 x 256 per step).

value: device-resident step (angles already in HBM: stab_set_params from a
device tensor, stab_run_generators, stab_expect_async), timed with CUDA events
per step on the context stream, L2 flushed between steps.
e2e:   the public host-buffer calls (stab_apply_circuit from host arrays,
stab_expect from host terms, stab_get_generators into host memory), wall
clock, transfers inside the timed region.
roofline: the generator launch against the FP64 rate measured on the same GPU
in the same run (stab_probe_fp64, DFMA chains), the pipe that bounds it.
sub:   bounded measurements of the other configurations in the same run, each
with its own clock record: the 4,096-circuit uneven batch against one launch
per circuit and the plain form, the n = 8 10,000-gate adjoint gradient
against batched parameter shift and the plain form, and the first requests
of the Poisson serving trace through both server engines and the plain form.

--impl reference times the CPU oracle (the plain FP64 C implementation used by
the tests) on the same workload on all host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Pauli-coefficient updates/s"
UNIT = "updates/s"


def workload_spec(name):
    from paper_2502_10685_gb300 import workloads as W
    if name == "layered-n4-60200":
        c = W.layered_ansatz(4, 60200, seed=1002)
        return c, W.obs_zz(4, 0, 1)
    if name == "layered-n4-2000":
        c = W.layered_ansatz(4, 2000, seed=1001)
        return c, W.obs_z(4, 0)
    if name.startswith("layered-n"):
        n, m = name[len("layered-n"):].split("-")
        c = W.layered_ansatz(int(n), int(m), seed=1000 + int(n))
        return c, W.obs_chain(int(n))
    raise SystemExit("unknown workload %s" % name)


def units_per_step(c):
    # generators (n vectors) forward + the observable backward
    return (c.n + 1) * c.m * 4 ** c.n


# DRAM bytes read + written by the generator phase's launches (k_batch first
# part + k_transfer_cols), per step, from one ncu capture of the 60,200-gate
# n = 4 workload: keyed by (n, gates, cut pass, transfer matrices)
GEN_TRAFFIC = {(4, 60200, 10535, 1): 3393024.0, (4, 60200, 9218, 2): 3195136.0}


def algorithmic_flops_generators(c):
    """FP64 flops of one generator launch: 6 per rotated pair (4^n / 4 pairs per
    rotation, per vector) and 15 per group for a composed 3x3 wire map."""
    from paper_2502_10685_gb300 import workloads as W
    n_rot = int(sum(1 for g in c.gates if g["op"] in W.ROTATIONS))
    return c.n * n_rot * 1.5 * 4 ** c.n


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev):
    import torch
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(dev.index if hasattr(dev, "index") else dev)


# ---------------------------------------------------------------- oracle timing

def host_cpu():
    """(nproc, CPU model) of the host the oracle runs on."""
    nproc = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return nproc, model or platform.processor() or platform.machine()


def oracle_units(c, obs):
    """The step's independent oracle jobs: each generator forward, <O> backward."""
    import oracle

    def gen(k):
        return lambda: oracle.forward(c.n, c.gates, c.thetas, oracle.generator(c.n, k))

    return [gen(k) for k in range(c.n)] + [lambda: oracle.expect(c.n, c.gates, c.thetas, obs)]


def run_oracle_jobs(jobs, threads):
    """Runs the jobs on `threads` host threads (ctypes releases the GIL);
    returns the wall time in seconds."""
    import concurrent.futures as cf
    t0 = time.perf_counter()
    if threads <= 1:
        for j in jobs:
            j()
    else:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            for f in [ex.submit(j) for j in jobs]:
                f.result()
    return time.perf_counter() - t0


def cpu_baseline(c, obs, runs=5):
    """The oracle on the host, two modes, median of `runs` each: one core (one
    full step, its n + 1 vectors one after another) and all cores (nproc
    steps' worth of independent vectors on nproc threads, the paper's
    one-vector-per-core scheme)."""
    import oracle
    oracle.build()
    nproc, model = host_cpu()
    units = oracle_units(c, obs)
    one = [run_oracle_jobs(units, 1) for _ in range(runs)]
    jobs = units * nproc
    many = [run_oracle_jobs(jobs, nproc) for _ in range(runs)]
    v1 = units_per_step(c) / statistics.median(one)
    vn = units_per_step(c) * nproc / statistics.median(many)
    return {"value": vn, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "all cores: %d full steps (%d vectors) on %d threads; one core: one full "
                      "step; median of %d runs each" % (nproc, len(jobs), nproc, runs),
            "single_core": {"value": v1, "ms_per_step": statistics.median(one) * 1e3},
            "all_cores": {"value": vn, "threads": nproc,
                          "ms_per_step": statistics.median(many) * 1e3 / nproc},
            "host": {"nproc": nproc, "cpu_model": model}, "runs": runs, "statistic": "median"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    c, obs = workload_spec(args.workload)
    import oracle
    oracle.build()
    nproc, model = host_cpu()
    units = oracle_units(c, obs)
    # warm-up steps, then the timed steps: every step's vectors are
    # independent jobs spread over all host cores
    run_oracle_jobs(units * args.warmup, nproc)
    dt = run_oracle_jobs(units * args.steps, nproc)
    value = units_per_step(c) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": c.n, "gates": c.m, "vectors_per_step": c.n + 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
                         "sample": "%d full steps of the workload, their %d vectors on %d threads"
                                   % (args.steps, len(units) * args.steps, nproc),
                         "host": {"nproc": nproc, "cpu_model": model}},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ranks

def combine_ranks(local_ms, units_per_rank, world, dist=None, device=None):
    """Whole-job figures for replicas: the slowest rank's time (barrier-bounded
    region, max over ranks) and the units of all ranks divided by it."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1 and dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    return total_ms, units_per_rank * world / (total_ms / 1e3)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def fp64_peak():
    """FP64 rate of this GPU, measured now: DFMA chains (the pipe the rotation
    passes use) and FP64 matrix-instruction chains, best of three launches."""
    from paper_2502_10685_gb300 import stab
    dfma = max(stab.stab_probe_fp64("dfma", 8192)[0] for _ in range(3))
    dmma = max(stab.stab_probe_fp64("dmma", 2048)[0] for _ in range(3))
    return dfma, dmma


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2502_10685_gb300 import stab
    c, obs = workload_spec(args.workload)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # the roofline's denominator, measured on this GPU before the timed region
    peak_dfma, peak_dmma = fp64_peak()
    # all work of this process is queued on one dedicated stream
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    s = stab.Stab(c.n, device=local)
    s.load_circuit(c.gates, c.thetas)
    s.set_observable(obs)
    th_dev = torch.tensor(c.thetas, dtype=torch.float64, device=dev)
    out_dev = torch.zeros(8, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        s.set_params(th_dev)
        s.run_generators()
        s.expect_async(out_dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_uuid(dev))
    clocks.start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = s.launch_count()
    for k in range(args.steps):
        flush.zero_()                       # untimed: evict L2 between steps
        e = ev[k]
        e[0].record(st)
        s.set_params(th_dev)
        e[1].record(st)
        s.run_generators()
        e[2].record(st)
        s.expect_async(out_dev)
        e[3].record(st)
    torch.cuda.synchronize()
    launches = s.launch_count() - l0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    gen_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms, value = combine_ranks(sum(step_ms), units_per_step(c) * args.steps, world,
                                    dist if world > 1 else None, dev)

    # check the device result against the host path once (same circuit)
    got = float(out_dev[0].item())

    # ---- e2e through host buffers
    gens_host = np.empty((c.n, 4 ** c.n))
    h0, d0 = s.transfer_bytes()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 4)
    for _ in range(e2e_steps):
        s.apply_circuit(c.gates, c.thetas)
        val = s.expect(obs)
        s.generators(out=gens_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h1, d1 = s.transfer_bytes()
    t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e2e_s = float(t.item())
    assert abs(val - got) <= 1e-12, (val, got)

    # ---- roofline of the dominant kernel (the generator launch)
    gen_avg_s = statistics.mean(gen_ms) / 1e3
    achieved = algorithmic_flops_generators(c) / gen_avg_s / 1e12
    cut, gen_units, _ = s.split_info()
    n_passes = s.plan_info()[1]
    if gen_units:
        # the generators' persistent launch: n vectors through passes [0, cut)
        # and the 4^n - 1 transfer-matrix columns through [cut, P), then one
        # product; FP64 work executed per algorithmic flop, counted in passes
        n_mats = (gen_units - (c.n + 1)) // (4 ** c.n - 1)
        if c.n == 4:
            kernel = ("k_transfer_cols (%d x 255 columns, %d per CTA) + k_batch (%d first-part "
                      "units) + k_apply_transfer" % (n_mats, 2 * n_mats, c.n + 1))
        else:
            kernel = "k_batch (split: %d units) + k_apply_transfer" % gen_units
        # every later part's columns together cover the passes after the cut once
        executed = ((c.n + 1) * cut + (4 ** c.n - 1) * (n_passes - cut)) / (c.n * n_passes)
        active_sms = min(sms, c.n + 1 + 128 if c.n == 4 else gen_units)
        note = ("one circuit: the generators' first part ends at pass %d of %d, %d later "
                "part(s) each through its transfer matrix; the n + 1 first-part vectors "
                "and the basis columns run at once (%s); passes are sequential within a "
                "vector" % (cut, n_passes, n_mats,
                            "%d columns per CTA" % (2 * n_mats) if c.n == 4
                            else "one CTA each"))
    else:
        kernel = "k_resident_stream (generators)"
        executed = 1.0
        active_sms = c.n
        note = "one circuit: n independent vectors, one CTA each; passes are sequential"
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_dfma, "unit": "TFLOP/s",
                "frac": achieved / peak_dfma,
                # DRAM bytes of the generator phase's two launches from one ncu
                # capture of this workload with this split (the staged streams);
                # another split stages other streams
                "traffic": GEN_TRAFFIC.get((c.n, c.m, cut, n_mats if gen_units else 0)),
                "kernel": kernel, "launch_ms": gen_avg_s * 1e3,
                "peak_source": "of measured: FP64 DFMA chains on this GPU in this run "
                               "(stab_probe_fp64, best of 3; %d SMs)" % sms,
                "peak_dmma_tflops": peak_dmma,
                "active_sms": active_sms,
                "executed_per_algorithmic": executed,
                "executed_frac": achieved * executed / peak_dfma,
                "note": note}

    # the plain GPU form: one launch per circuit, one pass per gate, no fusion, same step
    plain = None
    if not args.no_plain:
        sp = stab.Stab(c.n, kernel="plain", device=local)
        sp.load_circuit(c.gates, c.thetas)
        sp.set_observable(obs)
        out_p = torch.zeros(8, dtype=torch.float64, device=dev)

        def pstep():
            sp.set_params(th_dev)
            sp.run_generators()
            sp.expect_async(out_p)
        for _ in range(2):
            pstep()
        torch.cuda.synchronize()
        e0, e1 = _events()
        reps = 10
        e0.record(st)
        for _ in range(reps):
            pstep()
        e1.record(st)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / reps
        assert abs(float(out_p[0].item()) - got) <= 1e-10
        plain = {"value": units_per_step(c) / (pms / 1e3), "unit": UNIT, "ms_per_step": pms,
                 "speedup": pms / (total_ms / args.steps), "steps": reps,
                 "form": "one launch per circuit, one pass per gate, no fusion (STAB_KERNEL_PLAIN)"}
        sp.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": c.n, "gates": c.m,
                   "vectors_per_step": c.n + 1, "parallelism": "replicas" if world > 1 else "none",
                   "l2": "flushed between steps (512 MB write)"},
        "circuits_per_s": args.steps * world / (total_ms / 1e3),
        "e2e": {"value": units_per_step(c) * e2e_steps * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": (h1 - h0) // e2e_steps,
                "d2h_bytes_per_step": (d1 - d0) // e2e_steps},
        "gpu_launches": launches,
        "vs_plain_form": plain,
        "roofline": roofline,
        "path_choice": s.path_choice(),
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                   "reasons": clk.get("reasons"), "samples": clk.get("samples")},
        "expect": got,
    }
    s.close()
    del flush
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(c, obs)
    if rank == 0 and world == 1 and not args.no_sub:
        # the other configurations, bounded, each with its own clock record
        line["sub"] = {
            "c3_batch": measure_batch(steps=3, warmup=1, with_cpu=False),
            "c4_grad": measure_grad(steps=40, warmup=3, psr_slots=64, with_cpu=False),
            "c5_serve": measure_serve(requests=args.sub_requests),
        }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other configurations

def measure_batch(steps, warmup, with_cpu, small=False, world=1, rank=0, local=0, dist=None):
    """Uneven batch: 4,096 circuits (n ~ U{2..8}, depth ~ U[100, 20000]) including
    the 2m parameter-shift copies of a 6-qubit 2,000-gate circuit, one
    persistent launch per step; compared with one fused launch per circuit and
    the plain form, one pass per gate (both timed on a seeded sample of 16
    circuits, scaled by updates)."""
    import numpy as np
    import torch
    from paper_2502_10685_gb300 import stab, units, workloads as W
    torch.cuda.set_stream(torch.cuda.Stream())
    st = torch.cuda.current_stream()
    if small:
        # a small batch for profiler captures: 96 circuits, n ~ U{6..8}, 300..600 gates
        all_items = W.uneven_batch(96 * world, seed=1013, n_range=(6, 8), depth_range=(300, 600),
                                   psr_base=None)
    else:
        all_items = W.uneven_batch(4096 * world, seed=1003)   # weak scaling: 4,096 per GPU
    # units to ranks by longest processing time first on their coefficient updates
    costs = [units.unit_cost(it.circuit.n, it.circuit.m,
                             it.circuit.n if it.kind == "generators" else 1) for it in all_items]
    mine = units.lpt_partition(costs, world)[rank]
    items = [all_items[i] for i in mine]
    t0 = time.perf_counter()
    b = stab.Batch(items, device=local)
    create_s = time.perf_counter() - t0
    upd = sum((it.circuit.n if it.kind == "generators" else 1) * it.circuit.m * 4 ** it.circuit.n
              for it in items)
    for _ in range(warmup):
        b.run()
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    clocks = ClockSampler(gpu_uuid(torch.device("cuda", local)))
    clocks.start()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = _events()
        e0.record(st)
        b.run()
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    del flush
    ms, _ = combine_ranks(sum(times) / len(times), 0, world, dist,
                          torch.device("cuda", local))
    forms = {}
    rng = np.random.default_rng(0)
    sample = [items[i] for i in rng.choice(len(items), size=16, replace=False)]
    s_upd = sum((it.circuit.n if it.kind == "generators" else 1) * it.circuit.m * 4 ** it.circuit.n
                for it in sample)
    for kernel in ("auto", "plain"):
        tot = 0.0
        for it in sample:
            c = it.circuit
            sx = stab.Stab(c.n, kernel=kernel)
            sx.load_circuit(c.gates, c.thetas)
            out = torch.zeros(8, dtype=torch.float64, device="cuda")
            if it.kind == "expect":
                sx.set_observable(it.observable)
                fn = lambda: sx.expect_async(out)
            else:
                fn = sx.run_generators
            fn()
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
            sx.close()
        est = tot * upd / s_upd
        forms["fused_per_circuit" if kernel == "auto" else "plain_per_gate"] = {
            "extrapolated_ms": est, "batch_speedup": est / ms, "sample_circuits": len(sample)}
    info = b.info()
    # every item's <O> (NaN for generator items) back on rank 0, in item order
    full = units.gather_to_root(mine, [float(x) for x in b.expectations()], len(all_items), dist)
    b.close()
    total_upd = sum(costs)
    line = {
        "metric": "circuits/s", "value": len(all_items) / (ms / 1e3), "unit": "circuits/s",
        "n_gpus": world, "scaling": "weak", "steps": steps, "warmup": warmup,
        "ms_per_step": ms,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch-small" if small else "batch-c3",
                   "circuits": len(all_items),
                   "circuits_rank0": len(items), "units": info["units"],
                   "grid": info["grid"], "ctas_per_sm": info["ctas_per_sm"],
                   "smem_max_n": info["smem_max_n"],
                   "partition": "longest processing time first on coefficient updates",
                   "l2": "flushed between steps"},
        "updates_per_s": total_upd / (ms / 1e3), "create_s": create_s, "vs_forms": forms,
        "results_gathered": sum(1 for x in full if x is not None) if full else None,
        "clocks": clk}
    if world == 1 and with_cpu and len(items) >= 12:
        # the oracle on a seeded sample of small items, scaled by updates
        import oracle
        oracle.build()
        cand = [it for it in items if 4 ** it.circuit.n * it.circuit.m <= 2e7]
        pick = [cand[i] for i in np.random.default_rng(2).choice(len(cand),
                                                                  size=min(12, len(cand)),
                                                                  replace=False)]
        p_upd = sum((it.circuit.n if it.kind == "generators" else 1) * it.circuit.m *
                    4 ** it.circuit.n for it in pick)
        t0 = time.perf_counter()
        for it in pick:
            c = it.circuit
            if it.kind == "expect":
                oracle.expect(c.n, c.gates, c.thetas, it.observable)
            else:
                oracle.generators(c.n, c.gates, c.thetas)
        cpu_s = (time.perf_counter() - t0) * upd / p_upd
        line["cpu_baseline"] = {"value": len(items) / cpu_s, "unit": "circuits/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "12 seeded items with 4^n m <= 2e7, one core, scaled "
                                          "to the batch by coefficient updates"}
    return line


def run_batch(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = measure_batch(args.steps, args.warmup, not args.no_cpu_baseline,
                         small=args.workload == "batch-small", world=world, rank=rank,
                         local=local, dist=dist if world > 1 else None)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


def measure_grad(steps, warmup, psr_slots, with_cpu):
    """n=8, 10,000-gate layered ansatz, O = sum Z_i Z_{i+1} + 0.5 sum X_i: all
    gradients by one adjoint sweep, against parameter shift (2 evaluations per
    slot) in one batched launch, timed on psr_slots slots and scaled to all,
    and against the plain form's parameter shift (each shifted circuit one
    pass per gate), timed on 2 slots and scaled."""
    import numpy as np
    import torch
    from paper_2502_10685_gb300 import stab, workloads as W
    torch.cuda.set_stream(torch.cuda.Stream())
    st = torch.cuda.current_stream()
    c = W.layered_ansatz(8, 10000, seed=1004)
    obs = W.obs_chain(8)
    s = stab.Stab(8)
    s.load_circuit(c.gates, c.thetas)
    s.set_observable(obs)
    g = torch.zeros(c.n_params, dtype=torch.float64, device="cuda")
    e = torch.zeros(8, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        s.grad_async(e, g)
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_uuid(torch.device("cuda", torch.cuda.current_device())))
    clocks.start()
    time.sleep(0.2)
    times = []
    for _ in range(steps):
        e0, e1 = _events()
        e0.record(st)
        s.grad_async(e, g)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    adj_ms = sum(times) / len(times)
    grads = g.cpu().numpy()
    # parameter shift on a sample of slots, batched
    rng = np.random.default_rng(1)
    js = rng.choice(c.n_params, size=psr_slots, replace=False)
    items = []
    for j in js:
        for sgn in (1.0, -1.0):
            th = c.thetas.copy()
            th[j] += sgn * math.pi / 2
            items.append(W.BatchItem(c.with_thetas(th), "expect", obs))
    b = stab.Batch(items)
    b.run()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record(st)
    b.run()
    e1.record(st)
    torch.cuda.synchronize()
    psr_ms = e0.elapsed_time(e1)
    ex = b.expectations()
    b.close()
    psr = np.array([(ex[2 * k] - ex[2 * k + 1]) / 2 for k in range(len(js))])
    err = float(np.abs(psr - grads[js]).max())
    l1 = sum(abs(a) for a, _ in obs)
    assert err <= 1e-10 * l1, err
    psr_all_ms = psr_ms * c.n_params / len(js)
    # the plain form's parameter shift: each shifted circuit one pass per gate
    sp = stab.Stab(8, kernel="plain")
    sp.load_circuit(c.gates, c.thetas)
    sp.set_observable(obs)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    sp.expect_async(out)
    torch.cuda.synchronize()
    plain_vals = []
    e0, e1 = _events()
    e0.record(st)
    for j in js[:2]:
        for sgn in (1.0, -1.0):
            th = c.thetas.copy()
            th[j] += sgn * math.pi / 2
            sp.set_params(th)
            sp.expect_async(out)
            plain_vals.append(out[0].clone())
    e1.record(st)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) * c.n_params / 2
    pv = [float(v) for v in plain_vals]
    perr = max(abs((pv[2 * k] - pv[2 * k + 1]) / 2 - grads[js[k]]) for k in range(2))
    assert perr <= 1e-10 * l1, perr
    sp.close()
    s.close()
    line = {
        "metric": "gradient time", "value": adj_ms, "unit": "ms", "n_gpus": 1,
        "steps": steps, "warmup": warmup, "ms_per_step": adj_ms,
        "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "grad-c4", "n": 8, "gates": c.m, "params": c.n_params},
        "psr_batched_ms_all_params": psr_all_ms, "adjoint_speedup": psr_all_ms / adj_ms,
        "psr_sample_slots": int(psr_slots),
        "plain_form_psr_ms_all_params": plain_ms, "adjoint_speedup_vs_plain": plain_ms / adj_ms,
        "plain_form": "parameter shift, each shifted circuit one launch sequence of one pass "
                      "per gate (STAB_KERNEL_PLAIN); 2 slots timed, scaled to all",
        "max_abs_diff_vs_psr_sample": err, "clocks": clk}
    if with_cpu:
        # the oracle's parameter shift of one slot (two full propagations),
        # scaled to every slot: the CPU way to these gradients
        import oracle
        oracle.build()
        gi = int(np.nonzero([int(g["op"]) in W.ROTATIONS for g in c.gates])[0][0])
        t0 = time.perf_counter()
        oracle.psr_grad_gate(c.n, c.gates, c.thetas, obs, gi)
        one = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": one * 1e3 * c.n_params, "unit": "ms", "cores": 1,
                                "kind": "oracle",
                                "sample": "parameter shift of one slot (2 propagations of the "
                                          "full circuit), scaled to all %d slots" % c.n_params}
    return line


def run_grad(args):
    print(json.dumps(measure_grad(args.steps, args.warmup, 64, not args.no_cpu_baseline)))
    return 0


def run_grad_n(args):
    """All gradients by the adjoint on the layered ansatz with n, m from the
    workload name grad-n<N>-<M> (O = the ZZ chain + 0.5 X field); device time of
    a training step's set_params (angles from device memory) + grad_async with
    CUDA events, L2 flushed between steps (new angles every step, so nothing
    made for earlier angles is reused)."""
    import torch
    from paper_2502_10685_gb300 import stab, workloads as W
    n, m = (int(v) for v in args.workload[len("grad-n"):].split("-"))
    torch.cuda.set_stream(torch.cuda.Stream())
    st = torch.cuda.current_stream()
    c = W.layered_ansatz(n, m, seed=1000 + n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    s.set_observable(W.obs_chain(n))
    g = torch.zeros(max(1, c.n_params), dtype=torch.float64, device="cuda")
    e = torch.zeros(8, dtype=torch.float64, device="cuda")
    th = torch.tensor(c.thetas, dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        s.set_params(th)
        s.grad_async(e, g)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = _events()
        e0.record(st)
        s.set_params(th)
        s.grad_async(e, g)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    s.close()
    ms = sum(times) / len(times)
    print(json.dumps({
        "metric": "gradient time", "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "n": n, "gates": m,
                                        "params": c.n_params, "l2": "flushed between steps"}}))
    return 0


def _percentiles(lat):
    import numpy as np
    lat = np.asarray(lat)
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


def serve_trace(reqs, mine, form, max_active, aging_s, device=0, burst=False, server_kw=None):
    """Submits reqs[i] for i in mine at their arrival times and waits for all.
    form: ("iterate" | "contexts", policy) through stab.Server, or "plain":
    one request at a time in arrival order, each on a context of the plain
    form (one pass per gate; gradients by the library's streamed adjoint, the
    plain form having none of its own), results to the host before the next
    starts.  burst: every request submitted at time 0 (profiler captures).
    Returns (per request (latency s, <O>), makespan s, clocks)."""
    import torch
    from paper_2502_10685_gb300 import stab
    clocks = ClockSampler(gpu_uuid(torch.device("cuda", device)))
    clocks.start()
    if form == "plain":
        ctxs = {}
        t0 = time.perf_counter()
        out = []
        for i in mine:
            r = reqs[i]
            arrival = 0.0 if burst else r.arrival_s
            delay = arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            c = r.circuit
            sx = ctxs.get(c.n)
            if sx is None:
                sx = ctxs[c.n] = stab.Stab(c.n, kernel="plain", device=device)
            sx.load_circuit(c.gates, c.thetas)
            if r.kind == "expect":
                val = sx.expect(r.observable)
            else:
                val, _ = sx.grad(r.observable)
            out.append((time.perf_counter() - t0 - arrival, val))
        span = time.perf_counter() - t0
        for sx in ctxs.values():
            sx.close()
        return out, span, clocks.stop()
    engine, policy = form
    srv = stab.Server(max_active=max_active, policy=policy, engine=engine, aging_s=aging_s,
                      device=device, **(server_kw or {}))
    t0 = time.perf_counter()
    ids = []
    for i in mine:
        r = reqs[i]
        delay = (0.0 if burst else r.arrival_s) - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(r.circuit, r.kind, r.observable))
    res = [srv.wait(i) for i in ids]
    srv.close()
    clk = clocks.stop()
    assert all(x["status"] == 0 for x in res)
    span = (max(x["done_s"] for x in res) - min(x["submit_s"] for x in res)) if res else 0.0
    return [(x["done_s"] - x["submit_s"], x["expect"]) for x in res], span, clk


def serve_summary(reqs, out, span):
    p50, p99 = _percentiles([x[0] for x in out])
    upd = sum((1 if r.kind == "expect" else 2) * r.circuit.m * 4 ** r.circuit.n for r in reqs)
    return {"p50_s": p50, "p99_s": p99, "circuits_per_s": len(reqs) / span, "makespan_s": span,
            "updates_per_s": upd / span}


def serve_cpu_baseline(reqs, sample=8):
    """The oracle on the trace, one core: its update rate measured on a seeded
    sample of the trace's small requests (4^n m <= 2e7; <O> = one backward
    propagation, a gradient = the parameter shift of one slot, two
    propagations), then every request of the trace costed at that rate (a
    gradient two propagations per slot: the oracle has no adjoint)."""
    import numpy as np
    import oracle
    from paper_2502_10685_gb300 import workloads as W
    oracle.build()
    cand = [r for r in reqs if 4 ** r.circuit.n * r.circuit.m <= 2e7]
    rng = np.random.default_rng(5)
    pick = [cand[i] for i in rng.choice(len(cand), size=min(sample, len(cand)), replace=False)]
    t0 = time.perf_counter()
    upd = 0
    for r in pick:
        c = r.circuit
        rot = [i for i, g in enumerate(c.gates) if int(g["op"]) in W.ROTATIONS]
        if r.kind == "grad" and rot:
            oracle.psr_grad_gate(c.n, c.gates, c.thetas, r.observable, rot[0])
            upd += 2 * c.m * 4 ** c.n
        else:
            oracle.expect(c.n, c.gates, c.thetas, r.observable)
            upd += c.m * 4 ** c.n
    rate = upd / (time.perf_counter() - t0)
    work = sum((2 * max(r.circuit.n_params, 1) if r.kind == "grad" else 1) * r.circuit.m *
               4 ** r.circuit.n for r in reqs)
    nproc, model = host_cpu()
    return {"value": len(reqs) / (work / rate), "unit": "circuits/s", "cores": 1,
            "kind": "oracle", "host": {"nproc": nproc, "cpu_model": model},
            "sample": "%d seeded requests with 4^n m <= 2e7 on one core (%.3g updates/s), the whole "
                      "trace costed at that rate, gradients by parameter shift" % (len(pick), rate)}


def measure_serve(requests, max_active=256, aging_s=4.0, small=False,
                  forms_run=("iterate", "contexts", "plain"), burst=False, with_cpu=False,
                  server_kw=None):
    """The first `requests` requests of the Poisson serving trace (2,000 req/s,
    n ~ U{4..12}, depth log-uniform [100, 60,000], 50/50 <O> / gradient, seed
    1005), through the iteration engine and the context engine (both
    shortest-work-first with the aging bound) and the plain form, each with
    its own clock record; latency = completion - arrival."""
    from paper_2502_10685_gb300 import workloads as W
    if small:
        # the iteration engine's own range: n ~ U{4..8}, depth log-uniform [100, 20,000]
        reqs = W.serving_trace(requests, seed=1015, n_range=(4, 8), depth_range=(100, 20000))
    else:
        reqs = W.serving_trace(requests, seed=1005)
    mine = list(range(len(reqs)))
    # one context of every size first: the path tuner measures each n once per
    # process, which must not land inside the first form's timed trace
    from paper_2502_10685_gb300 import stab
    for n in sorted({r.circuit.n for r in reqs}):
        stab.Stab(n).close()
    forms = {}
    vals = {}
    for name, form in (("iterate", ("iterate", "shortest")), ("contexts", ("contexts", "shortest")),
                       ("plain", "plain")):
        if name not in forms_run:
            continue
        out, span, clk = serve_trace(reqs, mine, form, max_active, aging_s, burst=burst,
                                     server_kw=server_kw if name == "iterate" else None)
        forms[name] = dict(serve_summary(reqs, out, span), clocks=clk)
        vals[name] = [x[1] for x in out]
    first = next(iter(forms))
    worst = max([abs(a - b) for k in forms if k != first
                 for a, b in zip(vals[first], vals[k])] or [0.0])
    it = forms[first]
    line = {
        "metric": "p50/p99 latency", "value": it["p50_s"], "unit": "s", "p99_s": it["p99_s"],
        "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve-small" if small else "serve-c5", "requests": len(reqs),
                   "rate_per_s": 2000, "n_range": [4, 8] if small else [4, 12],
                   "max_active": max_active, "policy": "shortest estimated work first, aging "
                   "bound %g s" % aging_s, "arrivals": "all at 0" if burst else "Poisson",
                   "engine": "iteration engine for n <= 6, contexts above",
                   "iteration_engine_options": server_kw or "defaults"},
        "circuits_per_s": it["circuits_per_s"], "makespan_s": it["makespan_s"],
        "forms": forms,
        "speedup_vs_plain_circuits_per_s": (it["circuits_per_s"] / forms["plain"]["circuits_per_s"]
                                            if "plain" in forms else None),
        "max_abs_diff_between_forms": worst, "clocks": it["clocks"]}
    if with_cpu:
        line["cpu_baseline"] = serve_cpu_baseline(reqs)
    return line


def run_serve(args):
    """Serving trace: the line of measure_serve on one GPU; with several ranks
    each request is routed, in arrival order, to the rank with the least work
    assigned so far (the same routing on every rank, no exchange), every rank
    serves its share on its GPU through the iteration engine, and the
    per-request results are gathered to rank 0 (the trace is fixed: strong
    scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2502_10685_gb300 import units, workloads as W
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world == 1 or args.workload == "serve-small":
        print(json.dumps(measure_serve(args.requests, args.max_active, args.aging,
                                       small=args.workload == "serve-small",
                                       forms_run=tuple(args.serve_forms.split(",")),
                                       burst=args.burst, with_cpu=not args.no_cpu_baseline,
                                       server_kw={k: v for k, v in (
                                           ("iter_chunks", args.iter_chunks),
                                           ("iter_smem_kb", args.iter_smem_kb),
                                           ("iter_max_n", args.iter_max_n),
                                           ("iter_slice_us", args.iter_slice_us)) if v})))
        return 0
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    reqs = W.serving_trace(args.requests, seed=1005)
    # a gradient sweeps about three vectors where <O> sweeps one
    costs = [units.unit_cost(r.circuit.n, r.circuit.m, 1 if r.kind == "expect" else 3)
             for r in reqs]
    route = units.route_in_arrival_order(costs, world)
    mine = [i for i, r in enumerate(route) if r == rank]
    out, span, clk = serve_trace(reqs, mine, ("iterate", "shortest"), args.max_active, args.aging,
                                 device=local)
    full = units.gather_to_root(mine, out, len(reqs), dist)
    spans = [span] * world
    dist.all_gather_object(spans, span)
    dist.destroy_process_group()
    if rank != 0:
        return 0
    lat = np.array([x[0] for x in full])
    print(json.dumps({
        "metric": "p50/p99 latency", "value": float(np.percentile(lat, 50)), "unit": "s",
        "p99_s": float(np.percentile(lat, 99)), "n_gpus": world, "higher_is_better": False,
        "scaling": "strong", "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve-c5", "requests": len(reqs), "rate_per_s": 2000,
                   "max_active": args.max_active, "policy": "shortest estimated work first",
                   "routing": "arrival order, least assigned work"},
        "circuits_per_s": len(reqs) / max(spans), "makespan_s": max(spans), "clocks": clk}))
    return 0


def run_expect(args):
    """<O> only (one vector propagated backward) on the layered ansatz with
    n, m from the workload name expect-n<N>-<M>; device-resident steps timed
    with CUDA events, L2 flushed between steps."""
    import torch
    from paper_2502_10685_gb300 import stab, workloads as W
    n, m = (int(v) for v in args.workload[len("expect-n"):].split("-"))
    peak, _ = fp64_peak()
    torch.cuda.set_stream(torch.cuda.Stream())
    st = torch.cuda.current_stream()
    c = W.layered_ansatz(n, m, seed=1000 + n)
    obs = W.obs_chain(n)
    s = stab.Stab(n)
    s.load_circuit(c.gates, c.thetas)
    s.set_observable(obs)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        s.expect_async(out)
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tot = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = _events()
        e0.record(st)
        s.expect_async(out)
        e1.record(st)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    ms = tot / args.steps
    n_rot = int(sum(1 for g in c.gates if g["op"] in W.ROTATIONS))
    flops = n_rot * 1.5 * 4 ** n
    s.close()
    print(json.dumps({
        "metric": METRIC, "value": m * 4 ** n / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "gates": m, "vectors_per_step": 1},
        "fp64_tflops": flops / (ms / 1e3) / 1e12, "fp64_frac_of_peak": flops / (ms / 1e3) / 1e12 / peak,
        "peak_source": "of measured: DFMA chains on this GPU (stab_probe_fp64)"}))
    return 0


def run_fp64_peak(args):
    """The FP64 rates of this GPU (the roofline denominators of the rotation
    passes): DFMA and FP64 matrix-instruction chains at two launch lengths,
    with the clocks seen during the probes."""
    import torch
    from paper_2502_10685_gb300 import stab
    dev = torch.device("cuda", 0)
    props = torch.cuda.get_device_properties(dev)
    clocks = ClockSampler(gpu_uuid(dev))
    clocks.start()
    time.sleep(0.3)
    rows = []
    for kind, iters in (("dfma", 4096), ("dfma", 16384), ("dmma", 1024), ("dmma", 4096)):
        for _ in range(3):
            tf, ms = stab.stab_probe_fp64(kind, iters)
            rows.append({"kind": kind, "iters": iters, "tflops": tf, "ms": ms})
    clk = clocks.stop()
    best = {k: max(r["tflops"] for r in rows if r["kind"] == k) for k in ("dfma", "dmma")}
    mhz = clk.get("sm_mhz") or 2070.0
    print(json.dumps({
        "metric": "FP64 TFLOP/s", "value": best["dfma"], "unit": "TFLOP/s", "n_gpus": 1,
        "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fp64-peak", "sms": props.multi_processor_count,
                   "gpu": props.name},
        "dmma_tflops": best["dmma"],
        "dfma_per_clk_per_sm": best["dfma"] * 1e12 / 2 / props.multi_processor_count / (mhz * 1e6),
        "runs": rows, "clocks": clk}))
    return 0


def run_pass_latency(args):
    """Cycles per wire pass of the n = 4 register loop's pieces (one CTA, the
    SM's cycle counter; stab_probe_pass): what bounds a lone vector of the
    split generator sweep, against the FP64 pipe's six warp instructions per
    SMSP per pass."""
    import torch
    from paper_2502_10685_gb300 import stab
    dev = torch.device("cuda", 0)
    clocks = ClockSampler(gpu_uuid(dev))
    clocks.start()
    time.sleep(0.3)
    cases = [("register passes", 0, 256), ("+ layout switch every 2nd pass", 1, 256),
             ("+ four-CNOT pull walk every 4th pass", 2, 256),
             ("register passes, 128 threads", 0, 128),
             ("two entries per thread, one barrier per 4 passes (pull merged)", 3, 128),
             ("two-wire fused passes (per wire pass)", 4, 256)]
    rows = []
    for name, pattern, threads in cases:
        runs = [stab.stab_probe_pass(pattern, threads, 40000) for _ in range(3)]
        rows.append({"case": name, "pattern": pattern, "threads": threads,
                     "clk_per_pass": statistics.median(runs), "runs": runs})
    clk = clocks.stop()
    print(json.dumps({
        "metric": "cycles per wire pass", "value": rows[2]["clk_per_pass"], "unit": "clk",
        "n_gpus": 1, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "pass-latency", "passes": 40000, "ctas": 1},
        "rows": rows, "clocks": clk}))
    return 0


def run_paper_sweep(args):
    """The paper's experiment shape (Sec. V): time to the density matrix of
    the W_chain + ZXZ ansatz, n = 2, 3, 4, over #Layers (Repeats = 1) and
    #Repeats (Layers = 50), through the host-buffer calls (stab_load_circuit +
    stab_density_matrix to host memory), beside the CPU oracle's decode."""
    import numpy as np
    import oracle
    from paper_2502_10685_gb300 import stab, workloads as W
    oracle.build()
    rows = []
    points = [(L, 1) for L in (1, 10, 100, 1000)] + [(50, R) for R in (1, 10, 50, 100)]
    for n in (2, 3, 4):
        s = stab.Stab(n)
        for (layers, repeats) in points:
            c = W.paper_shaped_ansatz(n, layers, repeats, seed=7 + n)
            s.load_circuit(c.gates, c.thetas)
            s.density_matrix()
            reps = 5
            t0 = time.perf_counter()
            for _ in range(reps):
                s.load_circuit(c.gates, c.thetas)
                rho = s.density_matrix()
            gpu_s = (time.perf_counter() - t0) / reps
            t0 = time.perf_counter()
            ref = oracle.density_matrix(n, c.gates, c.thetas)
            cpu_s = time.perf_counter() - t0
            perm = np.zeros(2 ** n, dtype=int)
            for i in range(2 ** n):
                perm[i] = int(format(i, "0%db" % n)[::-1], 2)
            err = float(np.abs(rho[np.ix_(perm, perm)] - ref).max())
            rows.append({"n": n, "layers": layers, "repeats": repeats, "gates": c.m,
                         "todm_s": gpu_s, "oracle_todm_s": cpu_s, "max_abs_err": err})
        s.close()
    print(json.dumps({"metric": "time to density matrix", "unit": "s",
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "paper-sweep"}, "points": rows}))
    return 0


def _sparse_step_gates(c, backward=True):
    """Gates applied by each step of the sparse path: Clifford runs (in
    application order) and single rotations, as the library cuts them."""
    from paper_2502_10685_gb300 import workloads as W
    ops = [int(g["op"]) for g in (c.gates[::-1] if backward else c.gates)]
    steps, run = [], 0
    for op in ops:
        if op in W.ROTATIONS:
            if run:
                steps.append(("c", run))
                run = 0
            steps.append(("r", 1))
        else:
            run += 1
    if run:
        steps.append(("c", run))
    return steps


def _sparse_work(c, n0, history):
    """(term-gate updates, algorithmic bytes) of one backward propagation:
    every step reads its list (8 B key + 8 B coefficient per term) and writes
    its output list; a Clifford run maps each term once per gate."""
    steps = _sparse_step_gates(c)
    assert len(steps) == len(history), (len(steps), len(history))
    upd, nbytes, before = 0, 0, n0
    for (kind, g), after in zip(steps, history):
        upd += before * g
        nbytes += 16 * before + 16 * int(after)
        before = int(after)
    return upd, nbytes


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                               "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback 6.8 TB/s"


def run_sparse(args):
    """Term-list (sparse) path: n = 32, a 20,000-gate Clifford circuit with 28
    rotations; <O> for the open ZZ chain plus an X field, O propagated
    backward as a list (its order reaches ~5e6 terms).  Metric: term-gate
    updates/s (sum over steps of the list length times the gates the step
    applies).  The oracle is timed on the same circuit with fewer rotations."""
    import oracle
    import torch
    from paper_2502_10685_gb300 import stab, workloads as W
    n, m, n_rot = 32, 20000, 28
    c = W.clifford_plus_rotations(n, m, n_rot, seed=1006)
    obs = W.obs_chain(n)
    n0 = len(obs)
    sp = stab.Sparse(n, max_terms=1 << 26)
    sp.load_circuit(c.gates, c.thetas)
    for _ in range(args.warmup):
        val, info = sp.expect(obs)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        val, info = sp.expect(obs)
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    hist = sp.order_history()
    upd, nbytes = _sparse_work(c, n0, hist)
    dt = sum(times) / len(times)
    peak, src = _hbm_peak()
    achieved = nbytes / dt / 1e9
    line = {
        "metric": "term-gate updates/s", "value": upd / dt, "unit": "updates/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "sparse-n32", "n": n, "gates": m, "rotations": n_rot,
                   "observable_terms": n0, "l2": "list larger than L2 at its largest"},
        "expect": val, "order_max": info["order_max"], "steps_per_call": info["steps"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_source": src,
                     "kernel": "whole call (all sparse kernels), algorithmic bytes = "
                               "16 B per term read + 16 B per term written per step"},
        "clocks": clk,
    }
    sp.close()
    # where both representations apply (n = 12): term list (switching to the
    # dense vector past its threshold) against the dense path, same circuits
    cmp = []
    for n_rot in (8, 16, 24):
        c12 = W.clifford_plus_rotations(12, 4000, n_rot, seed=1016)
        o12 = W.obs_chain(12)
        sp12 = stab.Sparse(12, max_terms=1 << 22)
        sp12.load_circuit(c12.gates, c12.thetas)
        d12 = stab.Stab(12)
        d12.load_circuit(c12.gates, c12.thetas)
        for _ in range(3):
            vs, inf12 = sp12.expect(o12)
            vd = d12.expect(o12)
        t0 = time.perf_counter()
        for _ in range(5):
            vs, inf12 = sp12.expect(o12)
        ts = (time.perf_counter() - t0) / 5
        t0 = time.perf_counter()
        for _ in range(5):
            vd = d12.expect(o12)
        td = (time.perf_counter() - t0) / 5
        cmp.append({"n": 12, "gates": 4000, "rotations": n_rot, "sparse_ms": ts * 1e3,
                    "dense_ms": td * 1e3, "order_max": inf12["order_max"],
                    "dense_gates": inf12["dense_gates"], "abs_diff": abs(vs - vd)})
        sp12.close()
        d12.close()
    line["sparse_vs_dense_n12"] = cmp
    if not args.no_cpu_baseline:
        # oracle on the same circuit with fewer rotations (a bounded sample)
        k = 16
        cs = W.clifford_plus_rotations(n, m, k, seed=1006)
        sp2 = stab.Sparse(n, max_terms=1 << 22)
        sp2.load_circuit(cs.gates, cs.thetas)
        sp2.expect(obs)
        upd_s, _ = _sparse_work(cs, n0, sp2.order_history())
        sp2.close()
        oracle.build()
        t0 = time.perf_counter()
        oracle.sparse_expect(n, cs.gates, cs.thetas, obs)
        t_cpu = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": upd_s / t_cpu, "unit": "updates/s", "cores": 1,
                                "kind": "oracle",
                                "sample": "same n and gates, %d rotations (list up to ~5e4 "
                                          "terms), one call on one core" % k}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="layered-n4-60200")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-sub", action="store_true",
                    help="default line: skip the batch, gradient and serving sub-measurements")
    ap.add_argument("--sub-requests", type=int, default=64,
                    help="default line: serving trace length of the sub-measurement")
    ap.add_argument("--requests", type=int, default=200, help="serve-c5: trace length")
    ap.add_argument("--max-active", type=int, default=256, help="serve-c5: admitted at once")
    ap.add_argument("--aging", type=float, default=4.0, help="serve-c5: aging bound (s)")
    ap.add_argument("--burst", action="store_true",
                    help="serve-c5 / serve-small: submit every request at time 0")
    ap.add_argument("--iter-chunks", type=int, default=0,
                    help="serve workloads: the iteration engine's chunks per slice at n = 4")
    ap.add_argument("--iter-smem-kb", type=int, default=0,
                    help="serve workloads: KiB of shared memory per CTA for vectors")
    ap.add_argument("--iter-max-n", type=int, default=0,
                    help="serve workloads: largest n the iteration engine takes")
    ap.add_argument("--iter-slice-us", type=float, default=0.0,
                    help="serve workloads: target slice length (us; < 0: static budgets)")
    ap.add_argument("--serve-forms", default="iterate,contexts,plain",
                    help="serve-c5 / serve-small: which forms to run (comma list)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batch-c3", "batch-small"):
        return run_batch(args)
    if args.workload == "grad-c4":
        return run_grad(args)
    if args.workload.startswith("grad-n"):
        return run_grad_n(args)
    if args.workload in ("serve-c5", "serve-small"):
        return run_serve(args)
    if args.workload.startswith("expect-n"):
        return run_expect(args)
    if args.workload == "fp64-peak":
        return run_fp64_peak(args)
    if args.workload == "pass-latency":
        return run_pass_latency(args)
    if args.workload == "paper-sweep":
        return run_paper_sweep(args)
    if args.workload == "sparse-n32":
        return run_sparse(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
