#!/usr/bin/env python3
"""Benchmark: unique variables updated per second by the symmetry-adapted
HEOM RK4 step on B300.

Workload (default): w4, a batch of 512 independent seeded instances with
uneven N in 2..64, m in 1..2 plus the averaged static-disorder channel, L in
3..8, FP32 auxiliary variables with an FP64 physical density matrix, dt =
0.02.  One "step" is one classical RK4 step of the whole batch (four fused
right-hand-side + stage kernels).  Inputs are synthetic (seeded) and resident
in HBM; the four state-sized vectors (~0.6 GB) exceed the 126 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload w4|w5|w3|sec5]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own copy
of the batch (weak scaling, no data-path collective); the time is the max
over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "unique_vars_updated_per_s"
UNIT = "unique-variable RK4 updates/s"
FP32_BYTES_PER_VAR_STEP = 136    # 17 complex float accesses per variable per RK4 step
FP64_BYTES_PER_VAR_STEP = 272


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def max_over_ranks(value: float, dist) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's);
    the tensor lives where the process group's backend can reduce it."""
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(", ") for r in out.strip().splitlines() if r.strip()]
        sm = [float(r[0]) for r in rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 8:
                continue
            for n, v in zip(names, r[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_PHYS_BEGIN = "// -- begin: physical-representative kernels (outside the stage kernels' code)\n"
_PHYS_END = "// -- end: physical-representative kernels\n"
_PACK_BEGIN = "// -- begin: pack kernel (the opt-in packed layout; no list-kernel code)\n"
_PACK_END = "// -- end: pack kernel\n"


def _stage_sha(pack: bool = False) -> str:
    """Hash of the stage kernels' source: kernels.cu less its marked
    physical-representative sections (the FP64 rho_0, observables and init
    kernels and their launch wrappers) and, unless the packed layout's stage
    is meant, its pack-kernel section, which no other stage kernel calls."""
    src = open(os.path.join(ROOT, "paper_2608_20657_b300", "csrc", "kernels.cu"), encoding="utf-8").read()
    for b, e in ((_PHYS_BEGIN, _PHYS_END),) + (() if pack else ((_PACK_BEGIN, _PACK_END),)):
        src = re.sub(re.escape(b) + ".*?" + re.escape(e), "", src, flags=re.S)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _traffic(workload: str, kernel_name: str):
    """DRAM bytes per stage launch from the committed ncu summary of this
    kernel (variant and precision), if it was taken on the current kernel
    source."""
    p = os.path.join(ROOT, "profiles", f"{kernel_name.split('<')[0]}_{workload}_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("kernel_sha") != _stage_sha(kernel_name.startswith("pack")) or d.get("kernel") != kernel_name:
        return None
    return d.get("dram_bytes_per_launch")


def _params(workload):
    import paper_2608_20657_b300 as S

    if workload == "w4":
        ws = W.batch_w4()
        return ws, [S.params_from(w) for w in ws], S.SA_FP32_AUX, 0.02
    w = _single(workload)
    return [w], [S.params_from(w)], S.SA_FP32_AUX, w["dt_fs"] if workload == "sec5" else w["dt"]


def _single(workload):
    """A one-instance workload: w3, w5, or the paper's production set (Sec. V:
    N = 10^12, L = 25, one exponential plus the terminator, upper polariton)."""
    return W.sec5(10 ** 12, "up") if workload == "sec5" else W.WORKLOADS[workload]


def _rho0(ws):
    import paper_2608_20657_b300 as S

    draws = W.random_rho_draws()
    return np.stack([S.rho0_vars(w, draws) for w in ws])


# ------------------------------------------------------------ CPU baseline

def _oracle_sample(workload: str, budget_vars: int):
    """A bounded sample of the workload for the oracle: the first instances
    of the batch until budget_vars unique variables (w4), else the instance
    itself."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from tests._helpers import oracle_rho0, oracle_sa

    ws = W.batch_w4() if workload == "w4" else [_single(workload)]
    sample, total = [], 0
    for w in ws:
        sa = oracle_sa(w, cache=True)
        x = sa.initial_state(*oracle_rho0(w, W.random_rho_draws()))
        sample.append((sa, x))
        total += sa.nvar
        if total >= budget_vars:
            break
    return sample, total, len(ws)


def cpu_baseline(workload: str, seconds: float = 15.0, dt: float = 0.02) -> dict:
    import oracle

    sample, total, n_all = _oracle_sample(workload, 400_000 if workload == "w4" else 10 ** 12)
    steps, t0 = 0, time.perf_counter()
    while True:
        for sa, x in sample:
            sa.rk4(x, dt, 1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or (workload == "w5" and steps >= 1):
            break
    return {"value": total * steps / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "cpu": _cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{len(sample)} of {n_all} instances ({total} unique variables), {steps} RK4 steps, "
                      f"{el:.1f} s, FP64 C oracle with OpenMP over patterns"}


def _cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _workload_name(workload: str) -> str:
    if workload == "sec5":
        return "sec5 (Sec. V production set: N = 10^12, L = 25, m = 1 + terminator, UP start, dt 0.5 fs)"
    return workload + (" (512 seeded instances, FP32-aux + FP64 rho_0)" if workload == "w4" else "")


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return 0
    import oracle

    sample, total, n_all = _oracle_sample(args.workload, 400_000 if args.workload == "w4" else 10 ** 12)
    dt = 0.02
    for _ in range(args.warmup):
        for sa, x in sample:
            sa.rk4(x, dt, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for sa, x in sample:
            sa.rk4(x, dt, 1)
    el = time.perf_counter() - t0
    val = total * args.steps / el
    cb = {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
          "sample": f"{len(sample)} of {n_all} instances ({total} unique variables) per step"}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": _workload_name(args.workload), "n_instances": n_all,
                                 "sample": cb["sample"], "parallelism": "replicas1"},
                      "cpu_baseline": cb, "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                                                   "d2h_bytes_per_step": 0}}))
    return 0


# ------------------------------------------------------------ GPU arm

def _kernel_name(kernel, fp32, packed=False):
    """The stage kernel the step launches (the instantiation without index
    checks); on a packed handle the pack kernel, which also runs the list
    units of the unpacked instances."""
    args = "<float,true,false>" if fp32 else "<double,false,false>"
    if packed:
        return "pack_stage_kernel" + args
    return {1: "list_stage_kernel", 2: "ell_stage_kernel"}.get(kernel, "stage_kernel") + args


def run_ours(args):
    import torch

    import paper_2608_20657_b300 as S

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    ws, ps, precision, dt = _params(args.workload)
    if args.precision == "fp64":
        precision = S.SA_FP64
    h = S.Heom(ps, precision=precision, pack=args.layout == "packed")
    # a single instance, or a batch without a template of 16 members, has
    # no pack: its layout stays the canonical one
    pack = args.layout == "packed" and len(h.dump_packs()["packs"]) > 0
    st = h.new_state()
    h.init_state(st, _rho0(ws))
    stream = torch.cuda.current_stream()
    if args.tune:
        best = tuple(int(v) for v in args.tune.split(","))
        h.set_tuning(*best[:3])
        if len(best) > 3:
            h.set_kernel(best[3])
    else:
        h.autotune(st)
    tuning = h.tuning()
    h.init_state(st, _rho0(ws))
    torch.cuda.synchronize()

    # warm-up, and the CUDA graphs of the timed propagation built beforehand
    h.propagate(st, dt, args.warmup, observe=False)
    h.prepare(st, dt, args.steps)
    torch.cuda.synchronize()

    clocks = Clocks(torch.cuda.current_device()) if rank == 0 else None
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.propagate(st, dt, args.steps, observe=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if dist:
        dist.barrier()
    ck = clocks.stop() if clocks else None
    if dist:
        ms = max_over_ranks(ms, dist)
    ms_step = ms / args.steps
    n_vars = h.n_vars
    value = n_vars * world * args.steps / (ms / 1e3)

    # roofline of the stage kernel (4 launches per step; in FP32-aux mode the
    # small FP64 kernel of the physical density matrix overlaps each of them
    # on a side stream; on a packed handle the stage kernel is the pack
    # kernel, which runs the unpacked instances' list units after its packs)
    launch_ms = ms_step / 4.0
    bytes_launch = FP32_BYTES_PER_VAR_STEP * n_vars / 4.0 if precision == S.SA_FP32_AUX else \
        FP64_BYTES_PER_VAR_STEP * n_vars / 4.0
    achieved = bytes_launch / (launch_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    kname = _kernel_name(tuning["kernel"], precision == S.SA_FP32_AUX, pack)
    traffic = _traffic(args.workload, kname)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs",
            # DRAM bytes the kernel really moves (ncu, per launch) over the same live launch time
            "dram_achieved": traffic / (launch_ms / 1e3) / 1e9 if traffic else None,
            "dram_frac": traffic / (launch_ms / 1e3) / 1e9 / peak if traffic else None,
            "kernel": kname, "bytes_per_launch": bytes_launch}

    # end to end through the public API with host buffers: upload the state
    # from pinned host memory, K steps with the observables of every step read
    # back to the host, download the state
    e2e = None
    if not args.no_e2e:
        host_x = h.download(st)
        pinned = torch.from_numpy(host_x.view(np.float64)).pin_memory()
        hx = pinned.numpy().view(np.complex128)
        pinned_back = torch.empty_like(pinned).pin_memory()
        hb = pinned_back.numpy().view(np.complex128)
        k_e2e = max(1, min(args.steps, 50))
        h.prepare(st, dt, k_e2e, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.upload(st, hx)
        obs = h.propagate(st, dt, k_e2e, 1)
        back = h.download(st, out=hb)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        # bytes that cross the bus: the complex128 host state each way (the
        # device narrows / widens it), and the observables of every step
        e2e = {"value": n_vars * world * k_e2e / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(hx.nbytes / k_e2e),
               "d2h_bytes_per_step": int((back.nbytes + obs.nbytes) / k_e2e),
               "steps": k_e2e, "note": "state upload + propagate with observables every step + state download"}
        del back

    # FP64 comparison on the same workload: time per step and the population
    # error of the FP32-aux path against it
    extra = {}
    if rank == 0 and args.workload in ("w4", "w5") and not args.no_fp64 and precision == S.SA_FP32_AUX:
        extra = _fp64_comparison(S, torch, stream, args, h, ws, ps, dt, ms_step)

    if rank == 0 and not args.no_reconstruct:
        extra["reconstruct"] = _time_reconstruct(S, torch, stream)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if precision == S.SA_FP32_AUX else "f64",
                "data": "synthetic",
                "config": {"workload": _workload_name(args.workload),
                           "n_instances": h.count, "n_vars": n_vars, "n_patterns": h.n_patterns,
                           "state_bytes": h.state_bytes, "l2": "inputs larger than L2 (4 vectors)",
                           "tuning": tuning, "layout": "packed" if pack else "canonical",
                           "parallelism": f"replicas{world}"},
                "roofline": roof, "gpu_launches": h.launches_per_step() * args.steps, "clocks": ck, "e2e": e2e}
        line.update(extra)
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds, dt)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def _fp64_comparison(S, torch, stream, args, h32, ws, ps, dt, ms_step) -> dict:
    """The FP64 path on the same workload: ms per RK4 step, and the largest
    population error of the FP32-aux path against it over --err-steps steps
    (observed every tenth of them).  For the batch (w4) also the plain
    single-instance FP64 path: 32 seeded instances, each with its own handle
    and CUDA graph, run one after another and scaled to the batch; w5 is one
    instance, so its FP64 path is that path already."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h64 = S.Heom(ps, precision=S.SA_FP64, pack=args.layout == "packed")
    s64 = h64.new_state()
    if args.workload == "w4":
        h64.autotune(s64)
    else:  # one instance of 170 M variables: the list kernel's usual shape (no search)
        h64.set_tuning(128, 192, 1)
    h64.init_state(s64, _rho0(ws))
    h64.propagate(s64, dt, 3, observe=False)
    k64 = max(3, min(args.steps, 20))
    h64.prepare(s64, dt, k64)
    torch.cuda.synchronize()
    e0.record(stream)
    h64.propagate(s64, dt, k64, observe=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / k64
    nerr = args.err_steps
    a, b = h64.new_state(), h32.new_state()
    h64.init_state(a, _rho0(ws))
    h32.init_state(b, _rho0(ws))
    o64 = h64.propagate(a, dt, nerr, max(1, nerr // 10))
    o32 = h32.propagate(b, dt, nerr, max(1, nerr // 10))
    err = float(np.max(np.abs(o64[:, :, 1:7] - o32[:, :, 1:7])))
    del h64, s64, a, b
    torch.cuda.empty_cache()
    t_final = W.WORKLOADS["w5"]["steps"] if args.workload == "w5" else 10000
    out = {"fp64_ms_per_step": ms64, "fp32_over_fp64_speedup": ms64 / ms_step,
           "fp32_max_population_error_vs_fp64": err, "population_error_window_steps": nerr,
           "time_to_t_final_s": {"fp32_aux": ms_step * t_final / 1e3, "fp64": ms64 * t_final / 1e3,
                                 "steps": t_final}}
    if args.workload != "w4":
        return out
    rng = np.random.default_rng(2608)
    pick = np.sort(rng.choice(len(ps), size=min(32, len(ps)), replace=False))
    k1, ms_single = 20, 0.0
    for i in pick:
        h1 = S.Heom([ps[i]], precision=S.SA_FP64)
        s1 = h1.new_state()
        h1.init_state(s1, _rho0([ws[i]]))
        h1.propagate(s1, dt, 3, observe=False)
        h1.prepare(s1, dt, k1)
        torch.cuda.synchronize()
        e0.record(stream)
        h1.propagate(s1, dt, k1, observe=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_single += e0.elapsed_time(e1) / k1
        del h1, s1
    ms_single *= len(ps) / len(pick)
    out.update({"fp64_single_instance_ms_per_step": ms_single,
                "fp32_batched_over_fp64_single_speedup": ms_single / ms_step,
                "fp64_single_instance_note": f"{len(pick)} seeded instances run one at a time ({k1} steps each, "
                                             "own handle and CUDA graph), summed and scaled to the batch"})
    out["time_to_t_final_s"]["fp64_single_instance"] = ms_single * t_final / 1e3
    return out


def _time_reconstruct(S, torch, stream, n: int = 8192, reps: int = 10) -> dict:
    """Arbitrary initial operators (sa_heom_reconstruct_dense): the five
    representative propagations of an N = n - 1 instance (one exponential,
    L = 2, 20 steps), then the dense reconstruction of a seeded random
    operator, timed with CUDA events over `reps` calls.  Algorithmic bytes:
    A read twice and rho_S(t) written once, 48 per entry; FP64 work about 14
    operations per entry (2 complex FMAs in the bulk pass, ~4 adds per
    element in the partial sums)."""
    bath = {"c": np.array([0.3 + 0.05j]), "cc": np.array([0.3 - 0.05j]), "nu": np.array([0.6 + 0j])}
    h = S.Heom(S.make_params(n - 1, 1, 2, bath, g=0.01), representatives=True)
    st = h.new_state()
    h.init_representatives(st, stream)
    h.propagate(st, 0.05, 20, observe=False, stream=stream)
    gen = torch.Generator(device="cuda").manual_seed(2608)
    a = torch.randn(n, n, dtype=torch.complex128, device="cuda", generator=gen)
    out = torch.empty_like(a)
    for _ in range(3):
        h.reconstruct_dense(st, a, out, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        h.reconstruct_dense(st, a, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = 48.0 * n * n / (ms * 1e-3) / 1e9
    peak, peak_src = _peaks()
    # FP64 issue rate: 2 operations per clock per SM at the maximum SM clock
    mhz = 2032.0
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        mhz = float(json.load(open(pp)).get("sm_max_mhz", mhz))
    props = torch.cuda.get_device_properties(0)
    fp64_ops = 2.0 * props.multi_processor_count * mhz * 1e6
    out_ok = bool(torch.isfinite(out).all())
    del a, out, h, st
    return {"n": n, "ms_per_call": ms, "algorithmic_gbs": gbs, "hbm_frac": gbs / peak, "hbm_peak_source": peak_src,
            "bound": "alu (fp64)", "fp64_ops_per_entry": 14, "fp64_frac": 14.0 * n * n / (ms * 1e-3) / fp64_ops,
            "finite": out_ok}


def run_conv_scaling(args):
    """The conventional GPU hierarchy against the symmetry-adapted one as N
    grows (the w2 family: DL + 1 Matsubara pole, L = 6, g sqrt(N) =
    0.05, bright start), FP64 both: ms per RK4 step, the two state sizes, and
    the population agreement after the same steps.  Prints one JSON line."""
    import torch

    import paper_2608_20657_b300 as S

    rank, _ = _dist()
    if rank != 0:
        return 0
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rows = []
    for N in [int(v) for v in args.conv_n.split(",")]:
        w = dict(W.WORKLOADS["w2"], N=N)
        p = S.params_from(w)
        dt, k = w["dt"], 5
        t0 = time.perf_counter()
        cv = S.Conventional(p)
        t_build = time.perf_counter() - t0
        st = cv.new_state()
        rho = np.zeros((N + 1, N + 1), complex)
        rho[1:, 1:] = 1.0 / N  # |B><B|
        cv.set_rho0(st, rho)
        cv.step(st, dt, 2, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        cv.step(st, dt, k, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_conv = e0.elapsed_time(e1) / k
        rho_t = st[: (N + 1) ** 2 * 16].view(torch.float64).cpu().numpy().view(np.complex128).reshape(N + 1, N + 1)
        conv_bytes, nado = cv.state_bytes, cv.nado
        del cv, st
        h = S.Heom(p)
        s2 = h.new_state()
        h.init_state(s2, S.rho0_vars(w))
        h.propagate(s2, dt, 2, observe=False)
        torch.cuda.synchronize()
        e0.record(stream)
        h.propagate(s2, dt, k, observe=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_sa = e0.elapsed_time(e1) / k
        o = h.observables(s2)[0]
        rows.append({"N": N, "conventional_ados": nado, "conventional_bytes": conv_bytes,
                     "conventional_ms_per_step": ms_conv, "conventional_build_s": t_build,
                     "sa_vars": h.n_vars, "sa_bytes": h.n_vars * 16, "sa_ms_per_step": ms_sa,
                     "speedup": ms_conv / ms_sa,
                     "pop_diff": float(max(abs(o[1] - rho_t[0, 0].real),
                                           abs(o[2] - (np.trace(rho_t).real - rho_t[0, 0].real))))})
        del h, s2
    print(json.dumps({"conv_scaling": rows, "workload": "w2 family (DL + 1 Matsubara, L = 6), FP64, bright start",
                      "steps_timed": 5}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="w4", choices=["w3", "w4", "w5", "sec5"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--err-steps", type=int, default=2000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"],
                    help="fp32: FP32 auxiliary variables with FP64 rho_0 (default); fp64: everything in FP64")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-reconstruct", action="store_true")
    ap.add_argument("--conv-scaling", action="store_true",
                    help="time the conventional against the symmetry-adapted hierarchy over --conv-n, then exit")
    ap.add_argument("--conv-n", default="2,4,6,8,10,12")
    ap.add_argument("--reconstruct-only", action="store_true",
                    help="time only the dense reconstruction of arbitrary initial operators (N + 1 = 8192; "
                         "--steps calls), then exit")
    ap.add_argument("--tune", default="", help="block,chunk,queue[,kernel] (skips the autotuner; kernel 0 = "
                                                "connection records, 1 = term lists)")
    ap.add_argument("--layout", default="packed", choices=["packed", "canonical"],
                    help="packed (default, the faster on w4): instances of repeated templates interleaved in packs "
                         "of up to 32 (SA_BUILD_PACK_INSTANCES, the pack kernel); canonical: instance after instance, "
                         "the list kernel only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.conv_scaling:
        return run_conv_scaling(args)
    if args.reconstruct_only:
        import torch

        import paper_2608_20657_b300 as S

        print(json.dumps({"reconstruct": _time_reconstruct(S, torch, torch.cuda.current_stream(), reps=args.steps)}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
