"""Benchmark: parameter-configuration CV evaluations per second on one GB300.

A step is one pass of the whole hot path (gather, assembly, factorisation,
solves, refinement, prediction, local SSPE, combine) over one batch of B
parameter configurations of a device-resident dataset.  Default workload: the
paper-scale stand-in (2236^2 grid, 4,999,696 nodes with 10% missing, 80/10/10
split, 40 x 40 cores, shell 0.001, about 1600 subsets of 2250-2630 training
points), seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--workload paper5m|cluster262k|uniform4096] [--batch B]
                    [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is device-timed (CUDA events around each
step on the launching stream, L2 flushed between steps); `e2e` is the same metric
through the host-pointer C-ABI call (parameter upload and result download inside
the timed region); `roofline` uses the task kernel's own event-timed duration;
`cpu_baseline` times the FP64 oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1912_13132_gb300 import datagen  # noqa: E402

METRIC = "param-config CV evals/sec @5M obs: mixed vs FP64 at <=1e-6 rel err; p50/p99"
UNIT = "evals/s"
PEAKS_FALLBACK = dict(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0)
FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (SIMT and tensor), nominal


def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:  # pragma: no cover
            pass
    return dict(PEAKS_FALLBACK), "fallback"


def make_workload(name: str):
    if name == "paper5m":
        return datagen.config_paper_5m()
    if name == "paper-small":
        # same subset sizes as paper5m (56-node cores, shell 0.001 scaled), 100 subsets: profiling case
        return datagen.config_paper_5m(side=560, nx=10, delta=0.001 * 2236 / 560)
    if name == "cluster262k":
        return datagen.config_cluster_262k()
    if name == "uniform4096":
        return datagen.config_uniform_4096()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:  # pragma: no cover
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:  # pragma: no cover
            self.proc.kill()
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
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


def kernel_code_hash(sources) -> str:
    """sha256 of the kernel sources with // comments and blank lines removed (comment
    edits do not change the compiled kernel, code edits do)."""
    import hashlib
    h = hashlib.sha256()
    for src in sources:
        for line in open(os.path.join(ROOT, src)).read().splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def recorded_traffic(tasks_per_launch: int):
    """DRAM bytes of one task-kernel launch from the committed ncu record
    (profiles/task_kernel_traffic.txt), or None when the kernel sources changed since
    the counters were taken."""
    path = os.path.join(ROOT, "profiles", "task_kernel_traffic.txt")
    try:
        rec = json.load(open(path))
        if kernel_code_hash(rec["sources"]) != rec["source_sha256"]:
            return None, "kernel changed since the ncu capture"
        return rec["dram_bytes_per_task"] * tasks_per_launch, rec["note"]
    except Exception as e:  # pragma: no cover
        return None, f"no traffic record ({type(e).__name__})"


def task_sizes(ctx):
    k = np.diff(ctx.T_off)
    m = np.diff(ctx.V_off)
    act = m > 0
    return k[act].astype(np.float64), m[act].astype(np.float64)


def algorithmic_flops(k, m, B):
    """Per launch: B x sum over active subsets of k^3/3 (Cholesky) + 2k^2 (two
    triangular solves) + 2mk (prediction)."""
    return float(B * np.sum(k ** 3 / 3.0 + 2.0 * k ** 2 + 2.0 * m * k))


def cpu_baseline(w, params, budget_s: float, active, seed: int = 0):
    """FP64 oracle on a bounded random sample of the subsets with validation data,
    one configuration, a thread per host core.  Returns the wall time and the count
    done; a full configuration takes about elapsed * len(active) / n_done."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    cores = os.cpu_count() or 1
    allc = oracle.layout_cores(w.layout)
    order = np.random.default_rng(seed).permutation(np.asarray(active))
    s2, rho, tau = params

    def one(i):
        T, V = oracle.subset_members(w.xy, w.role, w.layout, int(i), allc)
        oracle.subset_cv(w.xy, w.v, T, V, s2, rho, tau)
        return 1

    t0 = time.perf_counter()
    n_done, pos = 0, 0
    with ThreadPoolExecutor(cores) as ex:
        while pos < len(order) and time.perf_counter() - t0 < budget_s:
            chunk = order[pos:pos + cores]
            pos += len(chunk)
            n_done += sum(ex.map(one, chunk))
    elapsed = time.perf_counter() - t0
    t_full = elapsed * len(order) / max(n_done, 1)
    return dict(elapsed=elapsed, n_done=n_done, n_total=len(order), cores=cores, value=1.0 / t_full,
                t_full=t_full)


def run_reference(args, rank: int, world: int):
    """The oracle as it stands on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    import oracle

    w = make_workload(args.workload)
    core = oracle.core_of(w.layout, w.xy[w.role == datagen.VALID])
    active = np.unique(core)
    vals = []
    for s in range(args.warmup + args.steps):
        cb = cpu_baseline(w, w.params[s % len(w.params)], args.ref_budget, active, seed=s)
        if s >= args.warmup:
            vals.append(cb)
    v = float(np.mean([c["value"] for c in vals]))
    cb = vals[-1]
    sample = (f"{cb['n_done']} of {cb['n_total']} subsets with validation data, one configuration per step "
              f"(~{args.ref_budget:.0f} s on {cb['cores']} threads), extrapolated by subset count")
    line = dict(metric=METRIC, value=v, unit=UNIT, impl="reference", n_gpus=world, steps=args.steps,
                warmup=args.warmup, higher_is_better=True, dtype="f64", data="synthetic",
                config=dict(workload=w.name, batch=1),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cb["cores"], kind="oracle", sample=sample),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                vs_baseline=None)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper5m")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--max-slots", type=int, default=0, help="limit concurrent tasks (profiling runs)")
    ap.add_argument("--engine", default="tensor", choices=["tensor", "simt"])
    ap.add_argument("--tc-stages", type=int, default=0, help="TMA ring depth of the tensor engine (2 or 3)")
    ap.add_argument("--refine-tol", type=float, default=0.0, help="refinement tolerance (0: library default)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_1912_13132_gb300 import pcv

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    t_setup = time.perf_counter()
    w = make_workload(args.workload)
    t_gen = time.perf_counter() - t_setup
    t0 = time.perf_counter()
    ctx = pcv.Context(w.xy, w.v, w.role, w.layout, device=local, max_slots=args.max_slots,
                      factor_engine=args.engine, tc_stages=args.tc_stages, refine_tol=args.refine_tol)
    t_create = time.perf_counter() - t0
    k, m = task_sizes(ctx)
    B = args.batch
    P = w.params
    nsteps = args.warmup + args.steps
    stream = torch.cuda.current_stream()
    d_params = [torch.tensor(np.stack([P[(s * B + j) % len(P)] for j in range(B)]), dtype=torch.float64,
                             device="cuda") for s in range(nsteps)]
    d_sspe = torch.empty(B, dtype=torch.float64, device="cuda")
    d_status = torch.empty(B, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > L2 (129 MB)
    ctx.set_timing(True)

    for s in range(args.warmup):
        ctx.cv_loss_device(d_params[s], d_sspe, precision=args.precision, d_status=d_status, stream=stream)
    torch.cuda.synchronize()
    st = d_status.cpu().numpy()
    if np.any(st != 0):
        print(f"warning: status {st.tolist()}", file=sys.stderr)

    clocks = ClockSampler(local)
    clocks.start()
    step_ms, task_ms = [], []
    pcv.pcv_launch_count(reset=True)
    barrier()
    torch.cuda.synchronize()
    for s in range(args.warmup, nsteps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.cv_loss_device(d_params[s], d_sspe, precision=args.precision, d_status=d_status, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        task_ms.append(ctx.kernel_time()[0])
    launches = pcv.pcv_launch_count()
    barrier()
    clk = clocks.stop()
    phases = ctx.phase_cycles() if args.precision == "mixed" else None
    total_s = sum(step_ms) / 1e3
    if dist is not None:
        t = torch.tensor([total_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * B * args.steps / total_s

    # end to end through the host-pointer call (params up, results down, per step)
    e2e_s = []
    host_P = [np.ascontiguousarray(d_params[s % nsteps].cpu().numpy()) for s in range(args.e2e_steps)]
    for s in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        out = ctx.cv_loss(host_P[s], precision=args.precision, stream=stream)
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = sum(e2e_s) if e2e_s else 1.0
    if dist is not None:
        t = torch.tensor([e2e_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_total = float(t.item())
    e2e_value = world * B * args.e2e_steps / e2e_total if args.e2e_steps > 0 else None

    peaks, peak_src = load_peaks()
    flops = algorithmic_flops(k, m, B)
    t_task = statistics.mean(task_ms) / 1e3
    achieved = flops / t_task / 1e12
    if args.precision == "fp64":
        bound, peak, peak_note = "alu", FP64_NOMINAL_TFLOPS, "FP64 nominal (no measured FP64 peak)"
    else:
        if args.engine == "tensor":
            # six BF16 products per FP32-accurate product: the useful-flop ceiling of the
            # split scheme is the measured sustained BF16 rate / 6
            bound = "tensor"
            peak = peaks["bf16_tflops_sustained"] / 6.0
            peak_note = f"bf16 sustained ({peak_src}) / 6 split products"
        else:
            bound = "alu"
            sm_max = (clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
            peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
            peak_note = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"
    traffic, traffic_note = (recorded_traffic(len(k) * B) if (args.precision == "mixed" and args.engine == "tensor")
                             else (None, "no ncu record for this kernel"))
    roof = dict(bound=bound, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak if peak else None,
                traffic=traffic, traffic_note=traffic_note, peak_source=peak_note,
                kernel="task kernel (persistent)", flops_per_launch=flops, launch_ms=t_task * 1e3)

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_s * 1e3 / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None,
                dtype="f64" if args.precision == "fp64" else
                ("bf16x6+f32+df32x2" if args.engine == "tensor" else "f32+df32x2"),
                data="synthetic",
                config=dict(workload=w.name, n_obs=int(len(w.v)), subsets=int(ctx.N), active_subsets=int(len(k)),
                            k_min=int(k.min()), k_max=int(k.max()), m_mean=float(m.mean()), batch=B,
                            precision=args.precision, engine=args.engine,
                            parallelism="replicas" if world > 1 else "single-gpu",
                            l2="flushed between steps (512 MB write)"),
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=24 * B, d2h_bytes_per_step=12 * B,
                         note="pcv_cv_loss host-pointer call; dataset resident since pcv_create"),
                gpu_launches=int(launches), roofline=roof, clocks=clk,
                setup=dict(datagen_s=t_gen, create_s=t_create))
    if phases and phases.get("task"):
        tot = phases["task"]
        line["phase_share"] = {k2: round(v / tot, 4) for k2, v in phases.items()
                               if v and k2 not in ("task", "residual_passes", "tasks")}
        line["residual_passes_per_task"] = phases["residual_passes"] / max(phases["tasks"], 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        active = np.nonzero(np.diff(ctx.V_off) > 0)[0]
        cb = cpu_baseline(w, P[0], args.cpu_budget, active)
        line["cpu_baseline"] = dict(value=cb["value"], unit=UNIT, cores=cb["cores"], kind="oracle",
                                    sample=f"{cb['n_done']} of {cb['n_total']} subsets with validation data, one "
                                           f"configuration ({cb['elapsed']:.1f} s), extrapolated by subset count "
                                           f"to {cb['t_full']:.0f} s per configuration")
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
