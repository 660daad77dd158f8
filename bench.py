"""Benchmark: parameter-configuration CV evaluations per second on one GB300.

A step is one pass of the whole hot path (gather, assembly, factorisation,
solves, refinement, prediction, local SSPE, combine) over one batch of B
parameter configurations of a device-resident dataset.  Default workload: the
paper-scale stand-in (2236^2 grid, 4,999,696 nodes with 10% missing, 80/10/10
split, 40 x 40 cores, shell 0.001, about 1600 subsets of 2250-2630 training
points), seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--workload paper5m|paper5m-recursive|cluster262k|uniform4096|serving] [--batch B]
                    [--impl ours|reference] [--serve-seconds S] [--hbm-budget-gb G]

Prints one JSON line (rank 0).  `value` is device-timed (CUDA events around each
step on the launching stream, L2 flushed between steps); `e2e` is the same metric
through the host-pointer C-ABI call (parameter upload and result download inside
the timed region); `roofline` uses the task kernel's own event-timed duration;
`cpu_baseline` times the FP64 oracle on a bounded sample of the same workload.
`serving` (rank 0, one GPU) runs the request loop over eight gridded datasets
(65,536 to 1,048,576 training points): Nelder-Mead clients submit CV evaluations
and prediction requests; capacity from a burst of the request mix first, then Poisson arrivals at
50/80/100% of it, with p50/p99 latency per load level.
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
# tensor engines: (operand terms x products, products per FP32-accurate product)
SCHEMES = {"tensor": ("f16x3", 3), "tensor-bf16": ("bf16x6", 6)}


def load_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:  # pragma: no cover
            pass
    return dict(PEAKS_FALLBACK), "fallback"


def load_device_peaks() -> dict:
    """FP64 / FP32 FMA and tcgen05 TF32 / BF16 / FP16 rates measured on this GPU model by
    `bench.py --peaks` (pcv_measure_peak), committed as JSON in
    profiles/device_peaks_gb300.txt; {} when absent."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "device_peaks_gb300.txt")))
        return rec.get("tflops", {})
    except Exception:  # pragma: no cover
        return {}


def measure_peaks(seconds: float) -> dict:
    """Peak probes with the clocks sampled during each."""
    import torch
    from paper_1912_13132_gb300 import pcv

    torch.cuda.set_device(0)
    out = dict(device=torch.cuda.get_device_name(0), sms=torch.cuda.get_device_properties(0).multi_processor_count,
               tflops={}, seconds={}, clocks={},
               how="pcv_measure_peak: FP64/FP32 = 8 independent FMA chains per thread, 8 x 256 threads per SM; "
                   "tensor = dense tcgen05 M=128 N=256 MMAs from fixed shared-memory tiles, one CTA per SM, "
                   "FP32 accumulators in TMEM; 2 flops per multiply-add; ~seconds per probe after calibration")
    for kind in ("fp64", "fp32", "tf32", "bf16", "fp16"):
        clk = ClockSampler(0)
        clk.start()
        r = pcv.pcv_measure_peak(kind, seconds)
        out["clocks"][kind] = clk.stop()
        out["tflops"][kind] = r["tflops"]
        out["seconds"][kind] = r["seconds"]
    return out


def make_workload(name: str):
    if name == "paper5m":
        return datagen.config_paper_5m()
    if name == "paper-small":
        # same subset sizes as paper5m (56-node cores, shell 0.001 scaled), 100 subsets: profiling case
        return datagen.config_paper_5m(side=560, nx=10, delta=0.001 * 2236 / 560)
    if name == "paper5m-recursive":
        # the paper's weak-scaling layout (Sec. 4.3.2): 512 recursive sub-domains, shells capped at 2000
        return datagen.config_paper_5m_recursive()
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


def recorded_traffic(tasks_per_launch: int, engine: str = "tensor"):
    """DRAM bytes of one task-kernel launch from the committed ncu record of the engine
    (profiles/task_kernel_traffic.txt, a JSON object per engine), or None when there is
    none or the kernel sources changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "task_kernel_traffic.txt")
    try:
        rec = json.load(open(path))
        if engine not in rec:
            return None, "no ncu record for this engine"
        rec = rec[engine]
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


def aggregate_rate(local_s: float, units_per_rank: float, world: int, dist=None, device=None):
    """Whole-job throughput of `world` replicas, each of which processed
    `units_per_rank` units in `local_s` seconds: the elapsed times are reduced by MAX
    over the ranks (the job ends with its slowest rank), value = world * units / max.
    Returns (value, max seconds)."""
    t = float(local_s)
    if dist is not None and world > 1:
        import torch
        x = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world * units_per_rank / t, t


def cpu_model() -> str:
    """The host CPU's model name (or its architecture when none is published)."""
    import platform
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "hardware")):
                return ln.split(":", 1)[1].strip()
    except OSError:  # pragma: no cover
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(w, params, budget_s: float, active, seed: int = 0, threads: int | None = None):
    """FP64 oracle on a bounded random sample of the subsets with validation data,
    one configuration, `threads` threads (default: one per host core).  Returns the
    wall time and the count done; a full configuration takes about
    elapsed * len(active) / n_done."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor

    cores = threads or os.cpu_count() or 1
    allc = oracle.layout_cores(w.layout, w.xy)
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


def nelder_mead(x0, step: float):
    """Ask/tell Nelder-Mead (a generator: yields a point, receives its loss) with the
    usual coefficients (reflection 1, expansion 2, contraction 1/2, shrink 1/2)."""
    n = len(x0)
    simplex = [np.asarray(x0, dtype=np.float64)] + [np.asarray(x0, dtype=np.float64) + step * e
                                                    for e in np.eye(n)]
    f = []
    for x in simplex:
        f.append((yield x))
    while True:
        order = np.argsort(f)
        simplex = [simplex[i] for i in order]
        f = [f[i] for i in order]
        c = np.mean(simplex[:-1], axis=0)
        xr = c + (c - simplex[-1])
        fr = yield xr
        if f[0] <= fr < f[-2]:
            simplex[-1], f[-1] = xr, fr
            continue
        if fr < f[0]:
            xe = c + 2.0 * (c - simplex[-1])
            fe = yield xe
            simplex[-1], f[-1] = (xe, fe) if fe < fr else (xr, fr)
            continue
        xc = c + 0.5 * (xr - c) if fr < f[-1] else c + 0.5 * (simplex[-1] - c)
        fc = yield xc
        if fc < min(fr, f[-1]):
            simplex[-1], f[-1] = xc, fc
            continue
        for i in range(1, n + 1):
            simplex[i] = simplex[0] + 0.5 * (simplex[i] - simplex[0])
            f[i] = yield simplex[i]


# projection of Nelder-Mead proposals, log(sigma2, rho, tau2)
LOG_LO = np.log([0.05, 0.005, 1e-3])
LOG_HI = np.log([20.0, 0.5, 1.0])


class ServingClient:
    """Serving workload over several datasets.  Each request goes to a dataset drawn
    uniformly at random; 80% are CV evaluations, 20% predictions of 10^3-10^5 uniform
    new locations at the dataset's best parameters so far.  A CV request evaluates the
    next point of an idle Nelder-Mead run (over log(sigma2, rho, tau2)) on that
    dataset; if all of the dataset's runs are waiting for a result it evaluates a probe
    near the best point found (log-normal perturbation, sd 0.1).  Requests go through
    pcv_server_*; each finished request reports its submit-to-completion latency."""

    def __init__(self, pcv, srv, workloads, n_runs: int, seed: int):
        from concurrent.futures import ThreadPoolExecutor
        self.srv = srv
        self.rng = np.random.default_rng(seed)
        self.ws = workloads
        self.lock = threading.Lock()
        self.cond = threading.Condition(self.lock)
        self.pool = ThreadPoolExecutor(64)
        self.runs = []
        for r in range(n_runs):
            d = r % len(workloads)
            s2, rho, tau2 = workloads[d].params[0]
            x0 = np.log([1.0, rho, tau2]) + self.rng.uniform(-1.0, 1.0, 3) * np.array([0.5, 1.0, 1.0])
            g = nelder_mead(np.clip(x0, LOG_LO, LOG_HI), 0.3)
            self.runs.append(dict(gen=g, dataset=d, x=next(g), busy=False))
        self.best = [(np.inf, np.log(w.params[0])) for w in workloads]
        self.records = []          # (phase, kind, latency_ms, status)
        self.outstanding = 0
        self.counts = dict(nm=0, probe=0, predict=0)
        self.phase = None

    @staticmethod
    def _params(x):
        return np.exp(np.clip(x, LOG_LO, LOG_HI))

    def _submit_one(self):
        """One request of the mix (called with the lock held)."""
        d = int(self.rng.integers(len(self.ws)))
        if self.rng.random() < 0.8:
            idle = [r for r, run in enumerate(self.runs) if run["dataset"] == d and not run["busy"]]
            if idle:
                r = idle[0]
                self.runs[r]["busy"] = True
                x = self.runs[r]["x"]
                self.counts["nm"] += 1
            else:
                r = -1
                x = self.best[d][1] + self.rng.normal(0.0, 0.1, 3)
                self.counts["probe"] += 1
            rid = self.srv.submit_cv(d, self._params(x))
            self.outstanding += 1
            self.pool.submit(self._wait_cv, r, d, x, rid, self.phase)
        else:
            m = int(round(np.exp(self.rng.uniform(np.log(1e3), np.log(1e5)))))
            rid = self.srv.submit_predict(d, self._params(self.best[d][1]), self.rng.random((m, 2)))
            self.outstanding += 1
            self.counts["predict"] += 1
            self.pool.submit(self._wait_pred, rid, self.phase)

    def _wait_cv(self, r, d, x, rid, phase):
        res = self.srv.wait(rid, timeout_s=600.0)
        with self.lock:
            loss = res["sspe"] if (res["status"] in (0, 7) and np.isfinite(res["sspe"])) else np.inf
            if loss < self.best[d][0]:
                self.best[d] = (loss, np.array(x, dtype=np.float64))
            if r >= 0:
                run = self.runs[r]
                run["x"] = run["gen"].send(loss)
                run["busy"] = False
            self.records.append((phase, "cv", res["latency_ms"], res["status"]))
            self.outstanding -= 1
            self.cond.notify_all()

    def _wait_pred(self, rid, phase):
        res = self.srv.wait(rid, timeout_s=600.0)
        with self.lock:
            self.records.append((phase, "predict", res["latency_ms"], res["status"]))
            self.outstanding -= 1
            self.cond.notify_all()

    def drain(self):
        with self.lock:
            self.cond.wait_for(lambda: self.outstanding == 0, timeout=900.0)

    def burst(self, n: int) -> float:
        """n requests of the mix submitted at once; returns requests/s to complete them
        (the capacity the open-loop loads are scaled to)."""
        t0 = time.perf_counter()
        with self.lock:
            self.phase = "burst"
            for _ in range(n):
                self._submit_one()
        self.drain()
        return n / (time.perf_counter() - t0)

    def open(self, rate: float, seconds: float, label: str) -> dict:
        """Poisson arrivals of the mix at `rate` requests/s for `seconds`, then drain."""
        with self.lock:
            self.phase = label
            before = dict(self.counts)
        t0 = time.perf_counter()
        t_next = t0 + self.rng.exponential(1.0 / rate)
        while t_next < t0 + seconds:
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            with self.lock:
                self._submit_one()
            t_next += self.rng.exponential(1.0 / rate)
        self.drain()
        elapsed = time.perf_counter() - t0
        n = {k: self.counts[k] - before[k] for k in self.counts}
        rec = [r for r in self.records if r[0] == label]
        lat = [r[2] for r in rec]
        lat_cv = [r[2] for r in rec if r[1] == "cv"]
        lat_pr = [r[2] for r in rec if r[1] == "predict"]

        def pct(v, q):
            return float(np.percentile(v, q)) if v else None
        return dict(rate_req_s=rate, seconds=seconds, cv_nelder_mead=n["nm"], cv_probe=n["probe"],
                    predict=n["predict"], failed=sum(1 for r in rec if r[3] not in (0, 7)),
                    cv_evals_per_s=(n["nm"] + n["probe"]) / elapsed, drain_s=elapsed - seconds,
                    p50_ms=pct(lat, 50), p99_ms=pct(lat, 99), cv_p50_ms=pct(lat_cv, 50),
                    cv_p99_ms=pct(lat_cv, 99), predict_p50_ms=pct(lat_pr, 50), predict_p99_ms=pct(lat_pr, 99))


def run_serving(pcv, device: int, seconds: float, hbm_budget_gb: float, max_batch: int, n_runs: int = 32,
                seed: int = 0, max_slots: int = 152, engine: str = "tensor", priorities: int = 0,
                lanes: int = 0) -> dict:
    """Serving measurement on the eight gridded datasets: capacity from a burst of the
    request mix, then Poisson arrivals at 50/80/100% of it."""
    t0 = time.perf_counter()
    ws = datagen.config_serving()
    t_gen = time.perf_counter() - t0
    # at most half of the GPU's task slots per dataset, so that two datasets' launches
    # run side by side
    ctxs = [pcv.Context(w.xy, w.v, w.role, w.layout, device=device, max_slots=max_slots, factor_engine=engine)
            for w in ws]
    # first call per dataset: work memory, tensor maps, one-time set-up
    for c, w in zip(ctxs, ws):
        c.cv_loss(w.params[:1])
    t_setup = time.perf_counter() - t0
    out = dict(workload="serving-8-grids-256..1024sq-32x32cores-8buf",
               datasets=[dict(name=w.name, n_obs=int(len(w.v)), subsets=int(c.N)) for w, c in zip(ws, ctxs)],
               nelder_mead_runs=n_runs, max_batch=max_batch, hbm_budget_gb=hbm_budget_gb or None,
               slots_per_dataset=max_slots, engine=engine, lanes=lanes or 2,
               priorities="by work per configuration" if priorities == 0 else "equal",
               setup_s=round(t_setup, 2), datagen_s=round(t_gen, 2))
    with pcv.Server(ctxs, max_batch=max_batch, precision="mixed",
                    hbm_budget_bytes=hbm_budget_gb * 1e9, lanes=lanes, priorities=priorities) as srv:
        cl = ServingClient(pcv, srv, ws, n_runs, seed)
        cap = cl.burst(20 * len(ws))
        out["capacity_req_s"] = cap
        out["loads"] = []
        for frac in (0.5, 0.8, 1.0):
            out["loads"].append(dict(load=frac, **cl.open(frac * cap, seconds, f"load{frac}")))
        st = srv.stats()
        out["server"] = dict(p50_ms=st["p50_ms"], p99_ms=st["p99_ms"], completed=st["completed"],
                             batches=st["batches"], evictions=st["evictions"])
        cl.pool.shutdown()
    for c in ctxs:
        c.close()
    return out


def run_cluster(pcv, device: int, steps: int = 3) -> dict:
    """The uneven-subset workload (262,144 Poisson-cluster points, 32 x 32 cores, k from
    about 100 to 900, many cores without validation data): all 64 configurations of its
    (rho, tau2) grid in one call, size-bucketed with autotuned engines against one launch
    over slots sized for the largest subset; device-timed, L2 flushed between steps."""
    import torch

    w = datagen.config_cluster_262k()
    d_p = torch.tensor(w.params, dtype=torch.float64, device="cuda")
    B = len(w.params)
    d_sspe = torch.empty(B, dtype=torch.float64, device="cuda")
    d_status = torch.empty(B, dtype=torch.int32, device="cuda")
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = dict(workload=w.name, batch=B)
    for label, bucketing in (("bucketed", 0), ("one_launch", 1)):
        t0 = time.perf_counter()
        ctx = pcv.Context(w.xy, w.v, w.role, w.layout, device=device, bucketing=bucketing)
        ctx.cv_loss_device(d_p, d_sspe, precision="mixed", d_status=d_status, stream=stream)   # tunes, allocates
        torch.cuda.synchronize()
        first_s = time.perf_counter() - t0
        ms = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.cv_loss_device(d_p, d_sspe, precision="mixed", d_status=d_status, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = sorted(set(d_status.cpu().numpy().tolist()))
        k = np.diff(ctx.T_off)[np.diff(ctx.V_off) > 0]
        out[label] = dict(value=B * steps / (sum(ms) / 1e3), unit=UNIT, ms_per_step=sum(ms) / steps, steps=steps,
                          status=st, setup_s=round(first_s, 2), buckets=ctx.buckets().strip().splitlines())
        # (the bucket lines, then the autotuner's per-class timings when this context tuned)
        out.update(active_subsets=int(len(k)), k_min=int(k.min()), k_max=int(k.max()))
        ctx.close()
    out["bucketed_over_one_launch"] = out["bucketed"]["value"] / out["one_launch"]["value"]
    return out


def run_reference(args, rank: int, world: int):
    """The oracle as it stands on the host cores, a bounded sample per step."""
    if rank != 0:
        return
    import oracle

    w = make_workload(args.workload)
    core = oracle.core_of(w.layout, w.xy[w.role == datagen.VALID], w.xy)
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
                config=dict(workload=w.name, n_obs=int(len(w.v)), batch=1, precision="fp64",
                            parallelism="host threads"),
                cpu_baseline=dict(value=v, unit=UNIT, cores=cb["cores"], kind="oracle", cpu=cpu_model(),
                                  sample=sample),
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
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end steps (0: as many as --steps)")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="steps of the FP64 arm on the same batches as the first timed steps (0: none)")
    ap.add_argument("--peaks", action="store_true", help="measure the device peaks (JSON) and exit")
    ap.add_argument("--cluster-steps", type=int, default=3,
                    help="steps of the 64-configuration cluster workload, bucketed and in one launch (0: none)")
    ap.add_argument("--peak-seconds", type=float, default=3.0)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-budget-1core", type=float, default=6.0)
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--max-slots", type=int, default=0, help="limit concurrent tasks (profiling runs)")
    ap.add_argument("--engine", default="tensor", choices=["tensor", "simt", "tensor-bf16"])
    ap.add_argument("--tc-stages", type=int, default=0, help="TMA ring depth of the tensor engine (2 or 3)")
    ap.add_argument("--refine-tol", type=float, default=0.0, help="refinement tolerance (0: library default)")
    ap.add_argument("--refine-loss-tol", type=float, default=0.0, help="loss-aware tolerance (0: default, <0: off)")
    ap.add_argument("--refine-loss-guard", type=float, default=0.0, help="loss-aware guard (0: default, <0: none)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="seconds per serving load level (0: no serving measurement)")
    ap.add_argument("--serve-batch", type=int, default=16, help="CV requests per serving batch")
    ap.add_argument("--hbm-budget-gb", type=float, default=0.0, help="serving work-memory budget (0: unlimited)")
    ap.add_argument("--serve-slots", type=int, default=152, help="task slots per serving lane")
    ap.add_argument("--serve-priorities", type=int, default=0, help="0: by work per configuration, 1: equal")
    ap.add_argument("--serve-lanes", type=int, default=0, help="lanes per serving dataset (0: default 2)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.peaks:
        if rank == 0:
            print(json.dumps(measure_peaks(args.peak_seconds)), flush=True)
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

    if args.workload == "serving":
        if rank == 0:
            sv = run_serving(pcv, local, args.serve_seconds or 10.0, args.hbm_budget_gb, args.serve_batch,
                             max_slots=args.serve_slots, engine=args.engine, priorities=args.serve_priorities,
                             lanes=args.serve_lanes)
            full = sv["loads"][-1]
            print(json.dumps(dict(metric=METRIC, value=full["cv_evals_per_s"], unit=UNIT, n_gpus=1, steps=0,
                                  warmup=0, higher_is_better=True, scaling="weak", vs_baseline=None,
                                  dtype=(SCHEMES[args.engine][0] + "+f32+df32x2" if args.engine in SCHEMES
                                         else "f32+df32x2"),
                                  data="synthetic",
                                  config=dict(workload=sv["workload"], precision="mixed"),
                                  serving=sv)), flush=True)
        return

    t_setup = time.perf_counter()
    w = make_workload(args.workload)
    t_gen = time.perf_counter() - t_setup
    t0 = time.perf_counter()
    ctx = pcv.Context(w.xy, w.v, w.role, w.layout, device=local, max_slots=args.max_slots,
                      factor_engine=args.engine, tc_stages=args.tc_stages, refine_tol=args.refine_tol,
                      refine_loss_tol=args.refine_loss_tol, refine_loss_guard=args.refine_loss_guard)
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
    value, total_s = aggregate_rate(sum(step_ms) / 1e3, B * args.steps, world, dist, "cuda")

    # end to end through the host-pointer call (params up, results down, per step), over
    # the same parameter batches as the timed steps
    e2e_steps = args.e2e_steps or args.steps
    e2e_s = []
    host_P = [np.ascontiguousarray(d_params[args.warmup + s % args.steps].cpu().numpy()) for s in range(e2e_steps)]
    for s in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        out = ctx.cv_loss(host_P[s], precision=args.precision, stream=stream)
        e2e_s.append(time.perf_counter() - t0)
    e2e_value, _ = aggregate_rate(sum(e2e_s), B * e2e_steps, world, dist, "cuda")

    # the FP64 arm of the metric: the same batches as the first timed steps, through the
    # same call, device-timed (one untimed single-configuration call allocates its work
    # memory first)
    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        ctx.cv_loss_device(d_params[0][:1], d_sspe, precision="fp64", d_status=d_status, stream=stream)
        torch.cuda.synchronize()
        f_ms, f_task = [], []
        for s in range(args.warmup, args.warmup + args.fp64_steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.cv_loss_device(d_params[s], d_sspe, precision="fp64", d_status=d_status, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            f_ms.append(e0.elapsed_time(e1))
            f_task.append(ctx.kernel_time()[0])
        f_st = d_status.cpu().numpy()
        f_value, f_total = aggregate_rate(sum(f_ms) / 1e3, B * args.fp64_steps, world, dist, "cuda")
        dev_peaks = load_device_peaks()
        f_peak = dev_peaks.get("fp64")
        f_ach = algorithmic_flops(k, m, B) / (statistics.mean(f_task) / 1e3) / 1e12
        fp64 = dict(value=f_value, unit=UNIT, steps=args.fp64_steps, ms_per_step=f_total * 1e3 / args.fp64_steps,
                    batches="the first timed steps' parameter batches", status=sorted(set(f_st.tolist())),
                    roofline=dict(bound="alu", achieved=f_ach, peak=f_peak, unit="TFLOP/s",
                                  frac=f_ach / f_peak if f_peak else None,
                                  peak_source="FP64 FMA probe (measured, profiles/device_peaks_gb300.txt)"
                                  if f_peak else "no committed FP64 measurement",
                                  kernel="k_cv_fp64 (persistent)", launch_ms=statistics.mean(f_task)))

    peaks, peak_src = load_peaks()
    flops = algorithmic_flops(k, m, B)
    t_task = statistics.mean(task_ms) / 1e3
    achieved = flops / t_task / 1e12
    dev_peaks = load_device_peaks()
    if args.precision == "fp64":
        if dev_peaks.get("fp64"):
            bound, peak, peak_note = "alu", dev_peaks["fp64"], "FP64 FMA probe (measured, profiles/device_peaks_gb300.txt)"
        else:
            bound, peak, peak_note = "alu", FP64_NOMINAL_TFLOPS, "FP64 nominal (no measured FP64 peak)"
    else:
        if args.engine in SCHEMES:
            # n 16-bit products per FP32-accurate product: the useful-flop ceiling of the
            # split scheme is the measured sustained BF16 rate / n (FP16 runs at the BF16
            # rate: nominal ratio 1)
            bound = "tensor"
            nprod = SCHEMES[args.engine][1]
            peak = peaks["bf16_tflops_sustained"] / nprod
            peak_note = f"bf16 sustained ({peak_src}) / {nprod} split products"
        else:
            bound = "alu"
            if dev_peaks.get("fp32"):
                peak, peak_note = dev_peaks["fp32"], "FP32 FMA probe (measured, profiles/device_peaks_gb300.txt)"
            else:
                sm_max = (clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
                peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12
                peak_note = "FP32 FMA: 152 SMs x 128 lanes x 2 flop x max SM clock"
    traffic, traffic_note = (recorded_traffic(len(k) * B, args.engine) if args.precision == "mixed"
                             else (None, "no ncu record for this kernel"))
    roof = dict(bound=bound, achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak if peak else None,
                traffic=traffic, traffic_note=traffic_note, peak_source=peak_note,
                kernel="task kernel (persistent)", flops_per_launch=flops, launch_ms=t_task * 1e3)
    if traffic:
        # the practical bound beside the algorithmic one: the recorded DRAM bytes of a
        # launch over its event-timed duration, against the measured copy bandwidth
        dram_gbs = traffic / t_task / 1e9
        roof.update(dram_gbs=dram_gbs, dram_frac=dram_gbs / peaks["hbm_gbs"],
                    dram_peak_source=f"hbm_gbs ({peak_src})")

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=total_s * 1e3 / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None,
                dtype="f64" if args.precision == "fp64" else
                (SCHEMES[args.engine][0] + "+f32+df32x2" if args.engine in SCHEMES else "f32+df32x2"),
                data="synthetic",
                config=dict(workload=w.name, n_obs=int(len(w.v)), subsets=int(ctx.N), active_subsets=int(len(k)),
                            k_min=int(k.min()), k_max=int(k.max()), m_mean=float(m.mean()), batch=B,
                            precision=args.precision, engine=args.engine,
                            parallelism="replicas" if world > 1 else "single-gpu",
                            l2="flushed between steps (512 MB write)"),
                e2e=dict(value=e2e_value, unit=UNIT, h2d_bytes_per_step=24 * B, d2h_bytes_per_step=12 * B,
                         steps=e2e_steps,
                         note="pcv_cv_loss host-pointer call over the timed steps' parameter batches; "
                              "dataset resident since pcv_create"),
                gpu_launches=int(launches), roofline=roof, clocks=clk,
                setup=dict(datagen_s=t_gen, create_s=t_create))
    if fp64 is not None:
        fp64["mixed_over_fp64"] = value / fp64["value"]
        line["fp64"] = fp64
    if phases and phases.get("task"):
        tot = phases["task"]
        counts = ("task", "residual_passes", "tasks", "fail_factor", "fail_nan", "fail_stall")
        line["phase_share"] = {k2: round(v / tot, 4) for k2, v in phases.items() if v and k2 not in counts}
        line["residual_passes_per_task"] = phases["residual_passes"] / max(phases["tasks"], 1)
        line["fp64_fallback_tasks"] = {k2: phases[k2] for k2 in ("fail_factor", "fail_nan", "fail_stall")}
    if rank == 0 and world == 1 and not args.no_cpu:
        active = np.nonzero(np.diff(ctx.V_off) > 0)[0]
        cb = cpu_baseline(w, P[0], args.cpu_budget, active)
        c1 = cpu_baseline(w, P[0], args.cpu_budget_1core, active, seed=1, threads=1)
        line["cpu_baseline"] = dict(value=cb["value"], unit=UNIT, cores=cb["cores"], kind="oracle",
                                    cpu=cpu_model(),
                                    sample=f"{cb['n_done']} of {cb['n_total']} subsets with validation data, one "
                                           f"configuration ({cb['elapsed']:.1f} s), extrapolated by subset count "
                                           f"to {cb['t_full']:.0f} s per configuration",
                                    one_core=dict(value=c1["value"], unit=UNIT,
                                                  sample=f"{c1['n_done']} subsets ({c1['elapsed']:.1f} s), "
                                                         f"extrapolated to {c1['t_full']:.0f} s per configuration"))
    ctx.close()
    if rank == 0 and world == 1 and args.cluster_steps > 0 and args.workload == "paper5m":
        line["cluster"] = run_cluster(pcv, local, args.cluster_steps)
    if rank == 0 and world == 1 and args.serve_seconds > 0:
        line["serving"] = run_serving(pcv, local, args.serve_seconds, args.hbm_budget_gb, args.serve_batch,
                                      max_slots=args.serve_slots, engine=args.engine,
                                      priorities=args.serve_priorities, lanes=args.serve_lanes)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
