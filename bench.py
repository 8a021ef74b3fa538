#!/usr/bin/env python
"""Benchmark of the fused fluctuating lattice Boltzmann step on GB300.

Metric: MLUPS (million lattice-site updates per second, all systems, all
ranks) of the batched FP32 ensemble, with the HBM-roofline fraction of the
fused step kernel.

Default workload ``fss_160``: the finite-size-scaling ensemble of 160 D3Q19
systems, L in {16, 24, 32, 48, 64}^3 x 8 values of a in [-0.004, 0.004] x 4
replicas, b = 0.1, kappa = 0.01, tau = 1, kT = 1e-4, FP32-deviation
populations, FP64 observables every 100 steps, CUDA-graph replay of 100-step
chunks.  One benchmark step = 100 fused LB steps + one observable pass (one
sampling interval of the hot path).  The populations (2 x 2.06 GB) are far
larger than L2, so no flush is needed between iterations.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
N > 1 runs under torch.distributed.run; each rank advances its own ensemble
(weak scaling, no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

LB_STEPS_PER_STEP = 100
METRIC = "MLUPS and % of HBM roofline (batched FP32 vs plain FP64) at stated Binder-cumulant error"
WORKLOADS = {
    "fss_160": dict(ensemble="fss_160", lattice="D3Q19", precision="fp32"),
    "fss_160_d2q9": dict(ensemble="fss_160", lattice="D2Q9", precision="fp32"),
    "single_64": dict(ensemble="single_64", lattice="D3Q19", precision="fp32"),
    "large_256": dict(ensemble="large_256", lattice="D3Q19", precision="fp32"),
    "fss_160_fp64": dict(ensemble="fss_160", lattice="D3Q19", precision="fp64"),
    "large_256_fp64": dict(ensemble="large_256", lattice="D3Q19", precision="fp64"),
    "large_256_d2q9": dict(ensemble="large_256", lattice="D2Q9", precision="fp32"),
    "fss_160_64": dict(ensemble="fss_160_64", lattice="D3Q19", precision="fp32"),
    "fss_60": dict(ensemble="fss_60", lattice="D3Q19", precision="fp32"),
    "fss_160_64_fp64": dict(ensemble="fss_160_64", lattice="D3Q19", precision="fp64"),
    "fss_160_modeq": dict(ensemble="fss_160", lattice="D3Q19", precision="fp32", coupling="modeq"),
    "fss_160_64_modeq": dict(ensemble="fss_160_64", lattice="D3Q19", precision="fp32", coupling="modeq"),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_kernel_traffic.txt")
KERNEL_SOURCES = ["paper_1202_4748_gb300/csrc/step_kernels.cuh", "paper_1202_4748_gb300/csrc/lb_device.cuh",
                  "paper_1202_4748_gb300/csrc/step_kernel_pair.cuh", "paper_1202_4748_gb300/csrc/collide_d3q19.cuh",
                  "paper_1202_4748_gb300/csrc/vec2.cuh", "paper_1202_4748_gb300/csrc/collide_d2q9.cuh",
                  "paper_1202_4748_gb300/csrc/step_kernel_strip_pair.cuh", "paper_1202_4748_gb300/csrc/lattice_tu.cuh",
                  "paper_1202_4748_gb300/csrc/lattice_d2q9.cu", "paper_1202_4748_gb300/csrc/lattice_d3q19.cu"]


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def describe(wl, systems):
    import synth
    sides = sorted({s["nx"] for s in systems})
    a = sorted({round(s["a"], 6) for s in systems})
    return {
        "workload": "%s: %d %s systems, sides %s, %d values of a in [%g, %g], %s populations"
                    % (wl["ensemble"], len(systems), wl["lattice"], sides, len(a), a[0], a[-1], wl["precision"]),
        "lattice": wl["lattice"], "coupling": systems[0]["coupling"], "precision": wl["precision"],
        "systems": len(systems), "sites": synth.sites(systems),
        "b": 0.1, "kappa": 0.01, "tau": 1.0, "kT": 1e-4,
        "lb_steps_per_step": LB_STEPS_PER_STEP, "obs_every": LB_STEPS_PER_STEP, "graph_chunk": LB_STEPS_PER_STEP,
        "l2": "working set larger than L2 (inputs larger than L2, no flush)",
    }


def q_of(lattice):
    return 9 if lattice == "D2Q9" else 19


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, fl in rows for k, v in enumerate(fl) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)
# ---------------------------------------------------------------------------
ORACLE_MAX_SITES = 1 << 18


def bounded_system(s):
    """The system itself, or, above ORACLE_MAX_SITES sites, the same parameters on
    a 64^3 (D3Q19) / 512^2 (D2Q9) lattice: the oracle's per-site rate is what is
    measured, and a 256^3 FP64 oracle state would not fit a bounded sample."""
    if s["nx"] * s["ny"] * s["nz"] <= ORACLE_MAX_SITES:
        return s
    if s["nz"] > 1:
        return dict(s, nx=64, ny=64, nz=64)
    return dict(s, nx=512, ny=512)


def oracle_sample_systems(wl):
    """One system per size class of the workload (the bounded CPU sample)."""
    import synth
    systems = synth.ensemble(wl["ensemble"], wl["lattice"], wl.get("coupling"))
    seen, out = set(), []
    for s in systems:
        if s["nx"] not in seen:
            seen.add(s["nx"])
            out.append(bounded_system(s))
    return out


def oracle_params(s):
    from oracle import lbm
    return lbm.Params(lattice=s["lattice"], coupling=s["coupling"], nx=s["nx"], ny=s["ny"], nz=s["nz"],
                      rho_c=s["rho_c"], a=s["a"], b=s["b"], kappa=s["kappa"], kT=s["kT"],
                      tau=tuple(s["tau"]), seed=s["seed"], system_id=s["system_id"])


def run_oracle_sample(wl, steps, warmup):
    """Time the FP64 oracle on the bounded sample; returns (MLUPS, sites, seconds)."""
    from oracle import lbm
    params_of = oracle_params
    systems = oracle_sample_systems(wl)
    ps = [params_of(s) for s in systems]
    fs = [lbm.initial_state(p) for p in ps]
    for k in range(len(ps)):
        fs[k] = lbm.run(fs[k], 0, warmup, ps[k])
    t0 = time.perf_counter()
    for k in range(len(ps)):
        fs[k] = lbm.run(fs[k], warmup, steps, ps[k])
    dt = time.perf_counter() - t0
    sites = sum(p.n_sites for p in ps)
    return sites * steps / dt / 1e6, sites, dt


def _oracle_worker(job):
    """One single-threaded process: time `steps` oracle LB steps of one system."""
    s, steps, warmup = job
    from oracle import lbm
    p = oracle_params(s)
    f = lbm.initial_state(p)
    f = lbm.run(f, 0, warmup, p)
    t0 = time.perf_counter()
    f = lbm.run(f, warmup, steps, p)
    return p.n_sites, time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_all_cores(wl, steps, warmup, nproc=None):
    """The FP64 oracle on every host core: one single-threaded process per core
    (spawned, never forked from a process that holds a GPU context), each
    stepping its own system of the workload (systems spread over the size
    classes).  Returns (MLUPS, processes, sites, seconds): all processes' site
    updates over the longest process's timed region."""
    import multiprocessing as mp
    import synth
    nproc = nproc or host_cores()
    systems = synth.ensemble(wl["ensemble"], wl["lattice"], wl.get("coupling"))
    picks = [systems[(k * len(systems)) // nproc] if len(systems) >= nproc else dict(systems[k % len(systems)],
             system_id=k) for k in range(nproc)]
    picks = [bounded_system(s) for s in picks]
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_oracle_worker, [(s, steps, warmup) for s in picks])
    sites = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return sites * steps / dt / 1e6, nproc, sites, dt


def cpu_baseline_subprocess(wl_name, steps, warmup):
    """Run the oracle sample in a fresh single-threaded process (not a fork of this one)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", wl_name, "--steps", str(steps),
           "--warmup", str(warmup)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


# ---------------------------------------------------------------------------
def load_peak():
    try:
        with open(PEAKS_FILE) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def load_traffic(workload):
    """DRAM bytes per step-kernel launch from the committed ncu summary ("key: value"
    lines; each "workload:" line starts the record of one workload), if it was
    taken on this kernel source and this workload; else None."""
    try:
        with open(TRAFFIC_FILE) as fh:
            lines = [ln for ln in fh if ":" in ln and not ln.startswith("#")]
    except OSError:
        return None
    common, records, cur = {}, {}, None
    for ln in lines:
        k, v = (x.strip() for x in ln.split(":", 1))
        if k == "workload":
            cur = records.setdefault(v, {})
        elif cur is None:
            common[k] = v
        else:
            cur[k] = v
    if common.get("kernel_source_hash") != kernel_source_hash() or workload not in records:
        return None
    try:
        return float(records[workload]["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fss_160", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the plain FP64 256^3 comparator")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = every rank advances the whole ensemble (its own noise streams); "
                         "strong = the ensemble is partitioned over the ranks (shard.partition)")
    ap.add_argument("--variant", default="default",
                    help="step-kernel variant: 'default', 'auto' (autotuner, timed on this ensemble) or a row index")
    ap.add_argument("--cpu-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()

    if args.cpu_sample:
        mlups, sites, dt = run_oracle_sample(WORKLOADS[args.cpu_sample], args.steps, args.warmup)
        print(json.dumps({"mlups": mlups, "sites": sites, "seconds": dt}))
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]

    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return

    import torch
    import synth
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1202_4748_gb300 as lb

    systems = synth.ensemble(wl["ensemble"], wl["lattice"], wl.get("coupling"))
    all_systems = [dict(s) for s in systems]
    n_sys = len(systems)
    all_sites = synth.sites(systems)
    if args.scaling == "strong":            # this rank's share of the one ensemble
        from paper_1202_4748_gb300 import shard
        systems = [systems[k] for k in shard.partition(systems, world)[rank]]
    else:
        for s in systems:                   # each rank draws its own noise streams
            s["system_id"] += rank * n_sys
    sites = synth.sites(systems)
    job_sites = all_sites if args.scaling == "strong" else all_sites * world
    q = q_of(wl["lattice"])
    es = 4 if wl["precision"] == "fp32" else 8

    stream = torch.cuda.current_stream()
    rows = lb.kernel_variants(wl["lattice"])
    if args.variant == "auto":
        from paper_1202_4748_gb300 import autotune
        best, _ = autotune.tune(systems, wl["precision"], cache=None)
        vindex = rows.index(best)
    elif args.variant == "default":
        vindex = -1                         # the library's choice, read back below
    else:
        vindex = int(args.variant)
    ens = lb.Ensemble(systems, precision=wl["precision"], obs_every=LB_STEPS_PER_STEP,
                      graph_chunk=LB_STEPS_PER_STEP, variant=vindex + 1)
    vindex = ens.kernel_variant()
    ens.init(amplitude=0.01)
    for _ in range(args.warmup):
        ens.step(LB_STEPS_PER_STEP)
    ens.sync()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    gpu_index = local_rank
    if os.environ.get("CUDA_VISIBLE_DEVICES"):
        vis = os.environ["CUDA_VISIBLE_DEVICES"].split(",")
        if local_rank < len(vis) and vis[local_rank].strip().isdigit():
            gpu_index = int(vis[local_rank])
    clocks = ClockSampler(gpu_index)

    # ---- timed region: K benchmark steps ---------------------------------
    launches0 = ens.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        ens.step(LB_STEPS_PER_STEP)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ens.sync()
    launches = ens.kernel_launches() - launches0
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    updates = job_sites * LB_STEPS_PER_STEP * args.steps
    mlups = updates / (ms_max * 1e-3) / 1e6

    # ---- step-kernel duration: 99 plain step launches, no observable pass ----
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    k0.record(stream)
    ens.step(LB_STEPS_PER_STEP - 1)
    k1.record(stream)
    torch.cuda.synchronize()
    kern_ms = k0.elapsed_time(k1) / (LB_STEPS_PER_STEP - 1)
    ens.step(1)
    ens.sync()
    bytes_per_launch = sites * q * 2 * es
    achieved = bytes_per_launch / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = load_peak()
    traffic = load_traffic(args.workload)

    # ---- end to end through the public API from pinned host memory -----------
    import numpy as np
    k_e2e = max(3, args.steps // 2)
    rho_host = torch.empty(sites, dtype=torch.float64, pin_memory=True)
    rho_host.copy_(torch.from_numpy(np.concatenate(
        [synth.random_density((s["nz"], s["ny"], s["nx"]), seed=s["system_id"]).ravel() for s in systems])))
    # each step's input density is copied from pinned host memory into one of
    # two device buffers on a side stream while the previous step runs, then
    # the context initialises from it (lb_init from device memory)
    side = torch.cuda.Stream()
    rho_dev = [torch.empty(sites, dtype=torch.float64, device="cuda") for _ in range(2)]
    landed = [torch.cuda.Event() for _ in range(2)]

    def stage(k):
        with torch.cuda.stream(side):
            rho_dev[k % 2].copy_(rho_host, non_blocking=True)   # H2D of step k's input density field
            landed[k % 2].record(side)

    barrier()
    t0 = time.perf_counter()
    d2h = 0
    stage(0)
    raw = None
    for k in range(k_e2e + 1):
        if k < k_e2e:
            stream.wait_event(landed[k % 2])
            ens.init(rho_device=rho_dev[k % 2])
            if k + 1 < k_e2e:
                stage(k + 1)                     # overlaps with this step's LB steps
            ens.step(LB_STEPS_PER_STEP)
        if raw is not None:                      # the previous step's records, unpacked while this one runs
            for levels, _ in ens.observables_all(raw):
                d2h += 64 * len(levels) + 64
            raw = None
        if k < k_e2e:
            raw = ens.observables_all_raw()      # D2H of the step's result (observables)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s_t = torch.tensor([e2e_s], device="cuda")
    d2h_t = torch.tensor([float(d2h)], device="cuda", dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(e2e_s_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(d2h_t, op=dist.ReduceOp.SUM)        # the job's read-back bytes
    d2h = int(d2h_t.item())
    e2e_mlups = job_sites * LB_STEPS_PER_STEP * k_e2e / float(e2e_s_t.item()) / 1e6

    ens.close()
    # ---- the plain FP64 single-system path on the 256^3 lattice of the same
    # model (the comparator of the metric: batched FP32 vs plain FP64), and the
    # FP32 path on that lattice, timed in this run -----------------------------
    fp64_plain = None
    if wl["precision"] == "fp32" and not args.no_fp64_arm:
        big = synth.ensemble("large_256", wl["lattice"])
        big_sites = synth.sites(big)
        arm = {"workload": "large_256: one %s system %dx%dx%d, a = %g, b = 0.1, kappa = 0.01, kT = 1e-4, tau = 1"
                           % (wl["lattice"], big[0]["nx"], big[0]["ny"], big[0]["nz"], big[0]["a"])}
        for prec, nsteps in (("fp64", 10), ("fp32", 100)):
            e = lb.Ensemble(big, precision=prec)
            e.init(amplitude=0.01)
            e.step(3)
            e.sync()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a0.record(stream)
            e.step(nsteps)
            a1.record(stream)
            torch.cuda.synchronize()
            ms_step = a0.elapsed_time(a1) / nsteps
            e.close()
            arm[prec] = {"value": round(big_sites / (ms_step * 1e-3) / 1e6, 1), "unit": "MLUPS",
                         "ms_per_step": round(ms_step, 4), "steps": nsteps}
        arm["fp32_over_fp64"] = round(arm["fp32"]["value"] / arm["fp64"]["value"], 1)
        fp64_plain = arm

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_baseline_subprocess(args.workload, steps=2, warmup=0)
        if "mlups" in r:
            n_cls = len(oracle_sample_systems(wl))
            cpu = {"value": r["mlups"], "unit": "MLUPS", "cores": 1, "kind": "oracle",
                   "sample": "FP64 numpy oracle, %d systems (one per size class, %d sites; sides above "
                             "2^18 sites run as 64^3 / 512^2 with the same parameters) x 2 LB steps, %.1f s"
                             % (n_cls, r["sites"], r["seconds"])}
        else:
            cpu = {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": r.get("error")}
        try:
            v, nproc, psites, pdt = run_oracle_all_cores(wl, steps=2, warmup=0)
            cpu["all_cores"] = {"value": round(v, 4), "unit": "MLUPS", "cores": nproc,
                                "sample": "one single-threaded oracle process per core, each one system of the "
                                          "workload (64^3 / 512^2 at most; %d sites in all) x 2 LB steps, %.1f s"
                                          % (psites, pdt)}
        except Exception as exc:          # the single-core figure stands on its own
            cpu["all_cores"] = {"value": None, "error": str(exc)[-200:]}

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
            "scaling": args.scaling, "vs_baseline": None,
            "dtype": "f32" if wl["precision"] == "fp32" else "f64", "data": "synthetic",
            "config": dict(describe(wl, all_systems), step_kernel_variant=list(rows[vindex]),
                           parallelism=("ensemble partitioned over %d ranks" % world if args.scaling == "strong"
                                        else "%d replicas of the ensemble" % world),
                           variant_choice=args.variant if args.variant in ("auto", "default") else "row"),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": traffic,
                         "kernel": "step_kernel", "kernel_ms": round(kern_ms, 5),
                         "bytes_per_launch": bytes_per_launch,
                         "peak_kind": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind,
                         "frac_of_8TBs": round(achieved / 8000.0, 4)},
            "e2e": {"value": round(e2e_mlups, 1), "unit": "MLUPS", "h2d_bytes_per_step": job_sites * 8,
                    "d2h_bytes_per_step": d2h // k_e2e},
            "fp64_plain": fp64_plain,
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args, wl, rank, world):
    """Reference arm: the FP64 oracle on the host cores, on a bounded sample."""
    if rank != 0:
        return
    mlups, nproc, sites, dt = run_oracle_all_cores(wl, args.steps, args.warmup)
    env_threads = nproc
    sample = ("FP64 numpy oracle on every host core: %d single-threaded processes, each one system of the %s "
              "workload (%d sites in all); one step = one LB step of every process's system"
              % (nproc, wl["ensemble"], sites))
    out = {
        "metric": METRIC,
        "value": round(mlups, 4), "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "%s (bounded oracle sample)" % wl["ensemble"], "lattice": wl["lattice"]},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": int(env_threads or 1),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
