"""Benchmark: Krylov MPS time steps at L = 16, D = 256 (apply_H TFLOP/s).

One step is one Krylov time step (paper Sec. 2.2.3; m = 10, dt = 0.05 a.u.,
D = 256, eps = 1e-8) of a 16-orbital, 15-electron, S_z = 1/2 state: fitted H
applications (environments, local matvecs, gauge moves and truncation),
fitted sums, the exact overlaps and H sandwiches of the Krylov matrices, and
the small FP64 exponential -- every stage of the hot path.  The state starts
as a seeded random block-sparse MPS at full D so every timed step runs at the
benchmark bond dimension; integrals are the seeded synthetic set standing in
for the paper's active spaces.  ``value`` is the algorithmic (block-sparse)
contraction FLOPs of the timed steps divided by their device time.

--impl reference times the CPU oracle instead (the only other place this file
runs oracle code).
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

import numpy as np  # noqa: E402

METRIC = "apply_H TFLOP/s at L=16, D=256 (Krylov step)"
METRIC_MATVEC = "local one-site matvec TFLOP/s at the centre site, L=16, D=256"
L, N_ELEC, TWO_SZ, D = 16, 15, 1, 256
M_KRYLOV, DT, EPS = 10, 0.05, 1e-8
SCHEDULE = (0, 2)   # two-site sweeps, one-site sweeps per fit


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


_ORACLE: dict = {}


def _oracle_workload(size):
    """The block-sparse oracle's copy of the workload: its own MPO of the
    seeded integrals and the seeded random state, normalised (built once)."""
    if _ORACLE.get("size") != size:
        import synth
        from oracle import bsmps as ob
        Ls, Ns, Ss, Ds = size
        big = Ls >= 24
        I = synth.make_integrals(Ls, seed=0, n_chol=64 if big else 16, localised_block=big)
        A, q = synth.random_mps(Ls, Ns, Ss, Ds, seed=0)
        psi = ob.from_dense(A, q)
        nrm = ob.norm(psi)
        psi.sites[0] = {k: v / nrm for k, v in psi.sites[0].items()}
        _ORACLE.clear()
        _ORACLE.update(size=size, ob=ob, mpo=ob.hamiltonian_mpo(I.h, I.eri, I.e0), psi=psi)
    return _ORACLE


def _krylov_step_oracle_flops(size):
    """Oracle FLOPs of one whole Krylov step of the default workload, counted
    when tests/golden/make_bench_golden.py ran the step (None otherwise)."""
    if size != (L, N_ELEC, TWO_SZ, D):
        return None
    try:
        path = os.path.join(ROOT, "tests", "golden", "krylov_L16_N15_D256.json")
        return float(json.load(open(path))["oracle_flops"])
    except Exception:
        return None


def cpu_baseline(seconds=20.0, size=None, with_fit=True):
    """The block-sparse FP64 oracle (oracle.bsmps) as it stands, on the host
    cores, on the benchmark's own workload (same L, N, D, integrals and
    state): a bounded sample of the Krylov step's operations -- one fitted
    H application with one one-site sweep (with_fit), then exact H
    sandwiches <psi|H|psi> until `seconds` have passed.  FLOPs are the
    oracle's algorithmic block-sparse count (the same definition as the
    GPU's: 8 per complex multiply-add of non-zero blocks, 4 per non-zero MPO
    entry times a complex number).  `cores` is the thread count the BLAS may
    use; `avg_busy_threads` is process CPU time / wall time."""
    size = size or (L, N_ELEC, TWO_SZ, D)
    o = _oracle_workload(size)
    ob, mpo, psi = o["ob"], o["mpo"], o["psi"]
    import resource
    fl = ob.Flops()
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    n_fit = n_sw = 0
    if with_fit:
        ob.apply_H(mpo, psi, -1j * DT, ob.Schedule(size[3], EPS, 0, 1), fl)
        n_fit = 1
    while n_sw == 0 or time.perf_counter() - t0 < seconds:
        ob.sandwich(mpo, psi, psi, fl)
        n_sw += 1
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    rate = fl.total / dt
    out = {"value": rate / 1e12, "unit": "TFLOP/s", "cores": int(threads), "kind": "oracle",
           "avg_busy_threads": round(cpu_s / dt, 2),
           "sample": "block-sparse FP64 oracle on the benchmark workload (L=%d N=%d 2Sz=%d "
                     "D=%d): %d fitted apply_H (one one-site sweep) + %d exact <psi|H|psi> "
                     "sandwiches, %.1f GFLOP in %.1f s"
                     % (size[0], size[1], size[2], size[3], n_fit, n_sw, fl.total / 1e9, dt)}
    kf = _krylov_step_oracle_flops(size)
    if kf:
        out["s_per_krylov_step_extrapolated"] = kf / rate
    return out


def dipole(gammas):
    """Synthetic dipole of each 1-RDM in a stack (..., L, L): mu = sum_i x_i
    Re gamma_ii with orbital coordinate x_i = i (there are no dipole
    integrals; charge density per orbital = gamma_ii, Sec. 3.2)."""
    g = np.asarray(gammas)
    occ = np.real(np.diagonal(g, axis1=-2, axis2=-1))
    return occ @ np.arange(g.shape[-1], dtype=np.float64)


def pinned_copies(arrays, torch):
    """Page-locked copies of host arrays, the e2e inputs, as numpy views of
    pinned torch tensors (kept alive in the returned list).  Where
    page-locking is unavailable (no driver) the arrays are returned as they
    are and the flag is False."""
    try:
        ts = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrays]
        return [t.numpy() for t in ts], ts, True
    except RuntimeError:
        return list(arrays), [], False


def fit_schedule(args):
    """Sweeps per fit: (two-site, one-site)."""
    if args.schedule:
        return tuple(int(x) for x in args.schedule.split(","))
    return SCHEDULE if args.mode == "krylov" else (0, 1)


def workload_size(args):
    """(L, N, 2Sz, D) of the krylov / apply workloads."""
    if args.size:
        Ls, Ns, Ds = (int(x) for x in args.size.split(","))
        return Ls, Ns, Ns % 2, Ds
    return L, N_ELEC, TWO_SZ, D


def workload_config(args, sched, size, world):
    """The `config` of the krylov / apply bench line (both arms)."""
    Ls, Ns, Ss, Ds = size
    if args.mode == "krylov":
        w = ("Krylov step, L=%d N=%d 2Sz=%d D=%d m=10 dt=0.05 eps=1e-8, fit schedule %d "
             "two-site + %d one-site sweeps, random seeded D=%d start"
             % (Ls, Ns, Ss, Ds, sched[0], sched[1], Ds))
    elif args.mode == "matvec":
        w = ("local one-site matvec L W x R (the fit's local product) at the centre site "
             "i = %d, L=%d N=%d 2Sz=%d D=%d, environments of <psi|H|psi> built once "
             "(untimed), %d applications per step, random seeded D=%d state"
             % (Ls // 2, Ls, Ns, Ss, Ds, args.reps, Ds))
    else:
        w = ("apply_H fit, L=%d N=%d 2Sz=%d D=%d, schedule %d two-site + %d one-site sweeps, "
             "random seeded D=%d state" % (Ls, Ns, Ss, Ds, sched[0], sched[1], Ds))
    if getattr(args, "start", "random") != "random":
        w = w.replace("random seeded D=%d start" % Ds, "start " + args.start)
        w = w.replace("random seeded D=%d state" % Ds, "state " + args.start)
        w += " (beta-hole determinant evolved K Krylov steps, schedule 1+1)"
    return {"workload": w,
            "l2": ("flushed before every application (a 256 MB write, outside the timed "
                   "intervals)" if args.mode == "matvec" else
                   "inputs larger than L2 (Krylov basis + environments, several GB)"),
            "inner_products": "serial" if args.serial_inner else "concurrent",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """The oracle on the host cores, on the native arm's workload: each step is
    a bounded sample of it (exact H sandwiches <psi|H|psi> of the seeded state
    by the block-sparse oracle, one per step, ~2-3 s each at L = 16, D = 256);
    each warm-up step is one untimed sandwich."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.mode == "batch":
        print(json.dumps({"impl": "reference",
                          "unavailable": "the oracle arm covers the krylov and apply modes"}))
        return
    size = workload_size(args)
    o = _oracle_workload(size)
    ob, mpo, psi = o["ob"], o["mpo"], o["psi"]
    if args.mode == "matvec":
        # the local operator at the centre site: environments once, untimed
        c = size[0] // 2
        Le, Re = ob.local_environments(mpo, psi, c)

        def unit(fl=ob.Flops()):
            ob.local_one(Le, Re, psi.sites[c], mpo.W[c], psi.bonds[c], psi.bonds[c + 1], fl=fl)
    else:
        def unit(fl=ob.Flops()):
            ob.sandwich(mpo, psi, psi, fl)
    for _ in range(args.warmup):
        unit()
    import resource
    fl = ob.Flops()
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        unit(fl)
    dt = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu_s = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    v = fl.total / dt / 1e12
    threads = os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    cb = {"value": v, "unit": "TFLOP/s", "cores": int(threads), "kind": "oracle",
          "avg_busy_threads": round(cpu_s / dt, 2),
          "sample": "block-sparse FP64 oracle on the benchmark workload (L=%d N=%d 2Sz=%d "
                    "D=%d): %s per step, %.1f GFLOP per step"
                    % (size[0], size[1], size[2], size[3],
                       "one application of the local operator at the centre site"
                       if args.mode == "matvec" else "one exact <psi|H|psi> sandwich",
                       fl.total / 1e9 / max(1, args.steps))}
    kf = _krylov_step_oracle_flops(size)
    if kf and args.mode != "matvec":
        cb["s_per_krylov_step_extrapolated"] = kf / (fl.total / dt)
    line = {"impl": "reference", "metric": METRIC_MATVEC if args.mode == "matvec" else METRIC,
            "value": v, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": reference_config(args, size),
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def reference_config(args, size):
    """`config` of the oracle arm: the native arm's workload, with the sample
    each timed step takes."""
    cfg = workload_config(args, fit_schedule(args), size, int(os.environ.get("WORLD_SIZE", "1")))
    if args.mode == "matvec":
        cfg["sample_per_step"] = ("one application of the local operator at the centre site "
                                  "(block-sparse FP64 oracle; environments built once, untimed)")
    else:
        cfg["sample_per_step"] = ("one exact <psi|H|psi> MPO sandwich of the seeded D=%d state "
                                  "(block-sparse FP64 oracle): the operation the Krylov step "
                                  "runs 55 times for its Hamiltonian matrix" % size[3])
    cfg["inner_products"] = "n/a (oracle)"
    return cfg


def replica_totals(ms, work, dist, device):
    """Whole-job timing of independent replicas (one process per GPU, no
    data-path collective): the slowest rank's timed region and the work of
    all ranks.  dist is torch.distributed (or None for one process)."""
    if dist is None:
        return ms, work
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def centre_site_matvec(td, ctx, mpo, A, q, torch, precision, reps=50, warmup=3):
    """The local one-site operator L W x R of the fit at the centre site of the
    seeded state (a micro-benchmark of the local product), after the timed region: its
    environments once, then `reps` applications, each after an L2 flush and
    timed on its own with CUDA events on the context stream."""
    L = len(A)
    state = td.mps_import(ctx, A, q)
    td.compress(ctx, state, max(len(x) for x in q), 0.0)
    op = td.local_hamiltonian(ctx, mpo, state, L // 2)
    y = state.copy()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(warmup):
        op.apply(state, y)
    torch.cuda.synchronize()
    ctx.stats_enable(True)
    ctx.stats_reset()
    ev = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        op.apply(state, y)
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    st = ctx.stats()
    ctx.stats_enable(False)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    flops = st["gemm"]["flops"] + st["gemm_fp64"]["flops"] + st["wstage"]["flops"]
    out = {"site": L // 2, "applications": reps, "us_per_application": 1e3 * ms / reps,
           "gflop_per_application": flops / reps / 1e9, "tflops": flops / (ms / 1e3) / 1e12,
           "env_bytes": op.env_bytes, "l2": "flushed before every application",
           "roofline": roofline(st, precision),
           "class_us_per_application": {k: 1e3 * v["ms"] / reps for k, v in st.items()
                                        if not k.startswith("host") and v["launches"]}}
    op.free()
    y.free()
    state.free()
    return out


def roofline(st, precision, cls=None):
    """Roofline entry of the kernel class with the largest live event time
    (or of class `cls`): achieved = its algorithmic work per launch / its
    average launch time."""
    peaks = _peaks()
    # the kernels run inside seconds-long steps: the sustained bf16 figure;
    # without the measured file, the earlier GB300 measurement (fallback)
    measured = "bf16_tflops_sustained" in peaks and "hbm_gbs" in peaks
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    fp64_peak = bf16 * 1.25 / 2250.0
    tag = "measured" if measured else "fallback"
    dev = {k: v for k, v in st.items() if not k.startswith("host")}
    top = cls if cls is not None else max(dev, key=lambda k: dev[k]["ms"])
    ks = st[top]
    per_launch_s = ks["ms"] / max(1, ks["launches"]) / 1e3
    per_launch = lambda x: x / max(1, ks["launches"])
    src64 = tag + " sustained bf16 x nominal FP64/bf16 (1.25/2250)"
    if top == "gemm":
        tf32 = bf16 * (1100.0 / 2250.0)
        if precision == "tf32x3":
            peak, src = tf32 / 3.0, tag + " sustained bf16 x nominal TF32/bf16 (1.1/2.25), /3 for split TF32"
        elif precision == "bf16":
            peak, src = bf16, tag + " sustained bf16"
        else:
            peak, src = tf32, tag + " sustained bf16 x nominal TF32/bf16 (1.1/2.25)"
        kern, bound, unit = "k_gemm_tc (tcgen05 grouped complex block GEMM)", "tensor", "TFLOP/s"
        achieved = per_launch(ks["flops"]) / per_launch_s / 1e12
    elif top in ("gemm_fp64", "qr", "svd"):
        kern = {"gemm_fp64": "k_gemm (FP64 grouped complex block GEMM)",
                "qr": "k_qr (FP64 Gram-Schmidt QR, one classical pass counted)",
                "svd": "k_svd (FP64 one-sided Jacobi SVD)"}[top]
        peak, src, bound, unit = fp64_peak, src64, "alu", "TFLOP/s"
        achieved = per_launch(ks["flops"]) / per_launch_s / 1e12
    else:
        kern = {"wstage": "k_wstage (sparse MPO-tensor stage)", "other": "k_copy/k_scatter"}[top]
        peak, src, bound, unit = hbm, tag + " HBM copy bandwidth", "hbm", "GB/s"
        achieved = per_launch(ks["bytes"]) / per_launch_s / 1e9
    return {"kernel": kern, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak, "traffic": None, "peak_source": src,
            "share_of_timed_device_time": ks["ms"] / max(1e-9, sum(v["ms"] for v in dev.values()))}


def batch_instances(n=64):
    """The uneven-instance workload: seeds 0..n-1, L uniform in {8,10,12,14}
    and D uniform in {32,64,128} drawn with default_rng(1000 + seed),
    electrons = L, S_z = 0."""
    out = []
    for seed in range(n):
        r = np.random.default_rng(1000 + seed)
        out.append((seed, int(r.choice([8, 10, 12, 14])), int(r.choice([32, 64, 128]))))
    return out


def run_batch(args, td, ctx, torch, local):
    import synth
    sched = (0, 2) if not args.schedule else tuple(int(x) for x in args.schedule.split(","))
    ctx.set_schedule(*sched)
    inst = batch_instances()
    mpos, states, Ds = [], [], []
    for seed, Lb, Db in inst:
        I = synth.make_integrals(Lb, seed=seed)
        mpos.append(td.build_mpo(ctx, I.h, I.eri, n_elec=Lb))
        A, q = synth.random_mps(Lb, Lb, 0, Db, seed=seed)
        s0 = td.mps_import(ctx, A, q)
        nrm = abs(td.overlap(ctx, s0, s0)) ** 0.5
        A[0] = A[0] / nrm
        s0.free()
        states.append(td.mps_import(ctx, A, q))
        Ds.append(Db)
    dtb = 0.01
    for _ in range(args.warmup):
        td.evolve_batch(ctx, mpos, states, dtb, 1, Ds, method="rk4", n_workers=args.workers)
    torch.cuda.synchronize()
    ctx.stats_enable(True)
    ctx.stats_reset()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            td.evolve_batch(ctx, mpos, states, dtb, 1, Ds, method="rk4", n_workers=args.workers)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    st = ctx.stats()
    ctx.stats_enable(False)
    flops = st["gemm"]["flops"] + st["gemm_fp64"]["flops"] + st["wstage"]["flops"]
    n = len(inst)
    line = {"metric": "instance RK4 steps/s, 64 uneven instances", "value": n * args.steps / (ms / 1e3),
            "unit": "instance-steps/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "tf32": "tf32", "tf32x3": "tf32x3", "bf16": "bf16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": "64 instances, seeds 0..63, L in {8,10,12,14}, N = L, D in "
                                   "{32,64,128}, RK4 dt=0.01, schedule %d two-site + %d one-site "
                                   "sweeps, random seeded start at D" % sched,
                       "workers": args.workers,
                       "l2": "inputs larger than L2 (64 states + environments)"},
            "tflops": flops / (ms / 1e3) / 1e12, "host_wall_s_per_step": wall / args.steps,
            "gpu_launches": int(sum(v["launches"] for k, v in st.items() if not k.startswith("host"))),
            "kernel_stats": {k: {"launches": v["launches"], "ms_summed_over_streams": round(v["ms"], 3),
                                 "gflop": round(v["flops"] / 1e9, 3)} for k, v in st.items()},
            "clocks": clk.summary()}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32", "tf32x3", "bf16"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64 run of the same steps (error and FP64 steps/s)")
    ap.add_argument("--no-traj-compare", action="store_true",
                    help="skip the mixed-vs-FP64 error on the physical beta-hole trajectory")
    ap.add_argument("--traj-steps", type=int, default=2,
                    help="Krylov steps of the beta-hole trajectory comparison (each takes "
                         "15-20 s per precision once the bonds reach D)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--mode", default="krylov", choices=["krylov", "apply", "matvec", "batch"],
                    help="krylov: one Krylov time step per step (default); apply: one "
                         "fitted H application (one one-site sweep) per step; matvec: "
                         "--reps applications of the local one-site operator at the "
                         "centre site per step (L2 flushed between applications); batch: "
                         "one RK4 step of each of 64 uneven instances (L in {8..14}, "
                         "D in {32, 64, 128}) on worker streams")
    ap.add_argument("--no-matvec", action="store_true",
                    help="krylov mode: skip the centre-site local matvec timed after the steps")
    ap.add_argument("--reps", type=int, default=50,
                    help="matvec mode: local operator applications per step")
    ap.add_argument("--workers", type=int, default=16, help="batch mode: worker streams")
    ap.add_argument("--compare-precisions", action="store_true",
                    help="apply mode: also run the fitted application in FP64, split TF32 "
                         "and BF16 and report each one's time and its error against FP64 "
                         "(fidelity, norm, 1-RDM of the normalised state)")
    ap.add_argument("--size", default=None,
                    help="apply/krylov modes: L,N,D of another workload (e.g. 32,23,512 for "
                         "the large active space: 64 Cholesky vectors and the localised "
                         "orbital block); the default is the L=16 workload")
    ap.add_argument("--schedule", default=None, help="two-site,one-site sweeps per fit")
    ap.add_argument("--start", default="random",
                    help="random (the seeded random D state, default) or hole:K (the beta-hole "
                         "determinant evolved K Krylov steps with schedule 1+1, the physical "
                         "timing state; needs N = L - 1)")
    ap.add_argument("--serial-inner", action="store_true",
                    help="run the Krylov inner products after each fit on the context "
                         "stream instead of beside it on a helper thread (for profilers "
                         "that serialise kernels across threads)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1902_08489_gb300 as td
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # The library's context runs on the current stream, and its helper stream
    # (the concurrent FP64 Krylov inner products) has the default, lowest,
    # priority.  On a high-priority stream the fits, which are the critical
    # path of a step, take the SMs first and the inner products fill in.
    hp_stream = torch.cuda.Stream(priority=-5)   # clamped to the highest priority
    torch.cuda.set_stream(hp_stream)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    ctx = td.Context(args.precision)
    if args.serial_inner:
        ctx.set_concurrent_inner(False)
    if args.mode == "batch":
        return run_batch(args, td, ctx, torch, local)
    sched = fit_schedule(args)
    ctx.set_schedule(*sched)
    global L, N_ELEC, TWO_SZ, D
    L, N_ELEC, TWO_SZ, D = workload_size(args)
    big = L >= 24
    I = synth.make_integrals(L, seed=0, n_chol=64 if big else 16, localised_block=big)
    mpo = td.build_mpo(ctx, I.h, I.eri, n_elec=N_ELEC)
    # replicas only: each rank evolves its own seeded state, no collective
    if args.start.startswith("hole:"):
        # the physical state: sudden beta hole in orbital L/2 - 1, evolved
        if N_ELEC != L - 1 or TWO_SZ != 1:
            raise SystemExit("--start hole:K needs N = L - 1 and 2Sz = 1")
        ctx.set_schedule(1, 1)
        s0 = td.mps_from_determinant(ctx, synth.hole_occupation(L, L, L // 2 - 1))
        for _ in range(int(args.start.split(":")[1])):
            td.krylov_step(ctx, mpo, s0, DT, M_KRYLOV, True, D, EPS)
        ctx.set_schedule(*sched)
        A, q = s0.export()
        s0.free()
    else:
        A, q = synth.random_mps(L, N_ELEC, TWO_SZ, D, seed=rank)
    nrm = None
    psi = td.mps_import(ctx, A, q)
    nrm = abs(td.overlap(ctx, psi, psi)) ** 0.5
    A[0] = A[0] / nrm
    h2d_bytes = sum(int(np.count_nonzero(t)) for t in A) * 16

    # matvec mode: the operator, its output state, an L2 flush buffer (a write
    # of twice the 129 MB L2 before every application) and the event pair of
    # every application (the flush stays outside the timed intervals)
    mv = {"op": None, "y": None, "flush": None, "events": []}

    def step(state):
        if args.mode == "krylov":
            td.krylov_step(ctx, mpo, state, DT, M_KRYLOV, True, D, EPS)
        elif args.mode == "matvec":
            for _ in range(args.reps):
                mv["flush"].zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                mv["op"].apply(state, mv["y"])
                e1.record()
                mv["events"].append((e0, e1))
        else:
            out = td.apply_H(ctx, mpo, state, -1j * DT, D, EPS)
            out.free()

    state = td.mps_import(ctx, A, q)
    if args.mode == "matvec":
        td.compress(ctx, state, D, 0.0)
        mv["op"] = td.local_hamiltonian(ctx, mpo, state, L // 2)
        mv["y"] = state.copy()
        mv["flush"] = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    if args.mode == "apply":
        # the gauge every state produced by the library is in (a fit or an
        # integrator step returns it right-canonical), so that the timed
        # application is the one an integrator makes; no truncation at D
        td.compress(ctx, state, D, 0.0)
    for _ in range(args.warmup):
        step(state)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.stats_enable(True)
    ctx.stats_reset()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        mv["events"].clear()
        ev0.record(stream)
        for _ in range(args.steps):
            step(state)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    if args.mode == "matvec":   # the applications alone, without the L2 flushes
        ms = sum(a.elapsed_time(b) for a, b in mv["events"])
    st = ctx.stats()
    ctx.stats_enable(False)
    flops = st["gemm"]["flops"] + st["gemm_fp64"]["flops"] + st["wstage"]["flops"]
    ms, flops_all = replica_totals(ms, flops, dist, "cuda")
    value = flops_all / (ms / 1e3) / 1e12
    g_mixed = td.one_rdm(ctx, state)
    e_mixed = td.expectation(ctx, mpo, state, state).real / td.overlap(ctx, state, state).real

    # the same steps in FP64 from the same start: steps/s and observable error
    fp64_cmp = None
    if args.precision != "fp64" and not args.no_fp64_compare and args.mode == "krylov":
        ctx.set_precision("fp64")
        ref = td.mps_import(ctx, A, q)
        for _ in range(args.warmup):
            step(ref)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(ref)
        t1.record(stream)
        torch.cuda.synchronize()
        ms64 = t0.elapsed_time(t1)
        g64 = td.one_rdm(ctx, ref)
        e64 = td.expectation(ctx, mpo, ref, ref).real / td.overlap(ctx, ref, ref).real
        ctx.set_precision(args.precision)
        fp64_cmp = {"steps_per_s_fp64": 1e3 * args.steps / ms64,
                    "speedup_vs_fp64": ms64 / ms,
                    "accuracy": "see vs_fp64_trajectory (the physical beta-hole trajectory)",
                    "random_start_divergence": {
                        "note": "the random start is chaotic: rounding of either precision "
                                "is amplified, so this is no accuracy measure",
                        "after_steps": args.warmup + args.steps,
                        "max_abs_diff_one_rdm": float(np.abs(g_mixed - g64).max()),
                        "abs_diff_energy": float(abs(e_mixed - e64))}}

    # Observable error of mixed precision on a well-conditioned trajectory:
    # the random D = 256 start has a broad energy spread, and the Gram-Schmidt
    # cancellation of its Krylov vectors amplifies any rounding, so the error
    # is taken on the physical problem of the same size instead: the neutral
    # 16-electron aufbau determinant minus the beta electron of orbital 7,
    # Krylov steps of m = 10, dt = 0.05, D = 256, eps = 1e-8 (one two-site +
    # one one-site sweep per fit so the bonds can grow), FP64 vs this
    # precision.  Observables of the normalised state (Sec. 3.2).
    traj = None
    if (args.precision != "fp64" and not args.no_traj_compare and args.mode == "krylov"
            and not args.size):
        occ = synth.hole_occupation(L, L, 7)
        obs = {}
        for p in ("fp64", args.precision):
            ctx.set_precision(p)
            ctx.set_schedule(1, 1)
            s0 = td.mps_from_determinant(ctx, occ)
            t0 = time.perf_counter()
            gs, es, ns = [], [], []
            for _ in range(args.traj_steps):
                td.krylov_step(ctx, mpo, s0, DT, M_KRYLOV, True, D, EPS)
                n2 = td.overlap(ctx, s0, s0).real
                gs.append(td.one_rdm(ctx, s0) / n2)
                es.append(td.expectation(ctx, mpo, s0, s0).real / n2)
                ns.append(n2)
            torch.cuda.synchronize()
            obs[p] = (np.array(gs), np.array(es), np.array(ns), time.perf_counter() - t0,
                      s0.info()["max_bond"])
            s0.free()
        ctx.set_precision(args.precision)
        ctx.set_schedule(*sched)
        g64, e64, n64, t64, b64 = obs["fp64"]
        gm, em, nm, tm, bm = obs[args.precision]
        dg = np.abs(gm - g64).reshape(len(gm), -1).max(axis=1)
        de = np.abs(em - e64)
        dmu = np.abs(dipole(gm) - dipole(g64)).reshape(len(gm), -1).max(axis=1)
        traj = {"workload": "beta-hole determinant, L=16 N=15, %d Krylov steps (m=10, dt=0.05, "
                            "D=256, eps=1e-8), schedule 1+1" % args.traj_steps,
                "observables": "of the normalised state; the Krylov result fit and inner "
                               "products in FP64, the basis fits in this precision",
                "max_abs_err_one_rdm": float(dg.max()),
                "max_abs_err_energy": float(de.max()),
                "max_abs_err_dipole": float(dmu.max()),
                "max_abs_err_norm2": float(np.abs(nm - n64).max()),
                "per_step_err_one_rdm": [float(x) for x in dg],
                "per_step_err_energy": [float(x) for x in de],
                "target_1e-6_met": bool(max(dg.max(), de.max(), dmu.max()) <= 1e-6),
                "s_per_step_fp64": t64 / args.traj_steps, "s_per_step": tm / args.traj_steps,
                "max_bond": int(bm)}

    # the same application in every precision against FP64 (apply mode)
    prec_cmp = None
    if args.compare_precisions and args.mode == "apply":
        res = {}
        for p in ("fp64", "tf32x3", "bf16"):
            ctx.set_precision(p)
            for rep in range(2):          # the first call carries one-time setup
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = td.apply_H(ctx, mpo, state, -1j * DT, D, EPS)
                torch.cuda.synchronize()
                dt_s = time.perf_counter() - t0
                if rep == 0:
                    out.free()
            res[p] = (out, dt_s)
        ctx.set_precision("fp64")
        ref = res["fp64"][0]
        n_ref = td.overlap(ctx, ref, ref).real
        g_ref = td.one_rdm(ctx, ref) / n_ref
        prec_cmp = {"fp64": {"s_per_apply": res["fp64"][1]}}
        for p in ("tf32x3", "bf16"):
            o = res[p][0]
            n_o = td.overlap(ctx, o, o).real
            x = td.overlap(ctx, ref, o)
            prec_cmp[p] = {"s_per_apply": res[p][1],
                           "speedup_vs_fp64": res["fp64"][1] / res[p][1],
                           "one_minus_fidelity": float(1.0 - abs(x) ** 2 / (n_ref * n_o)),
                           "norm2_ratio_minus_1": float(n_o / n_ref - 1.0),
                           "max_abs_err_one_rdm_normalised":
                               float(np.abs(td.one_rdm(ctx, o) / n_o - g_ref).max())}
        for p in res:
            res[p][0].free()
        ctx.set_precision(args.precision)

    # end-to-end through the public API with host buffers: import the state
    # from host memory, one Krylov step, read the 1-RDM back
    e2e = None
    if not args.no_e2e and args.mode != "matvec":
        A_host, _keep, pinned = pinned_copies(A, torch)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(1, args.steps)):
            s2 = td.mps_import(ctx, A_host, q)
            step(s2)
            g = td.one_rdm(ctx, s2)
            s2.free()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te, _ = replica_totals(te, 0.0, dist, "cuda")
        e2e = {"value": flops_all / te / 1e12,
               "unit": "TFLOP/s", "h2d_bytes_per_step": h2d_bytes,
               "d2h_bytes_per_step": int(g.nbytes), "pinned_inputs": pinned}

    # the local-product micro-benchmark beside the Krylov step (its own line in --mode matvec)
    k3 = None
    if args.mode == "krylov" and not args.size and not args.no_matvec:
        try:
            k3 = centre_site_matvec(td, ctx, mpo, A, q, torch, args.precision)
        except Exception as e:   # reported, never at the cost of the main line
            k3 = {"error": str(e)[:200]}
    # dominant kernel class: the largest live event time in the timed region
    roof = roofline(st, args.precision)
    config = dict(workload_config(args, sched, (L, N_ELEC, TWO_SZ, D), world),
                  stream_priority=int(hp_stream.priority))
    matvec = None
    if args.mode == "matvec":
        matvec = {"site": L // 2, "env_bytes": mv["op"].env_bytes,
                  "applications": len(mv["events"]),
                  "us_per_application": 1e3 * ms / max(1, len(mv["events"])),
                  "timed": "sum of per-application event intervals"}
        mv["op"].free()
        mv["y"].free()
    line = {
        "metric": METRIC_MATVEC if args.mode == "matvec" else METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "tf32": "tf32", "tf32x3": "tf32x3", "bf16": "bf16"}[args.precision],
        "data": "synthetic",
        "config": config,
        "steps_per_s": 1e3 * args.steps / ms,
        "matvec": matvec,
        "centre_site_matvec": k3,
        "vs_fp64": fp64_cmp,
        "vs_fp64_trajectory": traj,
        "precision_compare": prec_cmp,
        "gpu_launches": int(sum(v["launches"] for k, v in st.items() if not k.startswith("host"))),
        "kernel_stats": {k: {"launches": v["launches"], "ms": round(v["ms"], 3),
                             "gflop": round(v["flops"] / 1e9, 3), "gb": round(v["bytes"] / 1e9, 3)}
                         for k, v in st.items()},
        "roofline": roof,
        # the tensor-core GEMM class on its own (the contraction kernel of the
        # metric), whichever class dominates the step
        "roofline_tensor_core": (roofline(st, args.precision, "gemm")
                                 if args.precision != "fp64" and st["gemm"]["launches"] else None),
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(20.0, (L, N_ELEC, TWO_SZ, D))
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
