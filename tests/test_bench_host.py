"""Host logic of the benchmark: the roofline entry of the dominant kernel
class and the uneven-instance recipe (no GPU)."""
import bench


def _st(**ms):
    base = {k: {"launches": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}
            for k in ("gemm", "wstage", "qr", "svd", "other", "gemm_fp64",
                      "host_plan", "host_launch", "host_sync")}
    for k, (launches, t, fl, by) in ms.items():
        base[k] = {"launches": launches, "ms": t, "flops": fl, "bytes": by}
    return base


def test_roofline_picks_the_largest_device_class_and_ignores_host_time():
    st = _st(gemm_fp64=(10, 100.0, 50e9, 1e9), gemm=(100, 60.0, 1e12, 1e9),
             host_plan=(1000, 5000.0, 0.0, 0.0))
    r = bench.roofline(st, "tf32x3")
    assert r["kernel"].startswith("k_gemm (FP64")
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 50 GFLOP in 100 ms = 0.5 TFLOP/s over the FP64 peak (bf16 x 1.25/2250)
    assert abs(r["achieved"] - 0.5) < 1e-12
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-15
    assert abs(r["share_of_timed_device_time"] - 100.0 / 160.0) < 1e-12


def test_roofline_tensor_and_memory_classes():
    r = bench.roofline(_st(gemm=(4, 40.0, 4e12, 1e9)), "tf32x3")
    assert r["bound"] == "tensor"
    tf32 = r["peak"] * 3.0
    r1 = bench.roofline(_st(gemm=(4, 40.0, 4e12, 1e9)), "tf32")
    assert abs(r1["peak"] - tf32) < 1e-9
    r2 = bench.roofline(_st(wstage=(2, 10.0, 1e9, 20e9)), "tf32x3")
    assert r2["bound"] == "hbm" and r2["unit"] == "GB/s"
    assert abs(r2["achieved"] - 2000.0) < 1e-9   # 20 GB in 10 ms


def test_batch_instances_recipe():
    inst = bench.batch_instances()
    assert len(inst) == 64 and [s for s, _, _ in inst] == list(range(64))
    assert {L for _, L, _ in inst} <= {8, 10, 12, 14}
    assert {D for _, _, D in inst} <= {32, 64, 128}
    assert inst == bench.batch_instances()   # seeded


def test_both_arms_describe_the_same_workload():
    """The native line and the oracle (reference) line build `config` with
    the same helper from the same arguments."""
    from types import SimpleNamespace
    a = SimpleNamespace(mode="krylov", schedule=None, size=None, serial_inner=False)
    sched = bench.fit_schedule(a)
    assert sched == bench.SCHEDULE
    cfg = bench.workload_config(a, sched, bench.workload_size(a), 1)
    assert "L=16 N=15 2Sz=1 D=256" in cfg["workload"]
    assert "0 two-site + 2 one-site" in cfg["workload"]
    assert cfg["parallelism"] == "single" and cfg["inner_products"] == "concurrent"
    b = SimpleNamespace(mode="apply", schedule="1,1", size="32,23,512", serial_inner=True)
    assert bench.workload_size(b) == (32, 23, 1, 512)
    cfg = bench.workload_config(b, bench.fit_schedule(b), bench.workload_size(b), 2)
    assert cfg["workload"].startswith("apply_H fit, L=32 N=23 2Sz=1 D=512, schedule 1 two-site")
    assert cfg["parallelism"] == "replicas" and cfg["inner_products"] == "serial"


def test_synthetic_dipole():
    """mu = sum_i i * gamma_ii: a determinant's 1-RDM gives the sum of the
    occupied orbital indices weighted by occupation; stacks work per matrix."""
    import numpy as np
    g = np.diag([2.0, 2.0, 1.0, 0.0]).astype(complex)
    assert bench.dipole(g) == 0 * 2 + 1 * 2 + 2 * 1
    g2 = np.stack([g, np.diag([0.0, 1.0, 2.0, 2.0]).astype(complex) + 0.3j])
    assert np.allclose(bench.dipole(g2), [4.0, 1 + 4 + 6])


def test_reference_arm_json_line():
    """`bench.py --impl reference` prints one JSON line with the contract's
    keys, the native arm's metric and config, and an e2e entry without
    host-device traffic (the oracle's MPO build and two sandwiches at the
    benchmark size, about 15 s on the host cores)."""
    import json
    import subprocess
    import sys
    from types import SimpleNamespace
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "TFLOP/s" and line["steps"] == 1
    a = SimpleNamespace(mode="krylov", schedule=None, size=None, serial_inner=False)
    native = bench.workload_config(a, bench.fit_schedule(a), bench.workload_size(a), 1)
    assert line["config"]["workload"] == native["workload"]
    assert "sandwich" in line["config"]["sample_per_step"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "L=16 N=15 2Sz=1 D=256" in cb["sample"]
    assert 0.0 < cb["avg_busy_threads"] <= cb["cores"] + 0.5
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_native_arm_json_assembly_with_a_stand_in_library(monkeypatch, capsys):
    """Runs bench.main() on the CPU with a stand-in for the library and for
    torch.cuda (test double only: every number it prints is meaningless).  It
    checks the control flow and the JSON line of the native arm in the krylov,
    apply, local-matvec and serial-inner-product modes, so that a Python-level mistake there
    shows up without a GPU.  The real library is exercised by the GPU tests."""
    import json
    import sys
    import time
    import types
    import numpy as np
    import torch

    class Ev:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = time.perf_counter()

        def elapsed_time(self, other):
            return 1e3 * (other.t - self.t) + 1e-3

    class Stream:
        def __init__(self, priority=0):
            self.priority = max(priority, -3)

    for name, fn in (("Event", Ev), ("synchronize", lambda *a, **k: None),
                     ("set_device", lambda *a, **k: None), ("Stream", Stream),
                     ("set_stream", lambda *a, **k: None),
                     ("current_stream", lambda *a, **k: object())):
        monkeypatch.setattr(torch.cuda, name, fn)
    classes = ["gemm", "wstage", "qr", "svd", "other", "gemm_fp64", "host_plan", "host_launch",
               "host_sync"]
    seen = []

    class MPS:
        def __init__(self, L=16):
            self.L = L

        def info(self):
            return {"L": self.L, "n_elec": 15, "two_sz": 1, "max_bond": 256}

        def free(self):
            pass

        def copy(self):
            return MPS(self.L)

        def export(self):
            return ([np.ones((1, 4, 1), dtype=complex) for _ in range(self.L)],
                    [np.zeros((1, 2), dtype=np.int64) for _ in range(self.L + 1)])

    class Ctx:
        def __init__(self, prec):
            self.prec = prec

        def set_precision(self, p):
            self.prec = p

        def set_schedule(self, a, b):
            pass

        def set_concurrent_inner(self, on):
            seen.append(on)

        def stats_enable(self, on=True):
            pass

        def stats_reset(self):
            pass

        def stats(self):
            return {k: dict(launches=10, ms=5.0 * (i + 1), flops=1e10 * (i + 1), bytes=1e8)
                    for i, k in enumerate(classes)}

    lib = types.ModuleType("paper_1902_08489_gb300")
    lib.Context = Ctx
    lib.build_mpo = lambda ctx, h, eri, L=None, n_elec=0, e0=0.0: object()
    lib.mps_import = lambda ctx, A, q: MPS(len(A))
    lib.mps_from_determinant = lambda ctx, occ: MPS(len(occ))
    lib.overlap = lambda ctx, a, b: 1.0 + 0j
    lib.expectation = lambda ctx, mpo, a, b: -20.6 + 0j
    lib.one_rdm = lambda ctx, m: np.eye(m.L, dtype=complex) * (15.0 / m.L)
    lib.krylov_step = lambda *a, **k: None
    lib.apply_H = lambda *a, **k: MPS()
    lib.compress = lambda *a, **k: 0.0
    applied = []

    class Op:
        env_bytes = 12345

        def apply(self, x, y):
            applied.append((x, y))

        def free(self):
            pass

    lib.local_hamiltonian = lambda ctx, mpo, m, site: (applied.append(site), Op())[1]
    empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, **k: empty(16, dtype=k.get("dtype")))
    monkeypatch.setitem(sys.modules, "paper_1902_08489_gb300", lib)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    for argv, mode in ((["--steps", "2", "--warmup", "3"], "krylov"),
                       (["--mode", "apply", "--steps", "2", "--warmup", "3"], "apply"),
                       (["--mode", "apply", "--steps", "1", "--warmup", "3",
                         "--compare-precisions"], "apply-cmp"),
                       (["--mode", "apply", "--steps", "1", "--warmup", "3",
                         "--start", "hole:2"], "apply-hole"),
                       (["--mode", "matvec", "--steps", "2", "--warmup", "3", "--reps", "2"],
                        "matvec"),
                       (["--steps", "1", "--warmup", "3", "--serial-inner", "--no-traj-compare",
                         "--no-fp64-compare", "--no-e2e"], "serial")):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--no-cpu-baseline", *argv])
        applied.clear()
        bench.main()
        line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                  "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                  "roofline", "clocks", "e2e", "gpu_launches"):
            assert k in line, (mode, k)
        assert line["metric"] == (bench.METRIC_MATVEC if mode == "matvec" else bench.METRIC)
        assert line["gpu_launches"] > 0
        assert line["config"]["stream_priority"] == -3
        assert line["config"]["inner_products"] == ("serial" if mode == "serial" else "concurrent")
        rt = line["roofline_tensor_core"]
        assert rt["kernel"].startswith("k_gemm_tc") and rt["bound"] == "tensor"
        if mode == "krylov":
            traj = line["vs_fp64_trajectory"]
            assert traj["max_abs_err_dipole"] == 0.0 and line["vs_fp64"] is not None
            assert len(traj["per_step_err_one_rdm"]) == 2 and traj["target_1e-6_met"]
            assert line["e2e"]["h2d_bytes_per_step"] > 0
            assert line["e2e"]["pinned_inputs"] is False      # no driver here
            # the centre-site local matvec after the steps: 3 warm-up + 50 timed
            k3 = line["centre_site_matvec"]
            assert k3["site"] == 8 and k3["applications"] == 50 and "roofline" in k3
            assert applied[0] == 8 and len(applied) == 1 + 3 + 50
        else:
            assert line["vs_fp64_trajectory"] is None
        if mode not in ("krylov", "serial"):      # the serial run is a Krylov run too
            assert line["centre_site_matvec"] is None
        if mode == "matvec":
            # the operator at the centre site, (3 warm-up + 2 timed) x 2 applications,
            # only the timed ones in the line; no e2e in this mode
            assert applied[0] == 8 and len(applied) == 1 + 5 * 2
            assert line["matvec"]["applications"] == 4 and line["matvec"]["site"] == 8
            assert line["matvec"]["env_bytes"] == 12345 and line["e2e"] is None
            assert "flushed" in line["config"]["l2"]
        if mode == "apply-hole":
            assert "hole:2" in line["config"]["workload"]
        if mode == "apply-cmp":
            assert set(line["precision_compare"]) == {"fp64", "tf32x3", "bf16"}
            assert line["precision_compare"]["bf16"]["one_minus_fidelity"] == 0.0
    assert seen == [False]


def test_reference_arm_of_the_local_matvec_mode():
    """The oracle arm of --mode matvec times the oracle's local operator at
    the centre site of the benchmark state (environments once, untimed)."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--mode", "matvec",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["metric"] == bench.METRIC_MATVEC and line["value"] > 0
    assert "centre site" in line["config"]["sample_per_step"]
    assert "local operator at the centre site" in line["cpu_baseline"]["sample"]
    assert "s_per_krylov_step_extrapolated" not in line["cpu_baseline"]
