"""Host-side logic of bench.py: the recorded DRAM traffic (it applies only to the code it was
captured on and is scaled from the captured launches to the timed steps by algorithmic
bytes), the roofline arithmetic, the config object both arms report, the cooling schedule,
and the whole default run against a stand-in library (the JSON contract line)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_traffic_needs_matching_sources(monkeypatch):
    bench = _bench()
    key = ("heis8", "tf32", "kb_gemm_tc")
    rec = {"dram_bytes": 3.0e9, "alg_bytes": 2.0e9, "sources_sha256": bench.sources_sha256(),
           "source": "test"}
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, rec)
    assert bench.recorded_traffic(*key) is rec
    assert bench.recorded_traffic("heis8", "tf32", "kb_gemm") is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, dict(rec, sources_sha256="0" * 64))
    assert bench.recorded_traffic(*key) is None


def test_traffic_scales_by_algorithmic_bytes():
    bench = _bench()
    rec = {"dram_bytes": 3.0e9, "alg_bytes": 2.0e9}
    assert bench.traffic_per_launch(rec, 1.0e8) == 1.5e8


def test_recorded_entries_are_well_formed():
    bench = _bench()
    for key, rec in bench.NCU_TRAFFIC.items():
        assert len(key) == 3 and key[1] in ("fp32", "tf32", "fp64")
        assert rec["dram_bytes"] > 0 and rec["alg_bytes"] > 0 and rec["launches"] > 0
        assert rec["chains"] > 0
        assert len(rec["sources_sha256"]) == 64 and rec["source"]


def test_source_hash_ignores_comments_only():
    bench = _bench()
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* no overflow check */ }\n"
    b = "int f(int x) {\n  // a different comment\n  return 2 * x;\n}\n"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text(c)


def test_kernel_roofline_arithmetic():
    # the tensor-core contraction: achieved = algorithmic flops per launch / mean launch time,
    # frac against the TF32 peak (measured sustained BF16 x the nominal TF32/BF16 ratio), with
    # its HBM view beside it; a kernel with bytes only is HBM-bound; the dominant kernel is the
    # one with the most event time
    bench = _bench()

    class B:
        PEPS_FP64 = 0

    ks = {"kb_gemm_tc": (100, 50.0, 100 * 2.0e8, 100 * 4.0e9), "kb_gemm": (40, 10.0, 40 * 1.0e7, 0.0)}
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1700.0}
    roof, kernels = bench.kernel_roofline(ks, peaks, 2, B)
    assert roof["kernel"] == "kb_gemm_tc" and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(4.0e9 / 0.5e-3 / 1e12)
    assert roof["peak"] == pytest.approx(1700.0 * 1.1 / 2.25)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["hbm_view"]["achieved_GB_s"] == pytest.approx(2.0e8 / 0.5e-3 / 1e9)
    assert roof["mean_launch_us"] == 500.0 and roof["launches"] == 100
    assert abs(roof["share_of_kernel_time"] - 50.0 / 60.0) < 1e-15
    assert list(kernels) == ["kb_gemm_tc", "kb_gemm"]
    ks = {"k_gv": (10, 5.0, 10 * 3.0e9, 0.0)}
    roof, _ = bench.kernel_roofline(ks, peaks, 2, B)
    assert roof["bound"] == "hbm" and roof["achieved"] == pytest.approx(3.0e9 / 0.5e-3 / 1e9)
    # the Jacobi truncation: FMA-bound against the derived FP32 (FP64) rate
    ks = {"kb_trunc": (30, 200.0, 30 * 1.0e8, 30 * 4.0e11), "kb_gemm": (10, 1.0, 1.0e7, 0.0)}
    roof, _ = bench.kernel_roofline(ks, peaks, 2, B)
    assert roof["kernel"] == "kb_trunc" and roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["achieved"] == pytest.approx(4.0e11 / (200.0 / 30 / 1e3) / 1e12)
    assert roof["peak"] == pytest.approx(bench.PEAK_FP32_TFLOPS)
    roof, _ = bench.kernel_roofline(ks, peaks, 0, B)
    assert roof["peak"] == pytest.approx(bench.PEAK_FP64_TFLOPS)


def test_both_arms_share_the_config_object():
    bench = _bench()
    from paper_2409_05285_gb300.workloads import WORKLOADS
    wl = WORKLOADS["heis8"]
    c = bench.workload_config(wl, wl.n_samples, 1)
    assert "chains=8192 per GPU" in c["workload"] and c["global_batch"] == 8192
    assert bench.workload_config(wl, wl.n_samples, 4)["global_batch"] == 4 * 8192


def test_cooling_starts_from_the_warm_start_time():
    # the sampling exponent switches from 1 to 2 at beta_obs = 4t = 0.3, counting the
    # imaginary time of a simple-update warm start
    bench = _bench()

    class Ctx:
        def __init__(self):
            self.ps = []

        def step(self, n_sweeps, p, tau, eps, max_cg, cg_tol):
            self.ps.append(p)

    c = Ctx()
    assert bench.cooled_state(c, 5, 0.02, 0.3) == 5 * 0.02
    assert c.ps == [1, 1, 1, 1, 2]
    c = Ctx()
    t = bench.cooled_state(c, 3, 0.02, 0.3, t_start=0.1)
    assert abs(t - 0.16) < 1e-12 and c.ps == [2, 2, 2]


def _stand_in_cuda(monkeypatch, bench, Ctx, argv):
    # stand-in CUDA events, stream, clocks and library build for bench.py's arms on the CPU
    import sys as _sys
    import torch
    from paper_2409_05285_gb300 import binding, build as build_mod

    class Ev:
        n = 0

        def __init__(self, enable_timing=True):
            Ev.n += 1
            self.t = float(Ev.n)

        def record(self, stream=None):
            Ev.n += 1
            self.t = float(Ev.n)

        def elapsed_time(self, other):
            return 100.0 * (other.t - self.t)

        def synchronize(self):
            pass

    class Stream:
        cuda_stream = 0

    class Clocks:
        def __init__(self, index):
            pass

        def start(self):
            pass

        def stop(self):
            return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}

    monkeypatch.setattr(torch.cuda, "set_device", lambda i: None)
    monkeypatch.setattr(torch.cuda, "Stream", Stream)
    monkeypatch.setattr(torch.cuda, "Event", Ev)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(torch.cuda.profiler, "start", lambda: None)
    monkeypatch.setattr(torch.cuda.profiler, "stop", lambda: None)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(build_mod, "build", lambda *a, **k: None)
    monkeypatch.setattr(binding, "Context", Ctx)
    monkeypatch.setattr(bench, "Clocks", Clocks)
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6794.1})
    monkeypatch.setattr(_sys, "argv", argv)


def test_default_run_prints_the_contract_line(monkeypatch, capsys):
    # bench.py's own arm end to end on the CPU with a stand-in library and stand-in CUDA
    # events: the JSON line carries every key of the contract, with the recorded traffic
    import numpy as np
    bench = _bench()

    class Ctx:
        def __init__(self, L1, L2, D, chi, n, **kw):
            self.n, self.N = n, L1 * L2
            self.Np, self.No = 4 * self.N * D ** 4, self.N * D ** 4
            self.k = 0

        def mc_sweep(self, n_sweeps=1, p=2):
            self.k += 10

        def step(self, **kw):
            self.k += 30
            return {"cg_iters": 5, "E_site": -0.1, "beta_obs": 0.1, "cg_resid": 1e-3}

        def autotune(self, reps=1):
            return {"grid_pct": 100, "db_bytes": 12288, "ffma_g": 16, "kc_max": 32,
                    "ms_before": 2.0, "ms_after": 1.0}

        def profile(self, on, gemm_only=False):
            pass

        def set_graphs(self, on):
            pass

        def launches(self):
            return self.k

        def counters(self):
            return 1.0e9, 100.0 * self.n

        def eval_chains(self):
            self.k += 20

        def sr_step(self, tau, eps, max_cg, cg_tol, p):
            return {"cg_iters": 7, "E_site": -0.05, "beta_obs": 0.56, "cg_resid": 1e-3}

        def profile_read(self):
            return {"kb_gemm_tc": (3288, 400.0, 3288 * 2.9584155e8, 3288 * 1.0e9),
                    "kb_gemm": (1221, 40.0, 1221 * 1.0e7, 1221 * 1.0e6)}

        def get_theta(self):
            return np.zeros(self.Np)

        def get_configs(self):
            return np.zeros((self.n, self.N), dtype=np.uint8)

        def set_theta(self, th):
            pass

        def set_configs(self, S):
            pass

        def close(self):
            pass

    _stand_in_cuda(monkeypatch, bench, Ctx, ["bench.py", "--steps", "2", "--no-cpu-baseline",
                                             "--no-fp64-check", "--largest", "1"])
    bench.main()
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in out, key
    assert out["n_gpus"] == 1 and out["steps"] == 2 and out["warmup"] == 3
    assert out["config"]["workload"].startswith("8x8 OBC Heisenberg") and out["unit"] == "samples/s"
    assert out["value"] == pytest.approx(8192 / (out["ms_per_step"] / 1e3))
    roof = out["roofline"]
    assert roof["kernel"] == "kb_gemm_tc" and roof["bound"] == "tensor"
    assert roof["hbm_view"]["peak_GB_s"] == 6794.1
    big = out["largest_workload"]
    assert "10x10" in big["config"]["workload"] and "chains=16384" in big["config"]["workload"]
    assert big["value"] == pytest.approx(16384 / (big["ms_per_step"] / 1e3))
    assert big["roofline"]["bound"] == "tensor"
    rec = bench.recorded_traffic("heis8", "tf32", "kb_gemm_tc")
    if rec is not None:
        assert roof["traffic"] == pytest.approx(rec["dram_bytes"] / rec["alg_bytes"] * roof["bytes_per_launch"], rel=1e-9)
    assert set(out["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert out["gpu_launches"] > 0


def test_direct_run_prints_the_contract_line(monkeypatch, capsys):
    # bench.py --direct end to end on the CPU with a stand-in library: draw, evaluation and
    # p = 0 SR per step, b_d carried between steps by the library's rule, the truncation's
    # roofline on the FMA rate
    import numpy as np
    bench = _bench()
    from paper_2409_05285_gb300 import binding
    calls = []

    class Ctx:
        def __init__(self, L1, L2, D, chi, n, **kw):
            self.n, self.N = n, L1 * L2
            self.No = self.N * D ** 4
            self.k = 0
            assert kw["block_mode"] == binding.PEPS_BLOCKS_BATCHED

        def set_graphs(self, on):
            pass

        def su_warm_start(self, tau, n_steps):
            calls.append(("su", tau, n_steps))

        def direct_step(self, b_d, exponent=0.5, **kw):
            self.k += 50
            return {"diag_frac": 0.9}, b_d * 0.9

        def direct_draw(self, u=None, b_d=1.0, exponent=0.5):
            calls.append(("draw", None if u is None else u.shape, b_d))
            self.k += 40
            return np.zeros(self.n)

        def eval_chains(self):
            self.k += 20

        def sr_step(self, tau, eps, max_cg, cg_tol, p):
            assert p == 0
            return {"cg_iters": 7, "E_site": -0.05, "E_err": 1e-3, "beta_obs": 0.9,
                    "cg_resid": 1e-9, "diag_frac": 0.75}

        def profile(self, on, gemm_only=False):
            pass

        def profile_read(self):
            return {"kb_trunc": (30, 200.0, 30 * 1.0e8, 30 * 4.0e11),
                    "kb_gemm_tc2": (384, 150.0, 384 * 5.0e8, 384 * 2.5e9)}

        def counters(self):
            return 2.0e12, 5.0 * self.n

        def launches(self):
            return self.k

        def close(self):
            pass

    _stand_in_cuda(monkeypatch, bench, Ctx, ["bench.py", "--direct", "--steps", "2",
                                             "--no-cpu-baseline"])
    bench.main()
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in out, key
    assert "6x6" in out["config"]["workload"] and "30000 direct samples" in out["config"]["workload"]
    assert out["value"] == pytest.approx(30000 / (out["ms_per_step"] / 1e3))
    assert out["roofline"]["kernel"] == "kb_trunc" and out["roofline"]["bound"] == "alu"
    assert not any(c[0] == "su" for c in calls)   # direct6 starts from the beta = 0 state
    # warm-up steps lower b_d by the stand-in's 0.9; then the library's rule on diag 0.75
    b = [c[2] for c in calls if c[0] == "draw"]
    assert b[0] == pytest.approx(0.81)
    assert b[1] == pytest.approx(binding.direct_next_bd(0.81, 0.75, 36))
    assert out["b_d"][0] == pytest.approx(b[1])
    assert out["e2e"]["h2d_bytes_per_step"] == 30000 * 36 * 8
    assert any(c[0] == "draw" and c[1] == (30000, 36) for c in calls)


def test_fermion_run_prints_the_contract_line(monkeypatch, capsys):
    # bench.py --fermion end to end on the CPU with a stand-in evaluator: a sweep and an SR
    # step per timed step (p = 1 until beta_obs = 0.3, then 2), theta and the configurations
    # carried between steps, the contraction's roofline on the tensor pipe
    import numpy as np
    bench = _bench()
    from paper_2409_05285_gb300 import binding
    calls = []

    class FA:
        def __init__(self, L1, L2, D, chi, n, precision=None, stream=None):
            self.n, self.N, self.k = n, L1 * L2, 0
            self.prec = precision
            assert (L1, L2, D, chi) == (6, 6, 4, 16) and n in (1024, 608)
            calls.append(("create", n, precision))

        n_moves = 312

        def sweep(self, theta, S, p=2, n_sweeps=1, seed=0, sweep0=0, u=None):
            calls.append(("sweep", p, sweep0, n_sweeps))
            self.k += 100
            return S.copy(), np.ones(self.n, np.int32), np.zeros(self.n), np.ones(self.n, np.int8)

        def sr_step(self, theta, S, t_hop, U, mu, p=2, **kw):
            calls.append(("sr", p, (t_hop, U, mu)))
            self.k += 30
            return theta - 1e-3, {"E_site": -2.5, "E_err": 0.01, "docc": 0.2, "density": 1.0,
                                  "cg_iters": 40, "cg_resid": 1e-8, "cg_maxit": False}

        def local_energy(self, theta, S, t_hop, U, mu):
            m = len(S)
            shift = 0.0 if self.prec == binding.PEPS_FP64 else 1e-4
            return (np.zeros(m) + shift, np.ones(m, np.int8), np.full(m, -70.0 + shift),
                    np.full(m, -70.0))

        def profile(self, on):
            pass

        def profile_read(self):
            return {"kb_gemm_tc": (500, 300.0, 500 * 2.0e7, 500 * 1.0e9), "k_fsum": (10, 5.0, 0.0, 0.0)}

        def launches(self):
            return self.k

        def close(self):
            pass

    monkeypatch.setattr(binding, "FermionAmplitudes", FA)
    monkeypatch.setattr(binding, "famp_init_theta", lambda L1, L2, D, noise, seed: np.zeros(16 * 100))
    _stand_in_cuda(monkeypatch, bench, None, ["bench.py", "--fermion", "--steps", "2",
                                              "--no-cpu-baseline"])
    monkeypatch.setattr(bench, "l2_flusher", lambda stream: (lambda: calls.append(("flush",))))
    bench.main()
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in out, key
    assert "6x6 OBC Fermi-Hubbard t=1.0 U=8.0 mu=4.0" in out["config"]["workload"]
    assert out["value"] == pytest.approx(1024 / (out["ms_per_step"] / 1e3))
    assert out["roofline"]["kernel"] == "kb_gemm_tc" and out["roofline"]["bound"] == "tensor"
    assert out["gpu_launches"] == 2 * 130
    # burn-in (p = 1), three warm-up steps, two timed steps each after an L2 flush
    sweeps = [c for c in calls if c[0] == "sweep"]
    assert sweeps[0][1:] == (1, 0, 2)
    assert [c[2] for c in sweeps[1:6]] == [2, 3, 4, 5, 6]
    ps = [c[1] for c in calls if c[0] == "sr"]
    assert ps[:4] == [1, 1, 1, 1] and ps[4] == 2
    assert all(c[2] == (1.0, 8.0, 4.0) for c in calls if c[0] == "sr")
    assert sum(1 for c in calls if c[0] == "flush") == 2
    assert out["e2e"]["h2d_bytes_per_step"] == 2 * 1600 * 8 + 2 * 1024 * 36
    # the FP64 comparison on 608 of the chains: a second evaluator in FP64
    assert ("create", 608, binding.PEPS_FP64) in calls
    chk = out["fp64_check"]
    assert chk["chains"] == 608 and chk["sign_mismatch"] == 0
    assert chk["max_abs_dlog_amp"] == pytest.approx(1e-4)
    assert chk["dE_site"] == pytest.approx(1e-4 / 72)
