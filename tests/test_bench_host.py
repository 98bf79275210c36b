"""Host-side logic of bench.py: the recorded DRAM traffic (it applies only to the code it was
captured on and is scaled from the captured launches to the timed steps by algorithmic
bytes), the roofline arithmetic, and the config object both arms report."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_traffic_needs_matching_sources(monkeypatch):
    bench = _bench()
    key = ("heis8", "tf32", 8192, "kb_gemm_tc")
    rec = {"dram_bytes": 3.0e9, "alg_bytes": 2.0e9, "sources_sha256": bench.sources_sha256(),
           "source": "test"}
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, rec)
    assert bench.recorded_traffic(*key) is rec
    assert bench.recorded_traffic("heis8", "tf32", 4096, "kb_gemm_tc") is None
    monkeypatch.setitem(bench.NCU_TRAFFIC, key, dict(rec, sources_sha256="0" * 64))
    assert bench.recorded_traffic(*key) is None


def test_traffic_scales_by_algorithmic_bytes():
    bench = _bench()
    rec = {"dram_bytes": 3.0e9, "alg_bytes": 2.0e9}
    assert bench.traffic_per_launch(rec, 1.0e8) == 1.5e8


def test_recorded_entries_are_well_formed():
    bench = _bench()
    for key, rec in bench.NCU_TRAFFIC.items():
        assert len(key) == 4 and key[1] in ("fp32", "tf32", "fp64")
        assert rec["dram_bytes"] > 0 and rec["alg_bytes"] > 0 and rec["launches"] > 0
        assert len(rec["sources_sha256"]) == 64 and rec["source"]


def test_source_hash_ignores_comments_only():
    bench = _bench()
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* no overflow check */ }\n"
    b = "int f(int x) {\n  // a different comment\n  return 2 * x;\n}\n"
    c = "int f(int x) { return 3 * x; }"
    assert bench.code_text(a) == bench.code_text(b)
    assert bench.code_text(a) != bench.code_text(c)


def test_kernel_roofline_arithmetic():
    # achieved = algorithmic bytes per launch / mean launch time; frac against the measured
    # HBM copy bandwidth; the dominant kernel is the one with the most event time
    bench = _bench()

    class B:
        PEPS_FP64 = 0

    ks = {"kb_gemm_tc": (100, 50.0, 100 * 2.0e8, 0.0), "kb_gemm": (40, 10.0, 40 * 1.0e7, 0.0)}
    roof, kernels = bench.kernel_roofline(ks, {"hbm_gbs": 6000.0}, 2, B)
    assert roof["kernel"] == "kb_gemm_tc" and roof["bound"] == "hbm"
    assert roof["achieved"] == 2.0e8 / 0.5e-3 / 1e9
    assert roof["frac"] == roof["achieved"] / 6000.0
    assert roof["mean_launch_us"] == 500.0 and roof["launches"] == 100
    assert abs(roof["share_of_timed_kernels"] - 50.0 / 60.0) < 1e-15
    assert list(kernels) == ["kb_gemm_tc", "kb_gemm"]


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
