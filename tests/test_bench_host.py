"""Host logic of bench.py that turns kernel timings into the reported
rooflines, and the autotune selection (no GPU: synthetic inputs)."""
import pytest

import bench


def prof_entry(launches, ms_each, bytes_each=0.0, flops_each=0.0, issued=None):
    return {"launches": launches, "ms": ms_each * launches, "bytes": bytes_each * launches,
            "flops": flops_each * launches, "issued": launches if issued is None else issued}


def test_roofline_fractions_and_bounds():
    peak = 8000.0  # GB/s
    prof = {
        # 1 GB in 0.5 ms = 2000 GB/s; 1 GFLOP in 0.5 ms = 2 TFLOP/s: HBM-bound
        "wilson.k1.f32": prof_entry(10, 0.5, 1e9, 1e9, issued=100),
        # 0.5 GB in 0.25 ms = 2000 GB/s, 20 GFLOP in 0.25 ms = 80 TFLOP/s: ALU-bound
        "sw.k1.f32": prof_entry(4, 0.25, 0.5e9, 20e9, issued=40),
        # FP64 class: flops only
        "wilson.ru.f64": prof_entry(2, 4.0, 0.0, 2.5e9, issued=2),
    }
    kernels, roof, roof_hbm = bench.classify_kernels(prof, peak, "measured")
    k1 = kernels["wilson.k1.f32"]
    assert k1["GB/s"] == pytest.approx(2000.0) and k1["frac_hbm"] == pytest.approx(0.25)
    assert k1["bound"] == "hbm" and k1["issued"] == 100 and k1["ms_total_est"] == pytest.approx(50.0)
    s1 = kernels["sw.k1.f32"]
    assert s1["TFLOP/s"] == pytest.approx(80.0)
    assert s1["frac_fp32"] == pytest.approx(80.0 / bench.FP32_PEAK_TFLOPS, rel=1e-3)
    assert s1["bound"] == "alu-fp32"
    ru = kernels["wilson.ru.f64"]
    assert ru["bound"] == "alu-fp64"
    assert ru["frac_fp64"] == pytest.approx(2.5e9 / 4e-3 / 1e12 / bench.FP64_PEAK_TFLOPS, rel=1e-3)
    # the dominant class is the one with the most time: mean timed launch x issued launches
    # (wilson.k1: 0.5 ms x 100 = 50 ms; sw.k1: 10 ms; wilson.ru: 8 ms)
    assert roof["kernel"] == "wilson.k1.f32" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(2000.0) and roof["frac"] == pytest.approx(0.25)
    assert roof["bytes_per_launch"] == pytest.approx(1e9) and roof["peak"] == pytest.approx(peak)
    assert roof_hbm["kernel"] == "wilson.k1.f32"


def test_dominant_class_by_issued_launches_not_timed_ones():
    prof = {
        "a.k1.f32": prof_entry(50, 0.1, 1e8, issued=50),     # 5 ms issued
        "b.k1.f32": prof_entry(2, 0.2, 1e8, issued=1000),    # 200 ms issued, only 2 timed
    }
    _, roof, _ = bench.classify_kernels(prof, 8000.0, "measured")
    assert roof["kernel"] == "b.k1.f32"


def test_traffic_scaled_from_ncu_capture(monkeypatch):
    monkeypatch.setitem(bench.NCU_TRAFFIC, "x.k2.f32", {"bytes": 90e6, "algorithmic": 100e6, "systems": 12})
    prof = {"x.k2.f32": prof_entry(3, 1.0, 400e6, issued=3)}
    _, roof, _ = bench.classify_kernels(prof, 8000.0, "measured")
    # 0.9 of the algorithmic bytes in the capture -> 0.9 x 400 MB per bench launch
    assert roof["traffic"] == 360_000_000
    prof = {"y.k2.f32": prof_entry(3, 1.0, 400e6, issued=3)}
    _, roof, _ = bench.classify_kernels(prof, 8000.0, "measured")
    assert roof["traffic"] is None  # no capture of this kernel: null, never a guess


def test_iteration_fraction_sums_the_three_kernels():
    prof = {
        "wilson.k1.f32": prof_entry(4, 0.4, 1.2e9),
        "wilson.k2.f32": prof_entry(4, 0.5, 1.8e9),
        "wilson.k3.f32": prof_entry(4, 0.3, 2.0e9),
    }
    kernels, _, _ = bench.classify_kernels(prof, 8000.0, "measured")
    it = kernels["wilson.iteration"]
    assert it["ms"] == pytest.approx(1.2)
    assert it["GB/s"] == pytest.approx(5.0e9 / 1.2e-3 / 1e9, rel=1e-3)
    assert "sw.iteration" not in kernels


class FakeLib:
    """Stand-in for the binding: preset autotuner times, records the settings."""
    SW_PREC_F64, SW_PREC_F32_RELIABLE = 0, 1
    SW_OP_STAGGERED_WILSON, SW_OP_WILSON = 0, 1
    SW_PARAM_NS_SW, SW_PARAM_NS_WILSON, SW_PARAM_SITE_BLOCKING = 2, 3, 5
    SW_SITE_SHAPES = 3

    def __init__(self, times):
        self.times, self.params, self.calls = times, {}, []

    def sw_hypercube_build(self, *a, **k):
        self.calls.append("hypercube")

    def sw_autotune_layout(self, dims, op, U, W, nsys, prec, r, iters, stream=None):
        self.calls.append(("tune", op, nsys))
        t = self.times["sw" if op == self.SW_OP_STAGGERED_WILSON else "wilson"]
        best = min(t, key=t.get)
        return best, dict(t)

    def sw_set_param(self, key, value):
        self.params[key] = value


def test_autotune_keeps_the_shared_order_with_the_smallest_sum():
    # staggered Wilson prefers order 0, Wilson order 2; the sums of the best
    # widths per order: 0 -> 10 + 30 = 40, 1 -> 12 + 29 = 41, 2 -> 14 + 24 = 38
    sw_t = {(1, 0): 11.0, (2, 0): 10.0, (4, 0): 13.0, (1, 1): 13.0, (2, 1): 12.0, (4, 1): 15.0,
            (1, 2): 14.0, (2, 2): 16.0, (4, 2): 17.0}
    w_t = {(1, 0): 30.0, (2, 0): 35.0, (4, 0): 40.0, (1, 1): 29.0, (2, 1): 33.0, (4, 1): 45.0,
           (1, 2): 26.0, (2, 2): 24.0, (4, 2): 50.0}
    lib = FakeLib({"sw": sw_t, "wilson": w_t})
    res = bench.autotune_layout(lib, (4, 4, 4, 4), None, None, lib.SW_PREC_F32_RELIABLE, 12, 48, None)
    assert res["site_blocking"] == 2
    assert lib.params[lib.SW_PARAM_SITE_BLOCKING] == 2
    assert lib.params[lib.SW_PARAM_NS_SW] == 1       # fastest staggered Wilson width under order 2
    assert lib.params[lib.SW_PARAM_NS_WILSON] == 2   # fastest Wilson width under order 2
    assert ("tune", lib.SW_OP_STAGGERED_WILSON, 12) in lib.calls and ("tune", lib.SW_OP_WILSON, 48) in lib.calls
    assert lib.calls.index("hypercube") < lib.calls.index(("tune", lib.SW_OP_STAGGERED_WILSON, 12))
    assert res["ms"]["wilson"]["ns2_shape2"] == 24.0


def test_autotune_single_operator_and_fp64():
    w_t = {(w, b): 10.0 + w + (3 - b) for w in (1, 2, 4) for b in range(3)}
    lib = FakeLib({"wilson": w_t})
    res = bench.autotune_layout(lib, (4, 4, 4, 4), None, None, lib.SW_PREC_F32_RELIABLE, 0, 48, None)
    assert res["site_blocking"] == 2 and lib.params[lib.SW_PARAM_NS_WILSON] == 1
    assert lib.SW_PARAM_NS_SW not in lib.params and "hypercube" not in lib.calls
    lib = FakeLib({})
    assert "skipped" in bench.autotune_layout(lib, (4, 4, 4, 4), None, None, lib.SW_PREC_F64, 12, 48, None)
    assert lib.params == {}


def test_both_arms_name_the_same_config():
    """The reference arm and ours describe the workload with the same config
    object (the driver compares them); tuning details go elsewhere."""
    a = bench.workload_config(bench.WORKLOAD, bench.DIMS, bench.MASSES)
    b = bench.workload_config(bench.WORKLOAD, bench.DIMS, bench.MASSES)
    assert a == b and set(a) == {"workload", "lattice", "masses", "tol", "l2"}
    assert a["lattice"] == "16x16x16x32" and a["tol"] == 1e-8
