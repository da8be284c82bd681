"""Host-side accounting of bench.py: the per-unit algorithmic bytes, the layout bytes, the
kernel choice of the roofline and the source-hash guard on recorded DRAM traffic."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_algorithmic_bytes_follow_the_per_unit_figures(bench):
    # owner state 44 B each way (voxel form), 32 B per listed pair; FP64 144 B and 56 B
    a = bench.algorithmic_bytes("voxel_fp32", 1000, 250)
    assert a == {"integrate": 88000, "contact": 8000, "step": 96000}
    f = bench.algorithmic_bytes("fp64", 1000, 250)
    assert f["integrate"] == 144000 and f["contact"] == 14000
    assert bench.algorithmic_bytes("voxel_fp32", 10, 0, clumps=True)["integrate"] == 10 * (88 + 32)


def test_layout_bytes_exceed_the_algorithmic_figure(bench):
    for prec in ("voxel_fp32", "fp64"):
        a = bench.algorithmic_bytes(prec, 4_000_000, 1_590_000)
        lb = bench.layout_bytes(prec, 4_000_000, 2_090_000, 1_590_000)
        for k in ("integrate", "contact", "step"):
            assert lb[k] > a[k]
        # the fused step drops the force array and the second pass over busy owners
        assert lb["step"] < lb["integrate"] + lb["contact"]


def _prof(n_integrate, contact_ms=0.2, integrate_ms=0.15):
    return {"n_integrate": n_integrate, "n_contact": 100, "contact_ms": contact_ms, "integrate_ms": integrate_ms,
            "listed_pairs": 1.0e6, "with_entries": 1.5e6, "n_detect": 0, "detect_ms": 0.0}


def test_detection_bytes_follow_the_per_unit_figures(bench):
    # per sphere 20 + 24 + 48 + 4 B (voxel form; FP64 24 + 24 + 48 + 4), per listed pair
    # 8 B written plus the remap 2 (8 + 12) B (FP64 2 (8 + 24) B)
    assert bench.detection_bytes("voxel_fp32", 1000, 250) == 96 * 1000 + 48 * 250
    assert bench.detection_bytes("fp64", 1000, 250) == 100 * 1000 + 72 * 250


def test_roofline_reports_the_detection_phase_beside_the_kernels(bench):
    prof = dict(_prof(100, 0.15, 0.152), n_detect=10, detect_ms=3.0)
    r = bench.roofline("voxel_fp32", 4_000_000, prof, 6768.8, "measured", rebuilds_per_step=0.1)
    d = r["kernels"]["detect"]
    assert d["bytes"] == 96 * 4_000_000 + 48 * 1.0e6
    assert d["gbs"] == pytest.approx(d["bytes"] / 3.0e-3 / 1e9)
    assert d["ms_per_step"] == pytest.approx(0.3)
    # the detection phase is not a kernel: the dominant kernel stays a per-step kernel
    assert r["kernel"].startswith("k_integrate")


def test_roofline_picks_the_dominant_kernel(bench):
    r = bench.roofline("voxel_fp32", 4_000_000, _prof(100), 6768.8, "measured")
    assert r["kernel"].startswith("k_contact") and set(r["kernels"]) == {"contact", "integrate"}
    assert r["achieved"] == pytest.approx(32e6 / 0.2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6768.8)
    r = bench.roofline("voxel_fp32", 4_000_000, _prof(100, 0.1, 0.15), 6768.8, "measured")
    assert r["kernel"].startswith("k_integrate")
    # no integration launches: the fused step, whole force+integrate figure per launch
    r = bench.roofline("voxel_fp32", 4_000_000, _prof(0), 6768.8, "measured")
    assert r["kernel"].startswith("k_step_fused") and r["bytes_per_launch"] == 88 * 4_000_000 + 32e6


def test_contact_kernel_integration_moves_the_busy_owners_bytes(bench):
    # the owners with listed partners move from the integration kernel's figure to the
    # contact kernel's; the sum is the step's figure
    a = bench.algorithmic_bytes("voxel_fp32", 1000, 250, n_with_entries=300, contact_integrates=True)
    assert a == {"integrate": 88 * 700, "contact": 32 * 250 + 88 * 300, "step": 88 * 1000 + 32 * 250}
    lb0 = bench.layout_bytes("voxel_fp32", 4_000_000, 1_160_000, 710_000)
    lb1 = bench.layout_bytes("voxel_fp32", 4_000_000, 1_160_000, 710_000, contact_integrates=True)
    assert lb1["integrate"] + lb1["contact"] < lb0["integrate"] + lb0["contact"]
    r = bench.roofline("voxel_fp32", 4_000_000, _prof(100, 0.2, 0.1), 6768.8, "measured", contact_integrates=1)
    assert r["contact_integrates"] and r["kernel"].startswith("k_contact")
    assert r["bytes_per_launch"] == 32 * 1.0e6 + 88 * 1.5e6
    assert r["kernels"]["integrate"]["bytes"] == 88 * 2.5e6 and r["traffic"] is None


def test_recorded_traffic_is_dropped_when_the_kernel_source_changes(bench, monkeypatch):
    def current(rec):
        return all(bench.kernel_source_hash(sig, fn) == hv for fn, sig, hv in rec["source"])

    # the single contact kernel and the two-pass step each have their own record
    t, two = bench.MEASURED_TRAFFIC["contact"]
    assert t["tuning"]["contact_screen"] == 0 and two["tuning"] == {"contact_screen": 1}
    for r in (t, two):
        m = r["margin"]
        assert bench.measured_traffic("contact", r["n"], m, tuning=r["tuning"]) == (
            r["bytes"] if current(r) else None)
        assert bench.measured_traffic("contact", r["n"] + 1, m, tuning=r["tuning"]) is None   # another size
        assert bench.measured_traffic("contact", r["n"], 0.35 * m, tuning=r["tuning"]) is None  # another margin
        assert bench.measured_traffic("contact", r["n"], tuning=r["tuning"]) is None          # margin unknown
    # one build's record is not taken for the other
    assert bench.measured_traffic("contact", two["n"], two["margin"], tuning={"contact_screen": 0}) is None
    m = t["margin"]
    # each build of the integration has its own record; another build than the captured
    # ones has none
    plain, staged = bench.MEASURED_TRAFFIC["integrate"]
    assert plain["tuning"] == {"integrate_staged": 0} and staged["tuning"] == {"integrate_staged": 1}
    assert bench.measured_traffic("integrate", plain["n"], tuning={"integrate_staged": 0}) == (
        plain["bytes"] if current(plain) else None)
    assert bench.measured_traffic("integrate", staged["n"], tuning={"integrate_staged": 1}) == (
        staged["bytes"] if current(staged) else None)
    assert bench.measured_traffic("contact", t["n"], m, tuning={"contact_lean": 1}) is None
    # the integration's figure holds at any margin
    assert bench.measured_traffic("integrate", plain["n"], 0.35 * m, tuning={"integrate_staged": 0}) == (
        plain["bytes"] if current(plain) else None)
    # a forward declaration is not the definition it hashes
    assert bench.kernel_source_hash("integrate_core(const Dev<F> &d") == bench.kernel_source_hash(
        "integrate_core(const Dev<F> &d, DevStatus *stp")
    fn, sig, hv = t["source"][0]
    changed = dict(t, source=[(fn, sig, "0" * 16)] + t["source"][1:])
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "contact", [changed])
    assert bench.measured_traffic("contact", t["n"], m) is None
    fn, sig, hv = two["source"][0]
    changed = dict(two, source=[(fn, sig, "0" * 16)] + two["source"][1:])
    monkeypatch.setitem(bench.MEASURED_TRAFFIC, "contact", [changed])
    assert bench.measured_traffic("contact", two["n"], two["margin"], tuning={"contact_screen": 1}) is None


def test_bench_line_carries_the_contract_keys(bench, monkeypatch, capsys):
    """main() on a stand-in for the GPU run: one JSON line with the contract's keys, the
    roofline of the dominant kernel and the traffic guard keyed by the run's margin."""
    import json
    import sys
    prof = dict(_prof(100, 0.15, 0.152), n_detect=10, detect_ms=3.0, hash_ms=0.09, link_ms=0.2)
    stats = {"margin": 2.1e-5}
    res = {"chosen": {"ms": 1825.0, "steps": 5000, "rebuilds": 488, "fallbacks": 0, "stats": stats,
                      "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 30},
                      "first_step": 50, "contacts": (600_000, 700_000)},
           "window_start": 0,
           "profile": prof, "copy_gbs": 6700.0, "tuning": {"fused_block": 0, "margin": 2.1e-5},
           "e2e": {"seconds": 0.08, "steps": 8, "bytes_in": 416_000_000, "bytes_out": 416_000_000},
           "n_spheres": 4_000_000, "clumps": False,
           "plain": {"ms": 229.0, "steps": 40, "profile": dict(prof, n_integrate=5)}}
    monkeypatch.setattr(bench, "run_ours", lambda args, device: res)
    monkeypatch.setattr(bench, "cpu_baseline", lambda args: {"value": 8e4, "unit": "sphere-steps/s", "cores": 1,
                                                             "kind": "oracle", "sample": "stand-in"})
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] == pytest.approx(4_000_000 * 5000 / 1.825)
    assert line["gpu_launches"] == 3 * 5000 + 20 * 488
    r = line["roofline"]
    assert r["kernel"].startswith("k_integrate") and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert line["e2e"]["h2d_bytes_per_step"] == 416_000_000
    assert line["config"]["listed_pairs_per_sphere"] == pytest.approx(0.25)
    assert "detect" in r["kernels"]


def test_two_pass_contact_phase_competes_by_its_longer_pass(bench):
    # the contact phase of the two-pass step spans two kernels: the dominant kernel is the
    # single kernel with the largest time, so a 0.146 ms phase of 0.096 + 0.050 ms passes
    # loses to a 0.133 ms integration; the phase keeps its bytes and time, with both passes
    prof = dict(_prof(100, contact_ms=0.146, integrate_ms=0.133), eval_ms=0.050, n_eval=100)
    r = bench.roofline("voxel_fp32", 4_000_000, prof, 6686.5, "measured", tuning={"contact_screen": 1})
    assert r["kernel"].startswith("k_integrate") and r["contact_screen"]
    c = r["kernels"]["contact"]
    assert c["ms"] == 0.146 and c["passes"]["k_contact_eval_ms"] == 0.050
    assert abs(c["passes"]["k_contact_screen_ms"] - 0.096) < 1e-12
    # without the evaluation pass's time (one contact kernel) the phase competes whole
    r1 = bench.roofline("voxel_fp32", 4_000_000, _prof(100, contact_ms=0.146, integrate_ms=0.133), 6686.5,
                        "measured")
    assert r1["kernel"].startswith("k_contact") and "passes" not in r1["kernels"]["contact"]
