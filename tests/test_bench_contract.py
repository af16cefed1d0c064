"""bench.py's reference arm (the CPU oracle timed on a bounded sample) prints
one JSON line with the keys the benchmark contract names; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "pipe10", "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["unit"] == "s"
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1e3 * d["value"]) < 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_roofline_arithmetic_from_recorded_work():
    """The bench's per-kernel rooflines, recomputed by hand from the work the
    library records (launches, milliseconds, units): 18 flop per pair against
    the FP32 CUDA-core peak (152 SMs x 128 lanes x 2 x 2070 MHz), 129 FP32-pipe
    operations per double-float pair against the issue rate, 8 rest^2 bytes
    per rank-128 trailing update (units = 2 x 128 x rest^2 flop) against the
    HBM peak with the measured traffic ratio, and the coarse solve's factor
    bytes against the HBM peak."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_1609_04484_gb300 as S
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "test"}
    pairs = 1.855e10  # one operator application of the 136,192-node pipe
    rest = 67968.0
    prof = {S.STOKES_PROF_PAIRS_DF64: [2, 160.0, 2 * pairs],
            S.STOKES_PROF_LU_GEMM: [1, 8.0, 2.0 * 128 * rest * rest],
            S.STOKES_PROF_COARSE_SOLVE: [1, 10.0, 1.85e10]}
    r = {e["class"]: e for e in bench.kernel_rooflines(S, prof, peaks)}
    peak_fp32 = 152 * 128 * 2 * 2070e6 / 1e12
    gps = 2 * pairs / 0.160
    df = r["pairs_df64"]
    assert abs(df["achieved"] - 18 * gps / 1e12) < 1e-3 and abs(df["peak"] - round(peak_fp32, 2)) < 1e-9
    assert abs(df["frac"] - 18 * gps / 1e12 / peak_fp32) < 1e-4
    assert abs(df["fp32_issue"]["achieved"] - 129 * gps / 1e12) < 0.01
    assert abs(df["fp32_issue"]["frac"] - 129 * gps / 1e12 / (peak_fp32 / 2)) < 1e-4
    tc = r["lu_gemm"]
    gbs = 8 * rest * rest / 0.008 / 1e9
    assert tc["kernel"] == "k_tc_trailing" and tc["bound"] == "hbm"
    assert abs(tc["achieved"] - gbs) < 0.1 and abs(tc["frac"] - gbs / 6800.0) < 1e-4
    assert tc["traffic"] == round(bench.MEASURED_TRAFFIC_RATIO["k_tc_trailing"] * 8 * rest * rest)
    cs = r["coarse_solve"]
    assert abs(cs["achieved"] - 1.85e10 / 0.010 / 1e9) < 0.1 and abs(cs["frac"] - 1850.0 / 6800.0) < 1e-4
