"""Host logic of bench.py's roofline accounting (no GPU): the algorithmic
byte and flop counts per kernel class against the sizes they are built from,
the fractions of the peaks, the clock-record parsing, and the freshness of the
DRAM traffic records (each is tied to the sha256 of the sources it was
captured from)."""
import hashlib
import math
import os

import pytest

import bench
from paper_2110_02485_gb300 import synth


def test_gkb_bytes_is_the_sum_of_its_steps():
    # k steps: two passes over A-hat, the two CGS passes over the W (i - 1
    # vectors of m) and Q (i vectors of l) bases, two new vectors written
    h, l, m, k, c = 3, 5, 7, 4, 8
    want = sum(2 * c * h * l * m + 4 * c * h * ((i - 1) * m + i * l) + c * h * (l + m) for i in range(1, k + 1))
    assert bench.gkb_bytes(h, l, m, k, 4) == want
    # closed form of the same sum
    closed = k * (2 * c * h * l * m + c * h * (l + m)) + 4 * c * h * (m * k * (k - 1) // 2 + l * k * (k + 1) // 2)
    assert want == closed


def n256_work():
    cfg = synth.CONFIGS["n256"]
    rt = {"r": 96, "k": 86, "sweeps": 6}
    return cfg, bench.class_work(cfg, (rt, {"k": 23}, {"k": 23}))


def test_class_work_dft_bytes_are_the_transforms_of_a_step():
    cfg, w = n256_work()
    N = cfg.N
    h = N // 2 + 1
    real, cplx = 4 * N ** 3, 8 * h * N * N          # A read once, its half spectrum written once
    A = 3 * (real + cplx)                            # each of the three solves transforms A
    B = 3 * (4 * N * N + 8 * h * N)                  # and B (one lateral slice)
    Om = 4 * N * N * 96 + 8 * h * N * 96              # the r = 96 Gaussian slices the sketch uses
    inv = 3 * (8 * h * N + 4 * N * N)                # three inverse transforms of one slice
    assert w["dft"]["bytes"] == A + B + Om + inv
    assert w["dft"]["bound"] == "hbm"


def test_class_work_gemm_streams_a_hat_once_per_pass():
    cfg, w = n256_work()
    N, h = cfg.N, cfg.N // 2 + 1
    ahat = 8 * h * N * N                             # 67.6 MB at 256^3
    assert ahat == pytest.approx(67.6e6, rel=2e-3)
    nblk = 96 // cfg.block
    passes = nblk * (2 * cfg.q_power + 2) + math.ceil(96 / 32) + 2   # sketch/power/projection, K chunks, transpose
    r, c = 96, 8
    # the small products with r-column factors: V = Q_G U_R (reads Q_G and U_R, writes V), d = Q^H b (reads Q
    # and b) and X = V alpha (reads V, writes X)
    small = c * h * (N * r + r * r + N * r) + c * h * (r * N + N) + c * h * (N * r + N)
    assert w["gemm"]["bytes"] == passes * ahat + small
    assert w["gemm"]["bound"] == "hbm"


def test_class_work_orth_flops_of_the_deflation_dominate():
    cfg, w = n256_work()
    N, h, b, q = cfg.N, cfg.N // 2 + 1, cfg.block, cfg.q_power
    defl = sum(h * ((q + 1) * 32.0 * N * blk * b * b + 32.0 * N * blk * b * b) for blk in range(96 // b))
    assert defl < w["orth"]["flops"] < 1.5 * defl
    assert w["orth"]["bound"] == "alu" and w["svd"]["bound"] == "alu"


def test_roofline_entries_divide_work_by_time_and_peak():
    work = {"gemm": {"bytes": 2e9, "flops": None, "bound": "hbm"},
            "svd": {"bytes": None, "flops": 4e12, "bound": "alu"},
            "dp": {"bytes": 1e9, "flops": None, "bound": "hbm"}}
    per = {"gemm": (0.5, 10), "svd": (100.0, 1)}     # ms per step, launches; dp did not run
    out = bench.roofline_entries(work, per, 8000.0, "measured")
    assert set(out) == {"gemm", "svd", "peaks"}
    assert out["gemm"]["hbm_gbs"] == pytest.approx(4000.0)
    assert out["gemm"]["hbm_frac"] == pytest.approx(0.5)
    assert out["gemm"]["bytes_per_launch"] == pytest.approx(2e8)
    assert out["svd"]["tflops"] == pytest.approx(40.0)
    assert out["svd"]["fp32_simt_frac"] == pytest.approx(40.0 / bench.FP32_SIMT_TFLOPS)
    assert bench.FP32_SIMT_TFLOPS == pytest.approx(80.5, rel=1e-3)
    assert out["peaks"]["hbm_gbs"] == 8000.0


def test_clock_record_parsing():
    cs = bench.ClockSampler(0)
    cs.rows = [["2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["2055", "2070", "1300", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["1990", "2070", "1350", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["garbage"]]
    rec = cs.stop()
    assert rec["samples"] == 3
    assert rec["sm_mhz"] == 2055.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]


def test_traffic_record_reads_null_once_its_sources_change(monkeypatch):
    """A DRAM traffic record is reported only while every source it was
    captured from hashes to the recorded value, and only for the 256^3 step
    it was captured on."""
    cls = "orth"
    rec = bench.NCU_TRAFFIC[cls]
    cur = {}
    for src in rec["sources"]:
        with open(os.path.join(bench.ROOT, bench._SRC + src), "rb") as f:
            cur[src] = hashlib.sha256(f.read()).hexdigest()
    monkeypatch.setattr(bench, "_SHA", {**bench._SHA, **cur})
    assert bench.ncu_traffic(cls) == rec["bytes"]
    assert bench.ncu_traffic(cls, config="n512") is None
    monkeypatch.setattr(bench, "_SHA", {**bench._SHA, rec["sources"][0]: "0" * 64})
    assert bench.ncu_traffic(cls) is None
