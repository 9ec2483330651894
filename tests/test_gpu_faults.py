"""Failure detection on the GPU without a fault: the bounded device-side waits
are made to run out on purpose, and inputs carry NaNs.  The mbarrier waits of
the tensor-core product run out under a budget of one clock cycle (the copies
they wait for take longer); the grid-wide waits of the persistent tGKB kernels
are given an arrival that nothing makes (tp_wait_stall) and a budget of a few
thousand cycles, so that they run out whatever the timing of the other CTAs.  Every case must return promptly with a status word, leave
the context usable, and a following normal call must agree with the oracle.

The waits covered: the grid-wide waits of the persistent tGKB kernels (one
slice per CTA: k_gkb; eight lateral slices per launch: k_gkb_multi; the nested
basis: k_gkb_nested) and the mbarrier waits of the tensor-core product inside
the RT-tSVD.  The drains of work already in flight keep their own bound, so a
CTA never ends with copies or tensor-core operations outstanding.
"""
import time

import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_02485_gb300 import synth

pytestmark = pytest.mark.gpu

TP_ERR_TIMEOUT = -6
TP_ERR_NONFINITE = -8
STALL_BUDGET = 20000  # clock cycles, about 10 us
PROMPT_S = 0.5  # the default budgets are about 1 s (tensor-core product) and 2 s (grid waits)


@pytest.fixture(scope="module")
def tp():
    from paper_2110_02485_gb300 import build, tprod
    build.build()
    tprod.load()
    assert torch.cuda.is_available()
    return tprod


@pytest.fixture(scope="module")
def prob():
    P = synth.blur_problem("n32")
    d = {k: torch.from_numpy(P[k]).cuda() for k in ("A", "B", "Omega")}
    return P, d


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def with_budget(tp, cycles, fn):
    tp.wait_budget(cycles)
    try:
        return timed(fn)
    finally:
        tp.wait_budget(0)


def with_stall(tp, fn):
    """Grid-wide waits for an arrival that nothing makes, under a short budget."""
    tp.wait_budget(STALL_BUDGET)
    tp.wait_stall(True)
    try:
        return timed(fn)
    finally:
        tp.wait_stall(False)
        tp.wait_budget(0)


def rtsvd(tp, P, d, B=None):
    cfg = P["cfg"]
    return tp.rtsvd_solve(d["A"], d["B"] if B is None else B, d["Omega"], P["delta"], cfg.tau, cfg.p_over,
                          cfg.block, cfg.q_power, cfg.r_max, eps_rel=cfg.eps_rel)


def test_rtsvd_tensor_core_waits_run_out_and_the_next_call_is_exact(tp, prob):
    P, d = prob
    rtsvd(tp, P, d)  # first-use setup (tensor maps, shared-memory opt-in) outside the timed call
    (X, info), dt = with_budget(tp, 1, lambda: rtsvd(tp, P, d))
    assert info["status"] == TP_ERR_TIMEOUT
    assert dt < PROMPT_S
    cfg = P["cfg"]
    A64, B64, Om64 = (P[k].astype(np.float64) for k in ("A", "B", "Omega"))
    ref = O.rtsvd_solve(A64, B64, Om64, P["delta"], cfg.tau, cfg.eps_rel * np.sqrt(O.fro2(A64)), cfg.p_over,
                        cfg.block, cfg.q_power, cfg.r_max)
    X, info = rtsvd(tp, P, d)
    assert info["status"] == ref["status"] and info["k"] == ref["k"] and info["r"] == ref["r"]
    assert rel(X.cpu().numpy(), ref["X"]) <= 1e-5


def test_tgkb_grid_waits_run_out_and_the_next_call_is_exact(tp, prob):
    P, d = prob
    cfg = P["cfg"]
    tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max)
    (X, info), dt = with_stall(tp, lambda: tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max))
    assert info["status"] == TP_ERR_TIMEOUT
    assert dt < PROMPT_S
    ref = O.tgkb_solve(P["A"].astype(np.float64), P["B"].astype(np.float64), P["delta"], cfg.tau, cfg.k_max)
    X, info = tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max)
    assert info["status"] == ref["status"] and info["k"] == ref["k"]
    assert rel(X.cpu().numpy(), ref["X"]) <= 1e-5


def test_tgkt_reports_the_timeout_of_its_tgkb_part(tp, prob):
    P, d = prob
    cfg = P["cfg"]
    (X, info), dt = with_stall(tp, lambda: tp.tgkt_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max,
                                                         cfg.mu_lo, cfg.mu_hi))
    assert info["status"] == TP_ERR_TIMEOUT
    assert dt < PROMPT_S


def frames(P, d, p=3):
    """p lateral slices: the workload's image and shifted copies, each with its own noise norm."""
    B0 = P["B"].astype(np.float64)
    g = np.random.default_rng(3)
    Bs, deltas = [], []
    for j in range(p):
        b = np.roll(P["B_true"], j, axis=0) if j else P["B_true"]
        E = g.standard_normal(b.shape)
        E = 1e-2 * E / np.linalg.norm(E) * np.linalg.norm(b)
        Bs.append(b + E)
        deltas.append(float(np.linalg.norm(E)))
    B = np.concatenate(Bs, axis=2).astype(np.float32)
    return B, deltas, B0


def test_tgkb_p_grid_waits_run_out_and_the_next_call_is_exact(tp, prob):
    P, d = prob
    cfg = P["cfg"]
    B, deltas, _ = frames(P, d)
    Bd = torch.from_numpy(B).cuda()
    tp.tgkb_solve(d["A"], Bd, 0.0, cfg.tau, cfg.k_max, deltas=deltas)
    (X, infos), dt = with_stall(tp, lambda: tp.tgkb_solve(d["A"], Bd, 0.0, cfg.tau, cfg.k_max, deltas=deltas))
    assert all(i["status"] == TP_ERR_TIMEOUT for i in infos)
    assert dt < PROMPT_S
    ref = O.tgkb_p_solve(P["A"].astype(np.float64), B.astype(np.float64), deltas, cfg.tau, cfg.k_max)
    X, infos = tp.tgkb_solve(d["A"], Bd, 0.0, cfg.tau, cfg.k_max, deltas=deltas)
    assert [i["k"] for i in infos] == list(ref["k"])
    assert rel(X.cpu().numpy(), ref["X"]) <= 1e-5


def test_nested_tgkb_p_grid_waits_run_out_and_the_next_call_is_exact(tp, prob):
    P, d = prob
    cfg = P["cfg"]
    B, deltas, _ = frames(P, d)
    Bd = torch.from_numpy(B).cuda()
    tp.nested_tgkb_solve(d["A"], Bd, deltas, cfg.tau, cfg.k_max)
    (X, infos), dt = with_stall(tp, lambda: tp.nested_tgkb_solve(d["A"], Bd, deltas, cfg.tau, cfg.k_max))
    assert all(i["status"] == TP_ERR_TIMEOUT for i in infos)
    assert dt < PROMPT_S
    ref = O.nested_tgkb_p_solve(P["A"].astype(np.float64), B.astype(np.float64), deltas, cfg.tau, cfg.k_max)
    X, infos = tp.nested_tgkb_solve(d["A"], Bd, deltas, cfg.tau, cfg.k_max)
    assert [i["k"] for i in infos] == list(ref["k"])
    assert rel(X.cpu().numpy(), ref["X"]) <= 1e-5


def test_wait_budget_rejects_negative_values(tp):
    with pytest.raises(tp.TprodError):
        tp.wait_budget(-1)


def test_one_stalled_call_leaves_the_rest_of_a_batch_exact(tp, prob):
    """A timed-out call in the middle of a sequence: the calls before and
    after it give identical results (workspaces and grid counters are reset
    by every call)."""
    P, d = prob
    cfg = P["cfg"]
    X0, i0 = tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max)
    (_, it), _ = with_stall(tp, lambda: tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max))
    X1, i1 = tp.tgkb_solve(d["A"], d["B"], P["delta"], cfg.tau, cfg.k_max)
    assert it["status"] == TP_ERR_TIMEOUT and i0["status"] == i1["status"] == 0
    assert torch.equal(X0, X1)


@pytest.mark.parametrize("where", ["B", "A"])
def test_nan_inputs_end_within_the_caps_with_a_status(tp, prob, where):
    """A NaN in B (or in A): every solve runs within its caps (a NaN never
    meets the discrepancy bound) and reports TP_ERR_NONFINITE with a NaN
    residual, from the norms its DFTs form.  Nothing hangs or faults and the
    next call is exact."""
    P, d = prob
    cfg = P["cfg"]
    A, B = d["A"].clone(), d["B"].clone()
    (A if where == "A" else B)[3, 5, 0] = float("nan")
    calls = [lambda: tp.rtsvd_solve(A, B, d["Omega"], P["delta"], cfg.tau, cfg.p_over, cfg.block, cfg.q_power,
                                    cfg.r_max, eps_rel=cfg.eps_rel),
             lambda: tp.tgkb_solve(A, B, P["delta"], cfg.tau, cfg.k_max),
             lambda: tp.tgkt_solve(A, B, P["delta"], cfg.tau, cfg.k_max, cfg.mu_lo, cfg.mu_hi)]
    for fn in calls:
        (X, info), dt = timed(fn)
        assert dt < 2 * PROMPT_S
        assert info["status"] == TP_ERR_NONFINITE and not np.isfinite(info["residual"])
    X, info = rtsvd(tp, P, d)
    cfg_ref = O.rtsvd_solve(*(P[k].astype(np.float64) for k in ("A", "B", "Omega")), P["delta"], cfg.tau,
                            cfg.eps_rel * np.sqrt(O.fro2(P["A"].astype(np.float64))), cfg.p_over, cfg.block,
                            cfg.q_power, cfg.r_max)
    assert info["k"] == cfg_ref["k"] and rel(X.cpu().numpy(), cfg_ref["X"]) <= 1e-5
