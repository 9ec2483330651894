"""The tensor-core product's stage-count tuner: the stage count of the TMA
ring changes only the time of a product, never its result, so an RT-tSVD
solve gives bit-identical output under every stage count the tuner may pick,
and after rtsvd_autotune the table holds every product shape of the solve."""
import numpy as np
import pytest

from paper_2110_02485_gb300 import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_02485_gb300 import tprod
    tprod.load()
    return tprod


N, NT, BLOCK, R_MAX = 64, 16, 16, 48


def solve(tp, form):
    T, c = synth.blur_factors(N, 1.5, 4, 2.0, n=NT)
    A = synth.blur_tensor(T, c)
    g = np.random.default_rng(8)
    B = (A.astype(np.float64).sum(axis=2, keepdims=True) * 0.1 + 1e-3 * g.standard_normal((NT, N, 1))).astype(
        np.float32)
    Om = g.standard_normal((NT, N, R_MAX)).astype(np.float32)
    dev = lambda x: torch.from_numpy(x).cuda()
    kw = {"tf32": dict(tf32=True), "bf16": dict(bf16=True)}.get(form, {})
    X, info = tp.rtsvd_solve(dev(A), dev(B), dev(Om), 0.01, 1.1, 4, BLOCK, 1, R_MAX, eps_rel=1e-3, **kw)
    return X.cpu().numpy(), info


def shapes(form):
    h = NT // 2 + 1
    return [(0, form, BLOCK, N, N, h), (2, form, BLOCK, N, N, h), (2, "fp32", BLOCK, N, N, h),
            (0, "fp32", 32, N, N, h)]


@pytest.mark.parametrize("form", ["fp32", "tf32", "bf16"])
def test_every_stage_count_gives_the_same_solution(tp, form):
    tp.autotune_clear()
    X0, i0 = solve(tp, form)
    tried = 0
    for stages in range(2, 7):
        tp.autotune_clear()
        ok = True
        for sh in shapes(form):
            try:
                tp.autotune_set(*sh, stages)
            except tp.TprodError:
                ok = False  # more stages than this shape's ring holds
        if not ok:
            continue
        X, info = solve(tp, form)
        assert np.array_equal(X, X0) and info == i0, stages
        tried += 1
    tp.autotune_clear()
    assert tried >= 2


def test_autotune_tunes_every_product_shape_and_changes_no_result(tp):
    tp.autotune_clear()
    X0, i0 = solve(tp, "fp32")
    table = tp.rtsvd_autotune(NT, N, N, 1, BLOCK, R_MAX, "fp32")
    keys = {(e["op"], e["form"], e["columns"], e["M"], e["K"], e["batch"]) for e in table}
    h = NT // 2 + 1
    assert keys == {("A", "fp32", 16, N, N, h), ("conj(A)", "fp32", 16, N, N, h), ("A", "fp32", 32, N, N, h)}
    for e in table:
        assert 2 <= e["stages"] <= 6 and e["ms"] > 0 and e["ms"] <= e["ms_default"] * (1 + 1e-6)
    X1, i1 = solve(tp, "fp32")
    assert np.array_equal(X1, X0) and i1 == i0
    tp.autotune_clear()
    assert tp.autotune_table() == []
