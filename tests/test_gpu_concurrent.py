"""Independent solves on concurrent streams, as the bench step issues them: an
RT-tSVD, a tGKB and a Tikhonov-tGKB solve of the same problem (sharing the
read-only A and B) on three streams forked from the current stream and joined
back.  Every solve has its own workspace and its own grid counters, so the
results must be bit-identical to the same three solves on one stream, in
plain launches and in a CUDA-graph replay, at the small workload and at 256^3
(where the two cooperative tGKB launches cannot be co-resident and the second
waits for the first)."""
import numpy as np
import pytest
import torch

from paper_2110_02485_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    from paper_2110_02485_gb300 import build, tprod
    build.build()
    tprod.load()
    assert torch.cuda.is_available()
    return tprod


def three(tp, cfg, A, B, Om, delta):
    return [lambda: tp.rtsvd_solve(A, B, Om, delta, cfg.tau, cfg.p_over, cfg.block, cfg.q_power, cfg.r_max,
                                   eps_rel=cfg.eps_rel, sync=False)[:2],
            lambda: tp.tgkb_solve(A, B, delta, cfg.tau, cfg.k_max, sync=False)[:2],
            lambda: tp.tgkt_solve(A, B, delta, cfg.tau, cfg.k_max, cfg.mu_lo, cfg.mu_hi, sync=False)]


def on_streams(fns, side):
    main = torch.cuda.current_stream()
    out = []
    for fn, st in zip(fns, side):
        st.wait_stream(main)
        with torch.cuda.stream(st):
            out.append(fn())
    for st in side:
        main.wait_stream(st)
    return out


def host(res, tp):
    return [(X.cpu().numpy().copy(), tp._info_dict(i)) for X, i in res]


@pytest.mark.parametrize("name", ["n32", "n256"])
def test_three_solves_on_three_streams_equal_one_stream(tp, name):
    cfg = synth.CONFIGS[name]
    P = synth.blur_problem(cfg, seed=cfg.seed)
    A, B, Om = (torch.from_numpy(P[k]).cuda() for k in ("A", "B", "Omega"))
    fns = three(tp, cfg, A, B, Om, P["delta"])
    side = [torch.cuda.Stream() for _ in range(3)]
    ref = [f() for f in fns]
    torch.cuda.synchronize()
    ref = host(ref, tp)
    assert all(i["status"] == 0 for _, i in ref)
    par = on_streams(fns, side)
    torch.cuda.synchronize()
    for (x0, i0), (x1, i1) in zip(ref, host(par, tp)):
        assert np.array_equal(x0, x1) and i0 == i1
    g = tp.Captured(lambda: on_streams(fns, side), warmup=0)
    for X, _ in g.outputs:  # the checks below see the replay's results
        X.fill_(float("nan"))
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for (x0, i0), (x1, i1) in zip(ref, host(g.outputs, tp)):
            assert np.array_equal(x0, x1) and i0 == i1
