"""Parity of the uneven batch in the form bench.py times: several independent
problems of different sizes, one RT-tSVD and one tGKB solve each, recorded as
one CUDA graph over several streams and replayed.  Every problem's solutions
must equal the FP64 oracle's (truncation indices exactly, solutions within the
float32 bound), on the replay, not only on the captured calls."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2110_02485_gb300 import synth

pytestmark = pytest.mark.gpu

SIZES = (16, 24, 32, 20, 28)
TAU, P_OVER, Q_POWER, BLOCK, EPS_REL, K_MAX = 1.1, 3, 1, 4, 2e-2, 20


@pytest.fixture(scope="module")
def tp():
    from paper_2110_02485_gb300 import build, tprod
    build.build()
    tprod.load()
    assert torch.cuda.is_available()
    return tprod


def problems():
    rng = synth.rng_for(77)
    out = []
    for N in SIZES:
        T, c = synth.blur_factors(N, 1.5, 4, 2.0)
        img = synth.synthetic_image(N, N, 4, 1, rng)
        B, delta = synth.add_noise(synth.forward_blur(T, c, img), 1e-2, rng)
        out.append(dict(N=N, delta=delta, A=synth.blur_tensor(T, c), B=synth.lateral(B).astype(np.float32),
                        Omega=rng.standard_normal((N, N, N)).astype(np.float32)))
    return out


def test_uneven_batch_graph_over_streams_matches_oracle(tp):
    probs = problems()
    dev = [{k: torch.from_numpy(p[k]).cuda() for k in ("A", "B", "Omega")} for p in probs]

    def solve(p, d):
        X1, i1, _ = tp.rtsvd_solve(d["A"], d["B"], d["Omega"], p["delta"], TAU, P_OVER, BLOCK, Q_POWER, p["N"],
                                   eps_rel=EPS_REL, sync=False)
        X2, i2, _ = tp.tgkb_solve(d["A"], d["B"], p["delta"], TAU, min(K_MAX, p["N"]), sync=False)
        return X1, i1, X2, i2

    side = [torch.cuda.Stream() for _ in range(3)]

    def batch():
        main = torch.cuda.current_stream()
        outs = [None] * len(probs)
        for st in side:
            st.wait_stream(main)
        for i, (p, d) in enumerate(zip(probs, dev)):
            with torch.cuda.stream(side[i % len(side)]):
                outs[i] = solve(p, d)
        for st in side:
            main.wait_stream(st)
        return outs

    for p, d in zip(probs, dev):
        solve(p, d)
    torch.cuda.synchronize()
    g = tp.Captured(batch, warmup=0)
    for o in g.outputs:  # clear the captured results: the checks below see the replay's
        o[0].fill_(float("nan"))
        o[2].fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    for p, (X1, i1, X2, i2) in zip(probs, g.outputs):
        A, B, Om = (p[k].astype(np.float64) for k in ("A", "B", "Omega"))
        r1 = O.rtsvd_solve(A, B, Om, p["delta"], TAU, EPS_REL * np.sqrt(O.fro2(A)), P_OVER, BLOCK, Q_POWER, p["N"])
        r2 = O.tgkb_solve(A, B, p["delta"], TAU, min(K_MAX, p["N"]))
        i1, i2 = tp._info_dict(i1), tp._info_dict(i2)
        assert (i1["r"], i1["k"], i1["status"]) == (r1["r"], r1["k"], r1["status"]), p["N"]
        assert (i2["k"], i2["status"]) == (r2["k"], r2["status"]), p["N"]
        for X, r in ((X1, r1), (X2, r2)):
            x = X.cpu().numpy()
            assert np.linalg.norm(x - r["X"]) <= 1e-5 * np.linalg.norm(r["X"]), p["N"]
