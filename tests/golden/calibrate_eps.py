"""Calibrate eps_rel, the tolerance of Algorithm 3 relative to ||A||_F, for a
workload (the paper tunes the absolute eps per example by experiment, Table 0).

Reading taken: eps_rel is the largest value on the grid 10^(-j/10) for which
the oracle's RT-tSVD meets the discrepancy principle within [r - p, r] (Eq.
(kinit)), r being the rank at which eta falls below (eps_rel ||A||_F)^2.  One
block sketch to r_max gives eta after every block; each candidate rank is then
a prefix of that factorisation.  Calls only the oracle and the seeded input
generator:

    python tests/golden/calibrate_eps.py n512      # one named workload
    python tests/golden/calibrate_eps.py uneven    # each problem of the uneven batch
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2110_02485_gb300 import synth  # noqa: E402


def calibrate(A, B, Om, delta, tau, p_over, block, q_power, r_max, verbose=True):
    """(j, eps_rel, r, k) for the largest eps_rel = 10^(-j/10) that meets the
    discrepancy principle within [r - p, r], or None."""
    a2 = O.fro2(A)
    fac = O.rtsvd_block(A, Om, 0.0, block, q_power, r_max)
    etas = np.asarray(fac["etas"])
    if verbose:
        print("eta / ||A||^2 after each block:", (etas / a2).tolist(), flush=True)
    tried = set()
    for j in range(5, 61):
        e = 10.0 ** (-j / 10.0)
        below = np.nonzero(etas < e * e * a2)[0]
        if len(below) == 0:
            continue
        r = min(int(below[0]) * block, r_max)
        if r in tried:
            continue
        tried.add(r)
        out = O.rtsvd_solve(A, B, Om, delta, tau, e * np.sqrt(a2), p_over, block, q_power, r_max,
                            fac=O.rtsvd_prefix(fac, r, block))
        if verbose:
            print(f"eps_rel 10^(-{j}/10) = {e:.4g}: r = {r}, k = {out['k']}, status = {out['status']}, "
                  f"margin = {out['margin']:.3g}", flush=True)
        if out["status"] == O.STATUS_OK:
            return j, e, r, out["k"]
    return None


def main(name: str) -> None:
    if name == "uneven":
        res = []
        for i, p in enumerate(synth.uneven_problems(calibrated=False)):
            f64 = lambda x: x.astype(np.float64)
            c = calibrate(f64(p["A"]), f64(p["B"]), f64(p["Omega"]), p["delta"], synth.UNEVEN_TAU,
                          synth.UNEVEN_P_OVER, synth.UNEVEN_BLOCK, synth.UNEVEN_Q, p["r_max"], verbose=False)
            print(i, p["N"], c, flush=True)
            res.append(c[0] if c else None)
        print("UNEVEN_EPS_J =", tuple(res))
        return
    cfg = synth.CONFIGS[name]
    P = synth.blur_problem(cfg, seed=cfg.seed)
    A, B, Om = (P[k].astype(np.float64) for k in ("A", "B", "Omega"))
    print("calibrated:", calibrate(A, B, Om, P["delta"], cfg.tau, cfg.p_over, cfg.block, cfg.q_power, cfg.r_max))


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "n512")
