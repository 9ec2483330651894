"""Write <config>_oracle.json and <config>_oracle_X.npz: the FP64 oracle's
results on a full-size deblurring workload that bench.py times
(synth.CONFIGS[config], the seed of rank 0), for the full-size GPU parity tests
(tests/test_gpu_full_size.py) and the bench's error figures.

The .json holds the scalars (truncation indices, statuses, margins, residual
histories, mu, the float32 feasibility figures); the .npz holds the complete
float64 solutions X (n, N, 1) of the RT-tSVD, tGKB and Tikhonov-tGKB solves
(and, up to N = 256, of the T-tSVD).

Calls only the oracle and the seeded input generator:

    python tests/golden/make_goldens.py n256      # about a minute and a half
    python tests/golden/make_goldens.py n512      # several minutes
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2110_02485_gb300 import synth  # noqa: E402

N_SAMPLES = 1024


def sample_index(N: int) -> np.ndarray:
    """Seeded flat indices into an (N, N, 1) solution (the same on both sides)."""
    return np.random.default_rng(2024).choice(N * N, size=N_SAMPLES, replace=False)


def main(name: str) -> None:
    cfg = synth.CONFIGS[name]
    P = synth.blur_problem(cfg, seed=cfg.seed)
    A, B, Om = (P[k].astype(np.float64) for k in ("A", "B", "Omega"))
    idx = sample_index(cfg.N)
    out = {"config": name, "seed": cfg.seed, "delta": P["delta"], "sample_index": idx.tolist()}
    sols = {}

    def pack(method, r, extra):
        X = r["X"].reshape(-1)
        sols[method] = r["X"]
        d = {"k": int(r["k"]), "status": int(r["status"]), "tau_delta": float(r["tau_delta"]),
             "x_norm": float(np.linalg.norm(X)), "x_samples": X[idx].tolist()}
        d.update(extra)
        out[method] = d

    r1 = O.rtsvd_solve(A, B, Om, P["delta"], cfg.tau, cfg.eps_rel * np.sqrt(O.fro2(A)), cfg.p_over, cfg.block,
                       cfg.q_power, cfg.r_max)
    # FP32 feasibility: kappa_k = max_s sigma_1 / min_s sigma_k of the factorisation's singular values, and the
    # first-order float32 error of the truncated solution, u32 kappa_k sqrt(N)
    S = r1["S"]
    kappa = float(S[:, 0].max() / S[:, r1["k"] - 1].min())
    pack("rtsvd", r1, {"r": int(r1["r"]), "residual": float(r1["res"][r1["k"]]), "margin": float(r1["margin"]),
                       "res": {str(k): v for k, v in r1["res"].items()}, "kappa_k": kappa,
                       "fp32_error_prediction": float(np.finfo(np.float32).eps * kappa * np.sqrt(cfg.N))})
    r2 = O.tgkb_solve(A, B, P["delta"], cfg.tau, cfg.k_max)
    pack("tgkb", r2, {"residual": float(r2["res"][r2["k"]]), "margin": float(r2["margin"]),
                      "res": {str(k): v for k, v in r2["res"].items()}})
    r3 = O.tgkt_solve(A, B, P["delta"], cfg.tau, cfg.k_max, cfg.mu_lo, cfg.mu_hi)
    pack("tgkt", r3, {"mu": float(r3["mu"]), "residual": float(r3["residual"])})
    if cfg.N <= 256:  # the full tSVD (Section 4.1) of the comparison tables
        r4 = O.ttsvd_solve(A, B, P["delta"], cfg.tau)
        pack("ttsvd", r4, {"residual": float(r4["res"][r4["k"]]), "margin": float(r4["margin"])})
    with open(os.path.join(HERE, f"{name}_oracle.json"), "w") as f:
        json.dump(out, f)
    np.savez(os.path.join(HERE, f"{name}_oracle_X.npz"), **sols)
    print({m: {k: out[m].get(k) for k in ("k", "status", "margin", "mu", "r")} for m in sols})


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "n256")
