"""Write oracle results for the medium RPA + polarizability workload.

Calls only the CPU oracle (``oracle/``) on inputs from ``synth/``; nothing here
comes from the CUDA path.  Output: tests/golden/rpa_polar_medium.json with the
10 lowest Casida excitation energies, the 3x3 polarizability tensors at
omega = 0, 0.05, 0.1 Ha (rid preconditioner, FP64, threshold 1e-5), the
oracle's iteration / product counts and wall times, and checksums of the
generated inputs (so a changed generator is detected instead of read as a
parity failure).

    python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import davidson as DV  # noqa: E402
from oracle import operators as O  # noqa: E402
from synth.generator import CONFIGS, dipoles, make_config  # noqa: E402


def checksums(p, mu):
    return {"eps": float(p.eps_occ.sum() + p.eps_vir.sum()), "L_ov": float(p.L_ov.sum()),
            "L_vv_diag": float(np.einsum("paa->", p.L_vv)), "Lr_ov": float(p.Lr_ov.sum()),
            "mu": float(mu.sum())}


def main(name="rpa_polar_medium"):
    c = CONFIGS[name]
    p = make_config(name)
    mu = dipoles(c["mu_seed"], c["n_dip"], p.n_ov)
    op, T = O.exact_operator(p), O.ris_operator(p)
    out = {"config": name, "checksums": checksums(p, mu), "amplitude": p.amplitude}
    t0 = time.time()
    r = DV.solve_rpa(p, op, T, c["n_states"], precond="rid")
    out["rpa"] = {"omega": r.omega.tolist(), "resid": r.resid.tolist(), "n_iter": r.n_iter,
                  "n_mv": r.n_mv, "n_ris_mv": r.n_ris_mv, "converged": bool(r.converged),
                  "seconds": time.time() - t0}
    t0 = time.time()
    r = DV.solve_polar(p, op, T, mu, list(c["omegas"]), precond="rid")
    out["polar"] = {"alpha": r.alpha.tolist(), "omegas": list(c["omegas"]), "n_iter": r.n_iter,
                    "n_mv": r.n_mv, "n_ris_mv": r.n_ris_mv, "converged": bool(r.converged),
                    "seconds": time.time() - t0}
    # per-vector cost of the oracle's exact and ris pair products (for scaling samples)
    X = np.random.default_rng(0).standard_normal((4, p.n_ov))
    t0 = time.time()
    op.apb_amb(X)
    out["oracle_seconds_per_exact_pair_vector"] = (time.time() - t0) / 4
    t0 = time.time()
    T.apb_amb(X)
    out["oracle_seconds_per_ris_pair_vector"] = (time.time() - t0) / 4
    out["cpu_count"] = os.cpu_count()
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main(*sys.argv[1:])
