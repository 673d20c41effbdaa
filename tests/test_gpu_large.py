"""Full-size checks on the large mixed workload (n_occ=150, n_vir=1350,
ov=202,500, n_aux=6000, ris n_aux=1350) in the launch configuration of the
MIXED solves (tcgen05 BF16 hi+lo exact products, BF16 ris, rid).

The oracle cannot hold this problem (108 GB of FP64 factors over all
orbitals), so it works over P-chunks (tests/large_harness.py):
  * the exact pair products ((A+B)X, (A-B)X) of two random vectors, every
    element, against the oracle's FP64 products: 5e-5 relative (BF16 hi+lo, as
    for the medium workload);
  * the workload is well posed: lambda_min(A+B) and lambda_min(A-B) above
    0.02 Ha (Lanczos on the GPU products) and the diagonal-preconditioned Casida
    solve converging within 33 outer iterations, the input recipe's criterion;
  * TDA and Casida solves for the 20 lowest states with the rid preconditioner,
    each converged with its residuals re-certified below 1e-5 by the FP32
    operator, and rid taking no more outer iterations than diag;
  * the oracle's FP64 residuals of two converged TDA vectors: below 1.2e-5 (the
    FP32 re-certification itself is accurate to ~1e-7 relative).
"""
import numpy as np
import pytest

from oracle import operators as O
from synth.generator import CONFIGS, config_meta
from tests import large_harness as H

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
NAME = "large_mixed"


@pytest.fixture(scope="module")
def large():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api
    meta = config_meta(NAME)
    no, nv, na, nr = meta["n_occ"], meta["n_vir"], meta["n_aux"], meta["n_ris"]
    kidx = meta["ris_K_index"]
    dev = (torch.empty(na, no, no, device="cuda"), torch.empty(na, no, nv, device="cuda"),
           torch.empty(na, nv, nv, device="cuda"))
    X = np.random.default_rng(7).standard_normal((2, no * nv))
    parts = H.load_exact(NAME, meta, dev, X)
    rdev = (torch.empty(kidx.size, no, no, device="cuda"), torch.empty(nr, no, nv, device="cuda"),
            torch.empty(kidx.size, nv, nv, device="cuda"))
    H.load_ris(NAME, meta, rdev)
    cu = lambda a: torch.from_numpy(a).cuda()
    s = api.Solver(no, nv, cu(meta["eps_occ"]), cu(meta["eps_vir"]), dev[0], dev[1], dev[2], rdev[0],
                   rdev[1], rdev[2], cu(kidx), a_x=meta["a_x"], coulomb_factor=meta["coulomb_factor"],
                   t_cut_ha=meta["t_cut_ha"], precisions=2, dtype=api.F32)
    del dev, rdev
    torch.cuda.empty_cache()
    yield api, meta, s, X, parts
    s.close()


def _lanczos_min(api, s, which, steps=40):
    """Lowest eigenvalue of A+B (which=0) or A-B (1) by Lanczos with full
    reorthogonalisation on the MIXED tensor-core products."""
    import torch
    ov = s.n_ov
    q = torch.from_numpy(np.random.default_rng(11 + which).standard_normal((1, ov))).cuda()
    q /= q.norm()
    Q, alpha, beta = [q], [], []
    for _ in range(steps):
        y = s.apply(1, Q[-1], precision=api.MIXED, tensor_cores=True)[which]
        alpha.append(float((y * Q[-1]).sum()))
        for qq in Q:
            y = y - (y * qq).sum() * qq
        b = float(y.norm())
        if b < 1e-10:
            break
        beta.append(b)
        Q.append(y / b)
    n = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:n - 1], 1) + np.diag(beta[:n - 1], -1)
    return float(np.linalg.eigvalsh(T)[0])


def test_pair_products_full_size(large):
    api, meta, s, X, (J, K1, K2) = large
    d = O.delta(meta["eps_occ"], meta["eps_vir"])
    rp, rm = O.pair_from_parts(d, X, J, K1, K2, meta["a_x"], meta["coulomb_factor"])
    gp, gm = s.apply(1, X, precision=api.MIXED, tensor_cores=True)
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert rel(gp, rp) < 5e-5 and rel(gm, rm) < 5e-5


def test_workload_well_posed(large):
    api, _, s, _, _ = large
    lp, lm = _lanczos_min(api, s, 0), _lanczos_min(api, s, 1)
    print("\nlarge_mixed lambda_min(A+B) = %.4f Ha, lambda_min(A-B) = %.4f Ha" % (lp, lm))
    assert lp > 0.02 and lm > 0.02


def test_tda_and_casida_full_size(large):
    api, meta, s, _, _ = large
    k = CONFIGS[NAME]["n_states"]
    o = api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1)
    t = s.solve_tda(o, want_vectors=True)
    assert t["status"] == api.OK
    assert t["stats"]["max_resid_certified"] < 1e-5
    assert np.all(np.diff(t["omega"]) >= 0)
    r = s.solve_rpa(o, want_vectors=False)
    assert r["status"] == api.OK
    assert r["stats"]["max_resid_certified"] < 1e-5
    assert np.all(np.diff(r["omega"]) >= 0)
    od = api.default_opts(n_states=k, precond=api.DIAG, precision=api.MIXED, tensor_cores=1, max_iter=33)
    rd = s.solve_rpa(od, want_vectors=False)
    assert rd["status"] == api.OK, rd["stats"]
    print("\nlarge_mixed TDA rid: %d it %.2f s; Casida rid: %d it %.2f s; Casida diag: %d it %.2f s; "
          "omega_0 = %.8f Ha" % (t["stats"]["n_iter"], t["stats"]["t_total_s"], r["stats"]["n_iter"],
                                 r["stats"]["t_total_s"], rd["stats"]["n_iter"], rd["stats"]["t_total_s"],
                                 r["omega"][0]))
    assert r["stats"]["n_iter"] <= rd["stats"]["n_iter"]
    assert np.max(np.abs(rd["omega"] - r["omega"])) < 1e-5
    # the oracle's FP64 residuals of the lowest and the highest converged TDA state
    pick = [0, k - 1]
    Xs = np.ascontiguousarray(t["X"][pick])
    J, K1, _ = H.load_exact(NAME, meta, None, Xs)
    d = O.delta(meta["eps_occ"], meta["eps_vir"])
    AX = O.tda_from_parts(d, Xs, J, K1, meta["a_x"], meta["coulomb_factor"])
    om = np.asarray(t["omega"])[pick]
    res = np.linalg.norm(AX - om[:, None] * Xs, axis=1) / np.linalg.norm(Xs, axis=1)
    assert np.all(res < 1.2e-5), res
