"""Full-size checks on the large mixed workload (n_occ=150, n_vir=1350,
ov=202,500, n_aux=6000, ris n_aux=1350) in the launch configuration of the
MIXED solves (tcgen05 FP16 hi+lo exact products, BF16 ris, rid).

The oracle cannot hold this problem (108 GB of FP64 factors over all
orbitals), so it works over P-chunks (tests/large_harness.py):
  * the exact pair products ((A+B)X, (A-B)X) of two random vectors, every
    element, against the oracle's FP64 products: 1e-5 relative (FP16 hi+lo
    with power-of-two scales; FP32 accumulation over K = P x a terms);
  * the workload is well posed: lambda_min(A+B) and lambda_min(A-B) above
    0.02 Ha (Lanczos on the GPU products) and the diagonal-preconditioned Casida
    solve converging within 33 outer iterations, the input recipe's criterion;
  * TDA and Casida solves for the 20 lowest states with the rid preconditioner,
    each converged with its residuals, recomputed from fresh FP32-accurate
    products of the final vectors, below 1e-5, and rid taking no more outer
    iterations than diag;
  * the rid preconditioner on FP8 e4m3 ris factors (one scale per row):
    converged TDA and Casida energies within 1e-5 Ha of the BF16-ris solves;
  * every one of the 20 converged TDA vectors and the 20 Casida pairs is
    re-certified by the oracle in FP64 (one pass over the factors for all 60
    vectors X, X+Y, X-Y): the residual of Eq. residual below 1.2e-5, and the
    GPU energies within 1e-5 Ha of the oracle's Rayleigh quotients of the same
    vectors (x^T A x for TDA; sqrt(u^T(A+B)u w^T(A-B)w) / u^T w for Casida,
    u = X+Y, w = X-Y), which are exact to second order in the residual.
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
    print("\nlarge_mixed FP16 hi+lo tensor-core pair products: rel err %.2e, %.2e" % (rel(gp, rp), rel(gm, rm)))
    assert rel(gp, rp) < 1e-5 and rel(gm, rm) < 1e-5


def test_full_size_solves(large):
    """Well-posedness, the rid / diag / FP8-ris solves and the oracle's FP64
    certification of all 20 + 20 converged states.  The certification (one
    pass of the oracle over the factors on the host cores, several minutes)
    runs while the GPU does the diag and FP8 solves."""
    from concurrent.futures import ThreadPoolExecutor

    api, meta, s, _, _ = large
    k = CONFIGS[NAME]["n_states"]
    lp, lm = _lanczos_min(api, s, 0), _lanczos_min(api, s, 1)
    print("\nlarge_mixed lambda_min(A+B) = %.4f Ha, lambda_min(A-B) = %.4f Ha" % (lp, lm))
    assert lp > 0.02 and lm > 0.02
    o = api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1)
    t = s.solve_tda(o, want_vectors=True)
    assert t["status"] == api.OK
    assert t["stats"]["max_resid_certified"] < 1e-5
    assert np.all(np.diff(t["omega"]) >= 0)
    r = s.solve_rpa(o, want_vectors=True)
    assert r["status"] == api.OK
    assert r["stats"]["max_resid_certified"] < 1e-5
    assert np.all(np.diff(r["omega"]) >= 0)
    X = t["X"]
    U, W = r["X"] + r["Y"], r["X"] - r["Y"]
    assert np.max(np.abs(X @ X.T - np.eye(k))) < 1e-8
    assert np.max(np.abs(np.sum(U * W, axis=1) - 1.0)) < 1e-8
    V = np.ascontiguousarray(np.concatenate([X, U, W]))
    with ThreadPoolExecutor(1) as ex:
        cert = ex.submit(H.load_exact, NAME, meta, None, V)
        # meanwhile on the GPU: the diagonal preconditioner and the FP8 ris factors
        od = api.default_opts(n_states=k, precond=api.DIAG, precision=api.MIXED, tensor_cores=1, max_iter=33)
        rd = s.solve_rpa(od, want_vectors=False)
        of = api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1, ris_fp8=1)
        tf = s.solve_tda(of, want_vectors=False)
        rf = s.solve_rpa(of, want_vectors=False)
        J, K1, K2 = cert.result()
    print("large_mixed TDA rid: %d it %.2f s; Casida rid: %d it %.2f s; Casida diag: %d it %.2f s; "
          "omega_0 = %.8f Ha" % (t["stats"]["n_iter"], t["stats"]["t_total_s"], r["stats"]["n_iter"],
                                 r["stats"]["t_total_s"], rd["stats"]["n_iter"], rd["stats"]["t_total_s"],
                                 r["omega"][0]))
    print("large_mixed FP8 ris: TDA %d it %.2f s, Casida %d it %.2f s (BF16 ris: %d / %d)"
          % (tf["stats"]["n_iter"], tf["stats"]["t_total_s"], rf["stats"]["n_iter"], rf["stats"]["t_total_s"],
             t["stats"]["n_iter"], r["stats"]["n_iter"]))
    # diag: converges, same answer, no fewer outer iterations than rid
    assert rd["status"] == api.OK, rd["stats"]
    assert r["stats"]["n_iter"] <= rd["stats"]["n_iter"]
    assert np.max(np.abs(rd["omega"] - r["omega"])) < 1e-5
    # FP8 ris factors in the preconditioner: the converged answer does not move
    assert tf["status"] == api.OK and rf["status"] == api.OK
    assert tf["stats"]["max_resid_certified"] < 1e-5 and rf["stats"]["max_resid_certified"] < 1e-5
    assert np.max(np.abs(tf["omega"] - t["omega"])) < 1e-5
    assert np.max(np.abs(rf["omega"] - r["omega"])) < 1e-5
    # the oracle's FP64 certification of every converged vector
    d = O.delta(meta["eps_occ"], meta["eps_vir"])
    a_x, c_J = meta["a_x"], meta["coulomb_factor"]
    AX = O.tda_from_parts(d, X, J[:k], K1[:k], a_x, c_J)
    om = np.asarray(t["omega"])
    res_t = np.linalg.norm(AX - om[:, None] * X, axis=1) / np.linalg.norm(X, axis=1)
    rq_t = np.sum(X * AX, axis=1) / np.sum(X * X, axis=1)
    PU, _ = O.pair_from_parts(d, U, J[k:2 * k], K1[k:2 * k], K2[k:2 * k], a_x, c_J)
    _, MW = O.pair_from_parts(d, W, J[2 * k:], K1[2 * k:], K2[2 * k:], a_x, c_J)
    Om = np.asarray(r["omega"])
    res_r = np.sqrt(np.sum((PU - Om[:, None] * W) ** 2, axis=1) + np.sum((MW - Om[:, None] * U) ** 2, axis=1))
    rq_r = np.sqrt(np.sum(U * PU, axis=1) * np.sum(W * MW, axis=1)) / np.sum(U * W, axis=1)
    print("large_mixed oracle FP64 certification: TDA max |r| %.3e, max |omega - x^T A x| %.3e Ha; "
          "Casida max |r| %.3e, max |Omega - Rayleigh| %.3e Ha"
          % (res_t.max(), np.max(np.abs(om - rq_t)), res_r.max(), np.max(np.abs(Om - rq_r))))
    assert np.all(res_t < 1.2e-5), res_t
    assert np.all(res_r < 1.2e-5), res_r
    assert np.max(np.abs(om - rq_t)) < 1e-5
    assert np.max(np.abs(Om - rq_r)) < 1e-5
