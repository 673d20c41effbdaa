"""GPU parity of the variant terms of Eq. hessian: a second exchange factor set
with weight b_x (the long-range exchange of a range-separated hybrid) and a
low-rank response kernel sum_g w_g F^g_ia F^g_jb in place of f^xc.

Tolerances as for the base operator: products 1e-11 relative (PLAIN), 2e-5
(MIXED, FP32 SIMT), 2e-6 (MIXED, tcgen05 FP16 hi+lo); energies 1e-6 Ha (PLAIN)
/ 1e-5 Ha (MIXED); polarizabilities 1e-6 / 1e-5 relative, element by element
with the floor of tests/parity.py.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import dense as D
from oracle import operators as O
from synth.generator import dipoles, make_config, make_problem, with_variant_terms
from tests.parity import FLOOR, FLOOR_TC, alpha_excess

pytestmark = pytest.mark.gpu

OMEGAS = [0.0, 0.05]


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


PROBLEMS = {
    # hybrid with both terms
    "small_lr_kernel": lambda: with_variant_terms(make_config("tda_small"), 90, n_aux_lr=60, b_x=0.75,
                                                  n_kernel=30),
    # ragged tiles (n_vir = 33) for the tensor-core path
    "odd_lr_kernel": lambda: with_variant_terms(make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07),
                                                91, n_aux_lr=25, b_x=0.5, n_kernel=12),
    # no exchange in the base set: all exchange from the second set
    "lr_only": lambda: with_variant_terms(make_problem(10, 40, 200, 90, seeds=(0, 1, 2), a_x=0.0), 92,
                                          n_aux_lr=80, b_x=1.0),
    # kernel only
    "kernel_only": lambda: with_variant_terms(make_config("tda_small"), 93, n_kernel=20),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request, api):
    p = PROBLEMS[request.param]()
    s = api.Solver.from_problem(p)
    yield request.param, p, s
    s.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_variant_products(case, api):
    name, p, s = case
    X = np.random.default_rng(17).standard_normal((6, p.n_ov))
    op = O.exact_operator(p)
    rt = op.tda(X)
    rp, rm = op.apb_amb(X)
    assert _rel(s.apply(0, X), rt) < 1e-11
    gp, gm = s.apply(1, X)
    assert _rel(gp, rp) < 1e-11 and _rel(gm, rm) < 1e-11
    assert _rel(s.apply(0, X, precision=api.MIXED), rt) < 2e-5
    gp, gm = s.apply(1, X, precision=api.MIXED)
    assert _rel(gp, rp) < 2e-5 and _rel(gm, rm) < 2e-5
    assert _rel(s.apply(0, X, precision=api.MIXED, tensor_cores=True), rt) < 2e-6
    gp, gm = s.apply(1, X, precision=api.MIXED, tensor_cores=True)
    assert _rel(gp, rp) < 2e-6 and _rel(gm, rm) < 2e-6
    # the variant terms are really applied: the base operator differs
    base = O.Operator(p.eps_occ, p.eps_vir, p.L_ov, p.L_oo, p.L_ov, p.L_vv, p.a_x, p.coulomb_factor)
    assert _rel(base.apb_amb(X)[0], rp) > 1e-3


@pytest.mark.parametrize("mode", ["plain", "mixed_tc"])
def test_variant_solves(case, api, mode):
    name, p, s = case
    A, B = O.dense_exact_A_B(p)
    k = 5
    kw = dict(precond=api.RID, max_iter=100)
    if mode == "mixed_tc":
        kw.update(precision=api.MIXED, tensor_cores=1)
    tol_e = 1e-6 if mode == "plain" else 1e-5
    r = s.solve_tda(api.default_opts(n_states=k, **kw), want_vectors=False)
    assert r["status"] == api.OK
    assert np.max(np.abs(r["omega"] - D.tda(A, k)[0])) < tol_e
    r = s.solve_rpa(api.default_opts(n_states=k, **kw), want_vectors=False)
    assert r["status"] == api.OK
    assert np.max(np.abs(r["omega"] - D.casida(A, B, k)[0])) < tol_e
    mu = dipoles(5, 2, p.n_ov)
    r = s.solve_polar(api.default_opts(**kw), mu, OMEGAS)
    assert r["status"] == api.OK
    ref = D.polar(A, B, mu, OMEGAS)
    assert alpha_excess(r["alpha"], ref, tol_e, FLOOR_TC if mode == "mixed_tc" else FLOOR) <= 1.0


def test_variant_arguments(api):
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    try:
        q = with_variant_terms(p, 94, n_aux_lr=8, b_x=0.5, n_kernel=4)
        lr, ker = q.extra["exchange_lr"], q.extra["kernel"]
        s.add_exchange(lr["b_x"], lr["M_oo"], lr["M_ov"], lr["M_vv"])
        with pytest.raises(api.TddftError) as e:     # only one second set
            s.add_exchange(lr["b_x"], lr["M_oo"], lr["M_ov"], lr["M_vv"])
        assert e.value.status == api.ERR_ARG
        w = ker["w"].copy()
        w[1] = np.nan
        with pytest.raises(api.TddftError) as e:
            s.add_kernel(w, ker["F_ov"])
        assert e.value.status == api.ERR_ARG
        F = ker["F_ov"].copy()
        F[0, 0, 0] = np.inf
        with pytest.raises(api.TddftError) as e:
            s.add_kernel(ker["w"], F)
        assert e.value.status == api.ERR_INDEFINITE
        s.add_kernel(ker["w"], ker["F_ov"])
        # the allocation-free product does not apply the variant terms: refused
        import torch
        X = torch.zeros((1, p.n_ov), dtype=torch.float64, device="cuda")
        out = torch.empty_like(X)
        st = api.lib().tddft_apply_noalloc(s.h, 0, api.PLAIN, C.c_void_p(X.data_ptr()), 1,
                                           C.c_void_p(out.data_ptr()), None)
        assert st == api.ERR_ARG
        assert api.lib().tddft_add_exchange(s.h, 0.5, 0, None, None, None, 0, 0) == api.ERR_ARG
    finally:
        s.close()
