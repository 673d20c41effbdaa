"""FP8 (e4m3) ris factors with one scale per auxiliary row (the precision
growth step of the rid preconditioner, Eq. TDDFT-ris_approx): through the C ABI.

  * the ris products (T_A X and the pair (T_A+T_B)X, (T_A-T_B)X) with the
    exchange contractions in kind::f8f6f4 against the oracle's FP64 ris
    products: 1e-2 relative to the largest element (e4m3 keeps three
    mantissa bits, so a factor element is rounded by up to 2^-4 of itself;
    the products average those errors: 4e-4 to 4.3e-3 measured on GB300)
    -- a preconditioner only;
  * the preconditioner cannot move the converged answer: TDA, Casida and
    alpha(omega) solved with rid on FP8 ris factors match the oracle's dense
    results at the mixed tolerances (1e-5 Ha; alpha element by element, the
    tensor-core rule of tests/parity.py), on three shapes including ragged tiles and
    n_vir not a multiple of 16;
  * on the medium workload the FP8-ris Casida energies match the oracle's
    golden values to 1e-5 Ha and its outer iterations are printed beside the
    BF16-ris and diag counts.
"""
import json
import os

import numpy as np
import pytest

from oracle import dense as D
from oracle import operators as O
from synth.generator import dipoles, make_config, make_problem
from tests.parity import FLOOR_TC, alpha_excess

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "tda_small": lambda: make_config("tda_small"),
    "ragged": lambda: make_problem(3, 7, 5, 9, seeds=(30, 31, 32)),
    "odd": lambda: make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07),
}


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request, api):
    p = PROBLEMS[request.param]()
    s = api.Solver.from_problem(p)
    yield request.param, p, s
    s.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_fp8_ris_products(case, api):
    name, p, s = case
    T = O.ris_operator(p)
    for m in (1, 5, 23):
        X = np.random.default_rng(50 + m).standard_normal((m, p.n_ov))
        e = _rel(s.apply(2, X, precision=api.MIXED, tensor_cores=2), T.tda(X))
        tp, tm = s.apply(3, X, precision=api.MIXED, tensor_cores=2)
        rp, rm = T.apb_amb(X)
        ep, em = _rel(tp, rp), _rel(tm, rm)
        print("\n%s m=%d FP8 ris products: rel err %.3g (T), %.3g (T+), %.3g (T-)" % (name, m, e, ep, em))
        assert e < 1e-2 and ep < 1e-2 and em < 1e-2


def test_fp8_ris_solves_match_dense(case, api):
    name, p, s = case
    A, B = O.dense_A_B(p.eps_occ, p.eps_vir, O.eri_from_factors(p.extra["L_full"]), p.a_x, p.coulomb_factor)
    k = min(5, p.n_ov - 1)
    o = api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1, ris_fp8=1)
    r = s.solve_tda(o, want_vectors=False)
    assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.tda(A, k)[0])) < 1e-5
    r = s.solve_rpa(o, want_vectors=False)
    assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.casida(A, B, k)[0])) < 1e-5
    mu = dipoles(3, 3, p.n_ov)
    om = [0.0, 0.05, 0.1]
    r = s.solve_polar(api.default_opts(precond=api.RID, precision=api.MIXED, tensor_cores=1, ris_fp8=1), mu, om)
    assert r["status"] == api.OK and alpha_excess(r["alpha"], D.polar(A, B, mu, om), 1e-5, FLOOR_TC) <= 1.0


def test_fp8_needs_tensor_cores(api):
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    try:
        with pytest.raises(api.TddftError) as e:
            s.solve_tda(api.default_opts(n_states=3, precision=api.MIXED, ris_fp8=1))
        assert e.value.status == api.ERR_ARG
    finally:
        s.close()


def test_fp8_ris_medium(api):
    with open(os.path.join(os.path.dirname(__file__), "golden", "rpa_polar_medium.json")) as f:
        gold = json.load(f)
    p = make_config("rpa_polar_medium")
    s = api.Solver.from_problem(p, precisions=2, dtype=api.F32)
    try:
        it = {}
        for name, kw in (("fp8", dict(precond=api.RID, ris_fp8=1)), ("bf16", dict(precond=api.RID)),
                         ("diag", dict(precond=api.DIAG))):
            o = api.default_opts(n_states=10, precision=api.MIXED, tensor_cores=1, **kw)
            r = s.solve_rpa(o, want_vectors=False)
            assert r["status"] == api.OK, name
            assert np.max(np.abs(r["omega"] - np.array(gold["rpa"]["omega"]))) < 1e-5, name
            it[name] = r["stats"]["n_iter"]
        print("\nmedium Casida outer iterations: FP8 ris %d, BF16 ris %d, diag %d (oracle rid %d)"
              % (it["fp8"], it["bf16"], it["diag"], gold["rpa"]["n_iter"]))
        assert it["fp8"] <= it["diag"]
    finally:
        s.close()
