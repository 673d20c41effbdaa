"""Error behaviour of the C ABI on a GPU: bad arguments, budget overflow,
non-finite inputs, indefinite Hessians, iteration exhaustion, and the
asynchronous request queue (submit / poll with a bounded wait).  Every failure
is made on the host side (inputs or options); none faults or hangs the GPU."""
import ctypes as C
import time

import numpy as np
import pytest

from oracle import dense as D
from oracle import operators as O
from synth.generator import dipoles, make_config, make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


@pytest.fixture(scope="module")
def small(api):
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    yield p, s
    s.close()


def test_bad_options(api, small):
    p, s = small
    for kw in ({"n_states": 0}, {"precond": 7}, {"tol": -1.0}, {"precision": 5},
               {"tensor_cores": 1, "precision": 0}, {"n_states": 65}):
        with pytest.raises(api.TddftError) as e:
            s.solve_tda(api.default_opts(**kw))
        assert e.value.status == api.ERR_ARG


def test_budget_overflow_is_refused(api):
    p = make_config("tda_small")
    with pytest.raises(api.TddftError) as e:
        api.Solver.from_problem(p, hbm_budget_gb=1e-6)
    assert e.value.status == api.ERR_OOM


def test_non_finite_factors_are_refused(api):
    p = make_config("tda_small")
    p.L_vv[3, 1, 2] = np.nan
    with pytest.raises(api.TddftError) as e:
        api.Solver.from_problem(p)
    assert e.value.status == api.ERR_INDEFINITE


def test_unsorted_energies_are_refused(api):
    p = make_config("tda_small")
    p.eps_vir = p.eps_vir[::-1].copy()
    with pytest.raises(api.TddftError) as e:
        api.Solver.from_problem(p)
    assert e.value.status == api.ERR_ARG


def test_indefinite_casida_is_reported(api):
    """The literal 0.3 amplitude gives lambda_min(A-B) < 0: no real Casida solution."""
    p = make_config("tda_small", amplitude=0.3)
    s = api.Solver.from_problem(p)
    try:
        with pytest.raises(api.TddftError) as e:
            s.solve_rpa(api.default_opts(n_states=5, precond=api.DIAG))
        assert e.value.status == api.ERR_INDEFINITE
        # the Hermitian TDA problem is still well posed
        r = s.solve_tda(api.default_opts(n_states=5, precond=api.RID, max_iter=100))
        assert r["status"] == api.OK
        A, _ = O.dense_A_B(p.eps_occ, p.eps_vir, O.eri_from_factors(p.extra["L_full"]), p.a_x,
                           p.coulomb_factor)
        assert np.max(np.abs(r["omega"] - D.tda(A, 5)[0])) < 1e-6
    finally:
        s.close()


def test_iteration_exhaustion_returns_partial_results(api, small):
    p, s = small
    r = s.solve_tda(api.default_opts(n_states=5, precond=api.DIAG, max_iter=2))
    assert r["status"] == api.ERR_NOCONV
    assert np.all(np.isfinite(r["omega"])) and np.all(r["resid"] > 1e-5)
    assert r["stats"]["n_iter"] == 2 and r["stats"]["converged"] == 0


def test_submit_poll_matches_direct(api, small):
    p, s = small
    o = api.default_opts(n_states=5, precond=api.RID)
    direct = s.solve_tda(o)["omega"]
    mu = dipoles(3, 3, p.n_ov)
    t1 = s.submit(0, o)
    t2 = s.submit(2, api.default_opts(precond=api.RID), mu=mu, omegas=[0.0, 0.05])
    t0 = time.time()
    res = {}
    while len(res) < 2 and time.time() - t0 < 60:
        for t in (t1, t2):
            if t not in res:
                r = s.poll(t, timeout_ms=50)
                if r is not None:
                    res[t] = r
    assert len(res) == 2
    assert res[t1]["status"] == api.OK and np.allclose(res[t1]["omega"], direct, atol=1e-10)
    direct_a = s.solve_polar(api.default_opts(precond=api.RID), mu, [0.0, 0.05])["alpha"]
    assert res[t2]["status"] == api.OK and np.allclose(res[t2]["alpha"], direct_a, rtol=1e-10)


def test_poll_times_out_without_blocking(api, small):
    p, s = small
    t = s.submit(1, api.default_opts(n_states=5, precond=api.RID))
    t0 = time.time()
    first = s.poll(t, timeout_ms=1)      # most likely still running
    assert time.time() - t0 < 5.0
    while first is None:
        first = s.poll(t, timeout_ms=100)
    assert first["status"] == api.OK


def test_unknown_ticket(api, small):
    p, s = small
    assert api.lib().tddft_poll(s.h, 123456789, 0) == api.ERR_ARG
