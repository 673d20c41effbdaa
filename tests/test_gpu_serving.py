"""Concurrent serving through tddft_submit / tddft_poll.

Several contexts (different problem sizes, each with the resident factors and
the stream the library created for it) take TDA, Casida and polarizability
requests at once; each context's worker runs its queue on its own stream, so
requests of different contexts overlap on the device.  Every result must be
the same alone and in the mix: the kernels are deterministic (fixed-order
reductions, no atomics in the sums), so the comparison is to 1e-12 relative.
Every served result is also checked against the oracle's dense results for
its problem (LAPACK on the explicitly built A and B of Eq. hessian: Eq. TDA,
Eq. Casida, Eq. TDDFT_polar), at the tolerances of the other parity tests.
"""
import time

import numpy as np
import pytest

from oracle import dense as D
from oracle import operators as O
from synth.generator import dipoles, make_config, make_problem
from tests.parity import alpha_excess

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


def _requests(api, p):
    mu = dipoles(77, 2, p.n_ov)
    k = min(4, p.n_ov)
    return [
        (0, api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1), None, None),
        (1, api.default_opts(n_states=k, precond=api.RID), None, None),
        (2, api.default_opts(precond=api.RID, precision=api.MIXED), mu, [0.0, 0.07]),
        (1, api.default_opts(n_states=k, precond=api.DIAG, precision=api.MIXED, max_iter=200), None, None),
    ]


_DENSE = {}


def _dense(p):
    key = id(p)
    if key not in _DENSE:
        _DENSE[key] = (p, O.dense_A_B(p.eps_occ, p.eps_vir, O.eri_from_factors(p.extra["L_full"]), p.a_x,
                                      p.coulomb_factor))
    return _DENSE[key][1]


def _check_vs_oracle(api, p, kind, o, mu, om, r, key):
    """A converged served result against the dense oracle results of its problem."""
    if r["status"] != api.OK:
        return
    A, B = _dense(p)
    tol = 1e-6 if o.precision == api.PLAIN else 1e-5
    if kind == 0:
        ref = D.tda(A, o.n_states)[0]
        assert np.max(np.abs(r["omega"] - ref)) < tol, (key, np.max(np.abs(r["omega"] - ref)))
    elif kind == 1:
        ref = D.casida(A, B, o.n_states)[0]
        assert np.max(np.abs(r["omega"] - ref)) < tol, (key, np.max(np.abs(r["omega"] - ref)))
    else:
        ref = D.polar(A, B, mu, om)
        assert alpha_excess(r["alpha"], ref, tol) <= 1.0, (key, alpha_excess(r["alpha"], ref, tol))


def _run(solvers, reqs, together):
    """Submit the requests (all contexts at once when `together`, else one
    request at a time) and return every result, in request order."""
    out = {}
    pending = []
    for ci, (s, rl) in enumerate(zip(solvers, reqs)):
        for ri, (kind, o, mu, om) in enumerate(rl):
            t = s.submit(kind, o, mu=mu, omegas=om)
            if together:
                pending.append((ci, ri, s, t))
            else:
                out[(ci, ri)] = _wait(s, t)
    for ci, ri, s, t in pending:
        out[(ci, ri)] = _wait(s, t)
    return out


def _wait(s, t, limit_s=120.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = s.poll(t, timeout_ms=100)
        if r is not None:
            return r
    raise AssertionError("request did not finish within %.0f s" % limit_s)


def test_results_same_alone_and_in_the_mix(api):
    problems = [make_config("tda_small"), make_problem(3, 7, 5, 9, seeds=(30, 31, 32)),
                make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07)]
    solvers = [api.Solver.from_problem(p) for p in problems]
    try:
        reqs = [_requests(api, p) for p in problems]
        alone = _run(solvers, reqs, together=False)
        mixed = _run(solvers, reqs, together=True)
        assert set(alone) == set(mixed)
        for key in alone:
            a, b = alone[key], mixed[key]
            assert a["status"] == b["status"], (key, a["status"], b["status"])
            assert a["status"] in (api.OK, api.ERR_NOCONV), (key, a.get("error"))
            if key[1] != 3:   # every rid request converges (request 3 is the diag one)
                assert a["status"] == api.OK, (key, a.get("error"))
            for field in ("omega", "alpha"):
                if field in a and a[field] is not None:
                    x, y = np.asarray(a[field]), np.asarray(b[field])
                    assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(x))), (key, field)
            kind, o, mu, om = reqs[key[0]][key[1]]
            _check_vs_oracle(api, problems[key[0]], kind, o, mu, om, b, key)
    finally:
        for s in solvers:
            s.close()


# -- the server: admission of requests that bring their own problem -----------

def _server_requests(api, problems):
    out = []
    for pi, p in enumerate(problems):
        for ri, (kind, o, mu, om) in enumerate(_requests(api, p)):
            out.append(((pi, ri), p, kind, o, mu, om))
    return out


def _server_wait(srv, t, limit_s=180.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        r = srv.poll(t, timeout_ms=100)
        if r is not None:
            return r
    raise AssertionError("server request did not finish within %.0f s" % limit_s)


def _same(api, a, b, key):
    assert a["status"] == b["status"], (key, a["status"], b["status"], b.get("error"))
    for field in ("omega", "alpha"):
        if field in a and a[field] is not None:
            x, y = np.asarray(a[field]), np.asarray(b[field])
            assert np.max(np.abs(x - y)) <= 1e-12 * max(1.0, np.max(np.abs(x))), (key, field)


def test_server_admits_by_budget_and_matches_alone(api):
    """Twelve requests, each bringing its problem, queued at once on a server of
    four slots whose budget holds about two requests' charges: the requests
    start in submission order, the running charges never exceed the budget,
    some requests run at the same time, and every result equals the one the
    same request gives alone on its own context."""
    problems = [make_config("tda_small"), make_problem(3, 7, 5, 9, seeds=(30, 31, 32)),
                make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07)]
    solvers = [api.Solver.from_problem(p) for p in problems]
    try:
        alone = _run(solvers, [_requests(api, p) for p in problems], together=False)
    finally:
        for s in solvers:
            s.close()
    reqs = _server_requests(api, problems)
    charges = []
    for key, p, kind, o, mu, om in reqs:
        d = api._problem_args(**api._problem_kw(p))[0]
        f, w = api.estimate_bytes(d, kind, o, mu.shape[0] if mu is not None else 0,
                                  len(om) if om is not None else 0)
        charges.append(f + w)
    budget_gb = 2.2 * max(charges) / 1e9
    srv = api.Server(hbm_budget_gb=budget_gb, max_active=4)
    try:
        tickets = [(key, srv.submit(kind, o, problem=p, mu=mu, omegas=om)) for key, p, kind, o, mu, om in reqs]
        res = {key: _server_wait(srv, t) for key, t in tickets}
        info = srv.info()
    finally:
        srv.close()
    for key in alone:
        _same(api, alone[key], res[key], key)
    for key, p, kind, o, mu, om in reqs:
        _check_vs_oracle(api, p, kind, o, mu, om, res[key], key)
    order = [res[key] for key, _ in tickets]
    starts = [r["t_start_s"] for r in order]
    assert all(a <= b for a, b in zip(starts, starts[1:])), "admission is first in, first out"
    for i, r in enumerate(order):
        assert r["charged_bytes"] == charges[i]
        assert r["t_submit_s"] <= r["t_start_s"] <= r["t_end_s"]
    budget = info["budget_bytes"]
    most = 0
    for r in order:   # charges and slots in use at each admission instant
        live = [q for q in order if q["t_start_s"] <= r["t_start_s"] < q["t_end_s"]]
        assert sum(q["charged_bytes"] for q in live) <= budget
        assert len(live) <= 4
        most = max(most, len(live))
    assert most >= 2, "no two requests ran at the same time"
    assert info["peak_in_use_bytes"] <= budget
    assert info["in_use_bytes"] == 0 and info["active"] == 0 and info["queued"] == 0
    assert info["completed"] == len(reqs)
    print("\nserver: %d requests, budget %.3f GB, at most %d at once, peak charge %.3f GB, "
          "pool high-water %.3f GB above its use at creation" %
          (len(reqs), budget / 1e9, most, info["peak_in_use_bytes"] / 1e9,
           (info["pool_high_bytes"] - info["pool_used_at_create_bytes"]) / 1e9))


def test_server_charge_bounds_the_memory_a_request_takes(api):
    """One request at a time: the pool's high-water mark above its use at
    server creation stays below the request's charge (factor copies + work)."""
    p = make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07)
    for kind, o, mu, om in _requests(api, p):
        srv = api.Server(max_active=1)
        try:
            r = _server_wait(srv, srv.submit(kind, o, problem=p, mu=mu, omegas=om))
            info = srv.info()
        finally:
            srv.close()
        assert r["status"] in (api.OK, api.ERR_NOCONV), r.get("error")
        used = info["pool_high_bytes"] - info["pool_used_at_create_bytes"]
        assert used <= r["charged_bytes"], (kind, used, r["charged_bytes"])


def test_server_refuses_a_request_larger_than_its_budget(api):
    p = make_config("tda_small")
    srv = api.Server(hbm_budget_gb=0.01, max_active=2)
    try:
        with pytest.raises(api.TddftError) as e:
            srv.submit(0, api.default_opts(n_states=5), problem=p)
        assert e.value.status == api.ERR_OOM
        assert srv.info()["queued"] == 0
    finally:
        srv.close()


def test_server_on_resident_contexts(api):
    """Requests naming existing contexts reuse their resident factors and give
    the results of direct solves on those contexts."""
    problems = [make_config("tda_small"), make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07)]
    solvers = [api.Solver.from_problem(p) for p in problems]
    srv = api.Server(max_active=3)
    try:
        direct, tickets = {}, []
        for ci, (s, p) in enumerate(zip(solvers, problems)):
            for ri, (kind, o, mu, om) in enumerate(_requests(api, p)):
                tickets.append(((ci, ri), srv.submit(kind, o, solver=s, mu=mu, omegas=om)))
        res = {key: _server_wait(srv, t) for key, t in tickets}
        for ci, (s, p) in enumerate(zip(solvers, problems)):
            for ri, (kind, o, mu, om) in enumerate(_requests(api, p)):
                if kind == 0:
                    d = s.solve_tda(o, want_vectors=False)
                elif kind == 1:
                    d = s.solve_rpa(o, want_vectors=False)
                else:
                    d = s.solve_polar(o, mu, om)
                _same(api, d, res[(ci, ri)], (ci, ri))
                _check_vs_oracle(api, p, kind, o, mu, om, res[(ci, ri)], (ci, ri))
                # resident factors: only the work buffers are charged
                w = api.estimate_bytes(s.desc, kind, o, mu.shape[0] if mu is not None else 0,
                                       len(om) if om is not None else 0)[1]
                assert res[(ci, ri)]["charged_bytes"] == w
    finally:
        srv.close()
        for s in solvers:
            s.close()
