"""Concurrent serving through tddft_submit / tddft_poll.

Several contexts (different problem sizes, each with the resident factors and
the stream the library created for it) take TDA, Casida and polarizability
requests at once; each context's worker runs its queue on its own stream, so
requests of different contexts overlap on the device.  Every result must be
the same alone and in the mix: the kernels are deterministic (fixed-order
reductions, no atomics in the sums), so the comparison is to 1e-12 relative.
"""
import time

import numpy as np
import pytest

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


def _requests(api, p):
    mu = dipoles(77, 2, p.n_ov)
    k = min(4, p.n_ov)
    return [
        (0, api.default_opts(n_states=k, precond=api.RID, precision=api.MIXED, tensor_cores=1), None, None),
        (1, api.default_opts(n_states=k, precond=api.RID), None, None),
        (2, api.default_opts(precond=api.RID, precision=api.MIXED), mu, [0.0, 0.07]),
        (1, api.default_opts(n_states=k, precond=api.DIAG, precision=api.MIXED, max_iter=200), None, None),
    ]


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
    finally:
        for s in solvers:
            s.close()
