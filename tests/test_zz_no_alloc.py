"""tddft_apply_noalloc: the operator product for callers that cannot allocate
device memory at call time (another runtime owns the pool, a real-time loop, a
context where allocation calls are not allowed).  Its intermediates live in a
64 MiB array the library declares statically.  This file is collected last so a
run that stops at the first failure has already run every other test.

The checks, all through the C ABI:
  * two calls in a row of the no-allocation entry point give the products of
    the FP64 CPU oracle (Eq. hessian over the density-fitted factors) within
    the tolerances of the other GPU parity tests (FP64: 1e-11 relative; FP32
    exact factors: 2e-5; BF16 ris factors: 2e-2), and the products of
    tddft_apply (the allocating entry point) to the same tolerances;
  * on the medium workload (n_aux = 2000) the intermediates of 7 vectors need
    about fifty P-chunks of the static array, so the chunk offsets and the
    accumulation of later chunks into the first one are exercised too;
  * what one call leaves in the shared array does not leak into the next
    result (the second call of every pair uses other vectors and sizes);
  * the calls take nothing from the device's stream-ordered memory pool (its
    use and high-water mark are unchanged) and the device's free memory is
    unchanged;
  * sizes beyond the static array are refused with TDDFT_ERR_ARG.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import operators as O
from synth.generator import make_config

pytestmark = pytest.mark.gpu

TOL = {(0, "plain"): 1e-11, (1, "plain"): 1e-11, (2, "plain"): 1e-11, (3, "plain"): 1e-11,
       (0, "mixed"): 2e-5, (1, "mixed"): 2e-5, (2, "mixed"): 2e-2, (3, "mixed"): 2e-2}


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _oracle(p, kind, X):
    op = O.exact_operator(p) if kind < 2 else O.ris_operator(p)
    return op.apb_amb(X) if kind in (1, 3) else (op.tda(X), None)


def _check_problem(api, torch, p, sizes, kinds=(0, 1, 2, 3)):
    s = api.Solver.from_problem(p)
    lib = api.lib()
    try:
        # every device buffer of the test is made before the pool is watched
        cases = []
        for kind in kinds:
            for prec in (api.PLAIN, api.MIXED):
                for call, m in enumerate(sizes):
                    X = np.random.default_rng(100 * kind + 10 * prec + call).standard_normal((m, p.n_ov))
                    Xd = torch.from_numpy(X).cuda()
                    o0 = torch.full_like(Xd, float("nan"))
                    o1 = torch.full_like(Xd, float("nan")) if kind in (1, 3) else None
                    cases.append((kind, prec, call, X, Xd, o0, o1))
        torch.cuda.synchronize()   # inputs complete before the context's stream reads them

        def run_all():
            for kind, prec, call, X, Xd, o0, o1 in cases:
                st = lib.tddft_apply_noalloc(s.h, kind, prec, C.c_void_p(Xd.data_ptr()), X.shape[0],
                                             C.c_void_p(o0.data_ptr()),
                                             C.c_void_p(o1.data_ptr()) if o1 is not None else None)
                assert st == api.OK, lib.tddft_last_error(s.h)
            torch.cuda.synchronize()

        # a first pass loads every kernel the entry point launches (the driver
        # loads kernel code lazily, on first launch); the second pass is watched
        run_all()
        free0 = torch.cuda.mem_get_info()[0]
        used0, _ = api.pool_usage(torch.cuda.current_device(), reset_high=True)
        run_all()
        used1, high1 = api.pool_usage(torch.cuda.current_device())
        free1 = torch.cuda.mem_get_info()[0]
        assert used1 == used0 and high1 <= used0, (used0, used1, high1)
        assert free1 == free0, (free0, free1)
        for kind, prec, call, X, Xd, o0, o1 in cases:
            tol = TOL[(kind, "plain" if prec == api.PLAIN else "mixed")]
            ref0, ref1 = _oracle(p, kind, X)
            g0 = o0.cpu().numpy()
            assert _rel(g0, ref0) < tol, (kind, prec, call, _rel(g0, ref0))
            a = s.apply(kind, X, precision=prec)
            a0, a1 = a if kind in (1, 3) else (a, None)
            assert _rel(g0, a0) < tol, (kind, prec, call)
            if o1 is not None:
                g1 = o1.cpu().numpy()
                assert _rel(g1, ref1) < tol, (kind, prec, call, _rel(g1, ref1))
                assert _rel(g1, a1) < tol, (kind, prec, call)
    finally:
        s.close()


@pytest.fixture(scope="module")
def api_torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api
    return api, torch


def test_noalloc_matches_oracle_twice(api_torch):
    api, torch = api_torch
    _check_problem(api, torch, make_config("tda_small"), (7, 3))


def test_noalloc_many_chunks_match_oracle(api_torch):
    """Medium workload: 7 vectors in PLAIN need ~1.5 MB of intermediates per
    auxiliary row, so the 64 MiB array takes about 40 of the 2000 rows at a
    time; the second call (2 vectors) chunks differently."""
    api, torch = api_torch
    _check_problem(api, torch, make_config("rpa_polar_medium"), (7, 2), kinds=(0, 1, 3))


def test_noalloc_refuses_sizes_beyond_the_array(api_torch):
    api, torch = api_torch
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    lib = api.lib()
    try:
        big = torch.zeros((40000, p.n_ov), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(big)
        torch.cuda.synchronize()
        st = lib.tddft_apply_noalloc(s.h, 0, api.PLAIN, C.c_void_p(big.data_ptr()), big.shape[0],
                                     C.c_void_p(out.data_ptr()), None)
        assert st == api.ERR_ARG and b"static scratch" in lib.tddft_last_error(s.h)
    finally:
        s.close()
