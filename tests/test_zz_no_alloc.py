"""tddft_apply_noalloc: the operator product for callers that cannot allocate
device memory at call time (another runtime owns the pool, a real-time loop, a
context where allocation calls are not allowed).  Its intermediates live in a
64 MiB array the library declares statically.  This file is collected last so a
run that stops at the first failure has already run every other test.

The check: through the C ABI, two calls in a row of the no-allocation entry
point give the same products as tddft_apply (the allocating entry point)
within the tolerances the other GPU tests use (FP64: 1e-11 relative, FP32:
2e-5 relative); the second call also shows that what the first call left in
the shared array does not leak into the next result."""
import ctypes as C

import numpy as np
import pytest

from synth.generator import make_config

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_noalloc_matches_apply_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api

    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    try:
        lib = api.lib()
        for kind in (0, 1, 2, 3):
            for prec, tol in ((api.PLAIN, 1e-11), (api.MIXED, 2e-5)):
                for call, m in enumerate((7, 3)):
                    X = np.random.default_rng(10 * kind + call).standard_normal((m, p.n_ov))
                    ref = s.apply(kind, X, precision=prec)
                    ref0, ref1 = (ref if kind in (1, 3) else (ref, None))
                    Xd = torch.from_numpy(X).cuda()
                    o0 = torch.full_like(Xd, float("nan"))
                    o1 = torch.full_like(Xd, float("nan")) if kind in (1, 3) else None
                    torch.cuda.synchronize()   # inputs ready before the context's stream reads them
                    st = lib.tddft_apply_noalloc(s.h, kind, prec, C.c_void_p(Xd.data_ptr()), m,
                                                 C.c_void_p(o0.data_ptr()),
                                                 C.c_void_p(o1.data_ptr()) if o1 is not None else None)
                    assert st == api.OK, lib.tddft_last_error(s.h)
                    torch.cuda.synchronize()
                    assert _rel(o0.cpu().numpy(), ref0) < tol, (kind, prec, call)
                    if o1 is not None:
                        assert _rel(o1.cpu().numpy(), ref1) < tol, (kind, prec, call)
        # sizes beyond the static scratch are refused with a clear error
        big = torch.zeros((40000, p.n_ov), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(big)
        torch.cuda.synchronize()
        st = lib.tddft_apply_noalloc(s.h, 0, api.PLAIN, C.c_void_p(big.data_ptr()), big.shape[0],
                                     C.c_void_p(out.data_ptr()), None)
        assert st == api.ERR_ARG and b"static scratch" in lib.tddft_last_error(s.h)
    finally:
        s.close()
