"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (see the design notes for the derivation):
  * operator products, PLAIN (FP64): 1e-11 relative to max |out| -- rounding order only;
  * operator products, MIXED exact (FP32 factors, FP32 accumulation): 2e-5 relative;
  * ris products, MIXED (BF16 factors): 2e-2 relative (preconditioner only);
  * exact products, MIXED on the tensor cores (every operand scaled by a power
    of two and split into FP16 hi + lo, three products, FP32 accumulation):
    2e-6 relative (FP32-level); ris products on the tensor cores: 2e-2;
  * excitation energies: 1e-6 Ha (PLAIN), 1e-5 Ha (MIXED);
  * polarizabilities: 1e-6 relative (PLAIN), 1e-5 relative (MIXED), element
    by element with the floor of tests/parity.py.
"""
import numpy as np
import pytest

from oracle import davidson as DV
from oracle import dense as D
from oracle import operators as O
from synth.generator import dipoles, make_config, make_problem
from tests.parity import FLOOR, FLOOR_TC, alpha_excess, alpha_report

pytestmark = pytest.mark.gpu

OMEGAS = [0.0, 0.05, 0.1]


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    from paper_2404_17133_gb300 import api as a
    return a


def _dense(p):
    A, B = O.dense_A_B(p.eps_occ, p.eps_vir, O.eri_from_factors(p.extra["L_full"]), p.a_x,
                       p.coulomb_factor)
    return A, B


PROBLEMS = {
    "tda_small": lambda: make_config("tda_small"),
    "ragged": lambda: make_problem(3, 7, 5, 9, seeds=(30, 31, 32)),
    "odd": lambda: make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request, api):
    p = PROBLEMS[request.param]()
    s = api.Solver.from_problem(p)
    yield request.param, p, s
    s.close()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_operator_products(case, api):
    name, p, s = case
    X = np.random.default_rng(7).standard_normal((5, p.n_ov))
    op, T = O.exact_operator(p), O.ris_operator(p)
    ref_tda = op.tda(X)
    ref_p, ref_m = op.apb_amb(X)
    rt = T.tda(X)
    rtp, rtm = T.apb_amb(X)
    assert _rel(s.apply(0, X), ref_tda) < 1e-11
    gp, gm = s.apply(1, X)
    assert _rel(gp, ref_p) < 1e-11 and _rel(gm, ref_m) < 1e-11
    assert _rel(s.apply(2, X), rt) < 1e-11
    gp, gm = s.apply(3, X)
    assert _rel(gp, rtp) < 1e-11 and _rel(gm, rtm) < 1e-11
    # mixed: FP32 exact, BF16 ris
    assert _rel(s.apply(0, X, precision=api.MIXED), ref_tda) < 2e-5
    gp, gm = s.apply(1, X, precision=api.MIXED)
    assert _rel(gp, ref_p) < 2e-5 and _rel(gm, ref_m) < 2e-5
    assert _rel(s.apply(2, X, precision=api.MIXED), rt) < 2e-2


def test_tensor_core_products(case, api):
    name, p, s = case
    op = O.exact_operator(p)
    for m in (1, 5, 23):
        X = np.random.default_rng(m).standard_normal((m, p.n_ov))
        e0 = _rel(s.apply(0, X, precision=api.MIXED, tensor_cores=True), op.tda(X))
        gp, gm = s.apply(1, X, precision=api.MIXED, tensor_cores=True)
        rp, rm = op.apb_amb(X)
        print("\n%s m=%d FP16 hi+lo tensor-core products: rel err %.2e (A), %.2e (A+B), %.2e (A-B)"
              % (name, m, e0, _rel(gp, rp), _rel(gm, rm)))
        assert e0 < 2e-6 and _rel(gp, rp) < 2e-6 and _rel(gm, rm) < 2e-6
        # ris operator on the tensor cores: one BF16 product (preconditioner only)
        T = O.ris_operator(p)
        assert _rel(s.apply(2, X, precision=api.MIXED, tensor_cores=True), T.tda(X)) < 2e-2
        tp, tm = s.apply(3, X, precision=api.MIXED, tensor_cores=True)
        rtp, rtm = T.apb_amb(X)
        assert _rel(tp, rtp) < 2e-2 and _rel(tm, rtm) < 2e-2


def test_tensor_core_products_scale_with_the_input(case, api):
    """Every FP16 operand carries a power of two chosen from its own range, so
    scaling the trial vectors by 2^k scales the products by exactly 2^k, and
    inputs scaled by 1e-10 or 1e10 keep FP32-accurate products (no overflow of
    the FP16 range, no loss to its subnormals)."""
    name, p, s = case
    X = np.random.default_rng(9).standard_normal((4, p.n_ov))
    base = s.apply(1, X, precision=api.MIXED, tensor_cores=True)
    for k in (-30, 37):
        sc = s.apply(1, X * 2.0 ** k, precision=api.MIXED, tensor_cores=True)
        for a, b in zip(sc, base):
            assert np.array_equal(a, b * 2.0 ** k), k
    op = O.exact_operator(p)
    for c in (1e-10, 1e10):
        gp, gm = s.apply(1, X * c, precision=api.MIXED, tensor_cores=True)
        rp, rm = op.apb_amb(X * c)
        assert _rel(gp, rp) < 2e-6 and _rel(gm, rm) < 2e-6, c


@pytest.mark.parametrize("shape", [(6, 600, 24, 30), (6, 300, 20, 45)])
def test_tensor_core_products_in_clusters(api, shape, monkeypatch):
    """Wide virtual spaces put the second contractions (N = n_vir) on two or
    three 256-column tiles and m n_occ rows on two or three 128-row tiles, so
    they run in 2 x 2 CTA clusters that share A and B tiles by multicast, with a
    padding N tile (n_vir = 600: three tiles) or a padding M tile (270 rows).
    The products match the oracle and equal, bit for bit, those of the paired
    and of the unclustered launches."""
    no, nv, na, m = shape
    p = make_problem(no, nv, na, 18, seeds=(60, 61, 62), amplitude=0.07)
    s = api.Solver.from_problem(p)
    try:
        X = np.random.default_rng(13).standard_normal((m, p.n_ov))
        op = O.exact_operator(p)
        rp, rm = op.apb_amb(X)
        rt = op.tda(X)
        out = {}
        for pairs, quads in (("1", "1"), ("1", "0"), ("0", "1")):
            monkeypatch.setenv("TDDFT_TC_CLUSTER", pairs)
            monkeypatch.setenv("TDDFT_TC_QUAD", quads)
            out[pairs + quads] = (s.apply(1, X, precision=api.MIXED, tensor_cores=True),
                                  s.apply(0, X, precision=api.MIXED, tensor_cores=True))
        (gp, gm), gt = out["11"]
        assert _rel(gp, rp) < 2e-6 and _rel(gm, rm) < 2e-6 and _rel(gt, rt) < 2e-6
        for other in ("10", "01"):
            (op_, om_), ot_ = out[other]
            assert np.array_equal(gp, op_) and np.array_equal(gm, om_) and np.array_equal(gt, ot_), other
    finally:
        s.close()


@pytest.mark.parametrize("pc", ["diag", "rid"])
@pytest.mark.parametrize("prec", ["plain", "mixed", "mixed_tc"])
def test_tda(case, api, pc, prec):
    name, p, s = case
    A, _ = _dense(p)
    k = min(5, p.n_ov - 1)
    ref_w, ref_X = D.tda(A, k)
    o = api.default_opts(n_states=k, precond=api.RID if pc == "rid" else api.DIAG,
                         precision=api.PLAIN if prec == "plain" else api.MIXED,
                         tensor_cores=int(prec == "mixed_tc"))
    r = s.solve_tda(o)
    tol = 1e-6 if prec == "plain" else 1e-5
    assert r["status"] == api.OK
    assert np.max(np.abs(r["omega"] - ref_w)) < tol
    assert np.max(r["resid"]) < 1e-5
    ov = np.abs(np.sum(r["X"] * ref_X, axis=1))
    assert np.all(ov > 1 - 1e-6)


@pytest.mark.parametrize("pc", ["diag", "rid"])
@pytest.mark.parametrize("prec", ["plain", "mixed", "mixed_tc"])
def test_rpa(case, api, pc, prec):
    name, p, s = case
    A, B = _dense(p)
    k = min(5, p.n_ov - 1)
    ref_w, ref_X, ref_Y = D.casida(A, B, k)
    o = api.default_opts(n_states=k, precond=api.RID if pc == "rid" else api.DIAG,
                         precision=api.PLAIN if prec == "plain" else api.MIXED,
                         tensor_cores=int(prec == "mixed_tc"))
    r = s.solve_rpa(o)
    tol = 1e-6 if prec == "plain" else 1e-5
    assert r["status"] == api.OK
    assert np.max(np.abs(r["omega"] - ref_w)) < tol
    X, Y = r["X"], r["Y"]
    assert np.allclose(np.sum(X * X, 1) - np.sum(Y * Y, 1), 1.0, atol=1e-6)
    ovl = np.abs(np.sum(X * ref_X, 1) + np.sum(Y * ref_Y, 1))
    assert np.all(ovl > 1 - 1e-5)


@pytest.mark.parametrize("pc", ["diag", "rid"])
@pytest.mark.parametrize("prec", ["plain", "mixed", "mixed_tc"])
def test_polar(case, api, pc, prec):
    name, p, s = case
    A, B = _dense(p)
    mu = dipoles(3, 3, p.n_ov)
    ref = D.polar(A, B, mu, OMEGAS)
    o = api.default_opts(precond=api.RID if pc == "rid" else api.DIAG,
                         precision=api.PLAIN if prec == "plain" else api.MIXED,
                         tensor_cores=int(prec == "mixed_tc"))
    r = s.solve_polar(o, mu, OMEGAS)
    tol = 1e-6 if prec == "plain" else 1e-5
    assert r["status"] == api.OK
    print("\n%s %s %s alpha: max abs err %.3g, max per-element rel err %.3g" %
          ((name, pc, prec) + alpha_report(r["alpha"], ref)))
    assert alpha_excess(r["alpha"], ref, tol, FLOOR_TC if prec == "mixed_tc" else FLOOR) <= 1.0


def test_iterations_match_oracle_and_rid_wins(api):
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    op, T = O.exact_operator(p), O.ris_operator(p)
    try:
        for pc, code in (("diag", api.DIAG), ("rid", api.RID)):
            ref = DV.solve_tda(p, op, T, 5, precond=pc)
            r = s.solve_tda(api.default_opts(n_states=5, precond=code))
            assert abs(r["stats"]["n_iter"] - ref.n_iter) <= 1, (pc, r["stats"]["n_iter"], ref.n_iter)
        it = {pc: s.solve_tda(api.default_opts(n_states=5, precond=c))["stats"]["n_iter"]
              for pc, c in (("diag", api.DIAG), ("rid", api.RID))}
        assert it["rid"] <= it["diag"]
        it = {pc: s.solve_rpa(api.default_opts(n_states=5, precond=c))["stats"]["n_iter"]
              for pc, c in (("diag", api.DIAG), ("rid", api.RID))}
        assert it["rid"] <= it["diag"]
    finally:
        s.close()


def test_zero_factors_give_delta(api):
    p = make_problem(4, 9, 3, 9, seeds=(50, 51, 52), amplitude=0.0, ris_noise=0.0)
    d = np.sort(O.delta(p.eps_occ, p.eps_vir))
    s = api.Solver.from_problem(p)
    try:
        for pc in (api.DIAG, api.RID):
            r = s.solve_tda(api.default_opts(n_states=4, precond=pc))
            assert np.allclose(r["omega"], d[:4], atol=1e-10)
            r = s.solve_rpa(api.default_opts(n_states=4, precond=pc))
            assert np.allclose(r["omega"], d[:4], atol=1e-10)
    finally:
        s.close()


def test_single_state_and_T_equal_A(api):
    p = make_config("tda_small")
    # ris factors = exact factors, every row used for exchange, no window: T = A
    L = p.extra["L_full"]
    no = p.n_occ
    s = api.Solver(p.n_occ, p.n_vir, p.eps_occ, p.eps_vir, p.L_oo, p.L_ov, p.L_vv,
                   p.L_oo, p.L_ov, p.L_vv, np.arange(p.n_aux, dtype=np.int32), a_x=p.a_x,
                   coulomb_factor=p.coulomb_factor, t_cut_ha=1e9)
    try:
        r = s.solve_tda(api.default_opts(n_states=1, precond=api.RID, guess_tol=1e-9))
        A, _ = _dense(p)
        assert r["stats"]["n_iter"] == 1
        assert abs(r["omega"][0] - np.linalg.eigvalsh(A)[0]) < 1e-8
    finally:
        s.close()


def test_contraction_profile(api):
    """CUDA-event timing of the K1 contraction: one record per launch, the
    records' flops add up to the totals, and the algorithmic bytes of a launch
    are those of its operands and result (hi+lo Z and L_vv, FP32 output)."""
    p = make_config("tda_small")
    s = api.Solver.from_problem(p)
    try:
        X = np.random.default_rng(3).standard_normal((4, p.n_ov))
        s.profile(True)
        s.apply(1, X, precision=api.MIXED, tensor_cores=True)
        tot = s.profile_read(0)
        ms, fl, by = s.profile_records(0)
        assert tot["launches"] == len(ms) >= 1
        assert abs(fl.sum() - tot["flops"]) <= 1e-9 * tot["flops"]
        assert abs(ms.sum() - tot["ms"]) <= 1e-6 * max(tot["ms"], 1e-9) and np.all(ms > 0)
        no, nv, na = p.n_occ, p.n_vir, p.n_aux
        M = 4 * no
        assert fl.sum() == 2.0 * M * nv * na * nv          # one chunk covers every P here
        assert by[0] == 4.0 * M * na * nv + 4.0 * na * nv * nv + 4.0 * M * nv
        s.profile(False)
        assert s.profile_read(0)["launches"] == 0 and s.profile_records(0)[0].size == 0
    finally:
        s.close()


def test_printed_coulomb_prefactor(api):
    """c_J = 1 (Eq. hessian as printed) against the dense Hessians of the same prefactor."""
    p = make_problem(7, 33, 37, 27, seeds=(40, 41, 42), amplitude=0.07)
    A, B = O.dense_A_B(p.eps_occ, p.eps_vir, O.eri_from_factors(p.extra["L_full"]), p.a_x, 1.0)
    s = api.Solver(p.n_occ, p.n_vir, p.eps_occ, p.eps_vir, p.L_oo, p.L_ov, p.L_vv, p.Lr_oo[p.ris_K_index],
                   p.Lr_ov, p.Lr_vv[p.ris_K_index], p.ris_K_index, a_x=p.a_x, coulomb_factor=1.0,
                   t_cut_ha=p.t_cut_ha)
    try:
        for prec in (api.PLAIN, api.MIXED):
            tol = 1e-6 if prec == api.PLAIN else 1e-5
            r = s.solve_tda(api.default_opts(n_states=4, precision=prec), want_vectors=False)
            assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.tda(A, 4)[0])) < tol
            r = s.solve_rpa(api.default_opts(n_states=4, precision=prec), want_vectors=False)
            assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.casida(A, B, 4)[0])) < tol
    finally:
        s.close()


def test_tight_subspace_restarts_often(api):
    """The smallest subspace the rid solves accept (2 N_init for TDA, 4 N_init
    for Casida, N_init = n_states + 3) forces a thick restart almost every
    iteration; a restart keeps the previous solutions only where they and the
    new directions fit, and the converged answer is unchanged."""
    p = make_config("tda_small")
    A, B = _dense(p)
    s = api.Solver.from_problem(p)
    try:
        k = 4
        r = s.solve_tda(api.default_opts(n_states=k, precond=api.RID, max_subspace=2 * (k + 3), max_iter=300),
                        want_vectors=False)
        assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.tda(A, k)[0])) < 1e-6
        assert r["stats"]["n_restart"] >= 1
        r = s.solve_rpa(api.default_opts(n_states=k, precond=api.RID, max_subspace=4 * (k + 3), max_iter=300),
                        want_vectors=False)
        assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.casida(A, B, k)[0])) < 1e-6
        assert r["stats"]["n_restart"] >= 1
        # polarizability: the cap must hold four rows per system
        mu = dipoles(3, 3, p.n_ov)
        with pytest.raises(api.TddftError) as e:
            s.solve_polar(api.default_opts(precond=api.RID, max_subspace=20), mu, OMEGAS)
        assert e.value.status == api.ERR_ARG
    finally:
        s.close()


def test_most_states_of_a_tiny_space(api):
    """n_states close to the dimension of the space (ov = 21, 18 states): the
    subspace fills the whole space and the solve still matches dense results."""
    p = make_problem(3, 7, 5, 9, seeds=(30, 31, 32))
    A, B = _dense(p)
    s = api.Solver.from_problem(p)
    try:
        k = 18
        for pc in (api.DIAG, api.RID):
            r = s.solve_tda(api.default_opts(n_states=k, precond=pc, max_iter=100), want_vectors=False)
            assert r["status"] == api.OK and np.max(np.abs(r["omega"] - D.tda(A, k)[0])) < 1e-6
    finally:
        s.close()
