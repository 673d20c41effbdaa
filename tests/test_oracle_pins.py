"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each pin checks the oracle against something other than itself: brute force on
tiny inputs, closed forms of special cases, an independent numerical route
(secular equations by bracketing, the non-Hermitian Casida matrix, the
sum-over-states polarizability, Cholesky), and the paper's invariants
(the preconditioner does not change converged results; T = A converges at the
first iteration).  ``test_planted_mistakes`` plants typical mistakes in copies
of the oracle's operator and checks that the pins catch each of them.
"""
import numpy as np
import pytest
from scipy.linalg import cho_factor, cho_solve
from scipy.optimize import brentq

from oracle import davidson as DV
from oracle import dense as D
from oracle import operators as O
from synth.generator import Problem, dipoles, make_config, make_problem, with_variant_terms

TOL = 1e-5


def _problem_from_full(eo, ev, L, Lr=None, K_index=None, a_x=0.25, c_J=2.0, t_cut=1e9):
    no = eo.size
    if Lr is None:
        Lr = L
    if K_index is None:
        K_index = np.arange(Lr.shape[0], dtype=np.int32)
    o, v = slice(0, no), slice(no, None)
    return Problem(n_occ=no, n_vir=ev.size, n_aux=L.shape[0], n_ris=Lr.shape[0],
                   eps_occ=eo, eps_vir=ev,
                   L_oo=L[:, o, o].copy(), L_ov=L[:, o, v].copy(), L_vv=L[:, v, v].copy(),
                   Lr_ov=Lr[:, o, v].copy(), Lr_oo=Lr[:, o, o].copy(), Lr_vv=Lr[:, v, v].copy(),
                   ris_K_index=np.asarray(K_index, dtype=np.int32), a_x=a_x, coulomb_factor=c_J,
                   t_cut_ha=t_cut, extra={"L_full": L, "Lr_full": Lr})


@pytest.fixture(scope="module")
def small():
    return make_config("tda_small")


# ---------------------------------------------------------------------------
# brute force: Hessian elements by explicit loops over orbitals and P

def _brute_A_B(eo, ev, L, a_x, c_J):
    no, nv, naux = eo.size, ev.size, L.shape[0]

    def eri(p, q, r, s):
        tot = 0.0
        for P in range(naux):
            tot += L[P, p, q] * L[P, r, s]
        return tot

    ov = no * nv
    A = np.zeros((ov, ov))
    B = np.zeros((ov, ov))
    for i in range(no):
        for a in range(nv):
            for j in range(no):
                for b in range(nv):
                    I, J = i * nv + a, j * nv + b
                    A_, B_ = no + a, no + b
                    A[I, J] = (ev[a] - eo[i]) * (i == j) * (a == b) \
                        + c_J * eri(i, A_, j, B_) - a_x * eri(i, j, A_, B_)
                    B[I, J] = c_J * eri(i, A_, j, B_) - a_x * eri(i, B_, j, A_)
    return A, B


@pytest.mark.parametrize("c_J", [1.0, 2.0])
def test_dense_hessian_brute_force(c_J):
    rng = np.random.default_rng(5)
    no, nv, naux = 2, 3, 2
    eo = np.sort(rng.uniform(-0.8, -0.3, no))
    ev = np.sort(rng.uniform(0.05, 1.5, nv))
    L = rng.standard_normal((naux, no + nv, no + nv))
    L = L + L.transpose(0, 2, 1)
    A, B = O.dense_A_B(eo, ev, O.eri_from_factors(L), 0.25, c_J)
    Ab, Bb = _brute_A_B(eo, ev, L, 0.25, c_J)
    assert np.allclose(A, Ab, atol=1e-13) and np.allclose(B, Bb, atol=1e-13)
    # Eq. hessian: A+B and A-B contain (ib|ja) with opposite signs, (ij|ab) with the same
    assert np.allclose(A, A.T) and np.allclose(B, B.T)


def test_eri_symmetry(small):
    eri = O.eri_from_factors(small.extra["L_full"])
    assert np.allclose(eri, eri.transpose(1, 0, 2, 3))
    assert np.allclose(eri, eri.transpose(2, 3, 0, 1))
    assert np.allclose(eri, eri.transpose(0, 1, 3, 2))


def test_matrix_free_equals_dense(small):
    """Block-factor products vs Hessians read off the four-index tensor."""
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    op = O.exact_operator(small)
    X = np.random.default_rng(1).standard_normal((3, small.n_ov))
    assert np.allclose(op.tda(X), X @ A, atol=1e-12)
    p, m = op.apb_amb(X)
    assert np.allclose(p, X @ (A + B), atol=1e-12)
    assert np.allclose(m, X @ (A - B), atol=1e-12)
    TA, TB = O.dense_ris_A_B(small)
    T = O.ris_operator(small)
    assert np.allclose(T.tda(X), X @ TA, atol=1e-12)
    p, m = T.apb_amb(X)
    assert np.allclose(p, X @ (TA + TB), atol=1e-12)
    assert np.allclose(m, X @ (TA - TB), atol=1e-12)


# ---------------------------------------------------------------------------
# closed forms

def test_zero_factors_give_delta():
    """L = 0: A = B + Delta, B = 0, so Omega = sorted Delta and
    alpha(w) = sum_ia 2 mu_ia^2 Delta_ia / (Delta_ia^2 - w^2)."""
    rng = np.random.default_rng(2)
    eo = np.sort(rng.uniform(-0.8, -0.3, 4))
    ev = np.sort(rng.uniform(0.05, 1.5, 9))
    L = np.zeros((3, 13, 13))
    p = _problem_from_full(eo, ev, L)
    d = O.delta(eo, ev)
    op = O.exact_operator(p)
    T = O.ris_operator(p)
    ref = np.sort(d)[:4]
    for pc in ("diag", "rid"):
        assert np.allclose(DV.solve_tda(p, op, T, 4, precond=pc).omega, ref, atol=1e-10)
        assert np.allclose(DV.solve_rpa(p, op, T, 4, precond=pc).omega, ref, atol=1e-10)
    mu = rng.normal(0, 0.1, (2, d.size))
    om = [0.0, 0.05, 0.1]
    ref_a = np.array([[[np.sum(2 * mu[v] * mu[u] * d / (d * d - w * w)) for u in range(2)]
                       for v in range(2)] for w in om])
    for pc in ("diag", "rid"):
        r = DV.solve_polar(p, op, T, mu, om, precond=pc)
        assert np.allclose(r.alpha, ref_a, rtol=1e-9)


@pytest.mark.parametrize("c_J", [1.0, 2.0])
def test_tda_secular_equation(c_J):
    """One auxiliary function and a_x = 0: A = Delta + c_J l l^T, whose eigenvalues
    solve 1 = c_J sum_ia l_ia^2 / (Omega - Delta_ia) (found here by bracketing)."""
    rng = np.random.default_rng(3)
    eo = np.sort(rng.uniform(-0.8, -0.3, 3))
    ev = np.sort(rng.uniform(0.05, 1.5, 7))
    L = 0.3 * rng.standard_normal((1, 10, 10))
    L = L + L.transpose(0, 2, 1)
    p = _problem_from_full(eo, ev, L, a_x=0.0, c_J=c_J)
    d = O.delta(eo, ev)
    ell = p.L_ov[0].reshape(-1)
    order = np.argsort(d)
    ds, ls = d[order], ell[order]
    f = lambda w: 1.0 - c_J * np.sum(ls ** 2 / (w - ds))
    roots = [brentq(f, ds[k] + 1e-12, ds[k + 1] - 1e-12) for k in range(3)]
    A, _ = O.dense_A_B(eo, ev, O.eri_from_factors(L), 0.0, c_J)
    assert np.allclose(D.tda(A, 3)[0], roots, atol=1e-10)
    r = DV.solve_tda(p, O.exact_operator(p), O.ris_operator(p), 3, precond="diag")
    assert np.allclose(r.omega, roots, atol=1e-9)


def test_casida_secular_equation_without_exchange():
    """a_x = 0: A-B = Delta and A+B = Delta + 2 c_J l l^T, so Omega^2 solves
    1 = 2 c_J sum_ia Delta_ia l_ia^2 / (Omega^2 - Delta_ia^2)."""
    rng = np.random.default_rng(4)
    eo = np.sort(rng.uniform(-0.8, -0.3, 3))
    ev = np.sort(rng.uniform(0.05, 1.5, 6))
    L = 0.3 * rng.standard_normal((1, 9, 9))
    L = L + L.transpose(0, 2, 1)
    c_J = 2.0
    p = _problem_from_full(eo, ev, L, a_x=0.0, c_J=c_J)
    d = O.delta(eo, ev)
    ell = p.L_ov[0].reshape(-1)
    order = np.argsort(d)
    ds, ls = d[order], ell[order]
    f = lambda w2: 1.0 - 2 * c_J * np.sum(ds * ls ** 2 / (w2 - ds ** 2))
    roots = [np.sqrt(brentq(f, ds[k] ** 2 + 1e-12, ds[k + 1] ** 2 - 1e-12)) for k in range(3)]
    r = DV.solve_rpa(p, O.exact_operator(p), O.ris_operator(p), 3, precond="diag")
    assert np.allclose(r.omega, roots, atol=1e-9)


def test_exchange_sign_closed_form():
    """One P with L_oo = s I, L_vv = t I, L_ov = 0: (ij|ab) = s t d_ij d_ab and every
    Coulomb-type term vanishes, so TDA and Casida give Omega = Delta - a_x s t."""
    rng = np.random.default_rng(6)
    no, nv = 3, 5
    eo = np.sort(rng.uniform(-0.8, -0.3, no))
    ev = np.sort(rng.uniform(0.05, 1.5, nv))
    s, t = 0.4, 0.7
    L = np.zeros((1, no + nv, no + nv))
    L[0, :no, :no] = s * np.eye(no)
    L[0, no:, no:] = t * np.eye(nv)
    p = _problem_from_full(eo, ev, L, a_x=0.25)
    ref = np.sort(O.delta(eo, ev) - 0.25 * s * t)[:4]
    op = O.exact_operator(p)
    T = O.ris_operator(p)
    assert np.allclose(DV.solve_tda(p, op, T, 4, precond="diag").omega, ref, atol=1e-10)
    assert np.allclose(DV.solve_rpa(p, op, T, 4, precond="diag").omega, ref, atol=1e-10)


def test_k2_equals_coulomb_for_separable_ov():
    """One P with L_oo = L_vv = 0 and L_ov = u v^T: (ib|ja) = (ia|jb), so with
    c_J = a_x the B matrix vanishes and Casida equals TDA, whose roots solve
    1 = c_J sum l^2/(Omega - Delta)."""
    rng = np.random.default_rng(7)
    no, nv = 3, 6
    eo = np.sort(rng.uniform(-0.8, -0.3, no))
    ev = np.sort(rng.uniform(0.05, 1.5, nv))
    u, v = rng.standard_normal(no), rng.standard_normal(nv)
    L = np.zeros((1, no + nv, no + nv))
    L[0, :no, no:] = 0.4 * np.outer(u, v)
    L[0, no:, :no] = L[0, :no, no:].T
    p = _problem_from_full(eo, ev, L, a_x=0.5, c_J=0.5)
    d = O.delta(eo, ev)
    ell = p.L_ov[0].reshape(-1)
    order = np.argsort(d)
    ds, ls = d[order], ell[order]
    f = lambda w: 1.0 - 0.5 * np.sum(ls ** 2 / (w - ds))
    roots = [brentq(f, ds[k] + 1e-12, ds[k + 1] - 1e-12) for k in range(3)]
    r = DV.solve_rpa(p, O.exact_operator(p), O.ris_operator(p), 3, precond="diag")
    assert np.allclose(r.omega, roots, atol=1e-9)


def test_zero_ov_block_makes_rpa_equal_tda(small):
    """L_ov = 0 kills every (ia|jb) and (ib|ja): B = 0 and Casida = TDA."""
    L = small.extra["L_full"].copy()
    no = small.n_occ
    L[:, :no, no:] = 0.0
    L[:, no:, :no] = 0.0
    p = _problem_from_full(small.eps_occ, small.eps_vir, L)
    op = O.exact_operator(p)
    T = O.ris_operator(p)
    a = DV.solve_tda(p, op, T, 5, precond="diag").omega
    b = DV.solve_rpa(p, op, T, 5, precond="diag").omega
    assert np.allclose(a, b, atol=1e-9)


def test_window_selection():
    """Sec. 3.1: drop virtuals above eps_HOMO + t_cut and occupieds below eps_LUMO - t_cut."""
    eo = np.array([-3.0, -1.0, -0.5])
    ev = np.array([0.1, 0.9, 1.0, 2.0])
    ko, kv = O.window(eo, ev, 1.5)
    assert ko.tolist() == [False, True, True]       # bound 0.1 - 1.5 = -1.4
    assert kv.tolist() == [True, True, True, False]  # bound -0.5 + 1.5 = 1.0 (kept at equality)


# ---------------------------------------------------------------------------
# independent numerical routes

def test_casida_hermitian_form_equals_nonhermitian(small):
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    om, X, Y = D.casida(A, B, 5)
    big = np.block([[A, B], [-B, -A]])
    ev = np.linalg.eigvals(big)
    pos = np.sort(ev.real[ev.real > 0])[:5]
    assert np.allclose(om, pos, atol=1e-10)
    # X^T X - Y^T Y = 1
    assert np.allclose(np.sum(X * X, 1) - np.sum(Y * Y, 1), 1.0)


def test_polar_sum_over_states_and_cholesky(small):
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    mu = dipoles(3, 3, small.n_ov)
    om = [0.0, 0.05, 0.1]
    alpha = D.polar(A, B, mu, om)
    # symmetric in (v, u)
    assert np.allclose(alpha, alpha.transpose(0, 2, 1))
    # static limit by Cholesky: alpha(0) = 2 mu^T (A+B)^-1 mu
    c = cho_factor(A + B)
    assert np.allclose(alpha[0], 2 * mu @ cho_solve(c, mu.T), rtol=1e-10)
    # sum over all Casida states: alpha = sum_n 2 Omega_n (mu.(X+Y)_n)^2 / (Omega_n^2 - w^2)
    w, X, Y = D.casida(A, B, small.n_ov)
    t = mu @ (X + Y).T
    for f, ww in enumerate(om):
        sos = np.einsum("n,vn,un->vu", 2 * w / (w * w - ww * ww), t, t)
        assert np.allclose(alpha[f], sos, rtol=1e-9)
    # below the first excitation alpha grows with omega
    assert np.all(np.diagonal(alpha[1]) > np.diagonal(alpha[0]))
    assert np.all(np.diagonal(alpha[2]) > np.diagonal(alpha[1]))


# ---------------------------------------------------------------------------
# invariants of the method

@pytest.mark.parametrize("pc", ["diag", "rid"])
def test_davidson_equals_dense(small, pc):
    """The preconditioner does not change the converged result (abstract, Sec. 1)."""
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    op = O.exact_operator(small)
    T = O.ris_operator(small)
    r = DV.solve_tda(small, op, T, 5, precond=pc)
    assert r.converged and r.resid.max() < TOL
    assert np.allclose(r.omega, D.tda(A, 5)[0], atol=1e-8)
    r = DV.solve_rpa(small, op, T, 5, precond=pc)
    assert r.converged and np.allclose(r.omega, D.casida(A, B, 5)[0], atol=1e-8)
    mu = dipoles(3, 3, small.n_ov)
    r = DV.solve_polar(small, op, T, mu, [0.0, 0.05, 0.1], precond=pc)
    ref = D.polar(A, B, mu, [0.0, 0.05, 0.1])
    assert r.converged and np.allclose(r.alpha, ref, rtol=1e-8)


def test_rid_no_more_iterations_than_diag(small):
    op = O.exact_operator(small)
    T = O.ris_operator(small)
    mu = dipoles(3, 3, small.n_ov)
    for f in (lambda pc: DV.solve_tda(small, op, T, 5, precond=pc),
              lambda pc: DV.solve_rpa(small, op, T, 5, precond=pc),
              lambda pc: DV.solve_polar(small, op, T, mu, [0.0, 0.05, 0.1], precond=pc)):
        assert f("rid").n_iter <= f("diag").n_iter


def test_T_equal_A_converges_at_first_iteration(small):
    """Sec. 2.1: with T = A the residual of the initial guess (eigenvectors of T) is zero."""
    L = small.extra["L_full"]
    p = _problem_from_full(small.eps_occ, small.eps_vir, L, Lr=L,
                           K_index=np.arange(L.shape[0]), t_cut=1e9)
    op = O.exact_operator(p)
    T = O.ris_operator(p)
    assert DV.solve_tda(p, op, T, 5, precond="rid", guess_tol=1e-9).n_iter == 1
    assert DV.solve_rpa(p, op, T, 5, precond="rid", guess_tol=1e-9).n_iter == 1


def test_hessians_positive_definite(small):
    """The generator's amplitude keeps A-B and A+B definite (margin 0.02 Ha)."""
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    assert np.linalg.eigvalsh(A - B)[0] > 0.02
    assert np.linalg.eigvalsh(A + B)[0] > 0.02


def test_n_init_rule():
    """Sec. 3.2: N_init = N_states + min(N_states, 3) for rid, N_states + 8 otherwise."""
    assert [DV.n_init(n, "rid") for n in (1, 2, 5, 20)] == [2, 4, 8, 23]
    assert [DV.n_init(n, "diag") for n in (1, 5, 20)] == [9, 13, 28]


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by at least one pin above

class _Mutant(O.Operator):
    def __init__(self, base, kind):
        super().__init__(np.zeros(1), np.zeros(1), base.Lj_ov, base.Lx_oo, base.Lx_ov, base.Lx_vv,
                         base.a_x, base.c_J)
        self.d, self.n_occ, self.n_vir, self.kind = base.d, base.n_occ, base.n_vir, kind

    def _parts(self, X, need_k2):
        X, J, K1, K2 = super()._parts(X, True)
        if self.kind == "k1_sign":
            K1 = -K1
        elif self.kind == "drop_k2":
            K2 = np.zeros_like(K2)
        elif self.kind == "k2_as_coulomb":
            K2 = J
        elif self.kind == "k1_transposed":
            m = X.shape[0]
            Xt = X.reshape(m, self.n_occ, self.n_vir)
            K1 = np.einsum("pji,nja,pba->nib", self.Lx_oo, Xt,
                           self.Lx_vv[:, ::-1, :]).reshape(m, -1)
        elif self.kind == "coulomb_half":
            J = 0.5 * J
        return X, J, K1, K2


@pytest.mark.parametrize("kind", ["k1_sign", "drop_k2", "k2_as_coulomb", "k1_transposed",
                                  "coulomb_half"])
def test_planted_mistakes(small, kind):
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    mut = _Mutant(O.exact_operator(small), kind)
    X = np.random.default_rng(1).standard_normal((2, small.n_ov))
    p, m = mut.apb_amb(X)
    caught = not (np.allclose(mut.tda(X), X @ A, atol=1e-10)
                  and np.allclose(p, X @ (A + B), atol=1e-10)
                  and np.allclose(m, X @ (A - B), atol=1e-10))
    assert caught, kind


# ---------------------------------------------------------------------------
# variant terms of Eq. hessian: a second (range-separated) exchange factor set
# and a low-rank response kernel standing in for f^xc

def _brute_variant(eo, ev, L, M, b_x, F, w, a_x, c_J):
    """Elements of A and B by explicit loops: the base terms plus
    -b_x (ij|ab)_M, -b_x (ib|ja)_M and +c_J sum_g w_g F^g_ia F^g_jb."""
    A, B = _brute_A_B(eo, ev, L, a_x, c_J)
    no, nv = eo.size, ev.size
    for i in range(no):
        for a in range(nv):
            for j in range(no):
                for b in range(nv):
                    I, J = i * nv + a, j * nv + b
                    A_, B_ = no + a, no + b
                    lr_ijab = sum(M[Q, i, j] * M[Q, A_, B_] for Q in range(M.shape[0]))
                    lr_ibja = sum(M[Q, i, B_] * M[Q, j, A_] for Q in range(M.shape[0]))
                    f = sum(w[g] * F[g, i, A_] * F[g, j, B_] for g in range(F.shape[0]))
                    A[I, J] += -b_x * lr_ijab + c_J * f
                    B[I, J] += -b_x * lr_ibja + c_J * f
    return A, B


def test_variant_terms_brute_force():
    rng = np.random.default_rng(8)
    no, nv = 2, 3
    eo = np.sort(rng.uniform(-0.8, -0.3, no))
    ev = np.sort(rng.uniform(0.05, 1.5, nv))
    sym = lambda n: (lambda t: t + t.transpose(0, 2, 1))(rng.standard_normal((n, no + nv, no + nv)))
    L, M, F = sym(2), sym(3), sym(2)
    w = np.array([-0.7, 0.4])
    A, B = O.dense_A_B(eo, ev, O.eri_from_factors(L), 0.25, 2.0, eri_lr=O.eri_from_factors(M), b_x=0.6,
                       F_full=F, w=w)
    Ab, Bb = _brute_variant(eo, ev, L, M, 0.6, F, w, 0.25, 2.0)
    assert np.allclose(A, Ab, atol=1e-12) and np.allclose(B, Bb, atol=1e-12)


@pytest.fixture(scope="module")
def variant(small):
    return with_variant_terms(small, 90, n_aux_lr=60, b_x=0.75, n_kernel=30)


def test_variant_matrix_free_equals_dense(variant):
    A, B = O.dense_exact_A_B(variant)
    op = O.exact_operator(variant)
    X = np.random.default_rng(4).standard_normal((3, variant.n_ov))
    assert np.allclose(op.tda(X), X @ A, atol=1e-12)
    p, m = op.apb_amb(X)
    assert np.allclose(p, X @ (A + B), atol=1e-12)
    assert np.allclose(m, X @ (A - B), atol=1e-12)
    # both terms change the operator
    A0, _ = O.dense_exact_A_B(variant.__class__(**{**variant.__dict__, "extra": {"L_full": variant.extra["L_full"]}}))
    assert np.max(np.abs(A - A0)) > 1e-2


def test_variant_special_cases(small):
    """M = L with weight b_x is the base operator with a_x + b_x; a kernel of
    the Coulomb rows themselves with w = 1 doubles the Coulomb prefactor, with
    w = -1 cancels it."""
    L = small.extra["L_full"]
    no = small.n_occ
    o, v = slice(0, no), slice(no, None)
    eri = O.eri_from_factors(L)
    X = np.random.default_rng(6).standard_normal((2, small.n_ov))
    base = lambda a_x, c_J: O.Operator(small.eps_occ, small.eps_vir, small.L_ov, small.L_oo, small.L_ov,
                                       small.L_vv, a_x, c_J)
    lr = O.Operator(small.eps_occ, small.eps_vir, small.L_ov, small.L_oo, small.L_ov, small.L_vv, 0.25, 2.0,
                    lr=(small.L_oo, small.L_ov, small.L_vv, 0.5))
    for u, r in zip(lr.apb_amb(X), base(0.75, 2.0).apb_amb(X)):
        assert np.allclose(u, r, atol=1e-12)
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, eri, 0.25, 2.0, eri_lr=eri, b_x=0.5)
    A2, B2 = O.dense_A_B(small.eps_occ, small.eps_vir, eri, 0.75, 2.0)
    assert np.allclose(A, A2, atol=1e-12) and np.allclose(B, B2, atol=1e-12)
    n_aux = L.shape[0]
    for wv, cj in ((1.0, 4.0), (-1.0, 0.0)):
        k = O.Operator(small.eps_occ, small.eps_vir, small.L_ov, small.L_oo, small.L_ov, small.L_vv, 0.25, 2.0,
                       kernel=(small.L_ov, np.full(n_aux, wv)))
        for u, r in zip(k.apb_amb(X), base(0.25, cj).apb_amb(X)):
            assert np.allclose(u, r, atol=1e-12)
        A, B = O.dense_A_B(small.eps_occ, small.eps_vir, eri, 0.25, 2.0, F_full=L, w=np.full(n_aux, wv))
        A2, B2 = O.dense_A_B(small.eps_occ, small.eps_vir, eri, 0.25, cj)
        assert np.allclose(A, A2, atol=1e-12) and np.allclose(B, B2, atol=1e-12)


@pytest.mark.parametrize("pc", ["diag", "rid"])
def test_variant_davidson_equals_dense(variant, pc):
    """The preconditioner (T without the variant terms) changes the path, not
    the converged TDA, Casida and polarizability results."""
    A, B = O.dense_exact_A_B(variant)
    op, T = O.exact_operator(variant), O.ris_operator(variant)
    r = DV.solve_tda(variant, op, T, 5, precond=pc)
    assert np.allclose(r.omega, D.tda(A, 5)[0], atol=1e-8)
    r = DV.solve_rpa(variant, op, T, 5, precond=pc)
    assert np.allclose(r.omega, D.casida(A, B, 5)[0], atol=1e-8)
    mu = dipoles(3, 2, variant.n_ov)
    r = DV.solve_polar(variant, op, T, mu, [0.0, 0.05], precond=pc)
    assert np.allclose(r.alpha, D.polar(A, B, mu, [0.0, 0.05]), rtol=1e-7)


def test_tight_cap_restarts_still_converge(small):
    """With the smallest caps (2 N_init for TDA, 4 N_init for Casida) a thick
    restart cannot keep the previous solutions and the new directions; it
    keeps the current ones only, and the rid solves still reach the dense
    results (just in more iterations)."""
    op, T = O.exact_operator(small), O.ris_operator(small)
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]), small.a_x,
                       small.coulomb_factor)
    k = 4
    r = DV.solve_tda(small, op, T, k, precond="rid", max_subspace=2 * (k + 3), max_iter=300)
    assert r.converged and np.max(np.abs(r.omega - D.tda(A, k)[0])) < 1e-8
    r = DV.solve_rpa(small, op, T, k, precond="rid", max_subspace=4 * (k + 3), max_iter=300)
    assert r.converged and np.max(np.abs(r.omega - D.casida(A, B, k)[0])) < 1e-8


# ---------------------------------------------------------------------------
# mid-size: the matrix-free Davidson against dense LAPACK at ov = 3,456

def test_dense_blocks_equal_four_index_route(small):
    """The blockwise dense Hessians (used where the four-index tensor over all
    orbitals does not fit) equal the element-by-element read of (pq|rs)."""
    A, B = O.dense_A_B(small.eps_occ, small.eps_vir, O.eri_from_factors(small.extra["L_full"]),
                       small.a_x, small.coulomb_factor)
    A2, B2 = O.dense_A_B_blocks(small)
    assert np.allclose(A, A2, rtol=0, atol=1e-13) and np.allclose(B, B2, rtol=0, atol=1e-13)


@pytest.fixture(scope="module")
def mid():
    """n_occ=24, n_vir=144 (ov=3,456), n_aux=840 = 5 n_mo, ris n_aux=108 (12
    atoms); amplitude scale 0.7^3 of the default, between the small (1) and
    the medium (0.7^5) workloads as sqrt(n_occ n_vir) is."""
    from synth.generator import default_amplitude
    p = make_problem(24, 144, 840, 108, seeds=(60, 61, 62), amplitude=0.7 ** 3 * default_amplitude(840))
    A, B = O.dense_A_B_blocks(p)
    return p, A, B


@pytest.mark.slow
def test_davidson_equals_dense_mid_size(mid):
    """TDA (both preconditioners), Casida and alpha(omega) of the oracle's
    matrix-free Davidson at ov = 3,456 against eigh / solve of the dense
    Hessians: the converged results agree to 1e-8 Ha (||R|| <= 1e-5 puts the
    eigenvalue error near ||R||^2 / gap), alpha to 1e-8 relative element by
    element (one shared Galerkin subspace: second order in the residuals),
    and rid takes no more outer iterations than diag for TDA."""
    p, A, B = mid
    op, T = O.exact_operator(p), O.ris_operator(p)
    k = 10
    ref = D.tda(A, k)[0]
    it = {}
    for pc in ("diag", "rid"):
        r = DV.solve_tda(p, op, T, k, precond=pc)
        assert r.converged and np.max(np.abs(r.omega - ref)) < 1e-8, (pc, np.max(np.abs(r.omega - ref)))
        it[pc] = r.n_iter
    assert it["rid"] <= it["diag"], it
    r = DV.solve_rpa(p, op, T, k, precond="rid")
    assert r.converged and np.max(np.abs(r.omega - D.casida(A, B, k)[0])) < 1e-8
    mu = dipoles(63, 2, p.n_ov)
    r = DV.solve_polar(p, op, T, mu, [0.0, 0.1], precond="rid")
    ref = D.polar(A, B, mu, [0.0, 0.1])
    assert r.converged and np.max(np.abs(r.alpha - ref) / np.abs(ref)) < 1e-8
