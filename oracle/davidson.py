"""Preconditioned Davidson solver for the TDDFT response problems (oracle, FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The outer algorithm follows Sec. 2.1 step by step, in the paper's notation:
  V^(0)    initial subspace from the low-lying eigenvectors of the
           preconditioner T (Sec. 2.1; N_init rule of Sec. 3.2)
  Eq. 1    a^(k) = V^T A V
  Eq. 2    a^(k) x_n = Omega_n x_n
  Eq. 3    X = V x
  Eq. residual  R_n = A X_n - X_n Omega_n; converged when |R_n| < threshold
  Eq. precondition  v_n = (T - Omega_n)^-1 R_n for every unconverged n
           (element-wise division for the diagonal T; an inner Krylov solve
           for the ris T)
  then     modified Gram-Schmidt of the new directions against V and each
           other, append to V.

The same scheme serves the Casida problem (Eq. Casida) in the paired form
(A+B)(X+Y) = Omega (X-Y), (A-B)(X-Y) = Omega (X+Y) with one shared subspace
for X+Y and X-Y, and the polarizability linear systems (Eq. TDDFT_polar) by
Galerkin projection in the same paired subspace.

Readings where the paper is silent (each listed in the design notes):
  * convergence norm: TDA |R_n|_2 of unit-norm X_n; Casida
    sqrt(|R+|^2 + |R-|^2) with (X+Y)^T(X-Y) = 1; polarizability the same
    pair norm divided by |2 mu|
  * diagonal T = Delta_ia (eps_a - eps_i); |Delta - Omega| below 1e-8 is
    replaced by +-1e-8
  * the inner Krylov solve of Eq. precondition with the ris T is a block
    Galerkin projection shared by all roots, seeded and expanded with
    diagonal-preconditioned residuals, stopped at |res_n| <= inner_tol |R_n|
    or inner_max_iter iterations (1e-2 and 20, Sec. 3.1)
  * initial guesses: diagonal T -> unit vectors at the N_init smallest
    Delta (N_init = N_states + 8); ris T -> its N_init = N_states +
    min(N_states, 3) lowest eigenvectors converged to 1e-3 (Sec. 3.1-3.2);
    for the polarizability the solution of the T system to 1e-3 (diag:
    (Delta -+ omega)^-1 mu)
  * vectors whose norm after two Gram-Schmidt passes is below 1e-8 of the
    input norm are dropped; the subspace holds at most MAX_SUBSPACE vectors:
    before it would overflow it is rebuilt from the current and the
    previous iteration's solutions (thick restart with the previous Ritz
    vectors, as in Stathopoulos and Saad's GD+k): an eigen solve keeps the
    Ritz vectors of the wanted roots (Casida: their X+Y and X-Y), a
    polarizability solve its current and previous U and W; an inner solve
    stops with its current solution
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DROP_TOL = 1e-8
SHIFT_GUARD = 1e-8
MAX_SUBSPACE = 160   # subspace vectors kept before a collapse / restart


@dataclass
class Result:
    omega: np.ndarray
    X: np.ndarray
    Y: np.ndarray | None
    resid: np.ndarray
    n_iter: int
    n_mv: int
    converged: bool
    history: list = field(default_factory=list)
    n_ris_mv: int = 0
    alpha: np.ndarray | None = None


def _guard(den):
    small = np.abs(den) < SHIFT_GUARD
    return np.where(small, np.where(den < 0, -SHIFT_GUARD, SHIFT_GUARD), den)


def mgs(V: np.ndarray, cand: np.ndarray, drop_tol: float = DROP_TOL) -> np.ndarray:
    """Modified Gram-Schmidt (Sec. 2.1, last step): orthogonalise each candidate
    against the rows of V and the accepted candidates, two passes, normalise;
    drop a candidate whose remaining norm is below drop_tol of its input norm.
    Returns the accepted, orthonormal new rows."""
    basis = [V[r] for r in range(V.shape[0])] if V is not None else []
    out = []
    for v in np.atleast_2d(cand):
        v = v.astype(np.float64, copy=True)
        n0 = np.linalg.norm(v)
        if not np.isfinite(n0) or n0 == 0.0:
            continue
        for _ in range(2):
            for u in basis:
                v -= (u @ v) * u
            for u in out:
                v -= (u @ v) * u
        n1 = np.linalg.norm(v)
        if n1 < drop_tol * n0:
            continue
        if len(basis) + len(out) >= v.size:   # the space is already spanned
            break
        out.append(v / n1)
    if not out:
        return np.zeros((0, np.atleast_2d(cand).shape[1]))
    return np.array(out)


# ----------------------------------------------------------------------------
# Small subspace problems (Eq. 2 and its Casida / linear-system analogues)

def _paired_factors(ap, am):
    """With a- = Q diag(l) Q^T: S = a-^(1/2), S^-1, a-^-1, and eig of S a+ S."""
    l, Q = np.linalg.eigh(0.5 * (am + am.T))
    if l[0] <= 0.0:
        raise np.linalg.LinAlgError("projected A-B is not positive definite")
    S = (Q * np.sqrt(l)) @ Q.T
    Si = (Q / np.sqrt(l)) @ Q.T
    Ai = (Q / l) @ Q.T
    H = S @ ap @ S
    lam, Z = np.linalg.eigh(0.5 * (H + H.T))
    return S, Si, Ai, lam, Z


def _paired_solve(fac, hp, hm, s):
    """Solve t+ u - s w = hp, t- w - s u = hm in the subspace (one shift s).

    Substituting u = S u~, w = S^-1 w~ gives (S t+ S - s^2) u~ = S hp + s S^-1 hm,
    then u = S u~ and w = s S^-1 u~ + t-^-1 hm."""
    S, Si, Ai, lam, Z = fac
    rhs = S @ hp + s * (Si @ hm)
    ut = Z @ ((Z.T @ rhs) / _guard(lam - s * s))
    return S @ ut, s * (Si @ ut) + Ai @ hm


# ----------------------------------------------------------------------------
# Inner solves of Eq. precondition with the ris operator T

def inner_solve_tda(T, d, R, omega, tol=1e-2, max_iter=20):
    """(T - Omega_n) v_n = R_n for all n by one block Galerkin subspace.

    Returns (v [n][ov], number of T products)."""
    R = np.atleast_2d(R)
    S = mgs(None, R / _guard(d[None, :] - omega[:, None]))
    TS = T.tda(S)
    n_mv = S.shape[0]
    rn = np.linalg.norm(R, axis=1)
    for it in range(max_iter):
        t = S @ TS.T
        lam, Q = np.linalg.eigh(0.5 * (t + t.T))
        h = S @ R.T                                  # [k][n]
        y = Q @ ((Q.T @ h) / _guard(lam[:, None] - omega[None, :]))
        v = y.T @ S
        res = y.T @ TS - omega[:, None] * v - R
        ok = np.linalg.norm(res, axis=1) <= tol * rn
        if ok.all() or it == max_iter - 1:
            break
        if S.shape[0] + int((~ok).sum()) > MAX_SUBSPACE:
            break
        new = mgs(S, res[~ok] / _guard(d[None, :] - omega[~ok, None]))
        if new.shape[0] == 0:
            break
        S = np.vstack([S, new])
        TS = np.vstack([TS, T.tda(new)])
        n_mv += new.shape[0]
    return v, n_mv


def _diag_paired(d, gp, gm, s):
    """Diagonal T in the (X, Y) picture: x = r_X/(Delta - s), y = r_Y/(Delta + s),
    with r_X = (g+ + g-)/2, r_Y = (g+ - g-)/2; returns (x+y, x-y)."""
    rx = 0.5 * (gp + gm)
    ry = 0.5 * (gp - gm)
    x = rx / _guard(d[None, :] - s[:, None])
    y = ry / _guard(d[None, :] + s[:, None])
    return x + y, x - y


def inner_solve_paired(T, d, gp, gm, shifts, tol=1e-2, max_iter=20):
    """T+ u - s w = g+, T- w - s u = g- (T+- = T_A +- T_B) for all right-hand
    sides by one shared Galerkin subspace.  This is Eq. precondition for the
    Casida problem (s = Omega_n) and the ris linear system of Eq. TDDFT_polar
    (s = omega).  Returns (u, w, number of T pair products)."""
    gp = np.atleast_2d(gp)
    gm = np.atleast_2d(gm)
    u0, w0 = _diag_paired(d, gp, gm, shifts)
    S = mgs(None, np.vstack([u0, w0]))
    TP, TM = T.apb_amb(S)
    n_mv = S.shape[0]
    gn = np.sqrt(np.linalg.norm(gp, axis=1) ** 2 + np.linalg.norm(gm, axis=1) ** 2)
    for it in range(max_iter):
        fac = _paired_factors(S @ TP.T, S @ TM.T)
        hp = S @ gp.T
        hm = S @ gm.T
        U = np.zeros_like(gp)
        W = np.zeros_like(gp)
        rp = np.zeros_like(gp)
        rm = np.zeros_like(gp)
        for n, s in enumerate(shifts):
            uc, wc = _paired_solve(fac, hp[:, n], hm[:, n], s)
            U[n], W[n] = uc @ S, wc @ S
            rp[n] = uc @ TP - s * W[n] - gp[n]
            rm[n] = wc @ TM - s * U[n] - gm[n]
        rn = np.sqrt(np.linalg.norm(rp, axis=1) ** 2 + np.linalg.norm(rm, axis=1) ** 2)
        ok = rn <= tol * gn
        if ok.all() or it == max_iter - 1:
            break
        if S.shape[0] + 2 * int((~ok).sum()) > MAX_SUBSPACE:
            break
        nu, nw = _diag_paired(d, rp[~ok], rm[~ok], shifts[~ok])
        new = mgs(S, np.vstack([nu, nw]))
        if new.shape[0] == 0:
            break
        S = np.vstack([S, new])
        p, m = T.apb_amb(new)
        TP = np.vstack([TP, p])
        TM = np.vstack([TM, m])
        n_mv += new.shape[0]
    return U, W, n_mv


# ----------------------------------------------------------------------------
# Preconditioners

class DiagPrecond:
    """T = A^diag approximated by Delta_ia (Sec. 2.1: element-wise division)."""

    name = "diag"

    def __init__(self, d):
        self.d = d
        self.n_mv = 0

    def tda(self, R, omega):
        return R / _guard(self.d[None, :] - omega[:, None])

    def paired(self, gp, gm, s):
        return _diag_paired(self.d, gp, gm, s)


class RidPrecond:
    """T = the ris operator, applied by an inner Krylov solve (Sec. 2.1, Sec. 3.1)."""

    name = "rid"

    def __init__(self, T, d, inner_tol=1e-2, inner_max_iter=20):
        self.T, self.d = T, d
        self.tol, self.max_iter = inner_tol, inner_max_iter
        self.n_mv = 0

    def tda(self, R, omega):
        v, n = inner_solve_tda(self.T, self.d, R, omega, self.tol, self.max_iter)
        self.n_mv += n
        return v

    def paired(self, gp, gm, s):
        u, w, n = inner_solve_paired(self.T, self.d, gp, gm, s, self.tol, self.max_iter)
        self.n_mv += n
        return u, w


def n_init(n_states, precond):
    """N_init = N_states + min(N_states, 3) for rid, N_states + 8 otherwise (Sec. 3.2)."""
    return n_states + (min(n_states, 3) if precond == "rid" else 8)


def unit_guess(d, k):
    """Unit vectors at the k smallest Delta_ia (ties broken by index)."""
    order = np.argsort(d, kind="stable")[:k]
    G = np.zeros((k, d.size))
    G[np.arange(k), order] = 1.0
    return G


# ----------------------------------------------------------------------------
# Outer solvers

def davidson_tda(op, n_states, precond, guess, tol=1e-5, max_iter=50, max_subspace=None,
                 n_keep=None):
    """Lowest eigenpairs of A (Eq. TDA) by the Davidson algorithm of Sec. 2.1."""
    V = mgs(None, guess)
    AV = op.tda(V)
    n_mv = V.shape[0]
    ov = V.shape[1]
    max_subspace = max_subspace or MAX_SUBSPACE
    hist = []
    X_prev = None
    for k in range(1, max_iter + 1):
        a = V @ AV.T                                  # Eq. 1
        w, x = np.linalg.eigh(0.5 * (a + a.T))        # Eq. 2
        om = w[:n_states]
        xs = x[:, :n_states]
        X = xs.T @ V                                  # Eq. 3
        AX = xs.T @ AV
        R = AX - om[:, None] * X                      # Eq. residual
        r = np.linalg.norm(R, axis=1)
        hist.append(float(r.max()))
        if r.max() < tol:
            return Result(om, X, None, r, k, n_mv, True, hist, precond.n_mv)
        todo = r >= tol
        cand = precond.tda(R[todo], om[todo])         # Eq. precondition
        new = mgs(V, cand)
        if new.shape[0] == 0:
            break
        if V.shape[0] + int(todo.sum()) > max_subspace:
            # thick restart: current Ritz vectors + those of the previous iteration,
            # the latter only where they and the new directions fit under the cap
            V, AV = X, AX
            if X_prev is not None and 2 * X.shape[0] + new.shape[0] <= max_subspace:
                extra = mgs(V, X_prev)
                V = np.vstack([V, extra])
                AV = np.vstack([AV, op.tda(extra)])
                n_mv += extra.shape[0]
            new = mgs(V, new)
        X_prev = X
        V = np.vstack([V, new])
        AV = np.vstack([AV, op.tda(new)])
        n_mv += new.shape[0]
    return Result(om, X, None, r, k, n_mv, False, hist, precond.n_mv)


def _rpa_ritz(V, P, M, n_states):
    ap = V @ P.T
    am = V @ M.T
    S, Si, Ai, lam, Z = _paired_factors(0.5 * (ap + ap.T), 0.5 * (am + am.T))
    if lam[0] <= 0.0:
        raise np.linalg.LinAlgError("projected Casida problem has non-positive Omega^2")
    om = np.sqrt(lam[:n_states])
    z = Z[:, :n_states]
    u = (S @ z) / np.sqrt(om)                         # (X+Y) coefficients, u^T w = 1
    w = (ap @ u) / om                                 # (X-Y) coefficients
    return om, u, w, S, Si, lam, Z


def davidson_rpa(op, n_states, precond, guess, tol=1e-5, max_iter=50, max_subspace=None,
                 n_keep=None):
    """Lowest positive eigenpairs of Eq. Casida by a paired Davidson algorithm.

    One subspace V holds both X+Y and X-Y; a+ = V^T (A+B) V, a- = V^T (A-B) V;
    the projected problem a- a+ u = Omega^2 u is solved in the symmetric form
    a-^(1/2) a+ a-^(1/2) z = Omega^2 z."""
    V = mgs(None, guess)
    P, M = op.apb_amb(V)
    n_mv = V.shape[0]
    max_subspace = max_subspace or MAX_SUBSPACE
    hist = []
    prev = None
    for k in range(1, max_iter + 1):
        om, u, w, S, Si, lam, Z = _rpa_ritz(V, P, M, n_states)
        U, W = u.T @ V, w.T @ V
        Rp = u.T @ P - om[:, None] * W                # (A+B)(X+Y) - Omega (X-Y)
        Rm = w.T @ M - om[:, None] * U                # (A-B)(X-Y) - Omega (X+Y)
        r = np.sqrt(np.linalg.norm(Rp, axis=1) ** 2 + np.linalg.norm(Rm, axis=1) ** 2)
        hist.append(float(r.max()))
        X, Y = 0.5 * (U + W), 0.5 * (U - W)
        if r.max() < tol:
            return Result(om, X, Y, r, k, n_mv, True, hist, precond.n_mv)
        todo = r >= tol
        nu, nw = precond.paired(Rp[todo], Rm[todo], om[todo])
        new = mgs(V, np.vstack([nu, nw]))
        if new.shape[0] == 0:
            break
        if V.shape[0] + 2 * int(todo.sum()) > max_subspace:
            # thick restart: X+Y and X-Y of the wanted roots, now and one iteration ago
            # (the latter only where they and the new directions fit under the cap,
            # and while the restart block stays within 112 rows)
            keep_prev = prev is not None and 4 * U.shape[0] <= 112 and \
                4 * U.shape[0] + new.shape[0] <= max_subspace
            V = mgs(None, np.vstack([U, W] + (list(prev) if keep_prev else [])))
            P, M = op.apb_amb(V)
            n_mv += V.shape[0]
            new = mgs(V, new)
        prev = (U, W)
        V = np.vstack([V, new])
        p, m = op.apb_amb(new)
        P, M = np.vstack([P, p]), np.vstack([M, m])
        n_mv += new.shape[0]
    return Result(om, X, Y, r, k, n_mv, False, hist, precond.n_mv)


def polar_solve(op, mu, omegas, precond, guess, tol=1e-5, max_iter=50):
    """Dynamic polarizability of Eq. TDDFT_polar by Galerkin projection.

    For every (omega_f, mu_u): (A+B) U - omega W = 2 mu_u and
    (A-B) W - omega U = 0 with U = X+Y, W = X-Y, solved in one shared
    subspace; alpha_vu(omega_f) = mu_v^T U_fu.  ``guess`` holds initial
    directions (U and W rows).  Returns Result with ``alpha[f][v][u]``."""
    mu = np.atleast_2d(mu)
    nd = mu.shape[0]
    nf = len(omegas)
    om_all = np.repeat(np.asarray(omegas, dtype=float), nd)     # rhs index = f*nd + u
    b = np.tile(2.0 * mu, (nf, 1))
    bn = np.linalg.norm(b, axis=1)
    V = mgs(None, guess)
    P, M = op.apb_amb(V)
    n_mv = V.shape[0]
    hist = []
    prev = None
    for k in range(1, max_iter + 1):
        fac = _paired_factors(V @ P.T, V @ M.T)
        hp = V @ b.T
        U = np.zeros_like(b)
        W = np.zeros_like(b)
        Rp = np.zeros_like(b)
        Rm = np.zeros_like(b)
        for n, s in enumerate(om_all):
            uc, wc = _paired_solve(fac, hp[:, n], np.zeros(V.shape[0]), s)
            U[n], W[n] = uc @ V, wc @ V
            Rp[n] = uc @ P - s * W[n] - b[n]
            Rm[n] = wc @ M - s * U[n]
        r = np.sqrt(np.linalg.norm(Rp, axis=1) ** 2 + np.linalg.norm(Rm, axis=1) ** 2) / bn
        hist.append(float(r.max()))
        alpha = np.einsum("vx,fux->fvu", mu, U.reshape(nf, nd, -1))
        if r.max() < tol:
            res = Result(om_all, U, W, r, k, n_mv, True, hist, precond.n_mv)
            res.alpha = alpha
            return res
        todo = r >= tol
        nu, nw = precond.paired(Rp[todo], Rm[todo], om_all[todo])
        if V.shape[0] + 2 * int(todo.sum()) > MAX_SUBSPACE:
            # thick restart from the current and the previous solutions of every system
            # (the previous ones only where they and the new directions fit under the cap)
            keep_prev = prev is not None and 4 * U.shape[0] <= 112 and \
                4 * U.shape[0] + 2 * int(todo.sum()) <= MAX_SUBSPACE
            V = mgs(None, np.vstack([U, W] + (list(prev) if keep_prev else [])))
            P, M = op.apb_amb(V)
            n_mv += V.shape[0]
        prev = (U.copy(), W.copy())
        new = mgs(V, np.vstack([nu, nw]))
        if new.shape[0] == 0:
            break
        V = np.vstack([V, new])
        p, m = op.apb_amb(new)
        P, M = np.vstack([P, p]), np.vstack([M, m])
        n_mv += new.shape[0]
    res = Result(om_all, U, W, r, k, n_mv, False, hist, precond.n_mv)
    res.alpha = alpha
    return res


# ----------------------------------------------------------------------------
# Complete solves: initial guess + outer Davidson (Sec. 2.1, Sec. 3.1-3.2)

def solve_tda(prob, op, T, n_states, precond="rid", tol=1e-5, guess_tol=1e-3,
              inner_tol=1e-2, inner_max_iter=20, max_iter=50, max_subspace=None):
    from .operators import delta
    d = delta(prob.eps_occ, prob.eps_vir)
    k0 = min(n_init(n_states, precond), d.size)
    if precond == "rid":
        g = davidson_tda(T, k0, DiagPrecond(d), unit_guess(d, min(k0 + 8, d.size)),
                         tol=guess_tol, max_iter=max_iter)
        guess = g.X
        pc = RidPrecond(T, d, inner_tol, inner_max_iter)
        pc.n_mv = g.n_mv
    else:
        guess = unit_guess(d, k0)
        pc = DiagPrecond(d)
    return davidson_tda(op, n_states, pc, guess, tol, max_iter, max_subspace, n_keep=k0)


def solve_rpa(prob, op, T, n_states, precond="rid", tol=1e-5, guess_tol=1e-3,
              inner_tol=1e-2, inner_max_iter=20, max_iter=50, max_subspace=None):
    from .operators import delta
    d = delta(prob.eps_occ, prob.eps_vir)
    k0 = min(n_init(n_states, precond), d.size)
    if precond == "rid":
        g = davidson_rpa(T, k0, DiagPrecond(d), unit_guess(d, min(k0 + 8, d.size)),
                         tol=guess_tol, max_iter=max_iter)
        guess = np.vstack([g.X + g.Y, g.X - g.Y])
        pc = RidPrecond(T, d, inner_tol, inner_max_iter)
        pc.n_mv = g.n_mv
    else:
        guess = unit_guess(d, k0)
        pc = DiagPrecond(d)
    return davidson_rpa(op, n_states, pc, guess, tol, max_iter, max_subspace, n_keep=k0)


def solve_polar(prob, op, T, mu, omegas, precond="rid", tol=1e-5, guess_tol=1e-3,
                inner_tol=1e-2, inner_max_iter=20, max_iter=50):
    from .operators import delta
    d = delta(prob.eps_occ, prob.eps_vir)
    mu = np.atleast_2d(mu)
    nd = mu.shape[0]
    s = np.repeat(np.asarray(omegas, dtype=float), nd)
    b = np.tile(2.0 * mu, (len(omegas), 1))
    if precond == "rid":
        u, w, n0 = inner_solve_paired(T, d, b, np.zeros_like(b), s, tol=guess_tol,
                                      max_iter=max_iter)
        pc = RidPrecond(T, d, inner_tol, inner_max_iter)
        pc.n_mv = n0
    else:
        u, w = _diag_paired(d, b, np.zeros_like(b), s)
        pc = DiagPrecond(d)
    return polar_solve(op, mu, omegas, pc, np.vstack([u, w]), tol, max_iter)
