"""Seeded synthetic inputs for the TDDFT response problem.

This module only draws numbers: orbital energies, three-index factors L^P_pq,
the minimal-auxiliary ("ris") factors and dipole vectors.  It contains none of
the response-method arithmetic, so both the CPU oracle and the CUDA path read
their inputs from here and share nothing else.

Shapes follow the paper's statement of the problem with the integral
generation abstracted away (Sec. 2.2, Eqs. hessian and pqrs_approx): the
Coulomb-type integral is (pq|rs) = sum_P L^P_pq L^P_rs, so every factor block
is an [n_aux][p][q] array, symmetric in (p, q) for each P.

Generator conventions (each one a stated reading, not taken from the paper):

* every random stream is numpy ``Generator(Philox(key=(seed, index)))`` so a
  P-slice of the factors can be regenerated on its own;
* L^P over all n_mo = n_occ + n_vir orbitals is a symmetric matrix whose upper
  triangle (diagonal included) is N(0, 1), scaled by amp * exp(-P / d) with the
  decay length d = 60 * n_aux / 200 ("decay scaled to n_aux");
* the amplitude is amp = scale * 0.1 * sqrt(S(200, 60) / S(n_aux, d)), S(n, d) =
  sum_{P<n} exp(-2P/d), with a per-workload scale 0.7^k: the smallest k that
  leaves lambda_min(A-B) and lambda_min(A+B) above 0.02 Ha and lets the
  diagonal-preconditioned Davidson converge 10 states within the iteration
  range the paper reports for the diagonal preconditioner (Table 1, at most
  33).  A dense random coupling grows like sqrt(n_occ n_vir) at fixed
  element size, so larger workloads need a smaller scale; the literal 0.3
  gives indefinite Hessians and is only kept as an optional TDA input;
* the ris Coulomb factors are sqrt(0.9) times the leading n_ris rows of the
  exact factors plus an independent symmetric N(0, (0.1 sigma_P)^2)
  perturbation; the ris exchange factors are the s-type rows, one per atom,
  which are rows 0, 9, 18, ... of the ris Coulomb set (9 functions per atom:
  one s, three p, five d).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

HARTREE_PER_EV = 1.0 / 27.211386245988


def _rng(seed: int, index: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=np.array([seed, index], dtype=np.uint64)))


def default_amplitude(n_aux: int) -> float:
    """Amplitude that keeps the synthetic Hessians positive definite."""
    d = 60.0 * n_aux / 200.0
    s_ref = sum(math.exp(-2.0 * p / 60.0) for p in range(200))
    s_n = sum(math.exp(-2.0 * p / d) for p in range(n_aux))
    return 0.1 * math.sqrt(s_ref / s_n)


@dataclass
class Problem:
    """One synthetic TDDFT response problem (all arrays float64, C order)."""

    n_occ: int
    n_vir: int
    n_aux: int
    n_ris: int
    eps_occ: np.ndarray            # [n_occ], ascending
    eps_vir: np.ndarray            # [n_vir], ascending
    L_oo: np.ndarray               # [n_aux][n_occ][n_occ]
    L_ov: np.ndarray               # [n_aux][n_occ][n_vir]
    L_vv: np.ndarray               # [n_aux][n_vir][n_vir]
    Lr_ov: np.ndarray              # [n_ris][n_occ][n_vir]   ris Coulomb rows
    Lr_oo: np.ndarray              # [n_ris][n_occ][n_occ]
    Lr_vv: np.ndarray              # [n_ris][n_vir][n_vir]
    ris_K_index: np.ndarray        # [n_ris_K] int32: rows of the ris set used for exchange
    a_x: float = 0.25
    coulomb_factor: float = 2.0
    t_cut_ha: float = 40.0 * HARTREE_PER_EV
    amplitude: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n_ov(self) -> int:
        return self.n_occ * self.n_vir

    @property
    def n_ris_K(self) -> int:
        return int(self.ris_K_index.shape[0])


def _symmetric_rows(seed: int, n_rows: int, n: int, scale: np.ndarray, row0: int = 0) -> np.ndarray:
    out = np.empty((n_rows, n, n))
    iu = np.triu_indices(n)
    for r in range(n_rows):
        g = _rng(seed, row0 + r).standard_normal(iu[0].size)
        m = np.zeros((n, n))
        m[iu] = g
        m = m + np.triu(m, 1).T
        out[r] = m * scale[r]
    return out


def orbital_energies(seed: int, n_occ: int, n_vir: int):
    g = _rng(seed, 0)
    eo = np.sort(g.uniform(-0.8, -0.3, n_occ))
    ev = np.sort(g.uniform(0.05, 1.5, n_vir))
    return eo, ev


def make_problem(n_occ: int, n_vir: int, n_aux: int, n_ris: int, seeds=(0, 1, 2),
                 a_x: float = 0.25, coulomb_factor: float = 2.0,
                 amplitude: Optional[float] = None, ris_noise: float = 0.1,
                 ris_scale: float = 0.9) -> Problem:
    """Draw one problem.  ``seeds`` = (orbital energies, exact factors, ris perturbation)."""
    if n_ris % 9 != 0:
        raise ValueError("n_ris must be 9 * n_atom (s, p, d functions per atom)")
    s_eps, s_L, s_ris = seeds
    eo, ev = orbital_energies(s_eps, n_occ, n_vir)
    n_mo = n_occ + n_vir
    amp = default_amplitude(n_aux) if amplitude is None else float(amplitude)
    d = 60.0 * n_aux / 200.0
    sigma = amp * np.exp(-np.arange(n_aux) / d)
    L = _symmetric_rows(s_L, n_aux, n_mo, sigma)
    o, v = slice(0, n_occ), slice(n_occ, n_mo)
    n_r = min(n_ris, n_aux)
    noise = _symmetric_rows(s_ris, n_ris, n_mo, ris_noise * np.resize(sigma[:n_r], n_ris))
    Lr = np.zeros((n_ris, n_mo, n_mo))
    Lr[:n_r] = math.sqrt(ris_scale) * L[:n_r]
    Lr += noise
    k_index = np.arange(0, n_ris, 9, dtype=np.int32)
    return Problem(
        n_occ=n_occ, n_vir=n_vir, n_aux=n_aux, n_ris=n_ris,
        eps_occ=eo, eps_vir=ev,
        L_oo=np.ascontiguousarray(L[:, o, o]), L_ov=np.ascontiguousarray(L[:, o, v]),
        L_vv=np.ascontiguousarray(L[:, v, v]),
        Lr_ov=np.ascontiguousarray(Lr[:, o, v]), Lr_oo=np.ascontiguousarray(Lr[:, o, o]),
        Lr_vv=np.ascontiguousarray(Lr[:, v, v]), ris_K_index=k_index,
        a_x=a_x, coulomb_factor=coulomb_factor, amplitude=amp,
        extra={"L_full": L if n_mo <= 80 else None, "Lr_full": Lr if n_mo <= 80 else None},
    )


def with_variant_terms(prob: Problem, seed: int, n_aux_lr: int = 0, b_x: float = 0.0, n_kernel: int = 0,
                       lr_scale: float = 0.6, kernel_amp: Optional[float] = None) -> Problem:
    """Attach the optional variant terms of the response operator to a problem.

    * a second exchange factor set M (``extra["exchange_lr"]``) standing in for the
      long-range exchange integrals of a range-separated hybrid: n_aux_lr symmetric
      rows over all orbitals, N(0, 1) upper triangles scaled by lr_scale * amp *
      exp(-Q / d), d = 60 n_aux_lr / 200, with weight b_x;
    * a low-rank response kernel (``extra["kernel"]``) standing in for f^xc:
      n_kernel symmetric rows F^g over all orbitals scaled by kernel_amp *
      exp(-g / 60), kernel_amp = 0.15 / sqrt(n_occ n_vir) by default (so that a
      row's contribution w_g |F^g_ov|^2 stays near 0.02 Ha at any size), and
      weights w_g ~ U(-1, 0.5) (mostly negative, as an exchange-correlation
      kernel is).
    Streams: Philox keyed (seed, row) for M, (seed + 1, row) for F, (seed + 2, 0)
    for w.  The problem's own arrays are shared, not copied."""
    n_mo = prob.n_occ + prob.n_vir
    o, v = slice(0, prob.n_occ), slice(prob.n_occ, n_mo)
    extra = dict(prob.extra)
    if n_aux_lr > 0:
        d = 60.0 * n_aux_lr / 200.0
        sig = lr_scale * prob.amplitude * np.exp(-np.arange(n_aux_lr) / d)
        M = _symmetric_rows(seed, n_aux_lr, n_mo, sig)
        extra["exchange_lr"] = dict(M_oo=np.ascontiguousarray(M[:, o, o]), M_ov=np.ascontiguousarray(M[:, o, v]),
                                    M_vv=np.ascontiguousarray(M[:, v, v]), b_x=float(b_x),
                                    M_full=M if n_mo <= 80 else None)
    if n_kernel > 0:
        ka = 0.15 / math.sqrt(prob.n_occ * prob.n_vir) if kernel_amp is None else kernel_amp
        sig = ka * np.exp(-np.arange(n_kernel) / 60.0)
        F = _symmetric_rows(seed + 1, n_kernel, n_mo, sig)
        w = _rng(seed + 2, 0).uniform(-1.0, 0.5, n_kernel)
        extra["kernel"] = dict(F_ov=np.ascontiguousarray(F[:, o, v]), w=w, F_full=F if n_mo <= 80 else None)
    return Problem(**{**prob.__dict__, "extra": extra})


def factor_rows(name: str, p0: int, p1: int, **over):
    """Rows [p0, p1) of a named workload's exact factors, drawn exactly as
    make_config draws them (per-row Philox streams), without building the
    whole [n_aux][n_mo][n_mo] array: returns (L_oo, L_ov, L_vv) float64 slices.
    For workloads too large to hold in host memory at once."""
    c = _config_args(name, over)
    n_occ, n_mo, n_aux = c["n_occ"], c["n_occ"] + c["n_vir"], c["n_aux"]
    d = 60.0 * n_aux / 200.0
    sigma = c["amplitude"] * np.exp(-np.arange(n_aux) / d)
    L = _symmetric_rows(c["seeds"][1], p1 - p0, n_mo, sigma[p0:p1], row0=p0)
    o, v = slice(0, n_occ), slice(n_occ, n_mo)
    return (np.ascontiguousarray(L[:, o, o]), np.ascontiguousarray(L[:, o, v]),
            np.ascontiguousarray(L[:, v, v]))


def ris_rows(name: str, r0: int, r1: int, **over):
    """Rows [r0, r1) of a named workload's ris factors (as make_config builds
    them): returns (Lr_oo, Lr_ov, Lr_vv) float64 slices."""
    c = _config_args(name, over)
    n_occ, n_mo, n_aux, n_ris = c["n_occ"], c["n_occ"] + c["n_vir"], c["n_aux"], c["n_ris"]
    d = 60.0 * n_aux / 200.0
    sigma = c["amplitude"] * np.exp(-np.arange(n_aux) / d)
    n_r = min(n_ris, n_aux)
    scale = 0.1 * np.resize(sigma[:n_r], n_ris)
    Lr = _symmetric_rows(c["seeds"][2], r1 - r0, n_mo, scale[r0:r1], row0=r0)
    hi = min(r1, n_r)
    if hi > r0:
        Lr[: hi - r0] += math.sqrt(0.9) * _symmetric_rows(c["seeds"][1], hi - r0, n_mo, sigma[r0:hi], row0=r0)
    o, v = slice(0, n_occ), slice(n_occ, n_mo)
    return (np.ascontiguousarray(Lr[:, o, o]), np.ascontiguousarray(Lr[:, o, v]),
            np.ascontiguousarray(Lr[:, v, v]))


def config_meta(name: str, **over) -> dict:
    """Sizes, orbital energies, amplitude and ris exchange rows of a named
    workload, without drawing its factors."""
    c = _config_args(name, over)
    eo, ev = orbital_energies(c["seeds"][0], c["n_occ"], c["n_vir"])
    return dict(n_occ=c["n_occ"], n_vir=c["n_vir"], n_aux=c["n_aux"], n_ris=c["n_ris"], eps_occ=eo,
                eps_vir=ev, amplitude=c["amplitude"], ris_K_index=np.arange(0, c["n_ris"], 9, dtype=np.int32),
                a_x=c.get("a_x", 0.25), coulomb_factor=c.get("coulomb_factor", 2.0),
                t_cut_ha=40.0 * HARTREE_PER_EV)


def dipoles(seed: int, n_dip: int, n_ov: int, sigma: float = 0.1) -> np.ndarray:
    """Dipole right-hand sides mu^u_ia ~ N(0, sigma^2), shape [n_dip][n_ov]."""
    return _rng(seed, 0).normal(0.0, sigma, size=(n_dip, n_ov))


# Named workloads.  Sizes are the response-problem shapes (occupied, virtual,
# exact auxiliary and ris auxiliary counts) of the paper's benchmark regime.
CONFIGS = {
    "tda_small": dict(n_occ=10, n_vir=40, n_aux=200, n_ris=90, seeds=(0, 1, 2),
                      n_states=5, mu_seed=3),
    # amplitude scale 0.7^5: at 1.0 lambda_min(A-B) = -0.26 Ha (0.7: +0.21 Ha); at
    # 0.7^2 .. 0.7^4 the diagonal preconditioner needs 40 to more than 80 iterations
    "rpa_polar_medium": dict(n_occ=60, n_vir=400, n_aux=2000, n_ris=360, seeds=(10, 11, 12),
                             n_states=10, mu_seed=13, omegas=(0.0, 0.05, 0.1), n_dip=3,
                             amplitude_scale=0.7 ** 5),
    # amplitude scale 0.7^7: the exchange coupling of a dense random factor set
    # grows like sqrt(n_occ n_vir) (2.9x the medium workload), so two more steps
    # of 0.7 than the medium keep the same margin; the full-size GPU test checks
    # lambda_min(A+B), lambda_min(A-B) > 0.02 Ha and the diagonal-preconditioned
    # convergence within 33 iterations
    "large_mixed": dict(n_occ=150, n_vir=1350, n_aux=6000, n_ris=1350, seeds=(20, 21, 22),
                        n_states=20, mu_seed=23, amplitude_scale=0.7 ** 7),
    # the large workload's orbital shape over 100 auxiliary rows (one P-chunk,
    # ~2.5 GB on the device): the small case for profiling its kernels
    "large_orbitals_short_aux": dict(n_occ=150, n_vir=1350, n_aux=100, n_ris=18, seeds=(70, 71, 72),
                                     n_states=20, mu_seed=73),
}


def _config_args(name: str, over: dict) -> dict:
    c = dict(CONFIGS[name])
    c.update(over)
    if "amplitude" not in c:
        c["amplitude"] = c.get("amplitude_scale", 1.0) * default_amplitude(c["n_aux"])
    return c


def make_config(name: str, **over) -> Problem:
    c = _config_args(name, over)
    return make_problem(c["n_occ"], c["n_vir"], c["n_aux"], c["n_ris"], seeds=c["seeds"],
                        **{k: c[k] for k in ("a_x", "coulomb_factor", "amplitude") if k in c})
