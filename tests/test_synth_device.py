"""The device-side generator of served problems, run on the CPU: shapes,
symmetry, the ris rows' relation to the exact rows, and the request mix."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth.device import problem_kw, serving_mix  # noqa: E402


def test_problem_shapes_symmetry_and_ris_rows():
    no, nv, na, nr = 6, 30, 180, 27
    kw = problem_kw(3, no, nv, na, nr, device="cpu")
    assert tuple(kw["L_oo"].shape) == (na, no, no) and tuple(kw["L_vv"].shape) == (na, nv, nv)
    assert tuple(kw["L_ov"].shape) == (na, no, nv) and tuple(kw["Lr_ov"].shape) == (nr, no, nv)
    assert list(kw["ris_K_index"].numpy()) == [0, 9, 18]
    assert tuple(kw["Lr_oo"].shape) == (3, no, no) and tuple(kw["Lr_vv"].shape) == (3, nv, nv)
    for k in ("L_oo", "L_vv", "Lr_oo", "Lr_vv"):
        t = kw[k]
        assert torch.equal(t, t.transpose(1, 2)), k
    assert np.all(np.diff(kw["eps_occ"].numpy()) >= 0) and np.all(np.diff(kw["eps_vir"].numpy()) >= 0)
    # ris Coulomb rows: sqrt(0.9) x the exact rows + a perturbation of 0.1 sigma_P
    d = kw["Lr_ov"] - math.sqrt(0.9) * kw["L_ov"][:nr]
    ratio = float(d.norm() / kw["L_ov"][:nr].norm())
    assert 0.03 < ratio < 0.3
    # decay exp(-P/60): row norms fall by e^-2 over 120 rows
    rn = kw["L_vv"].flatten(1).norm(dim=1).numpy()
    assert abs(math.log(rn[120:150].mean() / rn[:30].mean()) + 2.0) < 0.15


def test_request_mix():
    mix = serving_mix(7, 4000, max_occ=150)
    kinds = np.bincount([m["kind"] for m in mix], minlength=3) / len(mix)
    assert abs(kinds[0] - 0.60) < 0.03 and abs(kinds[1] - 0.25) < 0.03 and abs(kinds[2] - 0.15) < 0.03
    no = np.array([m["n_occ"] for m in mix])
    assert no.min() >= 10 and no.max() <= 150
    assert abs(np.median(np.log(no)) - 0.5 * (math.log(10) + math.log(150))) < 0.1   # log-uniform
    for m in mix[:200]:
        assert m["n_vir"] % m["n_occ"] == 0 and 4 <= m["n_vir"] // m["n_occ"] <= 9
        assert m["n_aux"] == 5 * (m["n_occ"] + m["n_vir"]) and m["n_ris"] == 9 * math.ceil(m["n_occ"] / 2)
        assert 5 <= m["n_states"] <= 20 and 1 <= m["n_freq"] <= 4


def test_served_problems_are_well_posed_for_rid():
    """The served-stream amplitude rule keeps A+B and A-B positive definite and
    lets the oracle's rid-preconditioned TDA solve converge in the paper's
    regime (at most 12 outer iterations on these samples)."""
    from oracle import davidson as DV
    from oracle import operators as O
    from synth.generator import Problem

    mix = serving_mix(2404, 60, max_occ=40)
    picked = [(i, m) for i, m in enumerate(mix) if m["n_occ"] <= 12][:2]
    assert picked
    for i, m in picked:
        kw = problem_kw(1000 + i, m["n_occ"], m["n_vir"], m["n_aux"], m["n_ris"], device="cpu")
        f = lambda t: t.double().numpy()
        nr, k = m["n_ris"], kw["ris_K_index"].numpy()
        Lr_oo = np.zeros((nr, m["n_occ"], m["n_occ"]))
        Lr_oo[k] = f(kw["Lr_oo"])
        Lr_vv = np.zeros((nr, m["n_vir"], m["n_vir"]))
        Lr_vv[k] = f(kw["Lr_vv"])
        p = Problem(n_occ=m["n_occ"], n_vir=m["n_vir"], n_aux=m["n_aux"], n_ris=nr, eps_occ=f(kw["eps_occ"]),
                    eps_vir=f(kw["eps_vir"]), L_oo=f(kw["L_oo"]), L_ov=f(kw["L_ov"]), L_vv=f(kw["L_vv"]),
                    Lr_ov=f(kw["Lr_ov"]), Lr_oo=Lr_oo, Lr_vv=Lr_vv, ris_K_index=k.astype(np.int32))
        op, T = O.exact_operator(p), O.ris_operator(p)
        E = np.eye(p.n_ov)
        apb, amb = op.apb_amb(E)
        assert np.linalg.eigvalsh(0.5 * (apb + apb.T))[0] > 0.02
        assert np.linalg.eigvalsh(0.5 * (amb + amb.T))[0] > 0.02
        r = DV.solve_tda(p, op, T, min(m["n_states"], 10), precond="rid")
        assert r.n_iter <= 12, (m, r.n_iter)
