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
