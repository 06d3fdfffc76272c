"""The oracle against its stored regression record (tests/golden/oracle_small.json, written by
tests/golden/make_golden.py from the oracle alone).  Inputs come from the file, not from the generator, so a
change of the random streams cannot move them; a change of the oracle's arithmetic shows up here and must come
with a regenerated record."""
import json
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_small.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


def cx(v):
    a = np.asarray(v, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


def fl(v):
    return np.array([-np.inf if t is None else t for t in v], dtype=np.float64)


def close(got, want, tol=1e-12):
    got, want = np.asarray(got), np.asarray(want)
    scale = max(1.0, float(np.max(np.abs(want[np.isfinite(want)]))) if np.any(np.isfinite(want)) else 1.0)
    np.testing.assert_array_equal(np.isfinite(got), np.isfinite(want))
    m = np.isfinite(want)
    assert np.max(np.abs(got[m] - want[m]), initial=0.0) <= tol * scale


@pytest.mark.parametrize("case", ["em_step_grid", "em_step_dense"])
def test_em_step_record(gold, case):
    g = gold[case]
    i, o = g["inputs"], g["outputs"]
    kw = dict(Lw=i["Lw"], l0=i["l0"], step=i.get("step", 1.0))
    if "gamma" in i:
        kw.update(gamma=i["gamma"], log_rho_bar=fl(i["log_rho_bar"]))
    if "shifts" in i:
        kw.update(shifts=np.array(i["shifts"]))
    st = O.em_step(cx(i["y"]), cx(i["x"]), fl(i["log_rho"]), i["L"], i["sigma2"], **kw)
    close(st.x, cx(o["x"]))
    close(st.log_rho, fl(o["log_rho"]))
    close(st.w, np.asarray(o["w"]))
    close([st.loglik], [o["loglik"]])
    close([st.step], [o["step"]])


def test_synchronize_and_match_record(gold):
    g = gold["synchronize_and_match"]
    sh, phi, rel = O.synchronize_and_match(cx(g["inputs"]["y"]), g["inputs"]["P"], g["inputs"]["L"])
    np.testing.assert_array_equal(sh, g["outputs"]["shifts"])
    np.testing.assert_array_equal(phi, g["outputs"]["phi"])
    np.testing.assert_array_equal(rel, g["outputs"]["rel"])


def test_template_match_record(gold):
    y = cx(gold["synchronize_and_match"]["inputs"]["y"])
    got = O.template_match(y, y[0], gold["template_match"]["inputs"]["L"])
    np.testing.assert_array_equal(got, gold["template_match"]["outputs"]["shifts"])


def test_fit_prior_record(gold):
    i, o = gold["fit_prior"]["inputs"], gold["fit_prior"]["outputs"]
    h, _ = O.fit_prior(np.array(i["counts"]), i["L"], i["Lw"], l0=i["l0"], kind=0)
    v, kap = O.fit_prior(np.array(i["counts"]), i["L"], i["Lw"], l0=i["l0"], kind=1)
    close(h, fl(o["hist_log_rho"]))
    close(v, fl(o["vm_log_rho"]))
    close([kap], [o["kappa"]], tol=1e-10)


def test_loglik_grad_record(gold):
    i, o = gold["loglik_grad"]["inputs"], gold["loglik_grad"]["outputs"]
    ll, dx, dl, dk = O.loglik_grad(cx(i["y"]), cx(i["x"]), fl(i["logits"]), i["kappa"], i["L"], i["sigma2"],
                                   l0=i["l0"])
    close([ll], [o["loglik"]])
    close(dx, cx(o["dx"]))
    close(dl, fl(o["dlogits"]))
    close([dk], [o["dkappa"]])


def test_record_cites_a_passage_for_every_case(gold):
    for name, g in gold.items():
        assert g["cite"], name
