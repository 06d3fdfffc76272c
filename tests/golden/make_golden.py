"""Writes tests/golden/oracle_small.json: small seeded inputs and the FP64 oracle's outputs on them.

The paper prints no worked numerical example, so these stored values are not the paper's: every expected value
here comes from the oracle (oracle/mra_oracle.py) and only from it, on inputs that are stored next to them.  The
fixture is a regression record of the oracle's arithmetic; the oracle itself is pinned to brute force, closed
forms and invariants in tests/test_oracle_pins.py.  A change to the oracle's arithmetic regenerates this file
in the same commit, whose message names the passage of the paper (or its reading) that justifies it.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")


def c2l(a):
    """complex array -> nested [re, im] lists (shape [..., 2])."""
    a = np.asarray(a, dtype=np.complex128)
    return np.stack([a.real, a.imag], axis=-1).tolist()


def f2l(a):
    a = np.asarray(a, dtype=np.float64)
    return [None if not np.isfinite(v) else float(v) for v in a.ravel()] if a.ndim == 1 else a.tolist()


def cases():
    out = {}
    # one EM step of Algorithm Synch-EM on a grid window with a prior weight (E-step Eq. weights_2d_em,
    # a-update Eq. coefficients_update, rho-update with gamma, step size of the stopping rule)
    inst = synth.make_instance(3, 2, 9, 13, sigma2=0.2, decay=6.0, seed=101)
    x = synth.make_signal(3, 2, 6.0, np.random.default_rng(102))
    rng = np.random.default_rng(103)
    lr = np.log(rng.random(5) + 0.2)
    lr -= np.log(np.exp(lr).sum())
    lrb = np.log(np.array([0.1, 0.2, 0.4, 0.2, 0.1]))
    st = O.em_step(inst.y, x, lr, 13, 0.2, Lw=5, l0=-2, gamma=2.0, log_rho_bar=lrb, shifts=inst.s)
    out["em_step_grid"] = {
        "cite": "Algorithm Synch-EM (E-step, W_t, a-update, rho-update with gamma, step); Eq. weights_2d_em; "
                "Eq. coefficients_update",
        "inputs": {"y": c2l(inst.y), "x": c2l(x), "log_rho": f2l(lr), "log_rho_bar": f2l(lrb),
                   "shifts": inst.s.tolist(), "L": 13, "sigma2": 0.2, "Lw": 5, "l0": -2, "gamma": 2.0},
        "outputs": {"x": c2l(st.x), "log_rho": f2l(st.log_rho), "w": f2l(st.w), "loglik": st.loglik,
                    "step": st.step},
    }
    # the same on the denser-resolution window (Sec. 3.3), off-grid rotations
    inst = synth.make_instance(2, 2, 7, 11, sigma2=0.3, decay=6.0, seed=111, offgrid=True)
    x = synth.make_signal(2, 2, 6.0, np.random.default_rng(112))
    lr = np.log(np.full(6, 1 / 6))
    st = O.em_step(inst.y, x, lr, 11, 0.3, Lw=6, l0=-3, step=0.4)
    out["em_step_dense"] = {
        "cite": "Algorithm Synch-EM on the denser window of Sec. 3.3 (angles 2 pi step (l0 + i) / L)",
        "inputs": {"y": c2l(inst.y), "x": c2l(x), "log_rho": f2l(lr), "L": 11, "sigma2": 0.3, "Lw": 6, "l0": -3,
                   "step": 0.4},
        "outputs": {"x": c2l(st.x), "log_rho": f2l(st.log_rho), "w": f2l(st.w), "loglik": st.loglik,
                    "step": st.step},
    }
    # Synchronize and Match (pairwise argmin, power iteration and PPM, matching)
    inst = synth.make_instance(4, 3, 30, 17, sigma2=0.02, decay=6.0, seed=121)
    sh, phi, rel = O.synchronize_and_match(inst.y, 10, 17)
    out["synchronize_and_match"] = {
        "cite": "Algorithm Synchronize and Match; Eq. relative_angle_2d_dist; Sec. 2.1.2 (PPM)",
        "inputs": {"y": c2l(inst.y), "P": 10, "L": 17},
        "outputs": {"shifts": np.asarray(sh).astype(int).tolist(), "phi": np.asarray(phi).astype(int).tolist(),
                    "rel": np.asarray(rel).astype(int).tolist()},
    }
    # template matching against the first observation (Sec. 2.1.1)
    tm = O.template_match(inst.y, inst.y[0], 17)
    out["template_match"] = {
        "cite": "Sec. 2.1.1 (template matching)",
        "inputs": {"y": "synchronize_and_match.inputs.y", "ref": "y[0]", "L": 17},
        "outputs": {"shifts": np.asarray(tm).astype(int).tolist()},
    }
    # the window prior from a residual histogram (Algorithm 1 pooled, histogram and von Mises fit)
    counts = np.array([40, 25, 9, 3, 1, 0, 0, 0, 0, 0, 1, 4, 12, 30], dtype=np.int64)
    h_lr, _ = O.fit_prior(counts, 14, 7, l0=-3, kind=0)
    v_lr, kap = O.fit_prior(counts, 14, 7, l0=-3, kind=1)
    out["fit_prior"] = {
        "cite": "Algorithm 1 (learned distribution), Eq. learned_distribution_formula; von Mises reading of the prior",
        "inputs": {"counts": counts.tolist(), "L": 14, "Lw": 7, "l0": -3},
        "outputs": {"hist_log_rho": f2l(h_lr), "vm_log_rho": f2l(v_lr), "kappa": kap},
    }
    # the marginal log-likelihood and its gradient (Sec. 2.2, Fisher identity)
    inst = synth.make_instance(2, 2, 8, 9, sigma2=0.25, decay=6.0, seed=131)
    x = synth.make_signal(2, 2, 6.0, np.random.default_rng(132))
    logits = np.array([0.1, -0.2, 0.3, 0.0, -0.1])
    ll, dx, dl, dk = O.loglik_grad(inst.y, x, logits, 1.3, 9, 0.25, l0=-2)
    out["loglik_grad"] = {
        "cite": "Sec. 2.2 (marginal log-likelihood); gradient by the Fisher identity",
        "inputs": {"y": c2l(inst.y), "x": c2l(x), "logits": f2l(logits), "kappa": 1.3, "L": 9, "sigma2": 0.25,
                   "l0": -2},
        "outputs": {"loglik": ll, "dx": c2l(dx), "dlogits": f2l(dl), "dkappa": dk},
    }
    return out


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(cases(), f, indent=None, separators=(",", ":"))
        f.write("\n")
    print(f"wrote {OUT}")
