"""The Synchronize-and-Match certifier on the CPU: the oracle's own chain certifies with no
mismatch, and a planted mistake in any stage (a relative rotation, a synchronized rotation
or a match that no near-tie explains) is reported as uncertified."""
import numpy as np
import pytest

import oracle as O
import synth
from sync_certify import certify_chain


@pytest.fixture(scope="module")
def chain():
    inst = synth.make_instance(6, 4, 240, 36, 1 / 10, 50.0, seed=77)
    y64 = inst.y
    P = 24
    s, phi, rel = O.synchronize_and_match(y64, P, inst.L)
    return y64, P, inst.L, rel, phi, s


def test_oracle_chain_certifies_itself(chain):
    y64, P, L, rel, phi, s = chain
    rep = certify_chain(y64, P, L, rel, phi, s, o_rel=rel)
    assert rep["mismatch"] == 0 and not rep["uncertified"]
    np.testing.assert_array_equal(rep["o_chain"], s)


def test_planted_match_error_is_uncertified(chain):
    y64, P, L, rel, phi, s = chain
    g = s.copy()
    i = P + 5
    dd = np.sum(np.abs(y64[i][None] - y64[:P]) ** 2, axis=(1, 2))
    far = int(np.argmax(dd))
    assert phi[far] != s[i]
    g[i] = phi[far]
    rep = certify_chain(y64, P, L, rel, phi, g, o_rel=rel)
    assert rep["mismatch"] == 1
    assert ("match", i) in rep["uncertified"]


def test_planted_ppm_error_is_uncertified(chain):
    y64, P, L, rel, phi, s = chain
    ph = phi.copy()
    n = 3
    ph[n] = (ph[n] + 1) % L
    n_star = O.match(y64, P, np.arange(P))
    g = ph[n_star]  # the match stage applied faithfully to the wrong phi
    rep = certify_chain(y64, P, L, rel, ph, g, o_rel=rel)
    assert ("ppm", n) in rep["uncertified"]
    assert rep["mismatch"] == int(np.sum(n_star == n))


def test_planted_pairwise_error_is_uncertified(chain):
    y64, P, L, rel, phi, s = chain
    r = rel.copy()
    r[0, 1] = (r[0, 1] + L // 2) % L
    r[1, 0] = (L - r[0, 1]) % L
    rep = certify_chain(y64, P, L, r, phi, s, o_rel=rel)
    assert ("pairwise", (0, 1)) in rep["uncertified"]
    r2 = rel.copy()
    r2[2, 5] = (r2[2, 5] + 1) % L  # breaks antisymmetry
    rep = certify_chain(y64, P, L, r2, phi, s, o_rel=rel)
    assert ("pairwise-antisym", (2, 5)) in rep["uncertified"]
