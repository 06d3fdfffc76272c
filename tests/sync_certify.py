"""Certification of a Synchronize-and-Match result against the FP64 oracle.

Algorithm Synchronize and Match chains three stages: the pairwise relative rotations
of the first P images (Eq. relative_angle_2d_dist), the projected power method on
their synchronization matrix (Sec. 2.1.2) and the nearest-neighbour match of every
image to the synchronized subset.  An FP32 implementation may take a different
decision than the FP64 oracle wherever the oracle's own margin between the best and
the second-best choice lies below the FP32 resolution of the arithmetic (a near-tie).

`certify_chain` takes the three stage outputs of the implementation under test and
explains every image whose final shift differs from the oracle's chain:

  pairwise  a relative rotation differs only where the two candidate distances are
            within TIE of the pair's distance scale;
  ppm       a synchronized rotation differs (by one grid step) only where the oracle's
            angle, run from the implementation's own relative rotations, lies within
            1e-3 grid steps of a rounding boundary;
  match     a shift differs only where the chosen reference is within TIE of the
            distance scale of the nearest one (given the implementation's own phi).

An image whose final shift differs is traced through its nearest reference n*: a
difference of the match stage, else of phi[n*] at the PPM stage, else of the oracle's
PPM on the implementation's relative rotations against the oracle's PPM on its own
(possible only when some relative rotation differs at a certified near-tie).
Anything else is uncertified.  This is test infrastructure and imports the oracle."""
from collections import Counter

import numpy as np

import oracle as O

TIE = 2e-5  # relative margin below which an FP32 decision may differ from the FP64 one
PPM_EDGE = 1e-3  # grid steps from a rounding boundary within which a PPM rounding may differ


def pair_dists(vi, vj, L):
    rvj = O.rotate(vj, -O.grid_angle(np.arange(L), L))
    diff = vi[None] - rvj
    return np.sum(diff.real ** 2 + diff.imag ** 2, axis=(1, 2))


def match_dists(y64, P, i):
    dd = np.sum(np.abs(y64[i][None] - y64[:P]) ** 2, axis=(1, 2))
    if i < P:
        dd[i] = np.inf
    return dd


def certify_chain(y64, P, L, g_rel, g_phi, g_match, n_power=50, n_ppm=100, o_rel=None):
    """Returns {"mismatch": images whose shift differs from the oracle chain, "causes": Counter of
    the stage each traces to, "uncertified": list of (stage, index) that no near-tie explains}."""
    y64 = np.asarray(y64)
    N = y64.shape[0]
    g_rel = np.asarray(g_rel, dtype=np.int64)
    g_phi = np.asarray(g_phi, dtype=np.int64)
    g_match = np.asarray(g_match, dtype=np.int64)
    bad = []
    # structure of the relative rotations: zero diagonal, antisymmetric mod L
    for i in range(P):
        if g_rel[i, i] != 0:
            bad.append(("pairwise-diag", i))
        for j in range(i + 1, P):
            if g_rel[j, i] != (L - g_rel[i, j]) % L:
                bad.append(("pairwise-antisym", (i, j)))
    # stage 1: pairwise, against the oracle's argmin
    if o_rel is None:
        o_rel = O.pairwise_relative(y64[:P], L)
    rel_ties = 0
    for i in range(P):
        for j in range(i + 1, P):
            if g_rel[i, j] != o_rel[i, j]:
                dd = pair_dists(y64[i], y64[j], L)
                scale = np.sum(np.abs(y64[i]) ** 2) + np.sum(np.abs(y64[j]) ** 2)
                if dd[g_rel[i, j]] - dd[o_rel[i, j]] <= TIE * scale:
                    rel_ties += 1
                else:
                    bad.append(("pairwise", (i, j)))
    # stage 2: PPM, the oracle run from the implementation's relative rotations
    ang = O.ppm_angles(g_rel, L, n_power, n_ppm)
    o_phi_g = O.ppm(g_rel, L, n_power, n_ppm)
    frac = ang * L / (2 * np.pi) + 0.5
    near_edge = np.abs(frac - np.round(frac)) < PPM_EDGE
    ppm_ok = np.ones(P, dtype=bool)
    for i in np.nonzero(g_phi != o_phi_g)[0]:
        if not (near_edge[i] and (g_phi[i] - o_phi_g[i]) % L in (1, L - 1)):
            ppm_ok[i] = False
            bad.append(("ppm", int(i)))
    # stage 3: match, the oracle's nearest reference given the implementation's phi
    n_star = O.match(y64, P, np.arange(P))  # identity phi: the index of the nearest reference
    o_match_g = g_phi[n_star]
    match_ok = np.ones(N, dtype=bool)
    for i in np.nonzero(g_match != o_match_g)[0]:
        dd = match_dists(y64, P, i)
        scale = np.sum(np.abs(y64[i]) ** 2) + np.max(np.sum(np.abs(y64[:P]) ** 2, axis=(1, 2)))
        cand = np.nonzero(dd - np.min(dd) <= TIE * scale)[0]
        if g_match[i] not in set(g_phi[cand].tolist()) or cand.size < 2:
            match_ok[i] = False
            bad.append(("match", int(i)))
    # the chain: every image that differs from the oracle's own Synchronize and Match
    o_phi = O.ppm(o_rel, L, n_power, n_ppm)
    o_chain = o_phi[n_star]
    causes = Counter()
    mism = np.nonzero(g_match != o_chain)[0]
    for i in mism:
        n = n_star[i]
        if g_match[i] != o_match_g[i]:
            causes["match"] += 1
            if not match_ok[i]:
                bad.append(("chain-match", int(i)))
        elif g_phi[n] != o_phi_g[n]:
            causes["ppm"] += 1
            if not ppm_ok[n]:
                bad.append(("chain-ppm", int(i)))
        elif o_phi_g[n] != o_phi[n]:
            causes["pairwise"] += 1
            if rel_ties == 0:
                bad.append(("chain-pairwise", int(i)))
        else:
            bad.append(("chain-unexplained", int(i)))
    return {"mismatch": int(mism.size), "causes": causes, "uncertified": bad, "rel_ties": rel_ties,
            "o_chain": o_chain}
