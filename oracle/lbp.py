"""Loopy belief propagation over the clusters of the Potts model (paper Sec. IV).

TEST INFRASTRUCTURE: only tests/, the smoke check and the bench's CPU
baseline use this module; the library never calls it.

The paper's two message updates and its marginal, with messages indexed by
the projected classes of Eq. (4):

  mu_{m->n}(a)  = sum over states x of m with P^{mn}(x) = a of
                  exp(-beta E_x) * prod over neighbours m' != n of nu_{m'->m}(P^{mm'}(x))
  nu_{m->n}(b)  = sum over a of exp(-beta Ebar^{mn}[a, b]) * mu_{m->n}(a)
  p(x_n)       ~  exp(-beta E_{x_n}) * prod over neighbours m of nu_{m->n}(P^{nm}(x_n))

Readings where the section is silent (the same in the CUDA path):
* neighbours are the sites joined by at least one coupling;
* synchronous schedule: every mu from the previous nu, then every nu;
* nu starts uniform (all ones) and is scaled to sum 1 after each update,
  which the marginals do not see; energies are shifted by their minima
  (constant factors, normalised away as well);
* a fixed number of iterations; the reported change is the largest
  |nu_new - nu_old| over all entries of the normalised messages of the last
  iteration (the paper quotes this quantity saturating near 1e-3);
* the reduced state set keeps the k states of largest marginal, ties to the
  smaller state index.
"""
from __future__ import annotations

import numpy as np

from .potts import DIRS, OPP, PottsModel


def neighbours(pm: PottsModel, s: int):
    """Directions from site s to the sites it shares at least one coupling with."""
    S = pm.sites[s]
    out = []
    for dname, (dr, dc) in DIRS.items():
        T = pm.site(S.r + dr, S.c + dc)
        if T is None:
            continue
        t = T.r * pm.C + T.c
        if pm.pair_edges.get((min(s, t), max(s, t))):
            out.append(dname)
    return out


def _weights(pm: PottsModel, s: int, beta: float) -> np.ndarray:
    E = pm.sites[s].E
    return np.exp(-beta * (E - E.min()) / pm.inst.denom)


def lbp(pm: PottsModel, beta: float, n_iter: int):
    """Run n_iter synchronous iterations.  Returns (marginals per site, last change)."""
    n_sites = len(pm.sites)
    nbr = [neighbours(pm, s) for s in range(n_sites)]
    # nu[(s, dname)]: message into site s from its neighbour in direction dname,
    # indexed by the classes of s toward that neighbour
    nu = {(s, d): np.ones(pm.sites[s].proj[d].n) for s in range(n_sites) for d in nbr[s]}
    w = [_weights(pm, s, beta) for s in range(n_sites)]
    change = 0.0
    for _ in range(n_iter):
        # site -> edge messages (first update of Sec. IV)
        mu = {}
        for s in range(n_sites):
            S = pm.sites[s]
            for d in nbr[s]:
                prod = w[s].copy()
                for d2 in nbr[s]:
                    if d2 != d:
                        prod = prod * nu[(s, d2)][S.proj[d2].of_state]
                mu[(s, d)] = np.bincount(S.proj[d].of_state, weights=prod, minlength=S.proj[d].n)
        # edge -> site messages (second update of Sec. IV)
        new = {}
        for s in range(n_sites):
            S = pm.sites[s]
            for d in nbr[s]:
                dr, dc = DIRS[d]
                t = (S.r + dr) * pm.C + (S.c + dc)
                Eb = pm.ebar(S.r, S.c, d)                      # [class of s, class of t]
                B = np.exp(-beta * (Eb - Eb.min()) / pm.inst.denom)
                v = B.T @ mu[(s, d)]
                new[(t, OPP[d])] = v / v.sum()
        change = max((float(np.max(np.abs(new[key] - nu[key]))) for key in nu), default=0.0)
        nu = new
    marg = []
    for s in range(n_sites):
        S = pm.sites[s]
        b = w[s].copy()
        for d in nbr[s]:
            b = b * nu[(s, d)][S.proj[d].of_state]
        marg.append(b / b.sum())
    return marg, change


def top_states(marginal: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k largest marginals, largest first, ties to the smaller index."""
    order = np.lexsort((np.arange(len(marginal)), -marginal))
    return order[:k]
