"""Excitation (droplet) bookkeeping of the branch and bound (paper Sec. III.A, Fig. 4).

TEST INFRASTRUCTURE: only tests/ and the bench's CPU legs use this module.

When the bounding step merges candidates with the same boundary (Eq. 7), the
most probable one stays as the main branch and the others differ from it
only inside the placed region: each difference is a low-energy excitation
(a droplet) above the main branch.  Droplets of a merged-away candidate are
carried over to the main branch as well, and the main branch keeps the
droplets it inherited from its parent.  Fig. 4 keeps only droplets that are
singly connected and pairwise farther apart than a Hamming threshold.

A droplet is (dE, F): F the set of flipped spins relative to the main
branch, dE the exact energy change (numerator over denom).  Because both
configurations agree on every spin coupled to an unplaced cluster, dE is the
difference of the energies restricted to the placed clusters and stays exact
for every completion.

Readings where the figure is silent (the same in the CUDA path):
* droplets with dE > max_dE are not kept (the figure speaks of low-energy
  excitations);
* "singly connected": F is connected in the interaction graph (couplings
  J != 0);
* the Hamming rule: a new droplet whose set is within min_hamming flips of
  kept ones replaces all of them if its dE is smaller than theirs, else it
  is dropped (ties keep what was there);
* order: a main branch first keeps its parent's droplets, then takes its
  merged-away candidates in order of (dE, configuration), each with its own
  droplet followed by its parent's droplets, transformed to the main branch
  (F xor F', dE + dE');
* only merges count (candidates removed by the top-M cut are discarded with
  their droplets).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from .energy import energy_num
from .peps import boundary_mps
from .potts import PottsModel
from .search import boundary_key, boundary_pairs, conditional_scores, merge_and_cut


def adjacency(inst):
    adj = [[] for _ in range(inst.n_spins)]
    for i, j, J in zip(inst.ei, inst.ej, inst.j_num):
        if J != 0:
            adj[i].append(j)
            adj[j].append(i)
    return adj


def connected(flips, adj):
    if not flips:
        return False
    fs = set(flips)
    start = next(iter(fs))
    seen = {start}
    todo = deque([start])
    while todo:
        u = todo.popleft()
        for v in adj[u]:
            if v in fs and v not in seen:
                seen.add(v)
                todo.append(v)
    return len(seen) == len(fs)


def try_insert(drops, cand, max_dE, min_hamming, adj):
    """Apply the Fig. 4 filters to candidate droplet (dE, frozenset) against the list ``drops``."""
    dE, F = cand
    if dE > max_dE or not connected(F, adj):
        return drops
    clash = [i for i, (_, G) in enumerate(drops) if len(F ^ G) <= min_hamming]
    if not clash:
        return drops + [cand]
    if dE < min(drops[i][0] for i in clash):
        gone = set(clash)
        return [d for i, d in enumerate(drops) if i not in gone] + [cand]
    return drops


def search_droplets(inst, beta, chi, M, max_dE, min_hamming, n_sweeps=2, states=None):
    """The oracle's branch and bound (search.search) with droplet bookkeeping.

    Returns dict(config, energy_num, droplets=[(dE, sorted flip list)] of the
    best final configuration, sorted by (dE, flips))."""
    pm = PottsModel(inst, states)
    _, psis, mpos = boundary_mps(pm, beta, chi, n_sweeps)
    adj = adjacency(inst)
    C = pm.C

    def spins(cfg):
        return pm.spins_of_config(cfg)

    def e_placed(cfg):
        return energy_num(inst, spins(cfg))          # unplaced spins are 0: only the placed part counts

    beam = [((), 0.0)]
    drops = {(): []}
    for n in range(pm.R * C):
        r, c = divmod(n, C)
        pairs = boundary_pairs(pm, n)
        cands = {}
        for cfg, lp in beam:
            s = np.maximum(conditional_scores(pm, beta, mpos[r], psis[r], cfg, r, c), 0.0)
            tot = s.sum()
            for x in np.nonzero(s > 0)[0]:
                cand = cfg + (int(x),)
                cands.setdefault(boundary_key(pm, pairs, cand), []).append((cand, lp + float(np.log(s[x] / tot))))
        new_beam, _ = merge_and_cut(cands, M)
        kept = {t[0] for t in new_beam}
        new_drops = {}
        for group in cands.values():
            win = [t for t in group if t[0] in kept]
            if not win:
                continue
            w = win[0][0]
            sw, ew = spins(w), e_placed(w)
            lst = list(drops[w[:-1]])
            losers = []
            for cand, _ in group:
                if cand == w:
                    continue
                losers.append((e_placed(cand) - ew, cand))
            for dE, cand in sorted(losers):
                F = frozenset(np.nonzero(spins(cand) != sw)[0].tolist())
                lst = try_insert(lst, (dE, F), max_dE, min_hamming, adj)
                for dE2, G in drops[cand[:-1]]:
                    lst = try_insert(lst, (dE + dE2, F ^ G), max_dE, min_hamming, adj)
            new_drops[w] = lst
        beam = new_beam
        drops = new_drops
    best = beam[0][0]
    out = sorted((dE, sorted(F)) for dE, F in drops[best])
    return dict(config=best, energy_num=pm.state_energy_num(best), droplets=out, pm=pm)
