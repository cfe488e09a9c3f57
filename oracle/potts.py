"""Clustering an Ising instance into a generalized Potts model (paper Sec. III).

Follows Eq. (2): H = sum_<m,n> E_{x_m x_n} + sum_n E_{x_n}, with the
compressed inter-cluster energies of Eqs. (3)-(4): E_{x_m x_n} =
Ebar[P^{mn}(x_m), P^{nm}(x_n)], where P^{mn} maps a cluster state to the
sub-configuration of the spins of m that are coupled to n.

Conventions (readings where the paper is silent):
* a cluster state x is a bit pattern over the cluster's spins, local bit j
  for the j-th spin in increasing global index; bit 0 means s = +1, bit 1
  means s = -1;
* the classes of a projector are the distinct restrictions present among the
  cluster's states, numbered in increasing bit-pattern order of the
  restriction (restricted bit j = j-th coupled spin in increasing local order);
* energies are kept as integer numerators over ``denom``.
"""
from __future__ import annotations

import numpy as np

from .energy import energy_num

# neighbour directions of site (r, c): name -> (dr, dc)
DIRS = {"r": (0, 1), "l": (0, -1), "d": (1, 0), "u": (-1, 0),
        "dr": (1, 1), "dl": (1, -1), "ur": (-1, 1), "ul": (-1, -1)}
OPP = {"r": "l", "l": "r", "d": "u", "u": "d", "dr": "ul", "ul": "dr", "dl": "ur", "ur": "dl"}


def restrict(states: np.ndarray, bits) -> np.ndarray:
    """Restriction of each state to the given local bit positions (bit j of result = bits[j])."""
    out = np.zeros(states.shape, dtype=np.int64)
    for j, b in enumerate(bits):
        out |= ((states >> b) & 1) << j
    return out


class Projection:
    """Classes of the restriction of a site's states to a set of local bits."""

    def __init__(self, states: np.ndarray, bits):
        self.bits = list(bits)
        vals = restrict(states, self.bits)
        self.values = np.unique(vals)            # restricted pattern of each class
        self.of_state = np.searchsorted(self.values, vals)
        self.n = len(self.values)

    def class_of_values(self, vals):
        idx = np.searchsorted(self.values, vals)
        assert np.all(self.values[idx] == vals)
        return idx


class Site:
    def __init__(self, r, c, spins, states=None):
        self.r, self.c = r, c
        self.spins = list(spins)                 # global spin ids, increasing
        self.local = {g: j for j, g in enumerate(self.spins)}
        k = len(self.spins)
        if states is None:
            states = np.arange(1 << k, dtype=np.int64)
        self.states = np.asarray(states, dtype=np.int64)
        self.d = len(self.states)
        self.E = None                            # int64 intra-cluster energy numerators
        self.coupled = {}                        # dir -> sorted local bits coupled to that neighbour
        self.proj = {}                           # dir -> Projection


class PottsModel:
    """Clusters, intra energies E_x, projectors and compressed energies Ebar (Eqs. 2-4)."""

    def __init__(self, inst, states_per_site=None):
        self.inst = inst
        R, C = inst.rows, inst.cols
        self.R, self.C = R, C
        spins_of = [[] for _ in range(R * C)]
        for i, s in enumerate(inst.site_of_spin.tolist()):
            spins_of[s].append(i)
        self.sites = []
        for s in range(R * C):
            st = None if states_per_site is None else states_per_site[s]
            self.sites.append(Site(s // C, s % C, spins_of[s], st))
        site_of = inst.site_of_spin
        # spin values of each state: s = 1 - 2 * bit
        for S in self.sites:
            k = len(S.spins)
            bits = ((S.states[:, None] >> np.arange(k)[None, :]) & 1) if k else np.zeros((S.d, 0), np.int64)
            S.spinvals = (1 - 2 * bits).astype(np.int64)      # [d, k]
            S.E = np.zeros(S.d, dtype=np.int64)
            if k:
                S.E += S.spinvals @ inst.h_num[S.spins].astype(np.int64)
        # edges: intra or inter
        self.pair_edges = {}                     # (s, t) with s < t -> list of (i, j, J)
        for i, j, J in zip(inst.ei.tolist(), inst.ej.tolist(), inst.j_num.tolist()):
            si, sj = int(site_of[i]), int(site_of[j])
            if si == sj:
                S = self.sites[si]
                S.E += J * S.spinvals[:, S.local[i]] * S.spinvals[:, S.local[j]]
            else:
                a, b = (si, sj) if si < sj else (sj, si)
                ii, jj = (i, j) if si < sj else (j, i)
                self.pair_edges.setdefault((a, b), []).append((ii, jj, J))
        # every inter-cluster pair must be a king's-graph neighbour
        for (a, b) in self.pair_edges:
            ra, ca = divmod(a, C)
            rb, cb = divmod(b, C)
            if max(abs(ra - rb), abs(ca - cb)) != 1:
                raise ValueError(f"clusters {a},{b} coupled but not neighbours on the grid")
        # coupled bit sets per direction
        for S in self.sites:
            me = S.r * C + S.c
            for dname, (dr, dc) in DIRS.items():
                rr, cc = S.r + dr, S.c + dc
                bits = []
                if 0 <= rr < R and 0 <= cc < C:
                    t = rr * C + cc
                    for (i, j, J) in self.pair_edges.get((min(me, t), max(me, t)), []):
                        mine = i if site_of[i] == me else j
                        bits.append(S.local[mine])
                S.coupled[dname] = sorted(set(bits))
                S.proj[dname] = Projection(S.states, S.coupled[dname])

    def site(self, r, c):
        if 0 <= r < self.R and 0 <= c < self.C:
            return self.sites[r * self.C + c]
        return None

    def ebar(self, r, c, dname):
        """Ebar[a, b]: a = class of site (r,c) toward dname, b = class of the neighbour toward us (Eq. 3)."""
        S = self.site(r, c)
        dr, dc = DIRS[dname]
        T = self.site(r + dr, c + dc)
        if S is None or T is None:
            return np.zeros((1, 1), dtype=np.int64)
        PS, PT = S.proj[dname], T.proj[OPP[dname]]
        out = np.zeros((PS.n, PT.n), dtype=np.int64)
        me, them = S.r * self.C + S.c, T.r * self.C + T.c
        for (i, j, J) in self.pair_edges.get((min(me, them), max(me, them)), []):
            mine, theirs = (i, j) if self.inst.site_of_spin[i] == me else (j, i)
            bs = PS.bits.index(S.local[mine])
            bt = PT.bits.index(T.local[theirs])
            sa = 1 - 2 * ((PS.values >> bs) & 1)
            sb = 1 - 2 * ((PT.values >> bt) & 1)
            out += J * np.outer(sa, sb)
        return out

    def joint(self, r, c, dnames):
        """Projection of site (r,c) onto the union of spins coupled toward ``dnames``."""
        S = self.site(r, c)
        bits = sorted(set(b for d in dnames for b in S.coupled[d]))
        return Projection(S.states, bits)

    def component(self, joint: "Projection", S: Site, dname):
        """Class (toward dname) of every class of a joint projection."""
        P = S.proj[dname]
        sub = [joint.bits.index(b) for b in P.bits]
        vals = restrict(joint.values, sub)
        return P.class_of_values(vals)

    def spins_of_config(self, config) -> np.ndarray:
        s = np.zeros(self.inst.n_spins, dtype=np.int64)
        for S, x in zip(self.sites, config):
            if len(S.spins):
                s[S.spins] = S.spinvals[x]
        return s

    def state_energy_num(self, config) -> int:
        """Energy numerator of a full Potts configuration (state index per site)."""
        return energy_num(self.inst, self.spins_of_config(config))
