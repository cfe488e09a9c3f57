"""Exhaustive enumeration over all 2^N spin states (N <= 24); test pins only.

Z = sum_s exp(-beta H(s)) (Eq. 9), marginals and the ground state by the
plain definitions, used to pin the oracle before anything is compared to it.
"""
from __future__ import annotations

import numpy as np


def all_spins(n):
    idx = np.arange(1 << n, dtype=np.int64)
    return (1 - 2 * ((idx[:, None] >> np.arange(n)[None, :]) & 1)).astype(np.int8)


def energies_num(inst, spins=None):
    s = all_spins(inst.n_spins) if spins is None else spins
    s = s.astype(np.int64)
    return (s[:, inst.ei] * s[:, inst.ej]) @ inst.j_num.astype(np.int64) + s @ inst.h_num.astype(np.int64)


def log_z(inst, beta):
    E = energies_num(inst) / inst.denom
    m = (-beta * E).max()
    return float(m + np.log(np.sum(np.exp(-beta * E - m))))


def ground_state(inst):
    S = all_spins(inst.n_spins)
    E = energies_num(inst, S)
    i = int(np.argmin(E))
    return S[i], int(E[i])


def correlators(inst, beta):
    """<s_i s_j> on every edge, <s_i>, <H> under the Boltzmann distribution."""
    S = all_spins(inst.n_spins).astype(np.float64)
    E = energies_num(inst) / inst.denom
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    ss = (S[:, inst.ei] * S[:, inst.ej]).T @ p
    m = S.T @ p
    return ss, m, float(E @ p)
