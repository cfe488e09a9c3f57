"""The Ising energy of Eq. (1), H(s) = sum_<ij> J_ij s_i s_j + sum_i h_i s_i, exactly.

Couplings and fields are integer numerators over a common denominator, so the
energy of a configuration is an exact integer numerator (int64); this is the
checker's energy for every configuration the oracle or the library returns.
TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def energy_num(inst, spins) -> int:
    """Exact energy numerator H(s) * denom of one configuration of +-1 spins (Eq. 1)."""
    s = np.asarray(spins, dtype=np.int64)
    pair = s[np.asarray(inst.ei)] * s[np.asarray(inst.ej)]
    return int(np.dot(np.asarray(inst.j_num, dtype=np.int64), pair) + np.dot(np.asarray(inst.h_num, dtype=np.int64), s))
