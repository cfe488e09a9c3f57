"""Gradient of log Z (paper Eq. 9) with respect to J_ij, h_i and beta.

d log Z / dJ_ij = -beta <s_i s_j>, d log Z / dh_i = -beta <s_i> and
d log Z / dbeta = -<H> are evaluated as environment correlators of the
approximately contracted network: for row r the sandwich

    Z_r = <E_r| T_r |psi_r>

joins the boundary MPS of the rows below (psi_r, bottom-up) and an upper
boundary MPS E_r of the rows above (top-down, same truncation algorithm on the
transposed row MPOs).  Every Boltzmann factor sits in exactly one row MPO, so
the expectation of a spin product carried by a factor of T_r is
<E_r| T_r' |psi_r> / Z_r with T_r' the row MPO whose factor is multiplied by
that spin product.  With exact contraction these are the exact Boltzmann
correlators; with truncation they are the standard environment estimates, and
their difference to the derivative of the computed log Z is at the truncation
error level.  Dense vectors are used for the sandwich (small instances only).
"""
from __future__ import annotations

import numpy as np

from .peps import RowMPO, boundary_mps, mps_dense, upper_boundary_mps
from .potts import OPP, PottsModel


def apply_row(mpo, psi):
    """T_r psi as a dense array over row r's up classes (psi dense over row r+1's)."""
    t = psi.reshape(1, 1, -1)
    shape_rest = list(psi.shape)
    for c in range(len(mpo.cols)):
        W = mpo.dense(c)                                # [bl, br, u, s]
        t = t.reshape(t.shape[0], t.shape[1], shape_rest[0], -1)
        t = np.einsum("dbsr,bBus->duBr", t, W, optimize=True)
        t = t.reshape(-1, t.shape[2], t.shape[3])
        shape_rest = shape_rest[1:]
    return t.reshape(-1)


def factor_of_edge(pm, i, j):
    """(row, modifier key, spin-product table) of the factor carrying coupling (i, j)."""
    si, sj = int(pm.inst.site_of_spin[i]), int(pm.inst.site_of_spin[j])
    C = pm.C
    if si == sj:
        S = pm.sites[si]
        a, b = S.local[i], S.local[j]
        return si // C, ("w", si % C), (S.spinvals[:, a] * S.spinvals[:, b]).astype(float)
    ri, ci = divmod(si, C)
    rj, cj = divmod(sj, C)
    name = {(0, 1): "r", (1, 0): "d", (1, 1): "dr", (1, -1): "dl",
            (0, -1): "l", (-1, 0): "u", (-1, -1): "ul", (-1, 1): "ur"}[(rj - ri, cj - ci)]
    if name in ("l", "u", "ul", "ur"):                   # the upper / left site owns the factor
        i, j, ri, ci, rj, cj, name = j, i, rj, cj, ri, ci, OPP[name]
    S, T = pm.site(ri, ci), pm.site(rj, cj)
    PS, PT = S.proj[name], T.proj[OPP[name]]
    sa = 1 - 2 * ((PS.values >> PS.bits.index(S.local[i])) & 1)
    sb = 1 - 2 * ((PT.values >> PT.bits.index(T.local[j])) & 1)
    return ri, ("B", ri, ci, name), np.outer(sa, sb).astype(float)


def logz_grad(inst, beta, chi, n_sweeps=2, states=None):
    """(log Z, dlogZ/dJ[n_edges], dlogZ/dh[n_spins], dlogZ/dbeta)."""
    pm = PottsModel(inst, states)
    logz, psis, mpos = boundary_mps(pm, beta, chi, n_sweeps)
    E = upper_boundary_mps(pm, mpos, chi, n_sweeps)
    R, C = pm.R, pm.C
    psi = [mps_dense(A) for (A, _) in psis]
    up = [mps_dense(A).reshape(-1) for (A, _) in E]
    Z = [float(up[r] @ apply_row(mpos[r], psi[r])) for r in range(R)]

    def expect(r, key, mult):
        return float(up[r] @ apply_row(RowMPO(pm, r, beta, {key: mult}), psi[r])) / Z[r]

    ss = np.array([expect(*factor_of_edge(pm, i, j)) for i, j in zip(inst.ei.tolist(), inst.ej.tolist())])
    m = np.zeros(inst.n_spins)
    for s in range(R * C):
        S = pm.sites[s]
        for j, g in enumerate(S.spins):
            m[g] = expect(s // C, ("w", s % C), S.spinvals[:, j].astype(float))
    J = inst.j_num / inst.denom
    h = inst.h_num / inst.denom
    return logz, -beta * ss, -beta * m, -float(J @ ss + h @ m)
