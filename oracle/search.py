"""Conditional marginals and the branch-and-bound search (paper Sec. III.A, Eqs. 5-8, Figs. 3 and 6).

Clusters are placed in row-major order (the sweep of Fig. 3, "row after
row"), top-left first.  For a branch k (a partial configuration) and the next
cluster n+1 = (r, c), the unnormalised conditional score of state x is the
contraction of Fig. 6(b):

    s_k(x) = < f_k | W_0^(x_0) ... W_{c-1}^(x_{c-1}) W_c^(x) W_{c+1} ... W_{C-1} | psi_r >

where W_j are the dense MPO columns of row r (see ``peps``), W^(x) the slice of
one cluster state, psi_r the boundary MPS of the rows below, and f_k the
product vector on the up legs that carries the Boltzmann factors between the
fixed row r-1 of branch k and row r.  The conditional is
p(x | x_n) = s_k(x) / sum_x' s_k(x'), and the chain rule (Eq. 6) gives
log p(x_{n+1}) = log p(x_n) + log p(x | x_n).

Bounding (Fig. 3d-e): candidates are grouped by their boundary
(Eq. 7: the classes P^{kl}(x_k) over coupled pairs with k placed, l not yet
placed); only the most probable of each group survives; then the M most
probable survive.  p_d is the largest log-probability ever discarded (Sec.
III.A, last paragraph).

Readings: negative scores (possible with an approximate boundary MPS) are
clamped to zero and counted.  "Keep the most probable" (Fig. 3d-e) needs a
rule for equal probabilities, and integer couplings make exactly degenerate
candidates common; their log-probabilities, computed along different
contraction paths, differ only by rounding, so "equal" is read as "within
TIE_REL (relative)", and equal candidates are ordered by configuration
(lexicographically smaller first, in placement order): in a merge group
every candidate within tolerance of the group's maximum is a tie and the
smallest configuration wins; at the top-M cut the candidates within tolerance
of the M-th value form a tie class filled in configuration order.  A winner
is therefore never less probable than the most probable candidate it beats
by more than the tolerance.
"""
from __future__ import annotations

import numpy as np

from .energy import energy_num
from .peps import boundary_mps
from .potts import DIRS, PottsModel


def _B(pm, beta, r, c, dname):
    E = pm.ebar(r, c, dname)
    return np.exp(-beta * (E - E.min()) / pm.inst.denom)


def upper_vectors(pm: PottsModel, beta, r, row_above_states):
    """f[c'][u]: Boltzmann factors between the fixed row r-1 and class u of the up exposure of (r, c')."""
    out = []
    for cc in range(pm.C):
        S = pm.site(r, cc)
        U = pm.joint(r, cc, ("u", "ul", "ur"))
        f = np.ones(U.n)
        if r > 0:
            xa = row_above_states
            pu = pm.component(U, S, "u")
            f = f * _B(pm, beta, r - 1, cc, "d")[pm.site(r - 1, cc).proj["d"].of_state[xa[cc]], pu]
            if cc - 1 >= 0:
                pul = pm.component(U, S, "ul")
                f = f * _B(pm, beta, r - 1, cc - 1, "dr")[pm.site(r - 1, cc - 1).proj["dr"].of_state[xa[cc - 1]], pul]
            if cc + 1 < pm.C:
                pur = pm.component(U, S, "ur")
                f = f * _B(pm, beta, r - 1, cc + 1, "dl")[pm.site(r - 1, cc + 1).proj["dl"].of_state[xa[cc + 1]], pur]
        out.append(f)
    return out


def conditional_scores(pm, beta, mpo, psi, cfg, r, c):
    """Unnormalised scores s_k(x) of every state x of cluster (r, c) for partial configuration cfg."""
    A, _ = psi
    C = pm.C
    above = [cfg[(r - 1) * C + j] for j in range(C)] if r > 0 else None
    f = upper_vectors(pm, beta, r, above)
    E = np.ones((1, 1))
    for j in range(c):
        x = cfg[r * C + j]
        Wx = mpo.state_term(j, x)
        E = f[j][mpo.cols[j]["u_x"][x]] * np.einsum("ai,abs,sij->bj", E, Wx, A[j], optimize=True)
    F = np.ones((1, 1))
    for j in range(C - 1, c, -1):
        Wf = np.einsum("u,abus->abs", f[j], mpo.dense(j))
        F = np.einsum("abs,sij,bj->ai", Wf, A[j], F, optimize=True)
    M = np.einsum("ai,sij,bj->abs", E, A[c], F, optimize=True)         # [bl, br, sigma]
    col = mpo.cols[c]
    d = col["T"].shape[0]
    Tr = col["T"].reshape(d, -1, col["nsig"])           # [x, br, sigma]
    sig = np.arange(col["nsig"])
    rows = col["lam_x"][:, None] * col["nGl"] + col["pul"][None, :]
    Mg = M[rows, :, sig[None, :]]                        # [x, sigma, br]
    return f[c][col["u_x"]] * np.einsum("xbs,xsb->x", Tr, Mg)


def boundary_pairs(pm: PottsModel, n):
    """Coupled ordered pairs (p, l, dir) with p placed (index <= n) and l not placed (Eq. 7)."""
    C = pm.C
    out = []
    for p in range(n + 1):
        r, c = divmod(p, C)
        for dname, (dr, dc) in DIRS.items():
            rr, cc = r + dr, c + dc
            if 0 <= rr < pm.R and 0 <= cc < C:
                l = rr * C + cc
                if l > n and pm.sites[p].coupled[dname]:
                    out.append((p, l, dname))
    return sorted(out)


TIE_REL = 1e-10


def tie_tol(lp):
    return TIE_REL * max(1.0, abs(lp))


def merge_and_cut(cands, M):
    """Bounding of Fig. 3(d-e) on a dict key -> list of (config, log p).

    Returns (kept beam sorted by (-log p, config), largest discarded log p).
    """
    pd = -np.inf
    surv = []
    for group in cands.values():
        top = max(lq for _, lq in group)
        tied = [t for t in group if t[1] >= top - tie_tol(top)]
        win = min(tied, key=lambda t: t[0])
        surv.append(win)
        for t in group:
            if t is not win:
                pd = max(pd, t[1])
    surv.sort(key=lambda t: (-t[1], t[0]))
    if len(surv) > M:
        T = surv[M - 1][1]
        tol = tie_tol(T)
        sure = [t for t in surv if t[1] > T + tol]
        tie = sorted([t for t in surv if T - tol <= t[1] <= T + tol], key=lambda t: t[0])
        keep = sure + tie[:M - len(sure)]
        kept = set(id(t) for t in keep)
        for t in surv:
            if id(t) not in kept:
                pd = max(pd, t[1])
        surv = sorted(keep, key=lambda t: (-t[1], t[0]))
    return surv, pd


def boundary_key(pm, pairs, cfg):
    return tuple(pm.sites[p].proj[d].of_state[cfg[p]] for (p, l, d) in pairs)


def search(inst, beta, chi, M, n_sweeps=2, states=None, psis=None, window=0, trace=None):
    """Branch and bound over all clusters; returns the final beam sorted by (-log p, configuration).

    ``trace`` (a list, optional) receives one (beam, largest log p discarded
    at that step) pair per step.
    """
    pm = PottsModel(inst, states)
    logz, psis_, mpos = boundary_mps(pm, beta, chi, n_sweeps, window)
    psis = psis_ if psis is None else psis
    C = pm.C
    beam = [((), 0.0)]
    pd = -np.inf
    clamps = 0
    evals = 0
    for n in range(pm.R * C):
        r, c = divmod(n, C)
        pairs = boundary_pairs(pm, n)
        cands = {}
        for cfg, lp in beam:
            s = conditional_scores(pm, beta, mpos[r], psis[r], cfg, r, c)
            evals += s.size
            clamps += int(np.sum(s < 0))
            s = np.maximum(s, 0.0)
            tot = s.sum()
            for x in np.nonzero(s > 0)[0]:
                cand = cfg + (int(x),)
                cands.setdefault(boundary_key(pm, pairs, cand), []).append(
                    (cand, lp + float(np.log(s[x] / tot))))
        beam, pd_step = merge_and_cut(cands, M)
        pd = max(pd, pd_step)
        if trace is not None:
            trace.append((list(beam), pd_step))
    configs = [b[0] for b in beam]
    spins = np.array([pm.spins_of_config(cfg) for cfg in configs], dtype=np.int8)
    energies = np.array([energy_num(inst, s) for s in spins], dtype=np.int64)
    return dict(configs=configs, logp=np.array([b[1] for b in beam]), pd=pd, spins=spins,
                energy_num=energies, logz=logz, clamps=clamps, evals=evals, pm=pm, psis=psis, mpos=mpos)
