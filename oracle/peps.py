"""Boundary-MPS contraction of the Boltzmann-weight PEPS (paper Sec. III.B, Figs. 5-8, Eq. 9).

Everything here is dense and plain.  For row r the transfer operator T_r is
an MPO whose column-c tensor is built directly from the definition (Fig. 5):
a sum over the states x of cluster (r, c) of its Boltzmann weight times the
bond factors exp(-beta Ebar) that touch it, with Kronecker deltas selecting
the projected classes (Eqs. 3-4).  Diagonal couplings are carried on the
horizontal MPO bond, which is the role of the mediating tensors of Fig. 5.

Index conventions (readings where the figures are missing):
* the boundary MPS psi_r stands for rows r+1..R-1; its physical index at
  column c is the class of cluster (r+1, c) restricted to the spins coupled to
  any cluster of row r (its "up exposure");
* MPO bond (c, c+1) of row r carries (lam, g): lam = class of cluster
  (r, c+1) restricted to the spins coupled to (r, c) or (r+1, c) ("left
  exposure"), g = class of cluster (r+1, c+1) toward (r, c);
* W_c[(lam, g), (lam', g'), u, sigma] =
    sum_{x : Lambda(x)=lam, U(x)=u} [g = pi_ul(sigma)] w(x)
      * Bv[P_d x, pi_u sigma] * Bh[P_r x, pi_l lam'] * Bdl[pi_dl lam', pi_ur sigma]
      * Bdr[P_dr x, g'],
  with w(x) = exp(-beta (E_x - min E)) and B = exp(-beta (Ebar - min Ebar));
  the removed minima are added back to log Z as one offset;
* MPS tensors are stored [sigma][chi_left][chi_right].

Contraction (Fig. 8): psi_{R-1} is the trivial MPS; psi_{r-1} ~ Trunc(T_r psi_r)
for r = R-1..1.  Each step (Sec. III.B, "Variational zipper algorithm"):
left-canonicalise psi_r; zipper right to left starting from a 1x1x1
connecting tensor, keeping the top 2 chi singular values of each dashed-box
tensor (dense SVD here: the plain definition of the optimal rank-k
truncation), and after EACH zipper step one sweep of one-site variational
optimisation of the instantaneous stage (Fig. 8d): the tensors built so far
(columns c..C-1, or the ``window`` columns next to the zipper centre) are
re-optimised to maximise their overlap with the product of the MPO and MPS
columns c..C-1, whose left bond is left open (the connecting tensor is the
centre of that stage); then the 2 chi -> chi cut by an SVD sweep and
``n_sweeps`` full sweeps at chi.  Singular values below ``RANK_TOL`` times
the largest are dropped, in truncations and in every orthonormalisation
(exact zeros would otherwise leave part of a bond basis arbitrary).
log Z = offset + log-norms + log <T_0 | psi_0>.
"""
from __future__ import annotations

import numpy as np

from .potts import PottsModel

RANK_TOL = 1e-12


class RowMPO:
    """Dense MPO columns of row r, plus per-state terms for the branch step."""

    def __init__(self, pm: PottsModel, r: int, beta: float, mods=None):
        """``mods`` (optional) multiplies factors entrywise: key ('w', c) -> array over the
        states of site (r, c); key ('B', r', c', dir) -> array shaped like that bond table."""
        self.pm, self.r, self.beta = pm, r, beta
        self.mods = mods or {}
        self.cols = [self._column(r, c) for c in range(pm.C)]

    def _B(self, r, c, dname):
        E = self.pm.ebar(r, c, dname)
        return np.exp(-self.beta * (E - E.min()) / self.pm.inst.denom) * self.mods.get(("B", r, c, dname), 1.0)

    def _column(self, r, c):
        pm = self.pm
        S = pm.site(r, c)
        below = pm.site(r + 1, c)
        right = pm.site(r, c + 1)
        below_right = pm.site(r + 1, c + 1)
        w = np.exp(-self.beta * (S.E - S.E.min()) / pm.inst.denom) * self.mods.get(("w", c), 1.0)
        U = pm.joint(r, c, ("u", "ul", "ur"))
        Lam = pm.joint(r, c, ("l", "dl"))
        # old physical index sigma: up exposure of (r+1, c)
        if below is not None:
            sig = pm.joint(r + 1, c, ("u", "ul", "ur"))
            n_sig = sig.n
            pu = pm.component(sig, below, "u")
            pul = pm.component(sig, below, "ul")
            pur = pm.component(sig, below, "ur")
            nG = below.proj["ul"].n
        else:
            n_sig, nG = 1, 1
            pu = pul = pur = np.zeros(1, dtype=np.int64)
        # right bond: (Lambda of (r, c+1), g' = class of (r+1, c+1) toward 'ul')
        if right is not None:
            lamR = pm.joint(r, c + 1, ("l", "dl"))
            nLR = lamR.n
            pl_of_lam = pm.component(lamR, right, "l")
            pdl_of_lam = pm.component(lamR, right, "dl")
        else:
            nLR = 1
            pl_of_lam = pdl_of_lam = np.zeros(1, dtype=np.int64)
        nGR = below_right.proj["ul"].n if below_right is not None else 1
        Bv = self._B(r, c, "d")
        Bh = self._B(r, c, "r")
        Bdl = self._B(r, c + 1, "dl") if right is not None else np.ones((1, 1))
        Bdr = self._B(r, c, "dr")
        Pd = S.proj["d"].of_state
        Pr = S.proj["r"].of_state
        Pdr = S.proj["dr"].of_state
        # per-state term T[x, lam', g', sigma]
        T = (w[:, None, None, None]
             * Bh[Pr][:, pl_of_lam][:, :, None, None]
             * Bdr[Pdr][:, None, :, None]
             * Bv[Pd][:, pu][:, None, None, :]
             * Bdl[pdl_of_lam][:, pur][None, :, None, :])
        # left bond (lam, g): g = pi_ul(sigma), the class of (r+1, c) toward (r, c-1)
        return dict(T=T, lam_x=Lam.of_state, u_x=U.of_state, nLam=Lam.n, nGl=nG, pul=pul,
                    nLR=nLR, nGR=nGR, nU=U.n, nsig=n_sig)

    def dense(self, c):
        """W_c[bl, br, u, sigma] with bl = lam * nGl + g, br = lam' * nGR + g'."""
        col = self.cols[c]
        if "W" in col:
            return col["W"]
        T = col["T"]
        W = np.zeros((col["nLam"] * col["nGl"], col["nLR"] * col["nGR"], col["nU"], col["nsig"]))
        sig = np.arange(col["nsig"])
        for x in range(T.shape[0]):
            rows = col["lam_x"][x] * col["nGl"] + col["pul"][sig]
            W[rows, :, col["u_x"][x], sig] += T[x].reshape(-1, col["nsig"]).T
        col["W"] = W
        return W

    def state_term(self, c, x):
        """Single-state slice W^(x)[bl, br, sigma] (its u index is U(x))."""
        col = self.cols[c]
        out = np.zeros((col["nLam"] * col["nGl"], col["nLR"] * col["nGR"], col["nsig"]))
        sig = np.arange(col["nsig"])
        rows = col["lam_x"][x] * col["nGl"] + col["pul"][sig]
        out[rows, :, sig] = col["T"][x].reshape(-1, col["nsig"]).T
        return out


class TransposedRowMPO:
    """T_r^T: the same dense columns with the up and down physical legs swapped."""

    def __init__(self, mpo: RowMPO):
        self.base = mpo
        self.cols = mpo.cols
        self._W = {}

    def dense(self, c):
        if c not in self._W:
            self._W[c] = np.ascontiguousarray(self.base.dense(c).transpose(0, 1, 3, 2))
        return self._W[c]


def upper_boundary_mps(pm: PottsModel, mpos, chi: int, n_sweeps: int = 2, window: int = 0):
    """E_0..E_{R-1}: E_r covers rows 0..r-1 as a function of row r's up classes.

    Built top-down with the same row step (zipper, sweeps, cut) applied to the
    transposed row MPOs: E_0 is trivial, E_{r+1} ~ Trunc(T_r^T E_r).
    """
    R, C = pm.R, pm.C
    E = [None] * R
    E[0] = trivial_mps(C)
    for r in range(R - 1):
        A, ln = E[r]
        E[r + 1] = row_step(TransposedRowMPO(mpos[r]), A, ln, chi, n_sweeps, window)
    return E


def log_offset(pm: PottsModel, beta: float) -> float:
    """Sum of the minima removed from the site weights and bond factors."""
    off = 0.0
    for S in pm.sites:
        off += -beta * S.E.min() / pm.inst.denom
    for r in range(pm.R):
        for c in range(pm.C):
            for dname in ("r", "d", "dr", "dl"):
                off += -beta * pm.ebar(r, c, dname).min() / pm.inst.denom
    return off


# --- dense MPS algebra -------------------------------------------------------

def trivial_mps(C):
    return [np.ones((1, 1, 1)) for _ in range(C)], 0.0


def orthonormalise(M):
    """M = Q R with Q an isometry, through the SVD, dropping directions below RANK_TOL.

    A QR would leave an arbitrary basis for exactly dependent columns, which a
    later variational update could then use; the trimmed SVD basis spans only
    the column space of M, so the result is fixed up to a rotation.
    """
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = keep_count(s, s.size)
    return U[:, :k], s[:k, None] * Vh[:k]


def left_canonical(A, lognorm):
    A = [a.copy() for a in A]
    for c in range(len(A) - 1):
        s, l, r = A[c].shape
        Q, R = orthonormalise(A[c].reshape(s * l, r))
        A[c] = Q.reshape(s, l, Q.shape[1])
        A[c + 1] = np.einsum("ij,sjk->sik", R, A[c + 1])
    n = np.linalg.norm(A[-1])
    A[-1] = A[-1] / n
    return A, lognorm + np.log(n)


def keep_count(s, cap):
    """Number of singular values kept: at most ``cap``, none below RANK_TOL * s[0]."""
    k = int(np.sum(s > RANK_TOL * s[0])) if s.size and s[0] > 0 else 0
    if k == 0:
        raise FloatingPointError("zero tensor in truncation")
    return min(cap, k)


def _opt(L, W, A, R):
    """Optimal one-site tensor phi_c[u, a, a'] = sum L[a,bl,i] W[bl,br,u,s] A[s,i,j] R[a',br,j]."""
    t = np.einsum("sij,cBj->siBc", A, R)                 # [s, i, br, a']
    t = np.einsum("bBus,siBc->buic", W, t, optimize=True)  # [bl, u, i, a']
    return np.einsum("abi,buic->uac", L, t, optimize=True)


def _upd_L(L, phi, W, A):
    """L_{c+1}[a', br, j] = sum L[a,bl,i] phi[u,a,a'] W[bl,br,u,s] A[s,i,j]."""
    t = np.einsum("abi,uac->biuc", L, phi, optimize=True)     # [bl, i, u, a']
    t = np.einsum("biuc,bBus->icBs", t, W, optimize=True)     # [i, a', br, s]
    return np.einsum("icBs,sij->cBj", t, A, optimize=True)


def _upd_R(R, phi, W, A):
    """R_{c-1}[a, bl, i] = sum phi[u,a,a'] W[bl,br,u,s] A[s,i,j] R[a',br,j]."""
    t = np.einsum("sij,cBj->siBc", A, R)                 # [s, i, br, a']
    t = np.einsum("bBus,siBc->buic", W, t, optimize=True)  # [bl, u, i, a']
    return np.einsum("uac,buic->abi", phi, t, optimize=True)


def stage_sweep(Ws, A, phi, K, c0, e):
    """One-site variational sweep of the zipper's instantaneous stage (Fig. 8d).

    At zipper column c0 the approximation of the target Y = (W_c0 A_c0) ...
    (W_{C-1} A_{C-1}) -- the MPO-MPS product of the columns done so far, its
    left bond (bl, al) left open -- is K phi[c0] ... phi[C-1], with K[bl, al, k]
    the connecting tensor (the centre) and phi right-canonical.  The sweep
    re-optimises phi[c0..e] one tensor at a time, left to right and back, each
    update being the exact maximiser of the overlap with Y given all other
    tensors (in canonical form); tensors right of e stay fixed.  Returns the
    new K = <phi[c0..] | Y> (the optimal centre for the new phi).
    """
    C = len(A)
    # right environments of the fixed tensors e+1..C-1, then of the window
    R = [None] * C
    Rt = np.ones((1, 1, 1))
    for j in range(C - 1, e, -1):
        Rt = _upd_R(Rt, phi[j], Ws[j], A[j])
    R[e] = Rt
    for j in range(e, c0, -1):
        R[j - 1] = _upd_R(R[j], phi[j], Ws[j], A[j])
    # the centre moves from K onto phi[c0]: K's orthonormal factor becomes
    # the left environment of column c0 (the open bond is its "basis")
    bl, al, k = K.shape
    Q, _ = orthonormalise(K.reshape(bl * al, k))
    L = [None] * C
    L[c0] = Q.reshape(bl, al, Q.shape[1]).transpose(2, 0, 1)      # [a, bl, i]
    for j in range(c0, e + 1):
        t = _opt(L[j], Ws[j], A[j], R[j])
        if j < e:
            u, a, b = t.shape
            Qj, _ = orthonormalise(t.reshape(u * a, b))
            phi[j] = Qj.reshape(u, a, Qj.shape[1])
            L[j + 1] = _upd_L(L[j], phi[j], Ws[j], A[j])
        else:
            phi[j] = t
    Rc = R[e]
    for j in range(e, c0 - 1, -1):
        t = _opt(L[j], Ws[j], A[j], Rc)
        u, a, b = t.shape
        Qr, _ = orthonormalise(t.transpose(1, 0, 2).reshape(a, u * b).T)
        phi[j] = Qr.T.reshape(Qr.shape[1], u, b).transpose(1, 0, 2)
        Rc = _upd_R(Rc, phi[j], Ws[j], A[j])
    return phi, Rc.transpose(1, 2, 0)                                 # [bl, al, k]


def zipper(mpo: RowMPO, A, lognorm, chi_cap, window=0, trace=None):
    """Right-to-left zipper of Fig. 8(c) with a variational sweep after each step.

    ``A`` must be left-canonical (Fig. 8c starts from that form).  At column c
    the dashed-box tensor Theta = (W_c A_c) K is truncated by an SVD to at most
    ``chi_cap`` values (new tensor V^T, right-canonical; K <- U S), then the
    instantaneous stage is swept (``stage_sweep``) over columns c..e with
    e = C-1 (``window`` <= 0: every tensor built so far) or
    e = min(C-1, c + window - 1).  Returns the right-canonical MPS with the
    norm of the last connecting tensor (a 1x1x1 tensor) in ``lognorm`` and its
    sign in column 0.  ``trace`` (a list, optional) receives (c, tensors of
    columns c..C-1, connecting tensor after the step's sweep, connecting
    tensor before it) after every zipper step, both connecting tensors on the
    scale of the input MPS.
    """
    C = len(A)
    Ws = [mpo.dense(c) for c in range(C)]
    K = np.ones((1, 1, 1))
    ln = lognorm
    out = [None] * C
    for c in range(C - 1, -1, -1):
        theta = np.einsum("abus,sij,bjk->aiuk", Ws[c], A[c], K, optimize=True)
        bl, al, u, kk = theta.shape
        Uu, s, Vh = np.linalg.svd(theta.reshape(bl * al, u * kk), full_matrices=False)
        k = keep_count(s, chi_cap)
        out[c] = Vh[:k].reshape(k, u, kk).transpose(1, 0, 2)
        K = (Uu[:, :k] * s[:k]).reshape(bl, al, k)
        e = C - 1 if window <= 0 else min(C - 1, c + window - 1)
        K_before = K * np.exp(ln - lognorm) if trace is not None else None
        if e > c:
            # the sweep's centre is computed from Y itself, so its scale is
            # relative to the input MPS alone
            out, K = stage_sweep(Ws, A, out, K, c, e)
            ln = lognorm
        if trace is not None:
            trace.append((c, [t.copy() for t in out[c:]], K * np.exp(ln - lognorm), K_before))
        n = np.linalg.norm(K)
        ln += np.log(n)
        K = K / n
    out[0] = out[0] * K.reshape(())         # K is 1x1x1 holding +-1
    return out, ln


def right_canonical(phi):
    phi = [p.copy() for p in phi]
    for c in range(len(phi) - 1, 0, -1):
        u, a, b = phi[c].shape
        Q, R = orthonormalise(phi[c].transpose(1, 0, 2).reshape(a, u * b).T)
        phi[c] = Q.T.reshape(Q.shape[1], u, b).transpose(1, 0, 2)
        phi[c - 1] = np.einsum("uab,bk->uak", phi[c - 1], R.T)
    return phi


def variational_sweep(mpo: RowMPO, A, phi):
    """One left-right-left sweep of one-site overlap maximisation (Fig. 8d).

    ``A`` is the (left-canonical) MPS being multiplied, ``phi`` the
    approximation; returns phi right-canonical with its centre at column 0
    (unnormalised: the centre holds the overlap coefficients).
    """
    C = len(A)
    phi = right_canonical(phi)
    Ws = [mpo.dense(c) for c in range(C)]
    R = [None] * C
    R[C - 1] = np.ones((1, 1, 1))
    for c in range(C - 1, 0, -1):
        R[c - 1] = _upd_R(R[c], phi[c], Ws[c], A[c])
    L = [None] * C
    L[0] = np.ones((1, 1, 1))
    for c in range(C):
        t = _opt(L[c], Ws[c], A[c], R[c])
        if c < C - 1:
            u, a, b = t.shape
            Q, _ = orthonormalise(t.reshape(u * a, b))
            phi[c] = Q.reshape(u, a, Q.shape[1])
            L[c + 1] = _upd_L(L[c], phi[c], Ws[c], A[c])
        else:
            phi[c] = t
    Rc = np.ones((1, 1, 1))
    for c in range(C - 1, -1, -1):
        t = _opt(L[c], Ws[c], A[c], Rc)
        if c > 0:
            u, a, b = t.shape
            Q, _ = orthonormalise(t.transpose(1, 0, 2).reshape(a, u * b).T)
            phi[c] = Q.T.reshape(Q.shape[1], u, b).transpose(1, 0, 2)
            Rc = _upd_R(Rc, phi[c], Ws[c], A[c])
        else:
            phi[c] = t
    return phi


def svd_cut(phi, chi):
    """Cut a right-canonical MPS (centre at column 0) to bond chi by a left-to-right SVD sweep."""
    phi = [p.copy() for p in phi]
    for c in range(len(phi) - 1):
        u, a, b = phi[c].shape
        Uu, s, Vh = np.linalg.svd(phi[c].reshape(u * a, b), full_matrices=False)
        k = keep_count(s, chi)
        phi[c] = Uu[:, :k].reshape(u, a, k)
        phi[c + 1] = np.einsum("ij,ujk->uik", s[:k, None] * Vh[:k], phi[c + 1])
    return phi


def normalise_centre(phi, lognorm, centre):
    n = np.linalg.norm(phi[centre])
    phi = list(phi)
    phi[centre] = phi[centre] / n
    return phi, lognorm + np.log(n)


def row_step(mpo: RowMPO, A, lognorm, chi, n_sweeps, window=0):
    """psi_{r-1} ~ T_r psi_r (Fig. 8; Sec. III.B): zipper at 2 chi with a sweep
    after every zipper step, cut to chi, ``n_sweeps`` sweeps at chi."""
    A, lognorm = left_canonical(A, lognorm)
    phi, ln = zipper(mpo, A, lognorm, 2 * chi, window)
    phi = svd_cut(phi, chi)
    phi, ln = normalise_centre(phi, ln, len(phi) - 1)
    for _ in range(n_sweeps):
        phi = variational_sweep(mpo, A, phi)
        phi, ln = normalise_centre(phi, lognorm, 0)
    return phi, ln


def boundary_mps(pm: PottsModel, beta: float, chi: int, n_sweeps: int = 2, window: int = 0):
    """All boundary MPSs psi_0..psi_{R-1} (psi_r covers rows below r) and log Z (Eq. 9)."""
    R, C = pm.R, pm.C
    mpos = [RowMPO(pm, r, beta) for r in range(R)]
    psis = [None] * R
    psis[R - 1] = trivial_mps(C)
    for r in range(R - 1, 0, -1):
        A, ln = psis[r]
        psis[r - 1] = row_step(mpos[r], A, ln, chi, n_sweeps, window)
    logz = log_offset(pm, beta) + top_row_log_overlap(mpos[0], *psis[0])
    return logz, psis, mpos


def top_row_log_overlap(mpo0: RowMPO, A, lognorm):
    """log <T_0 | psi_0>: the top row has no up legs, so this is a plain contraction."""
    E = np.ones((1, 1))
    for c in range(len(A)):
        W = mpo0.dense(c)
        E = np.einsum("ai,abs,sij->bj", E, W[:, :, 0, :], A[c], optimize=True)
    val = float(E.reshape(()))
    if not val > 0:
        # an approximate psi_0 (negative entries, Sec. V) can give a
        # non-positive overlap: log Z is undefined, the boundary MPSs remain
        # usable for the branch and bound (its scores are clamped at 0)
        return float("nan")
    return lognorm + np.log(val)


def mps_dense(A, lognorm=0.0):
    """Full vector of an MPS (tiny cases only), scaled by exp(lognorm)."""
    v = np.ones((1, 1))                     # [flattened physical, bond]
    shape = []
    for a in A:
        s, l, r = a.shape
        v = np.einsum("pl,slr->psr", v, a).reshape(-1, r)
        shape.append(s)
    return v[:, 0].reshape(shape) * np.exp(lognorm)
