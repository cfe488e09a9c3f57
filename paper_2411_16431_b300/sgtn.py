"""Thin ctypes binding of libsgtn.so (C ABI declared in include/sgtn.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  There is no CPU fallback: if the library cannot be loaded the
calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgtn.so")
_lib = None

FP64, TF32, BF16, FP32 = 0, 1, 2, 3

_I32P = ct.POINTER(ct.c_int32)
_I64P = ct.POINTER(ct.c_int64)
_F64P = ct.POINTER(ct.c_double)
_I8P = ct.POINTER(ct.c_int8)


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_2411_16431_b300/build.py (no CPU fallback exists)")
    L = ct.CDLL(LIB_PATH)
    L.sgtn_build_instance.argtypes = [ct.c_int32, ct.c_int64, _I32P, _I32P, _I32P, _I32P, ct.c_int32, _I32P,
                                      ct.c_int32, ct.c_int32, _I64P, _I64P, ct.c_void_p, ct.POINTER(ct.c_void_p)]
    L.sgtn_set_beta.argtypes = [ct.c_void_p, ct.c_double]
    L.sgtn_contract_boundary.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, _F64P, _F64P]
    L.sgtn_conditionals.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _I32P, _F64P]
    L.sgtn_branch_step.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, _I32P, _F64P, _I32P, _F64P,
                                   _I32P, _F64P]
    L.sgtn_set_search_precision.argtypes = [ct.c_void_p, ct.c_int32]
    L.sgtn_set_zipper_window.argtypes = [ct.c_void_p, ct.c_int32]
    L.sgtn_set_final_sweeps_fp64.argtypes = [ct.c_void_p, ct.c_int32]
    L.sgtn_set_sweep_orthonormalisation.argtypes = [ct.c_void_p, ct.c_int32]
    L.sgtn_sweep_orthonormalisations.argtypes = [ct.c_void_p, _I64P, _I64P]
    L.sgtn_kernel_names.argtypes = [ct.c_char_p, ct.c_int32]
    L.sgtn_kernel_names.restype = ct.c_int32
    L.sgtn_search.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _I8P, _I64P, _F64P, _F64P, _I32P]
    L.sgtn_conditionals_noalloc.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _I32P, _F64P]
    L.sgtn_energies.argtypes = [ct.c_void_p, ct.c_int32, _I8P, _I64P]
    L.sgtn_logz_grad.argtypes = [ct.c_void_p, _F64P, _F64P, _F64P]
    L.sgtn_lbp.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _I32P, _F64P, _I32P, _F64P]
    L.sgtn_search_droplets.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_int32, ct.c_int32, _I8P, _I64P,
                                       _F64P, _F64P, _I32P, _I64P, _I32P, _I32P]
    L.sgtn_batch_search.argtypes = [ct.POINTER(ct.c_void_p), ct.c_int32, ct.c_double, ct.c_int32, ct.c_int32,
                                    ct.c_int32, ct.c_int32, ct.c_int32, ct.POINTER(_I8P), ct.POINTER(_I64P),
                                    ct.POINTER(_F64P), _F64P, _F64P, _I32P, ct.c_int32, _I32P]
    L.sgtn_site_dims.argtypes = [ct.c_void_p, ct.c_int32, _I32P]
    L.sgtn_boundary_info.argtypes = [ct.c_void_p, _I32P, _I32P]
    L.sgtn_mps_shape.argtypes = [ct.c_void_p, ct.c_int32, _I32P, _I32P, _F64P]
    L.sgtn_mps_tensor.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _F64P]
    L.sgtn_stats.argtypes = [_I64P, _F64P, _I64P]
    L.sgtn_stats.restype = None
    L.sgtn_kernel_timing.argtypes = [ct.c_int32, ct.c_int32]
    L.sgtn_kernel_timing.restype = None
    L.sgtn_kernel_time.argtypes = [ct.c_char_p, _F64P, _I64P, _F64P]
    L.sgtn_last_error.argtypes = [ct.c_void_p]
    L.sgtn_last_error.restype = ct.c_char_p
    L.sgtn_destroy.argtypes = [ct.c_void_p]
    L.sgtn_destroy.restype = None
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def stats():
    """(kernel launches, algorithmic flops, marginal evaluations) issued by the library so far."""
    L = load()
    a, b, c = ct.c_int64(), ct.c_double(), ct.c_int64()
    L.sgtn_stats(ct.byref(a), ct.byref(b), ct.byref(c))
    return a.value, b.value, c.value


def gemm(X, Y, precision, stream=None):
    """C = X @ Y (torch float64 CUDA tensors) with the library's GEMM in the given precision."""
    import torch
    X, Y = X.contiguous(), Y.contiguous()
    m, k = X.shape
    k2, n = Y.shape
    assert k == k2 and X.dtype == Y.dtype == torch.float64 and X.is_cuda and Y.is_cuda
    C = torch.empty((m, n), dtype=torch.float64, device=X.device)
    L = load()
    L.sgtn_gemm.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                            ct.c_void_p]
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = L.sgtn_gemm(precision, m, n, k, X.data_ptr(), Y.data_ptr(), C.data_ptr(), st)
    if rc != 0:
        raise SgtnError(f"sgtn_gemm failed: {rc}")
    return C


def seg_gemm(X, Y, seg_ptr, xr, yr, coef, precision, stream=None):
    """O[g] = sum over the terms t of segment g of coef[t] X[xr[t]] Y[yr[t]] with the
    library's segmented contraction kernel.  X: (nx, p, q), Y: (ny, q, s) float64 CUDA
    tensors; seg_ptr (nseg + 1), xr, yr (nterm) int32 and coef (nterm) float64 CUDA
    tensors (coef may be None: all ones).  Returns O (nseg, p, s)."""
    import torch
    X, Y = X.contiguous(), Y.contiguous()
    nx, p, q = X.shape
    ny, q2, s = Y.shape
    assert q == q2 and X.dtype == Y.dtype == torch.float64 and X.is_cuda and Y.is_cuda
    nseg, nterm = seg_ptr.numel() - 1, xr.numel()
    O = torch.empty((nseg, p, s), dtype=torch.float64, device=X.device)
    cidx = torch.arange(nterm, dtype=torch.int32, device=X.device) if coef is not None else None
    L = load()
    L.sgtn_seg_gemm.argtypes = [ct.c_int32] * 8 + [ct.c_void_p] * 9
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = L.sgtn_seg_gemm(precision, p, q, s, nseg, nterm, nx, ny, seg_ptr.data_ptr(), xr.data_ptr(), yr.data_ptr(),
                         cidx.data_ptr() if cidx is not None else None,
                         coef.contiguous().data_ptr() if coef is not None else None, X.data_ptr(), Y.data_ptr(),
                         O.data_ptr(), st)
    if rc != 0:
        raise SgtnError(f"sgtn_seg_gemm failed: {rc}")
    return O


def cholesky(G, shift=0.0, stream=None):
    """(R, R^{-1}, status, minratio) of the library's FP64 Cholesky of G (+ shift I), a float64 CUDA tensor."""
    import torch
    G = G.contiguous()
    n = G.shape[0]
    R = torch.empty_like(G)
    Ri = torch.empty_like(G)
    stat = torch.zeros(1, dtype=torch.int32, device=G.device)
    mr = torch.zeros(1, dtype=torch.float64, device=G.device)
    L = load()
    L.sgtn_cholesky.argtypes = [ct.c_int32, ct.c_double] + [ct.c_void_p] * 6
    st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = L.sgtn_cholesky(n, shift, G.data_ptr(), R.data_ptr(), Ri.data_ptr(), stat.data_ptr(), mr.data_ptr(), st)
    if rc != 0:
        raise SgtnError(f"sgtn_cholesky failed: {rc}")
    return R, Ri, int(stat.item()), float(mr.item())


def device_allocations():
    """Number of cudaMalloc calls the library has made so far in this process."""
    L = load()
    L.sgtn_device_allocations.restype = ct.c_int64
    return int(L.sgtn_device_allocations())


def kernel_timing(enable, reset=False):
    load().sgtn_kernel_timing(int(enable), int(reset))


def kernel_time(name):
    """(device ms, launches, algorithmic flops) of a timed kernel, or None."""
    ms, n, fl = ct.c_double(), ct.c_int64(), ct.c_double()
    if load().sgtn_kernel_time(name.encode(), ct.byref(ms), ct.byref(n), ct.byref(fl)) != 0:
        return None
    return ms.value, n.value, fl.value


def kernel_names():
    """Labels of the timed kernels seen so far."""
    L = load()
    n = L.sgtn_kernel_names(None, 0)
    buf = ct.create_string_buffer(n + 1)
    L.sgtn_kernel_names(buf, n + 1)
    return [x for x in buf.value.decode().split(",") if x]


class SgtnError(RuntimeError):
    pass


class Handle:
    """One instance on one device/stream; wraps the C ABI calls one to one."""

    def __init__(self, inst, states_per_site=None, stream=None):
        L = load()
        self.L = L
        self.inst = inst
        ei = np.ascontiguousarray(inst.ei, np.int32)
        ej = np.ascontiguousarray(inst.ej, np.int32)
        jn = np.ascontiguousarray(inst.j_num, np.int32)
        hn = np.ascontiguousarray(inst.h_num, np.int32)
        site = np.ascontiguousarray(inst.site_of_spin, np.int32)
        offs = sts = None
        if states_per_site is not None:
            lens = [len(s) for s in states_per_site]
            offs = np.zeros(len(lens) + 1, np.int64)
            offs[1:] = np.cumsum(lens)
            sts = np.ascontiguousarray(np.concatenate([np.asarray(s, np.int64) for s in states_per_site]))
        h = ct.c_void_p()
        rc = L.sgtn_build_instance(inst.n_spins, inst.n_edges, _p(ei, _I32P), _p(ej, _I32P), _p(jn, _I32P),
                                   _p(hn, _I32P), inst.denom, _p(site, _I32P), inst.rows, inst.cols,
                                   _p(offs, _I64P), _p(sts, _I64P), stream, ct.byref(h))
        if rc != 0:
            raise SgtnError(f"sgtn_build_instance failed ({rc})")
        self.h = h
        self.d = []
        for s in range(inst.rows * inst.cols):
            d = ct.c_int32()
            self._ck(L.sgtn_site_dims(h, s, ct.byref(d)))
            self.d.append(d.value)

    def _ck(self, rc):
        if rc != 0:
            raise SgtnError(f"sgtn error {rc}: {self.L.sgtn_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            self.L.sgtn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_beta(self, beta):
        self._ck(self.L.sgtn_set_beta(self.h, float(beta)))

    def contract_boundary(self, chi, precision=FP64, n_sweeps=2):
        lz = ct.c_double()
        ws = ct.c_double()
        self._ck(self.L.sgtn_contract_boundary(self.h, chi, precision, n_sweeps, ct.byref(lz), ct.byref(ws)))
        return lz.value, ws.value

    def set_zipper_window(self, window):
        """Columns swept after each zipper step (0: all built so far, 1: no sweep)."""
        self._ck(self.L.sgtn_set_zipper_window(self.h, int(window)))

    def set_final_sweeps_fp64(self, on=True):
        """Mixed contractions: run the sweeps after the cut to chi in FP64."""
        self._ck(self.L.sgtn_set_final_sweeps_fp64(self.h, int(bool(on))))

    def set_sweep_orthonormalisation(self, mode):
        """1: CholeskyQR plus a polar correction in the sweeps where the SVD would keep every direction (default); 0: always the SVD."""
        self._ck(self.L.sgtn_set_sweep_orthonormalisation(self.h, int(mode)))

    def sweep_orthonormalisations(self):
        """(sweep orthonormalisations done by CholeskyQR, done by the SVD) on this handle so far."""
        q, v = ct.c_int64(), ct.c_int64()
        self._ck(self.L.sgtn_sweep_orthonormalisations(self.h, ct.byref(q), ct.byref(v)))
        return q.value, v.value

    def set_search_precision(self, precision):
        """Precision of conditionals / branch_step / search (-1: as the last contract_boundary)."""
        self._ck(self.L.sgtn_set_search_precision(self.h, precision))

    def boundary_info(self):
        """(iterative truncations stopped at their cap, precision of the boundary)."""
        u, p = ct.c_int32(), ct.c_int32()
        self._ck(self.L.sgtn_boundary_info(self.h, ct.byref(u), ct.byref(p)))
        return u.value, p.value

    def conditionals(self, step, configs):
        configs = np.ascontiguousarray(np.asarray(configs, np.int32).reshape(-1, step) if step else
                                       np.zeros((len(configs), 0), np.int32))
        count = configs.shape[0]
        out = np.zeros((count, self.d[step]))
        self._ck(self.L.sgtn_conditionals(self.h, step, count, _p(configs, _I32P), _p(out, _F64P)))
        return out

    def conditionals_noalloc(self, step, configs):
        """Same as conditionals(), through the allocation-free entry point."""
        configs = np.ascontiguousarray(np.asarray(configs, np.int32).reshape(-1, step) if step else
                                       np.zeros((len(configs), 0), np.int32))
        count = configs.shape[0]
        out = np.zeros((count, self.d[step]))
        self._ck(self.L.sgtn_conditionals_noalloc(self.h, step, count, _p(configs, _I32P), _p(out, _F64P)))
        return out

    def branch_step(self, step, M, configs, logp, pd=-np.inf):
        configs = np.ascontiguousarray(np.asarray(configs, np.int32).reshape(len(logp), step))
        logp = np.ascontiguousarray(logp, np.float64)
        oc = np.zeros((M, step + 1), np.int32)
        ol = np.zeros(M)
        cnt = ct.c_int32()
        pdv = ct.c_double(pd)
        self._ck(self.L.sgtn_branch_step(self.h, step, M, len(logp), _p(configs, _I32P), _p(logp, _F64P),
                                         _p(oc, _I32P), _p(ol, _F64P), ct.byref(cnt), ct.byref(pdv)))
        return oc[:cnt.value], ol[:cnt.value], pdv.value

    def search(self, M, n_out=1):
        N = self.inst.n_spins
        sp = np.zeros((n_out, N), np.int8)
        en = np.zeros(n_out, np.int64)
        lp = np.zeros(n_out)
        pd = ct.c_double()
        cnt = ct.c_int32()
        self._ck(self.L.sgtn_search(self.h, M, n_out, _p(sp, _I8P), _p(en, _I64P), _p(lp, _F64P), ct.byref(pd),
                                    ct.byref(cnt)))
        k = cnt.value
        return dict(spins=sp[:k], energy_num=en[:k], logp=lp[:k], pd=pd.value)

    def lbp(self, n_iter, k):
        """Loopy belief propagation (sgtn_lbp): per site the positions of its k most
        probable states and their marginals, and the last iteration's message change."""
        ns = self.inst.rows * self.inst.cols
        idx = np.zeros((ns, k), np.int32)
        marg = np.zeros((ns, k))
        cnt = np.zeros(ns, np.int32)
        chg = ct.c_double()
        self._ck(self.L.sgtn_lbp(self.h, n_iter, k, _p(idx, _I32P), _p(marg, _F64P), _p(cnt, _I32P),
                                 ct.byref(chg)))
        return [idx[s, :cnt[s]] for s in range(ns)], [marg[s, :cnt[s]] for s in range(ns)], chg.value

    def search_droplets(self, M, max_dE_num, min_hamming, cap=4096):
        """sgtn_search_droplets: the best configuration and its droplets (Fig. 4) as a
        list of (dE numerator, flipped spin ids), in order of (dE, spins)."""
        N = self.inst.n_spins
        sp = np.zeros(N, np.int8)
        en = ct.c_int64()
        lp = ct.c_double()
        pd = ct.c_double()
        nd = ct.c_int32()
        dE = np.zeros(max(cap, 1), np.int64)
        off = np.zeros(max(cap, 1) + 1, np.int32)
        fl = np.zeros(max(cap, 1) * N, np.int32)
        self._ck(self.L.sgtn_search_droplets(self.h, M, int(max_dE_num), min_hamming, cap, _p(sp, _I8P),
                                             ct.byref(en), ct.byref(lp), ct.byref(pd), ct.byref(nd), _p(dE, _I64P),
                                             _p(off, _I32P), _p(fl, _I32P)))
        k = min(cap, nd.value)
        drops = [(int(dE[i]), fl[off[i]:off[i + 1]].copy()) for i in range(k)]
        return dict(spins=sp, energy_num=en.value, logp=lp.value, pd=pd.value, droplets=drops, n_droplets=nd.value)

    def logz_grad(self):
        """(dlogZ/dJ[n_edges], dlogZ/dh[n_spins], dlogZ/dbeta) for the current beta and boundary."""
        dJ = np.zeros(max(self.inst.n_edges, 1))
        dh = np.zeros(self.inst.n_spins)
        db = ct.c_double()
        self._ck(self.L.sgtn_logz_grad(self.h, _p(dJ, _F64P), _p(dh, _F64P), ct.byref(db)))
        return dJ[:self.inst.n_edges], dh, db.value

    def energies(self, spins):
        spins = np.ascontiguousarray(np.asarray(spins, np.int8).reshape(-1, self.inst.n_spins))
        out = np.zeros(spins.shape[0], np.int64)
        self._ck(self.L.sgtn_energies(self.h, spins.shape[0], _p(spins, _I8P), _p(out, _I64P)))
        return out

    def mps(self, row):
        C = self.inst.cols
        phys = np.zeros(C, np.int32)
        bond = np.zeros(C + 1, np.int32)
        ln = ct.c_double()
        self._ck(self.L.sgtn_mps_shape(self.h, row, _p(phys, _I32P), _p(bond, _I32P), ct.byref(ln)))
        ts = []
        for c in range(C):
            t = np.zeros((phys[c], bond[c], bond[c + 1]))
            self._ck(self.L.sgtn_mps_tensor(self.h, row, c, _p(t, _F64P)))
            ts.append(t)
        return ts, ln.value


def logz(inst, J, h, beta, chi, n_sweeps=2, states_per_site=None, precision=FP64):
    """log Z (Eq. 9) as a differentiable torch function of the couplings J
    (float64 tensor, one per edge of ``inst`` in its ei/ej order), the fields h
    (one per spin) and beta (0-d tensor).  J and h must be multiples of
    1/inst.denom (the library works on integer numerators).  The forward pass
    contracts the boundary MPSs; the backward pass asks the library for
    dlogZ/dJ, dlogZ/dh and dlogZ/dbeta (environment correlators of the same
    boundary, upper boundary recomputed on the device)."""
    return _logz_function().apply(J, h, beta, inst, chi, n_sweeps, states_per_site, precision)


_LOGZ_FN = None


def _logz_function():
    global _LOGZ_FN
    if _LOGZ_FN is not None:
        return _LOGZ_FN
    import dataclasses

    import torch

    def numerators(x, denom, what):
        v = x.detach().to("cpu", torch.float64).numpy() * denom
        r = np.rint(v)
        if np.max(np.abs(v - r), initial=0.0) > 1e-9:
            raise ValueError(f"{what} must be multiples of 1/{denom}")
        return r.astype(np.int32)

    class _LogZ(torch.autograd.Function):
        @staticmethod
        def forward(ctx, J, hf, beta, inst, chi, n_sweeps, states, precision):
            inst2 = dataclasses.replace(inst, j_num=numerators(J, inst.denom, "J"),
                                        h_num=numerators(hf, inst.denom, "h"))
            H = Handle(inst2, states)
            H.set_beta(float(beta))
            lz, _ = H.contract_boundary(chi, precision=precision, n_sweeps=n_sweeps)
            ctx.handle = H
            ctx.like = (J, hf, beta)
            return torch.tensor(lz, dtype=torch.float64, device=J.device)

        @staticmethod
        def backward(ctx, g):
            H = ctx.handle
            dJ, dh, db = H.logz_grad()
            H.close()
            ctx.handle = None
            J, hf, beta = ctx.like
            return (g * torch.as_tensor(dJ, dtype=J.dtype, device=J.device),
                    g * torch.as_tensor(dh, dtype=hf.dtype, device=hf.device),
                    g * torch.as_tensor(db, dtype=beta.dtype, device=beta.device),
                    None, None, None, None, None)

    _LOGZ_FN = _LogZ
    return _LOGZ_FN


def lbp_reduce(inst, beta, n_iter, k, states_per_site=None, stream=None):
    """Local dimensional reduction (Sec. IV): the k most probable states of every
    cluster by loopy belief propagation at beta, as state lists (bit patterns) for
    a new Handle.  ``states_per_site`` is the pool to choose from (None: every
    state of each cluster).  Returns (state lists, marginals, last message change)."""
    h = Handle(inst, states_per_site, stream=stream)
    try:
        h.set_beta(beta)
        idx, marg, chg = h.lbp(n_iter, k)
    finally:
        h.close()
    out = []
    for s, ix in enumerate(idx):
        if states_per_site is None:
            out.append(np.asarray(ix, np.int64))   # full enumeration: position == bit pattern
        else:
            out.append(np.asarray(states_per_site[s], np.int64)[ix])
    return out, marg, chg


def batch_search(handles, beta, chi, M, precision=FP64, n_sweeps=2, n_out=1, threads=0, raise_on_error=True):
    """sgtn_batch_search: set_beta, contract_boundary and search on every
    handle, handles on distinct streams concurrently.  Returns a list of
    (log Z, search result) in handle order; raises if any handle failed, or,
    with raise_on_error=False, gives (NaN, None) for a failed handle (its
    error text stays in the handle)."""
    L = load()
    n = len(handles)
    hs = (ct.c_void_p * n)(*[h.h for h in handles])
    sps = [np.zeros((n_out, h.inst.n_spins), np.int8) for h in handles]
    ens = [np.zeros(n_out, np.int64) for _ in handles]
    lps = [np.zeros(n_out) for _ in handles]
    sp_p = (_I8P * n)(*[_p(a, _I8P) for a in sps])
    en_p = (_I64P * n)(*[_p(a, _I64P) for a in ens])
    lp_p = (_F64P * n)(*[_p(a, _F64P) for a in lps])
    lz = np.zeros(n)
    pd = np.zeros(n)
    cnt = np.zeros(n, np.int32)
    status = np.zeros(n, np.int32)
    rc = L.sgtn_batch_search(hs, n, float(beta), chi, precision, n_sweeps, M, n_out, sp_p, en_p, lp_p,
                             _p(lz, _F64P), _p(pd, _F64P), _p(cnt, _I32P), threads, _p(status, _I32P))
    bad = [i for i in range(n) if status[i] != 0]
    if rc != 0 and (raise_on_error or not bad):
        i = bad[0] if bad else 0
        raise SgtnError(f"sgtn_batch_search failed ({rc}); handle {i}: {L.sgtn_last_error(hs[i]).decode()}")
    return [(float(lz[i]), dict(spins=sps[i][:cnt[i]], energy_num=ens[i][:cnt[i]], logp=lps[i][:cnt[i]],
                                pd=float(pd[i]))) if status[i] == 0 else (float("nan"), None) for i in range(n)]


def logz_spread(runs):
    """Standard deviation of log Z over the grid symmetries of one instance (the
    stability test of App. C compares Z from the eight contraction corners; the
    spread of log Z is its relative spread, and stays finite where Z overflows).
    NaN entries (undefined log Z) are left out; NaN if fewer than two remain."""
    v = np.array([r[1] for r in runs], dtype=np.float64)
    v = v[np.isfinite(v)]
    return float(np.std(v)) if len(v) >= 2 else float("nan")


def search_transforms(inst, beta, chi, M, states_per_site=None, precision=FP64, n_sweeps=2, transforms=range(8),
                      streams=None):
    """Boundary contraction + search of the instance in each of the grid
    symmetries ``transforms`` (lattices.TRANSFORMS): the paper runs every
    instance in all of its orientations and keeps the best state (Sec. V).
    ``streams``: one CUDA stream (raw pointer) per transform, to run them
    concurrently through sgtn_batch_search; None runs them one after another
    on the default stream.  Spins keep their indices, so the returned states
    and energies are comparable.  Returns (index of the best, list of
    (transform, log Z, search result)); ``logz_spread(runs)`` gives the
    contraction-stability measure of App. C over them."""
    from . import lattices as L
    ks = list(transforms)
    if streams is not None and len(streams) != len(ks):
        raise ValueError("one stream per transform")
    hs = []
    try:
        for j, k in enumerate(ks):
            st = None if states_per_site is None else L.transform_states(inst, states_per_site, k)
            hs.append(Handle(L.transform(inst, k), st, stream=None if streams is None else streams[j]))
        res = batch_search(hs, beta, chi, M, precision=precision, n_sweeps=n_sweeps)
    finally:
        for h in hs:
            h.close()
    out = [(k, lz, r) for k, (lz, r) in zip(ks, res)]
    best = min(range(len(out)), key=lambda i: (int(out[i][2]["energy_num"][0]), i))
    return best, out
