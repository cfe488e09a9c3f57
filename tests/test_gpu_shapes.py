"""Parity at the benchmark's shapes, through the C ABI.

The largest benchmark truncates at chi = 64 (2 chi = 128 kept by the zipper)
and cuts the beam at M = 1024.  The dense oracle cannot hold 24-spin Pegasus
cells, so these shapes are checked on instances it can: Chimera grids with all
256 states per cell.  Also here: the library's GEMM (the building block of
every contraction) element by element against a float64 product, with the
error bound of each precision.
"""
import numpy as np
import pytest

from oracle import brute
from oracle.peps import boundary_mps
from oracle.potts import PottsModel
from oracle.search import boundary_key, boundary_pairs, conditional_scores, merge_and_cut
from oracle.search import search as oracle_search
from paper_2411_16431_b300 import lattices as L

pytestmark = pytest.mark.gpu

RTOL = 1e-10
CHI64 = L.chimera_grid(6, 6, 2)


@pytest.fixture(scope="module")
def chi64():
    from paper_2411_16431_b300.sgtn import Handle
    pm = PottsModel(CHI64)
    lz_o, psis, mpos = boundary_mps(pm, 1.0, 64, 1)
    h = Handle(CHI64)
    h.set_beta(1.0)
    lz, _ = h.contract_boundary(64, n_sweeps=1)
    yield dict(pm=pm, lz_o=lz_o, psis=psis, mpos=mpos, h=h, lz=lz)
    h.close()


def _overlap(A, B):
    E = np.ones((1, 1))
    for a, b in zip(A, B):
        E = np.einsum("ab,sai,sbj->ij", E, a, b, optimize=True)
    return float(E.reshape(()))


def test_chi64_boundary_matches_oracle(chi64):
    """log Z to 1e-10 and every boundary MPS equal as a unit vector (|<a|b>| = 1 to 1e-13),
    with bonds at the chi = 64 cap."""
    assert abs(chi64["lz"] - chi64["lz_o"]) < RTOL * abs(chi64["lz_o"])
    psis = chi64["psis"]
    assert max(max(t.shape[1] for t in p[0]) for p in psis) == 64
    for r in range(CHI64.rows):
        ts, _ = chi64["h"].mps(r)
        A = psis[r][0]
        assert [t.shape for t in ts] == [a.shape for a in A]
        ov = _overlap(ts, A) / np.sqrt(_overlap(ts, ts) * _overlap(A, A))
        assert abs(abs(ov) - 1.0) < 1e-13, (r, ov)


@pytest.mark.parametrize("prec", ["TF32", "BF16"])
def test_chi64_mixed_boundary_on_tensor_cores(chi64, prec):
    """At chi = 64 the sparse site diagrams and environment updates of a TF32 or BF16
    contraction run on the tensor cores (3xTF32, or three BF16 slices and six products):
    log Z within 1e-6 relative of the FP64 oracle."""
    from paper_2411_16431_b300 import sgtn
    h = sgtn.Handle(CHI64)
    h.set_beta(1.0)
    sgtn.kernel_timing(True, reset=True)
    lz, _ = h.contract_boundary(64, precision=getattr(sgtn, prec), n_sweeps=1)
    sgtn.kernel_timing(False)
    suffix = "_tc_bf16" if prec == "BF16" else "_tc"
    assert sgtn.kernel_time("site_diagram" + suffix) is not None
    assert abs(lz - chi64["lz_o"]) < 1e-6 * abs(chi64["lz_o"])
    h.close()


@pytest.mark.parametrize("step", [7, 12, 20])
def test_chi64_branch_step_with_1024_branches(chi64, step):
    """One branch step of 1024 seeded partial configurations x 256 states (262,144
    candidates), merged by Eq. (7) and cut to M = 1024: the kept beam, its log p and p_d
    equal the oracle's."""
    pm, psis, mpos, h = chi64["pm"], chi64["psis"], chi64["mpos"], chi64["h"]
    C = CHI64.cols
    r, c = divmod(step, C)
    rng = np.random.default_rng(100 + step)
    K, M = 1024, 1024
    cfgs = rng.integers(0, 256, size=(K, step)).astype(np.int32)
    logp = -rng.uniform(0.0, 30.0, K)
    pairs = boundary_pairs(pm, step)
    cands = {}
    for cf, l0 in zip(map(tuple, cfgs.tolist()), logp.tolist()):
        s = np.maximum(conditional_scores(pm, 1.0, mpos[r], psis[r], cf, r, c), 0)
        for x in np.nonzero(s > 0)[0]:
            cand = cf + (int(x),)
            cands.setdefault(boundary_key(pm, pairs, cand), []).append((cand, l0 + float(np.log(s[x] / s.sum()))))
    want, pd_o = merge_and_cut(cands, M)
    oc, ol, pd = h.branch_step(step, M, cfgs, logp)
    got = sorted(zip(map(tuple, oc.tolist()), ol.tolist()))
    want = sorted(want)
    assert len(got) == len(want) == M
    assert [g[0] for g in got] == [w[0] for w in want]
    assert np.allclose([g[1] for g in got], [w[1] for w in want], rtol=RTOL, atol=0)
    assert abs(pd - pd_o) <= RTOL * abs(pd_o)


def test_search_with_beam_1024_matches_oracle():
    """The full search at M = 1024 (the cached per-row environments of the search, not the
    stateless branch step): Chimera 4x4, all 256 states, chi = 16."""
    from paper_2411_16431_b300.sgtn import Handle
    inst = L.chimera_grid(4, 4, 5)
    ref = oracle_search(inst, 1.0, chi=16, M=1024, n_sweeps=1)
    h = Handle(inst)
    h.set_beta(1.0)
    h.contract_boundary(16, n_sweeps=1)
    res = h.search(1024)
    assert np.array_equal(res["spins"], ref["spins"])
    assert np.array_equal(res["energy_num"], ref["energy_num"])
    assert np.allclose(res["logp"], ref["logp"], rtol=RTOL, atol=0)
    assert abs(res["pd"] - ref["pd"]) <= RTOL * abs(ref["pd"])
    h.close()


@pytest.mark.parametrize("inst", [L.slice_cells(L.chimera_grid(4, 4, 1), 2, 1), L.kings_grid(4, 4, 3)],
                         ids=lambda i: i.name)
def test_exact_conditionals_relative_parity(inst):
    """Untruncated boundary (every term of a score positive): every conditional marginal with
    p > 1e-300 within 1e-10 relative of the oracle and of brute force, also the smallest ones."""
    from paper_2411_16431_b300.sgtn import Handle
    beta = 1.3
    pm = PottsModel(inst)
    _, psis, mpos = boundary_mps(pm, beta, 256, 1)
    h = Handle(inst)
    h.set_beta(beta)
    h.contract_boundary(256, n_sweeps=1)
    rng = np.random.default_rng(4)
    S = brute.all_spins(inst.n_spins)
    E = brute.energies_num(inst, S) / inst.denom
    for n in range(1, inst.rows * inst.cols):
        r, c = divmod(n, inst.cols)
        cfgs = [tuple(int(rng.integers(pm.sites[p].d)) for p in range(n)) for _ in range(4)]
        got = h.conditionals(n, np.array(cfgs, np.int32))
        for k, cf in enumerate(cfgs):
            s = conditional_scores(pm, beta, mpos[r], psis[r], cf, r, c)
            assert np.all(s > 0)
            po = s / s.sum()
            ok = po > 1e-300
            assert np.allclose(got[k][ok], po[ok], rtol=RTOL, atol=0)
            # brute force: p(x | placed) by summing exp(-beta H) over completions
            m = np.ones(len(S), bool)
            for p, x in enumerate(cf):
                m &= np.all(S[:, pm.sites[p].spins] == pm.sites[p].spinvals[x][None, :], axis=1)
            w = np.exp(-beta * (E[m] - E[m].min()))
            site = pm.sites[n]
            pb = np.array([w[np.all(S[m][:, site.spins] == site.spinvals[x][None, :], axis=1)].sum()
                           for x in range(site.d)])
            pb /= pb.sum()
            assert np.allclose(got[k], pb, rtol=1e-9, atol=0)


# --- the library's GEMM against a float64 product ---------------------------------------

# m >= 128, n >= 64, k >= 32 take the dense tensor-core GEMM in TF32 mode, smaller ones the
# segmented SIMT kernel (a k tail in 97 x 33 x 17; a long reduction split over CTAs in
# 64 x 48 x 300 and 100 x 100 x 2000)
GEMM_SHAPES = [(128, 64, 32), (1024, 512, 2048), (300, 200, 1000), (2048, 128, 128), (256, 128, 13568),
               (97, 33, 17), (64, 48, 300), (100, 100, 2000), (40, 127, 65)]


@pytest.mark.parametrize("shape", GEMM_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("prec", [0, 3, 1], ids=["fp64", "fp32", "tf32"])
def test_gemm_elementwise_error_bound(shape, prec):
    """|C - X Y| <= bound * (|X| |Y|) element by element, X Y in float64 on the host:
    FP64 k 2^-52; FP32 (2^-23 + k 2^-24); TF32 (3xTF32 tensor cores for m >= 128, n >= 64,
    k >= 32, else FP32) (2^-20 + k 2^-24) -- the split drops lo*lo (2^-22 of |x||y|), each
    split rounds (2^-22 twice), and the sum runs in FP32."""
    import torch
    from paper_2411_16431_b300.sgtn import gemm
    m, n, k = shape
    g = torch.Generator().manual_seed(m * 7 + n * 3 + k)
    X = torch.randn(m, k, generator=g, dtype=torch.float64)
    Y = torch.randn(k, n, generator=g, dtype=torch.float64)
    # a spread of magnitudes inside rows and columns, as in normalised MPS tensors
    X *= torch.exp(torch.randn(m, 1, generator=g, dtype=torch.float64))
    Y *= torch.exp(torch.randn(1, n, generator=g, dtype=torch.float64))
    ref = (X @ Y).numpy()
    absprod = (X.abs() @ Y.abs()).numpy()
    got = gemm(X.cuda(), Y.cuda(), prec).cpu().numpy()
    bound = {0: k * 2.0 ** -52, 3: 2.0 ** -23 + k * 2.0 ** -24, 1: 2.0 ** -20 + k * 2.0 ** -24}[prec]
    err = np.abs(got - ref)
    assert np.all(err <= bound * absprod + 1e-300), float(np.max(err / absprod))


# --- the segmented contraction kernel (sparse site diagram, Fig. 7b) ----------------------

# (p, q, s): chi 64 site diagram with a 2 chi right bond, chi 32 site diagram, an environment
# update, ragged tails in k (40 = 32 + 8) and columns (48, 200: partial column tiles), two row
# tiles (160), and blocks too small for a 128-row tensor-core tile (SIMT in TF32 mode)
SEG_SHAPES = [(64, 64, 128), (32, 32, 64), (128, 64, 64), (96, 40, 48), (160, 32, 200), (16, 16, 16), (40, 18, 30)]


@pytest.mark.parametrize("shape", SEG_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("prec", [0, 3, 1, 2], ids=["fp64", "fp32", "tf32", "bf16"])
def test_seg_gemm_elementwise_error_bound(shape, prec):
    """O[g] = sum_t c_t X[xr_t] Y[yr_t] against float64 on the host, element by element:
    FP64 within K 2^-52, FP32 within (2^-23 + K 2^-24), TF32 (3xTF32 tensor cores where the
    shape allows) and BF16 (three BF16 slices per operand, six products) within
    (2^-20 + K 2^-24), of sum_t |c_t| |X_t| |Y_t|, K = the summed length of the segment's
    reductions.  Segments of 0..7 terms (empty ones give zero blocks), operands shared
    between terms, coefficients spread over six orders."""
    import torch
    from paper_2411_16431_b300.sgtn import seg_gemm, kernel_timing, kernel_time
    p, q, s = shape
    g = torch.Generator().manual_seed(p * 131 + q * 17 + s)
    nx, ny, nseg = 37, 29, 300
    X = torch.randn(nx, p, q, generator=g, dtype=torch.float64)
    Y = torch.randn(ny, q, s, generator=g, dtype=torch.float64)
    X *= torch.exp(torch.randn(nx, p, 1, generator=g, dtype=torch.float64))
    Y *= torch.exp(torch.randn(ny, 1, s, generator=g, dtype=torch.float64))
    cnt = torch.randint(0, 8, (nseg,), generator=g)
    cnt[:3] = 0
    seg_ptr = torch.zeros(nseg + 1, dtype=torch.int64)
    seg_ptr[1:] = torch.cumsum(cnt, 0)
    nterm = int(seg_ptr[-1])
    xr = torch.randint(0, nx, (nterm,), generator=g)
    yr = torch.randint(0, ny, (nterm,), generator=g)
    coef = torch.exp(3.0 * torch.randn(nterm, generator=g, dtype=torch.float64))
    ref = np.zeros((nseg, p, s))
    absref = np.zeros((nseg, p, s))
    Xn, Yn, cn = X.numpy(), Y.numpy(), coef.numpy()
    for k in range(nseg):
        for t in range(int(seg_ptr[k]), int(seg_ptr[k + 1])):
            ref[k] += cn[t] * (Xn[xr[t]] @ Yn[yr[t]])
            absref[k] += abs(cn[t]) * (np.abs(Xn[xr[t]]) @ np.abs(Yn[yr[t]]))
    kernel_timing(True, reset=True)
    i32 = dict(dtype=torch.int32, device="cuda")
    got = seg_gemm(X.cuda(), Y.cuda(), seg_ptr.to(**i32), xr.to(**i32), yr.to(**i32), coef.cuda(), prec)
    torch.cuda.synchronize()
    kernel_timing(False)
    got = got.cpu().numpy()
    K = (cnt.numpy() * q).reshape(nseg, 1, 1)
    bound = {0: K * 2.0 ** -52, 3: 2.0 ** -23 + K * 2.0 ** -24, 1: 2.0 ** -20 + K * 2.0 ** -24,
             2: 2.0 ** -20 + K * 2.0 ** -24}[prec]
    err = np.abs(got - ref)
    assert np.all(err <= bound * absref + 1e-300), float(np.max(err / np.maximum(absref, 1e-300)))
    assert np.all(got[:3] == 0.0)
    tensor_cores = prec in (1, 2) and p >= 32 and q >= 16 and s >= 16 and q % 2 == 0 and s % 2 == 0
    label = "seg_gemm_tc_bf16" if prec == 2 else "seg_gemm_tc"
    assert (kernel_time(label) is not None) == tensor_cores


# --- the Cholesky factor and inverse of the CholeskyQR orthonormalisations ---------------

@pytest.mark.parametrize("n", [20, 48, 49, 64, 100, 128, 160, 176, 177, 240])
def test_cholesky_factor_and_inverse(n):
    """R^T R = G and R R^{-1} = I to FP64 rounding (relative to the condition of G) for the
    orders of the truncation's Gram matrices: one-CTA (n <= 48) and recursive blocked
    (n > 48, splits at 16-row multiples) forms; the pivot ratio is the smallest Schur-
    complement pivot over the diagonal of G (computed here from numpy's factor); a matrix
    with a negative pivot reports the first failing position."""
    import torch
    from paper_2411_16431_b300.sgtn import cholesky
    rng = np.random.default_rng(n)
    X = rng.standard_normal((3 * n, n)) * np.exp(rng.standard_normal(n))   # graded columns
    G = X.T @ X
    Rn = np.linalg.cholesky(G).T
    R, Ri, status, mr = cholesky(torch.tensor(G, device="cuda"))
    R, Ri = R.cpu().numpy(), Ri.cpu().numpy()
    assert status == 0
    assert np.allclose(np.tril(R, -1), 0.0) and np.allclose(np.tril(Ri, -1), 0.0)
    assert np.allclose(R, Rn, rtol=1e-9, atol=1e-12 * np.abs(Rn).max())
    assert np.abs(R.T @ R - G).max() <= 1e-13 * np.abs(G).max() * n
    assert np.abs(R @ Ri - np.eye(n)).max() <= 1e-10
    assert abs(mr - np.min(np.diag(Rn) ** 2 / np.diag(G))) <= 1e-9 * mr
    # an indefinite matrix: the first non-positive pivot is reported (position + 1)
    Gb = G.copy()
    j = n // 2
    Gb[j, j] = 0.5 * (Rn[:j, j] ** 2).sum()   # Schur complement at j becomes negative
    _, _, status_b, _ = cholesky(torch.tensor(Gb, device="cuda"))
    assert status_b == j + 1


def test_seg_gemm_rejects_indices_out_of_range():
    """An X or Y block index outside the operands is refused before any launch."""
    import torch
    from paper_2411_16431_b300.sgtn import seg_gemm, SgtnError
    X = torch.zeros(4, 32, 16, dtype=torch.float64, device="cuda")
    Y = torch.zeros(3, 16, 16, dtype=torch.float64, device="cuda")
    i32 = dict(dtype=torch.int32, device="cuda")
    seg_ptr = torch.tensor([0, 2], **i32)
    for xr, yr in (([0, 4], [0, 1]), ([0, 1], [3, 0]), ([-1, 0], [0, 0])):
        with pytest.raises(SgtnError):
            seg_gemm(X, Y, seg_ptr, torch.tensor(xr, **i32), torch.tensor(yr, **i32), None, 1)
    with pytest.raises(SgtnError):   # seg_ptr must end at the number of terms
        seg_gemm(X, Y, torch.tensor([0, 3], **i32), torch.tensor([0, 1], **i32), torch.tensor([0, 1], **i32), None, 0)
