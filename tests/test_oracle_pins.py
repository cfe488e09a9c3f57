"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test pins one part of the oracle to the mathematics or to numbers the
paper prints: brute-force enumeration (Eq. 9, Eq. 5), closed forms of 1D
chains, beta = 0, gauge invariance, decoupled rows, the Pegasus dimensions of
Sec. III.B.1, and the exact-dynamic-programming property of the search.
"""
import itertools

import numpy as np
import pytest

from oracle import brute
from oracle.peps import boundary_mps
from oracle.potts import PottsModel
from oracle.search import conditional_scores, search
from paper_2411_16431_b300 import lattices as L


# --- generators ------------------------------------------------------------

def test_chimera_counts():
    inst = L.chimera_grid(4, 4, 0)
    assert inst.n_spins == 128 and inst.n_edges == 352
    assert set(np.abs(inst.j_num)) <= set(range(1, 8))


def test_class_one_couplings():
    """Class I (Sec. IV): J uniform in [-1, 1], h = 0, hence a global reflection symmetry."""
    inst = L.kings_grid(6, 7, 2, couplings="uniform")
    assert inst.denom == 1000 and not inst.h_num.any()
    assert np.abs(inst.j_num).max() <= 1000 and len(set(inst.j_num.tolist())) > inst.n_edges // 2
    assert inst.n_edges == 6 * 6 + 5 * 7 + 2 * 5 * 6
    s = np.where(np.arange(inst.n_spins) % 3 == 0, 1, -1)
    assert inst.energy_num(s) == inst.energy_num(-s)


def test_pegasus_counts_and_degree():
    # nice subgraph of P_M has 24 (M-1)^2 nodes; max degree 15 (Sec. II)
    for m, n in ((4, 216), (6, 600), (16, 5400)):
        assert L.pegasus_nice(m, 0).n_spins == n
    q, e = L.pegasus_graph(8)
    deg = np.zeros(len(q), int)
    idx = {x: i for i, x in enumerate(q)}
    for a, b in e:
        deg[idx[a]] += 1
        deg[idx[b]] += 1
    assert deg.max() == 15
    # the 5616-qubit device has "over 40000" couplers; the full P16 fabric must have more
    assert len(L.pegasus_graph(16)[1]) > 40135


def _golden(name):
    import os
    out = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            out[key] = tuple(int(v) for v in vals)
    return out


def test_pegasus_dims_match_paper():
    """Site-tensor legs (l,u,r,d) and the mediating projector dims printed in
    Sec. III.B.1 (tests/golden/pegasus_dims.txt), for a bulk cell."""
    g = _golden("pegasus_dims.txt")
    inst = L.pegasus_nice(6, 0)
    pm = PottsModel(inst, states_per_site=[np.zeros(1, np.int64)] * 25)  # no enumeration needed
    S = pm.site(2, 2)
    k = {d: len(S.coupled[d]) for d in S.coupled}
    union = lambda *ds: len(set().union(*[S.coupled[d] for d in ds]))
    assert (union("l", "ul", "dl"), union("u", "ul", "ur"), union("r", "ur", "dr"), union("d", "dl", "dr")) == g["site"]
    assert (k["ur"], k["u"], k["ul"], k["dr"], k["d"], k["dl"]) == g["proj"]


def test_planted_energy_is_ground():
    base = L.slice_cells(L.chimera_grid(2, 2, 5), 2, 1)
    inst = L.planted(base, 11)
    _, e = brute.ground_state(inst)
    assert inst.planted_energy_num == e == inst.meta["loop_bound_num"]


# --- clustering (Eqs. 2-4) --------------------------------------------------

def test_cluster_energies_match_spin_energies():
    inst = L.kings_grid(3, 3, 7)
    inst2 = L.slice_cells(L.chimera_grid(2, 2, 3), 2, 1)
    rng = np.random.default_rng(0)
    for I in (inst, inst2):
        pm = PottsModel(I)
        for _ in range(50):
            cfg = [int(rng.integers(S.d)) for S in pm.sites]
            e = sum(int(pm.sites[i].E[x]) for i, x in enumerate(cfg))
            for r in range(pm.R):
                for c in range(pm.C):
                    for d, (dr, dc) in (("r", (0, 1)), ("d", (1, 0)), ("dr", (1, 1)), ("dl", (1, -1))):
                        T = pm.site(r + dr, c + dc)
                        if T is None:
                            continue
                        S = pm.site(r, c)
                        Eb = pm.ebar(r, c, d)
                        from oracle.potts import OPP
                        a = S.proj[d].of_state[cfg[r * pm.C + c]]
                        b = T.proj[OPP[d]].of_state[cfg[(r + dr) * pm.C + c + dc]]
                        e += int(Eb[a, b])
            assert e == I.energy_num(pm.spins_of_config(cfg))


def test_projector_classes_by_enumeration():
    inst = L.chimera_grid(2, 2, 1)
    pm = PottsModel(inst)
    S = pm.site(0, 0)
    # the cell's spins 4..7 couple right, 0..3 couple down (Chimera reading)
    assert S.coupled["r"] == [4, 5, 6, 7] and S.coupled["d"] == [0, 1, 2, 3]
    for x in range(S.d):
        bits = [(x >> b) & 1 for b in range(8)]
        assert S.proj["r"].of_state[x] == sum(bits[4 + j] << j for j in range(4))


# --- log Z (Eq. 9) -------------------------------------------------------------

SMALL = [L.square_grid(3, 3, 1), L.kings_grid(4, 4, 3), L.square_grid(4, 4, 4, fields=False),
         L.slice_cells(L.chimera_grid(4, 4, 0), 2, 1), L.slice_cells(L.chimera_grid(4, 4, 0), 1, 2),
         L.kings_grid(2, 5, 9), L.kings_grid(3, 4, 6, couplings="uniform")]


@pytest.mark.parametrize("inst", SMALL, ids=lambda i: i.name)
@pytest.mark.parametrize("beta", [0.3, 1.0, 2.5])
def test_exact_logz_equals_brute_force(inst, beta):
    lz, _, _ = boundary_mps(PottsModel(inst), beta, chi=64, n_sweeps=1)
    assert abs(lz - brute.log_z(inst, beta)) < 1e-11 * max(1.0, abs(lz))


def test_beta_zero_gives_two_to_n():
    inst = L.chimera_grid(3, 3, 2)
    lz, _, _ = boundary_mps(PottsModel(inst), 0.0, chi=4, n_sweeps=1)
    assert abs(lz - inst.n_spins * np.log(2)) < 1e-10


def test_open_chain_closed_form():
    # one row of single spins, h = 0: Z = 2 prod_i 2 cosh(beta J_i)
    inst = L.square_grid(1, 9, 5, fields=False)
    beta = 0.8
    lz, _, _ = boundary_mps(PottsModel(inst), beta, chi=2, n_sweeps=1)
    J = inst.j_num / 7.0
    assert abs(lz - (np.log(2) + np.sum(np.log(2 * np.cosh(beta * J))))) < 1e-12


def test_chain_with_fields_transfer_matrix():
    # a column of single spins with fields: 2x2 transfer-matrix product
    inst = L.square_grid(7, 1, 6)
    beta = 1.3
    lz, _, _ = boundary_mps(PottsModel(inst), beta, chi=2, n_sweeps=1)
    s = np.array([1.0, -1.0])
    h = inst.h_num / 7.0
    J = inst.j_num / 7.0
    v = np.exp(-beta * h[0] * s)
    for i in range(1, 7):
        T = np.exp(-beta * J[i - 1] * np.outer(s, s)) * np.exp(-beta * h[i] * s)[None, :]
        v = v @ T
    assert abs(lz - np.log(v.sum())) < 1e-12


def test_decoupled_rows_factorise():
    inst = L.square_grid(3, 4, 8)
    keep = np.array([(inst.site_of_spin[a] // 4) == (inst.site_of_spin[b] // 4) for a, b in zip(inst.ei, inst.ej)])
    inst.j_num = np.where(keep, inst.j_num, 0).astype(np.int32)
    beta = 1.1
    lz, _, _ = boundary_mps(PottsModel(inst), beta, chi=3, n_sweeps=1)
    rows = [L.slice_cells(inst, 1, 4)]
    tot = 0.0
    for r in range(3):
        sub = L.Instance(4, np.arange(3, dtype=np.int32), np.arange(1, 4, dtype=np.int32),
                         inst.j_num[[k for k in range(inst.n_edges) if inst.ei[k] // 4 == r and inst.ej[k] // 4 == r]],
                         inst.h_num[4 * r:4 * r + 4], 7, np.arange(4, dtype=np.int32), 1, 4)
        tot += brute.log_z(sub, beta)
    assert abs(lz - tot) < 1e-11


def test_gauge_invariance_truncated():
    inst = L.chimera_grid(4, 4, 0)
    rng = np.random.default_rng(3)
    g = rng.choice([-1, 1], inst.n_spins)
    inst2 = L.Instance(inst.n_spins, inst.ei, inst.ej, (inst.j_num * g[inst.ei] * g[inst.ej]).astype(np.int32),
                       (inst.h_num * g).astype(np.int32), 7, inst.site_of_spin, 4, 4)
    a, _, _ = boundary_mps(PottsModel(inst), 1.0, chi=6, n_sweeps=1)
    b, _, _ = boundary_mps(PottsModel(inst2), 1.0, chi=6, n_sweeps=1)
    assert abs(a - b) < 1e-10 * abs(a)


def test_truncation_converges_to_exact():
    inst = L.kings_grid(5, 5, 4)
    lz_ex, _, _ = boundary_mps(PottsModel(inst), 1.0, chi=64, n_sweeps=1)
    errs = [abs(boundary_mps(PottsModel(inst), 1.0, chi=c, n_sweeps=2)[0] - lz_ex) for c in (1, 2, 4, 32)]
    assert errs[-1] < 1e-10 and errs[0] > 1e-6


# --- conditionals (Fig. 6) and search (Fig. 3) -----------------------------------

def _brute_conditional(inst, pm, cfg, n, beta):
    """p(x_{n+1} | x_<=n) by summing exp(-beta H) over all completions."""
    S = brute.all_spins(inst.n_spins)
    E = brute.energies_num(inst, S) / inst.denom
    w = np.exp(-beta * (E - E.min()))
    site = pm.sites[n]
    # which spin states agree with cfg on the placed clusters
    ok = np.ones(len(S), bool)
    for p, x in enumerate(cfg):
        Sp = pm.sites[p]
        ok &= np.all(S[:, Sp.spins] == Sp.spinvals[x][None, :], axis=1)
    out = np.zeros(site.d)
    for x in range(site.d):
        m = ok & np.all(S[:, site.spins] == site.spinvals[x][None, :], axis=1)
        out[x] = w[m].sum()
    return out / out.sum()


@pytest.mark.parametrize("inst", [L.kings_grid(3, 3, 2), L.slice_cells(L.chimera_grid(4, 4, 1), 2, 1)], ids=lambda i: i.name)
def test_exact_conditionals_match_brute_force(inst):
    beta = 0.9
    pm = PottsModel(inst)
    _, psis, mpos = boundary_mps(pm, beta, chi=64, n_sweeps=1)
    rng = np.random.default_rng(1)
    for n in range(pm.R * pm.C):
        r, c = divmod(n, pm.C)
        cfg = tuple(int(rng.integers(pm.sites[p].d)) for p in range(n))
        s = conditional_scores(pm, beta, mpos[r], psis[r], cfg, r, c)
        p = s / s.sum()
        assert np.allclose(p, _brute_conditional(inst, pm, cfg, n, beta), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("inst", [L.kings_grid(4, 4, 3), L.square_grid(4, 4, 12),
                                  L.slice_cells(L.chimera_grid(4, 4, 0), 2, 1),
                                  L.planted(L.slice_cells(L.chimera_grid(2, 2, 5), 1, 2), 4),
                                  L.kings_grid(3, 4, 6, couplings="uniform")], ids=lambda i: i.name)
def test_exact_search_is_dynamic_programming(inst):
    """With exact marginals and no top-M cut, merging keeps the best completion of each boundary,
    so the search returns the brute-force ground state and log p = -beta E - log Z."""
    beta = 1.7
    res = search(inst, beta, chi=256, M=10 ** 9, n_sweeps=1)
    _, e = brute.ground_state(inst)
    assert int(res["energy_num"][0]) == e
    lz = brute.log_z(inst, beta)
    assert abs(res["logp"][0] + beta * e / inst.denom + lz) < 1e-9
    assert res["pd"] <= res["logp"][0] + 1e-12


def test_search_config1_smoke():
    res = search(L.chimera_grid(4, 4, 0), 1.0, chi=16, M=64, n_sweeps=2)
    assert res["energy_num"][0] == res["pm"].state_energy_num(res["configs"][0])
    assert res["pd"] < 0 and len(res["configs"]) == 1


def test_pegasus_restricted_logz_by_enumeration():
    """Pegasus P3 (2x2 cells of 24 spins, one diagonal) on reduced state sets: the exact
    contraction equals the brute-force sum of exp(-beta H) over the restricted product space."""
    inst = L.pegasus_nice(3, 4)
    states = L.hamming_ball_states(inst, 10, seed=1)
    pm = PottsModel(inst, states)
    beta = 0.7
    lz, _, _ = boundary_mps(pm, beta, chi=256, n_sweeps=1)
    # brute force over all 10^4 combinations, energies from spins only
    sp_of = [[i for i in range(inst.n_spins) if inst.site_of_spin[i] == s] for s in range(4)]
    E = []
    for combo in itertools.product(*[range(len(s)) for s in states]):
        spins = np.zeros(inst.n_spins, np.int64)
        for s, x in enumerate(combo):
            pat = int(states[s][x])
            spins[sp_of[s]] = [1 - 2 * ((pat >> j) & 1) for j in range(len(sp_of[s]))]
        E.append(inst.energy_num(spins))
    E = np.array(E) / 7.0
    m = (-beta * E).max()
    ref = m + np.log(np.exp(-beta * E - m).sum())
    assert abs(lz - ref) < 1e-11 * abs(ref)


def test_pegasus_restricted_search_finds_restricted_ground_state():
    inst = L.planted(L.pegasus_nice(3, 2), 5, loops_per_cell=4)
    states = L.hamming_ball_states(inst, 12)          # ball around the planted state
    res = search(inst, 2.0, chi=256, M=10 ** 6, n_sweeps=1, states=states)
    assert int(res["energy_num"][0]) == inst.planted_energy_num


# --- gradients (Eq. 9: d log Z/dJ = -beta<ss>, d/dh = -beta<s>, d/dbeta = -<H>) ---------

@pytest.mark.parametrize("inst", [L.kings_grid(3, 3, 2), L.kings_grid(4, 4, 3), L.square_grid(4, 3, 5),
                                  L.slice_cells(L.chimera_grid(4, 4, 0), 2, 1)], ids=lambda i: i.name)
def test_exact_gradient_equals_brute_force_correlators(inst):
    from oracle.grad import logz_grad
    beta = 0.9
    _, dJ, dh, db = logz_grad(inst, beta, chi=64, n_sweeps=1)
    ss, m, H = brute.correlators(inst, beta)
    assert np.allclose(dJ, -beta * ss, atol=1e-12)
    assert np.allclose(dh, -beta * m, atol=1e-12)
    assert abs(db + H) < 1e-11 * max(1, abs(H))


def test_truncated_gradient_close_to_finite_differences():
    """Environment correlators vs central differences (step 1e-4) of the truncated log Z:
    equal up to the truncation error, so the tolerance is loose; it catches a wrong
    sign, a dropped factor or a misplaced edge."""
    from oracle.grad import logz_grad
    inst, beta, chi = L.chimera_grid(3, 3, 1), 1.0, 4
    _, dJ, dh, db = logz_grad(inst, beta, chi, n_sweeps=2)

    def lz(jn=None, hn=None, b=beta):
        I = L.Instance(inst.n_spins, inst.ei, inst.ej, inst.j_num if jn is None else jn,
                       inst.h_num if hn is None else hn, 7, inst.site_of_spin, inst.rows, inst.cols)
        return boundary_mps(PottsModel(I), b, chi, 2)[0]

    eps = 1e-4
    assert abs(db - (lz(b=beta + eps) - lz(b=beta - eps)) / (2 * eps)) < 1e-3 * abs(db)
    # couplings and fields are integers over denom: refine the grid (denom 7 -> 7 K) and move one by 1/(7 K)
    K = 20000
    for kind, e in (("J", 0), ("J", 17), ("J", 45), ("h", 3), ("h", 50)):
        vals = []
        for sgn in (+1, -1):
            jn = inst.j_num.astype(np.int64) * K
            hn = inst.h_num.astype(np.int64) * K
            (jn if kind == "J" else hn)[e] += sgn
            I = L.Instance(inst.n_spins, inst.ei, inst.ej, jn, hn, 7 * K, inst.site_of_spin, inst.rows, inst.cols)
            vals.append(boundary_mps(PottsModel(I), beta, chi, 2)[0])
        fd = (vals[0] - vals[1]) / (2.0 / (7 * K))
        got = dJ[e] if kind == "J" else dh[e]
        assert abs(got - fd) < 1e-2 * max(1.0, abs(fd)), (kind, e, got, fd)


def test_grid_symmetries_keep_log_z_and_ground_state():
    """The eight symmetries of the cluster grid change only the direction of the
    contraction: exact log Z and the exact-DP ground state are unchanged (king's
    lattice: both diagonals trade places; Chimera: vertical and horizontal
    couplings trade places)."""
    for inst, beta in ((L.kings_grid(2, 3, 4), 0.7), (L.slice_cells(L.chimera_grid(3, 3, 6), 2, 1), 1.1)):
        ref = brute.log_z(inst, beta)
        e0 = brute.ground_state(inst)[1]
        for k in range(8):
            t = L.transform(inst, k)
            assert t.rows * t.cols == inst.rows * inst.cols
            assert len(set(t.site_of_spin.tolist())) == t.rows * t.cols
            lz, _, _ = boundary_mps(PottsModel(t), beta, 256, 1)
            assert abs(lz - ref) < 1e-12 * abs(ref)
            res = search(t, beta, chi=256, M=10 ** 6, n_sweeps=1)
            assert res["energy_num"][0] == e0


# --- loopy belief propagation (Sec. IV) -------------------------------------------

def _exact_cluster_marginals(inst, beta):
    """p(x_n) by enumeration: x_n = bits of the cluster's spins (bit j = j-th spin, 1 = down)."""
    S = brute.all_spins(inst.n_spins)
    E = brute.energies_num(inst, S) / inst.denom
    p = np.exp(-beta * (E - E.min()))
    p /= p.sum()
    out = []
    for site in range(inst.rows * inst.cols):
        spins = np.nonzero(inst.site_of_spin == site)[0]
        x = np.zeros(len(p), np.int64)
        for j, g in enumerate(spins):
            x |= ((1 - S[:, g].astype(np.int64)) // 2) << j
        out.append(np.bincount(x, weights=p, minlength=1 << len(spins)))
    return out


@pytest.mark.parametrize("inst", [L.slice_cells(L.chimera_grid(4, 4, 0), 1, 2), L.slice_cells(L.chimera_grid(4, 4, 3), 2, 1),
                                  L.kings_grid(1, 7, 4), L.square_grid(5, 1, 2, couplings="uniform")],
                         ids=lambda i: i.name)
def test_lbp_is_exact_on_a_chain_of_clusters(inst):
    """On a tree of clusters (a single row or column) belief propagation is exact once
    messages have crossed it: the marginals are the enumerated cluster marginals."""
    from oracle.lbp import lbp
    beta = 0.9
    marg, change = lbp(PottsModel(inst), beta, n_iter=inst.rows * inst.cols + 1)
    exact = _exact_cluster_marginals(inst, beta)
    for m, e in zip(marg, exact):
        assert np.allclose(m, e, rtol=1e-10, atol=1e-14)
    assert change < 1e-12


def test_lbp_limits():
    """beta = 0 gives uniform marginals; couplings of zero between clusters give the
    local Boltzmann weights of each cluster; marginals sum to one on a loopy grid."""
    from oracle.lbp import lbp, top_states
    inst = L.chimera_grid(3, 3, 5)
    marg, _ = lbp(PottsModel(inst), 0.0, n_iter=3)
    assert all(np.allclose(m, 1.0 / len(m), rtol=1e-13) for m in marg)
    dec = L.chimera_grid(2, 3, 6)
    inter = dec.site_of_spin[dec.ei] != dec.site_of_spin[dec.ej]
    dec.j_num = np.where(inter, 0, dec.j_num).astype(np.int32)
    pm = PottsModel(dec)
    marg, _ = lbp(pm, 1.3, n_iter=4)
    for S, m in zip(pm.sites, marg):
        w = np.exp(-1.3 * (S.E - S.E.min()) / dec.denom)
        assert np.allclose(m, w / w.sum(), rtol=1e-12)
    marg, change = lbp(PottsModel(L.kings_grid(4, 4, 3)), 1.0, n_iter=6)
    assert all(abs(m.sum() - 1) < 1e-12 and (m >= 0).all() for m in marg) and change > 0
    assert list(top_states(np.array([0.1, 0.3, 0.3, 0.05, 0.25]), 3)) == [1, 2, 4]


# --- droplets (Fig. 4) ----------------------------------------------------------------

@pytest.mark.parametrize("inst", [L.kings_grid(4, 4, 3), L.slice_cells(L.chimera_grid(4, 4, 0), 2, 1),
                                  L.kings_grid(3, 5, 6, couplings="uniform")], ids=lambda i: i.name)
def test_droplets_are_exact_excitations(inst):
    """Every droplet of the best configuration is an excitation whose energy, recomputed
    from scratch on the flipped configuration, is E_best + dE; it is connected, within the
    energy window and farther than the Hamming threshold from the others.  With exact
    marginals and no cut the main branch of a merge has the lowest interior energy, so
    every dE >= 0."""
    from oracle.droplets import adjacency, connected, search_droplets
    max_dE, hmin = 6 * inst.denom, 1
    res = search_droplets(inst, 1.2, chi=256, M=10 ** 6, max_dE=max_dE, min_hamming=hmin, n_sweeps=1)
    s = res["pm"].spins_of_config(res["config"])
    E0 = inst.energy_num(s)
    assert E0 == brute.ground_state(inst)[1]
    adj = adjacency(inst)
    assert res["droplets"]
    for dE, F in res["droplets"]:
        t = s.copy()
        t[F] *= -1
        assert inst.energy_num(t) == E0 + dE
        assert 0 <= dE <= max_dE and connected(F, adj)
    Fs = [set(F) for _, F in res["droplets"]]
    assert all(len(a ^ b) > hmin for i, a in enumerate(Fs) for b in Fs[i + 1:])


def test_droplet_filters():
    """The Fig. 4 filters on hand-made droplets: energy window, connectivity, and the
    Hamming rule (a closer, lower droplet replaces every droplet it clashes with)."""
    from oracle.droplets import try_insert
    adj = [[1], [0, 2], [1, 3], [2], []]          # path 0-1-2-3, isolated 4
    d = try_insert([], (5, frozenset({0, 1})), 10, 1, adj)
    assert d == [(5, frozenset({0, 1}))]
    assert try_insert(d, (11, frozenset({3})), 10, 1, adj) == d          # above the window
    assert try_insert(d, (1, frozenset({0, 2})), 10, 1, adj) == d        # not connected
    assert try_insert(d, (7, frozenset({1})), 10, 1, adj) == d           # clashes, not lower
    assert try_insert(d, (3, frozenset({1})), 10, 1, adj) == [(3, frozenset({1}))]
    assert try_insert(d, (3, frozenset({2, 3})), 10, 1, adj) == d + [(3, frozenset({2, 3}))]


def test_search_tie_rule_on_a_flat_landscape():
    """With every coupling and field zero all configurations are equally probable:
    every merge and the top-M cut are ties, which go to the lexicographically
    smallest configuration, so the search returns all-zero state indices
    (all spins up) with energy 0 and log p = -N log 2."""
    inst = L.kings_grid(3, 4, 2)
    inst.j_num = np.zeros_like(inst.j_num)
    inst.h_num = np.zeros_like(inst.h_num)
    res = search(inst, 1.0, chi=4, M=3, n_sweeps=1)
    assert res["configs"][0] == (0,) * (inst.rows * inst.cols)
    assert int(res["energy_num"][0]) == 0
    assert abs(res["logp"][0] + inst.n_spins * np.log(2)) < 1e-10


# --- the zipper's instantaneous-stage sweep and the cut (Sec. III.B, Fig. 8) ---------

def _chain(tensors, first_open):
    """Dense product of column tensors G_j[bond_in, bond_out, u] over the columns, the
    first bond_in left open when ``first_open`` (result [bond_in, physical...])."""
    Y = tensors[0]
    for G in tensors[1:]:
        Y = np.einsum("xbp,bcu->xcpu", Y, G).reshape(Y.shape[0], G.shape[1], -1)
    assert Y.shape[1] == 1
    return Y[:, 0, :] if first_open else Y[0, 0, :]


def _mpo_mps_columns(Ws, A, c0):
    """(W_j A_j)[(bl, i), (br, j), u] for the columns c0..C-1 (plain einsum of the definitions)."""
    out = []
    for W, a in zip(Ws[c0:], A[c0:]):
        G = np.einsum("abus,sij->aibju", W, a)
        out.append(G.reshape(G.shape[0] * G.shape[1], G.shape[2] * G.shape[3], G.shape[4]))
    return out


def _random_right_canonical(rng, dims, bonds):
    """phi[j][u, a, b] with orthonormal rows of the (a) x (u, b) matrix, right bond of the last = 1."""
    phi = []
    for j, u in enumerate(dims):
        a, b = bonds[j], bonds[j + 1]
        Q, _ = np.linalg.qr(rng.standard_normal((u * b, a)))
        phi.append(Q.T.reshape(a, u, b).transpose(1, 0, 2))
    return phi


@pytest.mark.parametrize("e_off", [None, 1], ids=["full", "window2"])
def test_stage_sweep_centre_is_projection_and_captured_weight_grows(e_off):
    """One sweep of the zipper's instantaneous stage (Fig. 8d) over columns c0..e with the
    left bond open: the returned centre is the projection <phi|Y> of the dense target Y
    (the MPO-MPS product of columns c0..C-1), the new phi are right-canonical, tensors right
    of e are untouched, and the captured weight |<phi|Y>|^2 never decreases (each one-site
    update maximises the overlap) and does grow from a random start."""
    from oracle.peps import RowMPO, left_canonical, stage_sweep
    inst = L.kings_grid(3, 5, 7)
    pm = PottsModel(inst)
    mpo = RowMPO(pm, 1, 0.9)
    C = pm.C
    Ws = [mpo.dense(c) for c in range(C)]
    rng = np.random.default_rng(5)
    bonds_A = [1, 2, 3, 3, 2, 1]
    A = [rng.standard_normal((mpo.cols[c]["nsig"], bonds_A[c], bonds_A[c + 1])) for c in range(C)]
    A, _ = left_canonical(A, 0.0)
    c0 = 1
    e = C - 1 if e_off is None else c0 + e_off
    dims = [mpo.cols[c]["nU"] for c in range(c0, C)]
    phi = [None] * c0 + _random_right_canonical(rng, dims, [2, 2, 2, 2, 1])
    Y = _chain(_mpo_mps_columns(Ws, A, c0), True)                    # [(bl, al), P]
    Phi = _chain([p.transpose(1, 2, 0) for p in phi[c0:]], True)    # [k, P]
    assert np.allclose(Phi @ Phi.T, np.eye(Phi.shape[0]), atol=1e-12)
    K0 = Y @ Phi.T
    bl, al = Ws[c0].shape[0], A[c0].shape[1]
    kept = [p.copy() for p in phi[e + 1:]]
    new, K = stage_sweep(Ws, A, list(phi), K0.reshape(bl, al, -1), c0, e)
    Phi2 = _chain([p.transpose(1, 2, 0) for p in new[c0:]], True)
    assert np.allclose(Phi2 @ Phi2.T, np.eye(Phi2.shape[0]), atol=1e-12)
    Kd = K.reshape(bl * al, -1)
    assert np.allclose(Kd, Y @ Phi2.T, rtol=0, atol=1e-12 * np.abs(Kd).max())
    for a, b in zip(kept, new[e + 1:]):
        assert np.array_equal(a, b)
    w0, w1 = np.sum(K0 ** 2), np.sum(Kd ** 2)
    assert w1 >= w0 * (1 - 1e-12) and w1 > w0 * (1 + 1e-6)
    # a second sweep from the first's output does not lose weight either
    _, K2 = stage_sweep(Ws, A, list(new), K, c0, e)
    assert np.sum(K2 ** 2) >= w1 * (1 - 1e-12)


def test_two_column_row_reaches_eckart_young():
    """A single two-column row applied to the trivial MPS is the matrix v[u0, u1] of the row's
    Boltzmann weights summed per pair of up-exposure patterns (by enumeration of the row's
    spins).  One bond is truncated, so the best bond-chi MPS is the truncated SVD of v
    (Eckart-Young); the zipper with its sweeps, the cut and repeated sweeps (block power
    iteration on v) must reach it: same direction to 1e-10, captured weight = the kept
    singular values' share."""
    inst = L.chimera_grid(2, 2, 3)
    beta = 0.6
    row = [i for i in range(inst.n_spins) if inst.site_of_spin[i] >= 2]           # row 1 spins
    in_row = np.zeros(inst.n_spins, bool)
    in_row[row] = True
    up = {c: [] for c in (0, 1)}
    for i, j in zip(inst.ei.tolist(), inst.ej.tolist()):
        for a, b in ((i, j), (j, i)):
            if in_row[a] and not in_row[b]:
                up[int(inst.site_of_spin[a]) - 2].append(a)
    up = {c: sorted(set(v)) for c, v in up.items()}
    S = brute.all_spins(len(row)).astype(np.int64)
    pos = {g: k for k, g in enumerate(row)}
    E = np.zeros(len(S), np.int64)
    for i, j, J in zip(inst.ei.tolist(), inst.ej.tolist(), inst.j_num.tolist()):
        if in_row[i] and in_row[j]:
            E += J * S[:, pos[i]] * S[:, pos[j]]
    for i in row:
        E += int(inst.h_num[i]) * S[:, pos[i]]
    w = np.exp(-beta * (E - E.min()) / inst.denom)
    pat = [sum(((S[:, pos[g]] < 0).astype(np.int64) << k) for k, g in enumerate(up[c])) for c in (0, 1)]
    v = np.zeros((1 << len(up[0]), 1 << len(up[1])))
    np.add.at(v, (pat[0], pat[1]), w)
    sv = np.linalg.svd(v, compute_uv=False)
    chi = next(k for k in range(1, len(sv) - 1) if sv[k] < 0.5 * sv[k - 1])
    U, s, Vh = np.linalg.svd(v)
    v_chi = (U[:, :chi] * s[:chi]) @ Vh[:chi]
    _, psis, _ = boundary_mps(PottsModel(inst), beta, chi=chi, n_sweeps=30)
    A, ln = psis[0]
    assert A[0].shape[2] == chi
    from oracle.peps import mps_dense
    phi = mps_dense(A)
    phi_hat = phi / np.linalg.norm(phi)
    assert np.allclose(phi_hat, v_chi / np.linalg.norm(v_chi), rtol=0, atol=1e-10)
    # the overlap with v captures exactly the kept share of the weight
    fid = np.sum(phi_hat * v) ** 2 / np.sum(v * v)
    assert abs(fid - np.sum(s[:chi] ** 2) / np.sum(s ** 2)) < 1e-10


# --- the bounding with a real top-M cut (Fig. 3d-e, Eq. 7) ------------------------------

def _site_states_of_spins(pm, S):
    """Cluster state index of every spin configuration, per site (full enumeration: index = pattern)."""
    X = np.zeros((len(S), len(pm.sites)), np.int64)
    for t, site in enumerate(pm.sites):
        for k, g in enumerate(site.spins):
            X[:, t] |= (S[:, g] < 0).astype(np.int64) << k
    return X


@pytest.mark.parametrize("M", [1, 3, 8])
@pytest.mark.parametrize("inst", [L.kings_grid(4, 4, 3), L.square_grid(3, 5, 12),
                                  L.slice_cells(L.chimera_grid(4, 4, 0), 2, 1)], ids=lambda i: i.name)
def test_top_m_cut_matches_brute_force_partial_marginals(inst, M):
    """With an exact contraction, every step's beam is a top-M set of the previous beam's
    extensions after merging by boundary (Eq. 7), with the exact partial marginals
    p(x_1..x_n) = sum over completions of exp(-beta H) / Z by enumeration: kept candidates
    lie in distinct boundary groups, each is its group's most probable, no discarded group
    is more probable than a kept one, min(M, #groups) are kept, and p_d is the most
    probable candidate not kept."""
    beta = 1.1
    trace = []
    res = search(inst, beta, chi=256, M=M, n_sweeps=1, trace=trace)
    pm = res["pm"]
    S = brute.all_spins(inst.n_spins)
    lw = -beta * brute.energies_num(inst, S) / inst.denom
    lz = float(np.logaddexp.reduce(lw))
    X = _site_states_of_spins(pm, S)
    nb = {}
    for i, j in zip(inst.ei.tolist(), inst.ej.tolist()):
        nb.setdefault(i, set()).add(j)
        nb.setdefault(j, set()).add(i)
    site_of = inst.site_of_spin
    tol = 1e-9
    beam = [()]
    for n, (kept, pd_step) in enumerate(trace):
        exposed = sorted(g for g in range(inst.n_spins) if site_of[g] <= n and any(site_of[q] > n for q in nb.get(g, ())))
        cand = {}
        for cfg in beam:
            m = np.all(X[:, :n] == np.array(cfg, np.int64)[None, :], axis=1) if n else np.ones(len(S), bool)
            for x in range(pm.sites[n].d):
                mm = m & (X[:, n] == x)
                lp = float(np.logaddexp.reduce(lw[mm])) - lz
                c = cfg + (x,)
                spins = pm.spins_of_config(c + (0,) * (len(pm.sites) - n - 1))
                cand[c] = (lp, tuple(int(spins[g]) for g in exposed))
        groups = {}
        for c, (lp, key) in cand.items():
            groups[key] = max(groups.get(key, -np.inf), lp)
        kcfg = [c for c, _ in kept]
        assert len(kcfg) == min(M, len(groups))
        assert len(set(cand[c][1] for c in kcfg)) == len(kcfg)
        for c, lp in kept:
            assert abs(lp - cand[c][0]) < tol
            assert cand[c][0] >= groups[cand[c][1]] - tol
        kept_keys = set(cand[c][1] for c in kcfg)
        worst_kept = min(cand[c][0] for c in kcfg)
        for key, top in groups.items():
            if key not in kept_keys:
                assert top <= worst_kept + tol
        rest = [lp for c, (lp, _) in cand.items() if c not in set(kcfg)]
        if rest:
            assert abs(pd_step - max(rest)) < tol
        else:
            assert pd_step == -np.inf
        beam = kcfg


def test_tie_rule_never_prefers_a_less_probable_candidate_beyond_the_tolerance():
    """merge_and_cut on random groups with exact and near ties (the rule that makes
    degenerate candidates deterministic): a merge winner is never less probable than its
    group's best by more than the tie tolerance, no discarded group beats a kept one by
    more than it, and where all log-probabilities are well separated the result is the
    plain argmax per group and the plain top-M."""
    from oracle.search import merge_and_cut, tie_tol
    rng = np.random.default_rng(11)
    for trial in range(300):
        M = int(rng.integers(1, 6))
        base = rng.choice([-3.0, -2.0, -2.0 + 1e-13, -1.5, -1.5 - 4e-12], size=int(rng.integers(1, 15)))
        sep = trial % 2 == 1
        if sep:
            base = -rng.permutation(np.arange(len(base))) * 0.37 - 1.0
        cands = {}
        for i, lp in enumerate(base):
            key = int(rng.integers(0, 4))
            cands.setdefault(key, []).append(((int(rng.integers(0, 9)), i), float(lp)))
        kept, pd = merge_and_cut(cands, M)
        best = {k: max(lp for _, lp in g) for k, g in cands.items()}
        key_of = {cfg: k for k, g in cands.items() for cfg, _ in g}
        assert len(kept) == min(M, len(cands))
        for cfg, lp in kept:
            assert lp >= best[key_of[cfg]] - tie_tol(best[key_of[cfg]])
        worst = min(lp for _, lp in kept)
        kept_keys = {key_of[c] for c, _ in kept}
        for k, b in best.items():
            if k not in kept_keys:
                assert b <= worst + tie_tol(worst)
        allc = [t for g in cands.values() for t in g]
        rest = [lp for cfg, lp in allc if cfg not in {c for c, _ in kept}]
        assert pd == (max(rest) if rest else -np.inf)
        if sep:
            winners = sorted(((max(g, key=lambda t: t[1])) for g in cands.values()), key=lambda t: -t[1])[:M]
            assert [c for c, _ in kept] == [c for c, _ in winners]


@pytest.mark.parametrize("window", [0, 2])
def test_every_zipper_step_is_followed_by_a_sweep_of_its_stage(window):
    """Sec. III.B: each zipper step is followed by a variational sweep of the instantaneous
    stage.  At every step the connecting tensor is the projection <phi[c..]|Y_c> of the
    stage's target Y_c (the dense MPO-MPS product of columns c..C-1) onto the tensors built
    so far -- the zipper's own truncation already gives that -- and the sweep can only raise
    the captured weight |<phi[c..]|Y_c>|^2; it does raise it on this truncated row, while a
    zipper without the sweeps (window 1) leaves every stage as the truncation made it."""
    from oracle.peps import RowMPO, left_canonical, zipper
    inst = L.kings_grid(3, 5, 7)
    pm = PottsModel(inst)
    mpo = RowMPO(pm, 1, 1.3)
    C = pm.C
    Ws = [mpo.dense(c) for c in range(C)]
    rng = np.random.default_rng(8)
    bonds_A = [1, 2, 4, 4, 2, 1]
    A = [rng.standard_normal((mpo.cols[c]["nsig"], bonds_A[c], bonds_A[c + 1])) for c in range(C)]
    A, ln = left_canonical(A, 0.0)

    def stages(w):
        trace = []
        zipper(mpo, A, ln, 2, window=w, trace=trace)
        gains = []
        for c, tens, K, Kb in trace:
            Y = _chain(_mpo_mps_columns(Ws, A, c), True)
            Phi = _chain([p.transpose(1, 2, 0) for p in tens], True)
            P = Y @ Phi.T
            assert np.allclose(K.reshape(P.shape), P, rtol=0, atol=1e-11 * np.abs(P).max())
            gains.append(np.sum(K ** 2) / np.sum(Kb ** 2) - 1.0)
        assert len(gains) == C
        return gains

    g = stages(window)
    assert min(g) > -1e-12 and max(g) > 1e-6
    assert max(abs(x) for x in stages(1)) < 1e-12     # no sweeps: nothing changes after the truncation


# --- the transposed row MPO as a column over (state, lower class) pairs -------
def _dense_column(col):
    """W[(lam,g)][(lam',g')][u][sigma] = sum_x [Lam x = lam, U x = u] [pul sigma = g] T[x, lam', g', sigma]."""
    T = col["T"]
    nG, nsig = col["nGl"], col["nsig"]
    W = np.zeros((col["nLam"] * nG, col["nLR"] * col["nGR"], col["nU"], nsig))
    for x in range(T.shape[0]):
        for sg in range(nsig):
            bl = col["lam_x"][x] * nG + col["pul"][sg]
            W[bl, :, col["u_x"][x], sg] += T[x, :, :, sg].reshape(-1)
    return W


@pytest.mark.parametrize("inst,states", [
    (L.pegasus_nice(4, 3), "ball12"), (L.kings_grid(3, 3, 5), None), (L.chimera_grid(3, 2, 4), None)],
    ids=["pegasus3x3_12states", "kings3x3", "chimera3x2"])
def test_transposed_column_as_virtual_states(inst, states):
    """The gradient's top-down pass applies T_r^T written as a forward-form column
    over virtual states y = (x, sigma): left bond Lam x nG + pul sigma, output
    sigma, input u_x through an identity table, right-bond factor
    Bh'[(pr, pur)][lam'] = Bh[pr][pl lam'] Bdl[pdl lam'][pur], Bdr unchanged,
    weight w_x Bv[pd_x][pu sigma].  Built here from the bond tables and
    compared element by element with the transpose (u <-> sigma) of the
    oracle's dense column."""
    from oracle.peps import RowMPO
    if states == "ball12":
        states = L.hamming_ball_states(inst, 12, seed=2)
    pm = PottsModel(inst, states)
    beta = 0.7
    mpo0 = RowMPO(pm, 0, beta)
    for r in range(pm.R - 1):
        mpo = RowMPO(pm, r, beta)
        for c in range(pm.C):
            col = mpo.cols[c]
            W = _dense_column(col)
            S, below, right = pm.site(r, c), pm.site(r + 1, c), pm.site(r, c + 1)
            w = np.exp(-beta * (S.E - S.E.min()) / inst.denom)
            sig = pm.joint(r + 1, c, ("u", "ul", "ur"))
            pu, pul, pur = (pm.component(sig, below, k) for k in ("u", "ul", "ur"))
            nPur = below.proj["ur"].n
            if right is not None:
                lamR = pm.joint(r, c + 1, ("l", "dl"))
                pl, pdl = pm.component(lamR, right, "l"), pm.component(lamR, right, "dl")
                Bdl = mpo._B(r, c + 1, "dl")
            else:
                pl = pdl = np.zeros(1, dtype=np.int64)
                Bdl = np.ones((1, 1))
            Bv, Bh, Bdr = mpo._B(r, c, "d"), mpo._B(r, c, "r"), mpo._B(r, c, "dr")
            nPr = S.proj["r"].n
            # Bh'[(pr, pur)][lam'] = Bh[pr][pl lam'] Bdl[pdl lam'][pur]
            Bhp = np.zeros((nPr * nPur, col["nLR"]))
            for pr in range(nPr):
                for q in range(nPur):
                    Bhp[pr * nPur + q] = Bh[pr, pl] * Bdl[pdl, q]
            nG, nU, nsig = col["nGl"], col["nU"], col["nsig"]
            Wt = np.zeros((col["nLam"] * nG, col["nLR"] * col["nGR"], nsig, nU))
            for x in range(S.d):
                for sg in range(nsig):
                    bl = col["lam_x"][x] * nG + pul[sg]                 # Lam' y
                    wy = w[x] * Bv[S.proj["d"].of_state[x], pu[sg]]      # w'_y
                    prp = S.proj["r"].of_state[x] * nPur + pur[sg]       # pr' y
                    right_factor = (Bhp[prp][:, None] * Bdr[S.proj["dr"].of_state[x]][None, :]).reshape(-1)
                    Wt[bl, :, sg, col["u_x"][x]] += wy * right_factor    # out sigma, in u_x (identity Bv')
            assert np.allclose(Wt, W.transpose(0, 1, 3, 2), rtol=1e-13, atol=0)
    assert mpo0.cols[0]["nU"] == 1   # the top row has no upper classes: E_0 is the trivial MPS
