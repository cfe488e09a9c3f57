"""Seeded synthetic Ising instances on quasi-2D lattices of unit cells.

This module only *draws inputs*: spins, couplings J_ij = j/denom, fields
h_i = k/denom and the assignment of spins to the R x C grid of clusters
(paper Sec. II, Eq. 1; clusters of Sec. III, Eq. 2).  It contains none of the
method's arithmetic, so the CPU oracle and the CUDA library can both be fed
from it.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), seeded per instance.  A draw
of a coupling or field picks one of the 14 values {+-1, ..., +-7} uniformly
(value/7), matching the i.i.d. workloads used for benchmarking; the square and
king's lattices can instead draw class I couplings (uniform in [-1, 1] on a
grid of step 1/1000, no fields; paper Sec. IV and App. B).

Lattices
--------
* ``chimera_grid``   R x C grid of K_{4,4} cells, 8 spins per cell.  Spins 0-3
  of a cell couple to the same-index spin of the cell below, spins 4-7 to the
  same-index spin of the cell to the right; the cell itself is the complete
  bipartite graph {0..3} x {4..7}.
* ``square_grid`` / ``kings_grid``  one spin per site, nearest-neighbour bonds
  (plus both diagonals for the king's lattice), paper App. B.
* ``pegasus_nice``   the Pegasus graph P_M (paper Sec. II, Fig. 1a) built
  from its geometric definition: every qubit is a straight segment of length
  12 on a 12M x 12M grid, perpendicular segments that cross are coupled
  (internal couplers), collinear neighbours are coupled (external couplers)
  and qubits 2j, 2j+1 of a segment pair are coupled (odd couplers).  The
  (M-1)^2 "nice" cells of 24 qubits -- three K_{4,4} tiles each -- become the
  clusters of the Potts model; qubits outside nice cells are dropped.
* ``planted``  any of the above with couplings replaced by frustrated 4-loop
  tiles consistent with a seeded planted state, so the ground energy is known.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele-Lea-Flood 2014) on Python ints."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        return self.next() % n

    def pm7(self) -> int:
        """Uniform on {-7..-1, 1..7}."""
        v = self.below(14)
        return (v % 7 + 1) * (1 if v < 7 else -1)

    def uniform01(self) -> float:
        return (self.next() >> 11) * (1.0 / (1 << 53))


@dataclass
class Instance:
    """An Ising instance H = sum J_ij s_i s_j + sum h_i s_i on an R x C grid of clusters.

    Couplings and fields are integers over ``denom`` (J_ij = j_num / denom).
    ``site_of_spin[i] = r * cols + c`` places spin i in cluster (r, c).
    ``ei < ej`` and edges are sorted lexicographically.
    """

    n_spins: int
    ei: np.ndarray
    ej: np.ndarray
    j_num: np.ndarray
    h_num: np.ndarray
    denom: int
    site_of_spin: np.ndarray
    rows: int
    cols: int
    name: str = ""
    planted: Optional[np.ndarray] = None      # planted state (+-1) if any
    planted_energy_num: Optional[int] = None  # its energy numerator
    meta: dict = field(default_factory=dict)

    @property
    def n_edges(self) -> int:
        return int(self.ei.shape[0])

    def energy_num(self, spins: np.ndarray) -> int:
        """Exact energy numerator (integer) of one configuration of +-1 spins."""
        s = np.asarray(spins, dtype=np.int64)
        return int(np.sum(self.j_num * s[self.ei] * s[self.ej]) + np.sum(self.h_num * s))


UNIFORM_DENOM = 1000


def _finish(n, edges, site_of_spin, rows, cols, rng, name, fields=True, couplings="pm7"):
    """``couplings``: "pm7" draws J and h from {+-1..+-7}/7; "uniform" draws J
    uniformly from the grid {-1000..1000}/1000 of [-1, 1] with no fields (the
    paper's class I, Sec. IV) -- ``fields`` is then ignored."""
    edges = sorted(set((min(a, b), max(a, b)) for a, b in edges if a != b))
    ei = np.array([a for a, _ in edges], dtype=np.int32)
    ej = np.array([b for _, b in edges], dtype=np.int32)
    if couplings == "uniform":
        jn = np.array([rng.below(2 * UNIFORM_DENOM + 1) - UNIFORM_DENOM for _ in edges], dtype=np.int32)
        hn = np.zeros(n, dtype=np.int32)
        return Instance(n, ei, ej, jn, hn, UNIFORM_DENOM, np.asarray(site_of_spin, dtype=np.int32), rows, cols,
                        name + "_classI")
    if couplings != "pm7":
        raise ValueError(f"unknown coupling distribution {couplings!r}")
    jn = np.array([rng.pm7() for _ in edges], dtype=np.int32)
    hn = np.array([rng.pm7() if fields else 0 for _ in range(n)], dtype=np.int32)
    return Instance(n, ei, ej, jn, hn, 7, np.asarray(site_of_spin, dtype=np.int32), rows, cols, name)


def chimera_grid(rows: int, cols: int, seed: int, fields: bool = True) -> Instance:
    """R x C grid of K44 cells (8 spins); vertical shore 0-3 links down, horizontal shore 4-7 links right."""
    rng = SplitMix64(seed)
    n = 8 * rows * cols
    site = [0] * n
    edges = []
    for r in range(rows):
        for c in range(cols):
            base = 8 * (r * cols + c)
            for k in range(8):
                site[base + k] = r * cols + c
            for a in range(4):
                for b in range(4, 8):
                    edges.append((base + a, base + b))
            if r + 1 < rows:
                below = 8 * ((r + 1) * cols + c)
                for k in range(4):
                    edges.append((base + k, below + k))
            if c + 1 < cols:
                right = 8 * (r * cols + c + 1)
                for k in range(4, 8):
                    edges.append((base + k, right + k))
    return _finish(n, edges, site, rows, cols, rng, f"chimera{rows}x{cols}_s{seed}", fields)


def square_grid(rows: int, cols: int, seed: int, fields: bool = True, kings: bool = False,
                couplings: str = "pm7") -> Instance:
    """One spin per site with nearest-neighbour bonds (and both diagonals if ``kings``)."""
    rng = SplitMix64(seed)
    n = rows * cols
    edges = []
    for r in range(rows):
        for c in range(cols):
            i = r * cols + c
            if c + 1 < cols:
                edges.append((i, i + 1))
            if r + 1 < rows:
                edges.append((i, i + cols))
                if kings and c + 1 < cols:
                    edges.append((i, i + cols + 1))
                if kings and c >= 1:
                    edges.append((i, i + cols - 1))
    kind = "kings" if kings else "square"
    return _finish(n, edges, list(range(n)), rows, cols, rng, f"{kind}{rows}x{cols}_s{seed}", fields, couplings)


def kings_grid(rows: int, cols: int, seed: int, fields: bool = True, couplings: str = "pm7") -> Instance:
    return square_grid(rows, cols, seed, fields, kings=True, couplings=couplings)


# --- Pegasus ---------------------------------------------------------------
# Segment offsets of the standard Pegasus lattice: vertical qubit k starts at
# y = 12 z + VOFF[k], horizontal qubit k at x = 12 z + HOFF[k].
_VOFF = (2, 2, 2, 2, 10, 10, 10, 10, 6, 6, 6, 6)
_HOFF = (6, 6, 6, 6, 2, 2, 2, 2, 10, 10, 10, 10)


def pegasus_graph(m: int) -> Tuple[List[tuple], List[tuple]]:
    """Qubits (u, w, k, z) and couplers of P_m from the segment geometry."""
    qubits = [(u, w, k, z) for u in (0, 1) for w in range(m) for k in range(12) for z in range(m - 1)]
    qset = set(qubits)
    edges = set()
    # internal couplers: vertical (x = 12w+k, y in [12z+VOFF, +12)) crosses
    # horizontal (y = 12w'+k', x in [12z'+HOFF, +12))
    horiz_at_y = {}
    for (u, w, k, z) in qubits:
        if u == 1:
            horiz_at_y.setdefault(12 * w + k, []).append((u, w, k, z))
    for (u, w, k, z) in qubits:
        if u != 0:
            continue
        x = 12 * w + k
        y0 = 12 * z + _VOFF[k]
        for y in range(y0, y0 + 12):
            for h in horiz_at_y.get(y, ()):
                x0 = 12 * h[3] + _HOFF[h[2]]
                if x0 <= x < x0 + 12:
                    edges.add(((u, w, k, z), h))
    for q in qubits:
        u, w, k, z = q
        nxt = (u, w, k, z + 1)
        if nxt in qset:
            edges.add((q, nxt))
        if k % 2 == 0:
            edges.add((q, (u, w, k + 1, z)))
    return qubits, sorted(edges)


def pegasus_nice_cell(q: tuple, m: int):
    """Nice cell (y, x) and tile t of qubit q, or None outside the (m-1)^2 nice cells.

    The three K44 tiles of P_m pair vertical group g with one horizontal group:
    g=0 (w, z) with horizontal group 2 at (w'=z, z'=w-1); g=1 with group 1 at
    (w'=z+1, z'=w); g=2 with group 0 at (w'=z+1, z'=w).  A nice cell (y, x)
    collects tile t=0 at w = x+1 and tiles t=1,2 at w = x, all with z = y.
    """
    u, w, k, z = q
    g = k // 4
    if u == 0:
        t = g
        y, x = (z, w - 1) if g == 0 else (z, w)
    else:
        t = {2: 0, 1: 1, 0: 2}[g]
        y, x = (w, z) if g == 2 else (w - 1, z)
    if 0 <= y < m - 1 and 0 <= x < m - 1:
        return (y, x), t
    return None


def pegasus_nice(m: int, seed: int, fields: bool = True) -> Instance:
    """Pegasus P_m restricted to its nice cells, clustered into an (m-1) x (m-1) grid of 24-spin cells.

    Spin order inside a cell: vertical qubits (u=0) of tiles t=0,1,2 then
    horizontal ones, 4 per tile in k order -- local index 12 u + 4 t + (k mod 4).
    """
    qubits, edges = pegasus_graph(m)
    R = C = m - 1
    gid = {}
    for q in qubits:
        nc = pegasus_nice_cell(q, m)
        if nc is None:
            continue
        (y, x), t = nc
        gid[q] = 24 * (y * C + x) + 12 * q[0] + 4 * t + (q[2] % 4)
    n = 24 * R * C
    site = [i // 24 for i in range(n)]
    e2 = [(gid[a], gid[b]) for a, b in edges if a in gid and b in gid]
    rng = SplitMix64(seed)
    return _finish(n, e2, site, R, C, rng, f"pegasusP{m}_s{seed}", fields)


def planted(inst: Instance, seed: int, loops_per_cell: int = 6, field_max: int = 7) -> Instance:
    """Planted variant: sum of frustrated 4-cycles, each consistent with a seeded state s*.

    Each loop gets a weight w in {1..7}/7; three of its edges get J = -w and one
    J = +w, then the whole loop is gauge-transformed by s* (J_ij <- J_ij s*_i s*_j).
    s* satisfies three edges and frustrates one, which is the best any state can
    do on a frustrated cycle, so each loop contributes exactly -2w at s*.  Fields
    h_i = -k_i s*_i with k_i in {0..field_max} are satisfied by s*.  Hence
    E(s*) = sum_loops(-2w) - sum_i k_i is the ground-state energy (numerator).
    Cycles are drawn from 4-cycles of the instance's own graph inside a cell or
    between a cell and its right / lower neighbour.
    """
    rng = SplitMix64(seed)
    n = inst.n_spins
    s_star = np.array([1 if rng.below(2) == 0 else -1 for _ in range(n)], dtype=np.int64)
    adj = [set() for _ in range(n)]
    for a, b in zip(inst.ei.tolist(), inst.ej.tolist()):
        adj[a].add(b)
        adj[b].add(a)
    C = inst.cols
    cells = {}
    for i, s in enumerate(inst.site_of_spin.tolist()):
        cells.setdefault(s, []).append(i)
    J = {}
    bound = 0
    for s in sorted(cells):
        r, c = divmod(s, C)
        pool = list(cells[s])
        for nb in ((r, c + 1), (r + 1, c)):
            if nb[0] < inst.rows and nb[1] < C:
                pool += cells.get(nb[0] * C + nb[1], [])
        pool_set = set(pool)
        for _ in range(loops_per_cell):
            cyc = None
            for _try in range(64):
                a = cells[s][rng.below(len(cells[s]))]
                nb_a = sorted(adj[a] & pool_set)
                if len(nb_a) < 2:
                    continue
                b = nb_a[rng.below(len(nb_a))]
                d = nb_a[rng.below(len(nb_a))]
                if b == d:
                    continue
                common = sorted((adj[b] & adj[d] & pool_set) - {a})
                if not common:
                    continue
                cc = common[rng.below(len(common))]
                cyc = [a, b, cc, d]
                break
            if cyc is None:
                continue
            w = 1 + rng.below(7)
            bad = rng.below(4)
            bound += -2 * w
            for e in range(4):
                i, j = cyc[e], cyc[(e + 1) % 4]
                val = (w if e == bad else -w) * int(s_star[i] * s_star[j])
                key = (min(i, j), max(i, j))
                J[key] = J.get(key, 0) + val
    ei = inst.ei.copy()
    ej = inst.ej.copy()
    jn = np.array([J.get((int(a), int(b)), 0) for a, b in zip(ei, ej)], dtype=np.int32)
    k = np.array([rng.below(field_max + 1) for _ in range(n)], dtype=np.int64)
    hn = (-k * s_star).astype(np.int32)
    out = Instance(n, ei, ej, jn, hn, 7, inst.site_of_spin.copy(), inst.rows, inst.cols,
                   inst.name + f"_planted{seed}")
    out.planted = s_star.astype(np.int8)
    out.planted_energy_num = out.energy_num(s_star)
    out.meta["loop_bound_num"] = bound - int(k.sum())
    return out


def slice_cells(inst: Instance, rows: int, cols: int) -> Instance:
    """The sub-instance on the top-left rows x cols clusters (spins renumbered)."""
    keep = [i for i in range(inst.n_spins)
            if (inst.site_of_spin[i] // inst.cols) < rows and (inst.site_of_spin[i] % inst.cols) < cols]
    new = {old: k for k, old in enumerate(keep)}
    sel = [(new[a], new[b], j) for a, b, j in zip(inst.ei.tolist(), inst.ej.tolist(), inst.j_num.tolist())
           if a in new and b in new]
    sel.sort()
    site = [(inst.site_of_spin[i] // inst.cols) * cols + (inst.site_of_spin[i] % inst.cols) for i in keep]
    return Instance(len(keep), np.array([a for a, _, _ in sel], dtype=np.int32),
                    np.array([b for _, b, _ in sel], dtype=np.int32),
                    np.array([j for _, _, j in sel], dtype=np.int32),
                    inst.h_num[keep].copy(), inst.denom, np.array(site, dtype=np.int32), rows, cols,
                    inst.name + f"_slice{rows}x{cols}")


# The eight symmetries of the rectangular grid of clusters (the paper runs
# every instance in all of its contraction orientations, Sec. V): cluster
# (r, c) of an R x C grid goes to the returned cell of the transformed grid.
TRANSFORMS = ("identity", "rot90", "rot180", "rot270", "flip_lr", "flip_ud", "transpose", "antitranspose")


def transformed_cell(k: int, r: int, c: int, rows: int, cols: int) -> Tuple[int, int, int, int]:
    """(r', c', rows', cols') of cluster (r, c) under grid symmetry k (see TRANSFORMS)."""
    R, C = rows, cols
    return [(r, c, R, C), (c, R - 1 - r, C, R), (R - 1 - r, C - 1 - c, R, C), (C - 1 - c, r, C, R),
            (r, C - 1 - c, R, C), (R - 1 - r, c, R, C), (c, r, C, R), (C - 1 - c, R - 1 - r, C, R)][k]


def transform(inst: Instance, k: int) -> Instance:
    """The same spins, couplings and fields with the cluster grid mapped by symmetry k.

    Only the placement of the clusters changes (spins keep their indices and
    their order inside a cluster), so H, Z and the ground states are the same;
    the boundary-MPS contraction and the exploration order run along
    different directions of the lattice.
    """
    site = np.empty_like(inst.site_of_spin)
    rows2 = cols2 = 0
    for i, s in enumerate(inst.site_of_spin.tolist()):
        r2, c2, rows2, cols2 = transformed_cell(k, s // inst.cols, s % inst.cols, inst.rows, inst.cols)
        site[i] = r2 * cols2 + c2
    out = Instance(inst.n_spins, inst.ei.copy(), inst.ej.copy(), inst.j_num.copy(), inst.h_num.copy(), inst.denom,
                   site, rows2, cols2, inst.name + ("" if k == 0 else "_" + TRANSFORMS[k]), inst.planted,
                   inst.planted_energy_num, dict(inst.meta))
    return out


def transform_states(inst: Instance, states_per_site, k: int):
    """Per-cluster state lists of ``inst`` reordered for ``transform(inst, k)``."""
    out = [None] * (inst.rows * inst.cols)
    for s, lst in enumerate(states_per_site):
        r2, c2, _, cols2 = transformed_cell(k, s // inst.cols, s % inst.cols, inst.rows, inst.cols)
        out[r2 * cols2 + c2] = lst
    return out


def hamming_ball_states(inst: Instance, d: int, seed: int = 0, reference: Optional[np.ndarray] = None):
    """Per-cluster state lists of (at most) d states nearest to a reference configuration.

    For cells too large to enumerate (24-spin Pegasus cells) the Potts model
    runs on a reduced state set.  This draws one synthetic such set: the d
    patterns closest in Hamming distance to the reference (the planted state
    if any, else a seeded random configuration), ordered by (distance,
    pattern).  Bit j of a pattern is 1 when the j-th spin of the cluster (in
    increasing global index) is -1.
    """
    import itertools
    if reference is None:
        if inst.planted is not None:
            reference = inst.planted
        else:
            rng = SplitMix64(seed)
            reference = np.array([1 if rng.below(2) == 0 else -1 for _ in range(inst.n_spins)], dtype=np.int8)
    spins_of = [[] for _ in range(inst.rows * inst.cols)]
    for i, s in enumerate(inst.site_of_spin.tolist()):
        spins_of[s].append(i)
    out = []
    for sp in spins_of:
        k = len(sp)
        ref = sum(1 << j for j, g in enumerate(sp) if reference[g] < 0)
        states = []
        for dist in range(k + 1):
            level = sorted(ref ^ sum(1 << b for b in flip) for flip in itertools.combinations(range(k), dist))
            states.extend(level)
            if len(states) >= d:
                break
        out.append(np.array(states[:d], dtype=np.int64))
    return out
