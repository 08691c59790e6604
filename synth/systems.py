"""Synthetic gapped model Hamiltonians shaped like the molecules and solids of
the paper's performance study (Sec. 3.3: H(C2H4)nH chains, clusters, slabs).

The paper's systems (FHI-aims geometries, NAO basis sets, DFPT first-order
Hamiltonians) are not available, so seeded stand-ins are drawn here:

* every model atom carries ``opa`` orthogonal orbitals, the first half
  occupied (onsite energies U(-1.0, -0.5) Ha), the second half virtual
  (onsite U(0.2, 0.8) Ha); intra-atom off-diagonal H0 elements are zero;
* atoms closer than ``cutoff`` bohr are coupled by a hopping block whose
  elements are iid N(0,1) * 0.05 * exp(-r / 1.5 bohr); H0[J,I] = H0[I,J]^T;
* the perturbation H1 for direction gamma (the dipole matrix D_gamma, i.e.
  dH/dlambda for H0 + lambda * D_gamma) is block-diagonal over atoms:
  r_gamma(I) * Identity + S, with S symmetric and its upper triangle
  (diagonal included) iid N(0, 0.1^2);
* coordinates are centred at the atom centroid; clusters and slabs are
  ordered along a Morton (Z-order) curve so that consecutive atoms, and
  therefore the b x b blocks that group them, are spatially compact.

Random draw order (numpy ``default_rng(seed)``), fixed so that a system is
reproducible bit for bit on any machine:
  1. positions (random sequential addition for clusters and slabs; chains
     draw nothing), then the Morton reordering;
  2. occupied onsite energies, shape (n_atoms, opa/2);
  3. virtual onsite energies, shape (n_atoms, opa/2);
  4. one standard normal (opa, opa) block per coupled pair (I < J), pairs in
     lexicographic order;
  5. for gamma = x, y, z in turn: one standard normal (opa, opa) block per
     atom, whose upper triangle defines S.
All three directions are always drawn so that H1_x does not depend on which
directions a caller asks for.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np
from scipy.spatial import cKDTree

WATER_DENSITY = 0.0148      # atoms / bohr^3  (~0.100 atoms / Angstrom^3)
MIN_DIST = 2.5              # bohr, random sequential addition exclusion radius
HOP_SCALE = 0.05            # Ha
HOP_DECAY = 1.5             # bohr
SIGMA_H1 = 0.1              # intra-atom dipole block noise
DIRS = ("x", "y", "z")


@dataclass
class Bsr:
    """Square block-sparse row matrix with b x b blocks.

    ``row_ptr`` (int32, nb+1), ``col_idx`` (int32, nnzb, strictly increasing
    within a row), ``vals`` (float64, (nnzb, b, b), each block row-major).
    ``n`` is the number of meaningful rows/cols; rows n..nb*b-1 are padding
    whose elements are all zero.
    """

    nb: int
    b: int
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    vals: np.ndarray

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def row_of_block(self) -> np.ndarray:
        return np.repeat(np.arange(self.nb, dtype=np.int64), np.diff(self.row_ptr))

    def to_dense(self, padded: bool = False) -> np.ndarray:
        b = self.b
        a = np.zeros((self.nb, b, self.nb, b), dtype=np.float64)
        a[self.row_of_block(), :, self.col_idx.astype(np.int64), :] = self.vals
        a = a.reshape(self.nb * b, self.nb * b)
        return a if padded else a[: self.n, : self.n]

    def submatrix_dense(self, idx: np.ndarray) -> np.ndarray:
        """Dense A[idx][:, idx] for sorted row/column indices, read from the
        blocks that intersect them (the full matrix is never formed)."""
        b = self.b
        idx = np.asarray(idx, dtype=np.int64)
        loc = np.full(self.nb * b, -1, dtype=np.int64)
        loc[idx] = np.arange(idx.size)
        blk_has = np.zeros(self.nb, dtype=bool)
        blk_has[idx // b] = True
        rows = self.row_of_block()
        sel = np.nonzero(blk_has[rows] & blk_has[self.col_idx])[0]
        out = np.zeros((idx.size, idx.size), dtype=np.float64)
        for k in sel:
            lr = loc[rows[k] * b + np.arange(b)]
            lc = loc[int(self.col_idx[k]) * b + np.arange(b)]
            mr, mc = lr >= 0, lc >= 0
            out[np.ix_(lr[mr], lc[mc])] = self.vals[k][np.ix_(mr, mc)]
        return out

    @staticmethod
    def from_dense(a: np.ndarray, b: int, drop_zero_blocks: bool = True,
                   keep_diagonal: bool = True) -> "Bsr":
        n = a.shape[0]
        nb = -(-n // b)
        ap = np.zeros((nb * b, nb * b), dtype=np.float64)
        ap[:n, :n] = a
        blocks = ap.reshape(nb, b, nb, b).transpose(0, 2, 1, 3)
        nz = np.abs(blocks).max(axis=(2, 3)) > 0 if drop_zero_blocks else np.ones((nb, nb), bool)
        if keep_diagonal:
            nz[np.arange(nb), np.arange(nb)] = True
        ii, jj = np.nonzero(nz)
        row_ptr = np.zeros(nb + 1, dtype=np.int32)
        np.add.at(row_ptr, ii + 1, 1)
        row_ptr = np.cumsum(row_ptr).astype(np.int32)
        vals = np.ascontiguousarray(blocks[ii, jj])
        return Bsr(nb, b, n, row_ptr, jj.astype(np.int32), vals)


@dataclass
class System:
    """One synthetic system: geometry, H0 and the dipole perturbations."""

    name: str
    kind: str
    coords: np.ndarray           # (n_atoms, 3) bohr, centroid at 0, Morton order
    opa: int                     # orbitals per atom
    n_occ: int                   # occupied orbitals (= electrons / 2)
    b: int
    h0: Bsr
    h1: List[Bsr]                # one per entry of ``dirs``
    dirs: Sequence[str]
    cutoff: float
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n(self) -> int:
        return self.n_atoms * self.opa

    @property
    def n_electrons(self) -> int:
        return 2 * self.n_occ


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def _part1by2(v: np.ndarray) -> np.ndarray:
    """Spread the low 21 bits of v so that bit k lands at bit 3k."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_order(pos: np.ndarray) -> np.ndarray:
    """Permutation that sorts points along a 3-D Z-order curve (21 bits/axis)."""
    lo = pos.min(axis=0)
    span = max(float((pos.max(axis=0) - lo).max()), 1e-12)
    q = np.floor((pos - lo) / span * ((1 << 21) - 1)).astype(np.int64)
    code = _part1by2(q[:, 0]) | (_part1by2(q[:, 1]) << np.uint64(1)) | (_part1by2(q[:, 2]) << np.uint64(2))
    return np.argsort(code, kind="stable")


def _rsa(rng: np.random.Generator, n: int, box: np.ndarray, dmin: float) -> np.ndarray:
    """Random sequential addition of n points in an axis-aligned box with a
    minimum pair distance ``dmin``.  Candidates are drawn in batches; a
    candidate is accepted if it is farther than dmin from every accepted point
    and from every earlier candidate accepted in its batch."""
    acc = np.zeros((0, 3))
    tries = 0
    while acc.shape[0] < n:
        tries += 1
        if tries > 10000:
            raise RuntimeError("random sequential addition did not reach the requested count")
        m = max(256, int(1.3 * (n - acc.shape[0])))
        cand = rng.uniform(0.0, 1.0, size=(m, 3)) * box
        if acc.shape[0]:
            d, _ = cKDTree(acc).query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[d >= dmin]
        if cand.shape[0] == 0:
            continue
        # resolve conflicts inside the batch: keep the earlier candidate
        pairs = cKDTree(cand).query_pairs(dmin, output_type="ndarray")
        drop = np.zeros(cand.shape[0], dtype=bool)
        if pairs.size:
            pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
            for a, c in pairs:
                if not drop[a]:
                    drop[c] = True
        cand = cand[~drop]
        need = n - acc.shape[0]
        acc = np.vstack([acc, cand[:need]])
    return acc


# --------------------------------------------------------------------------
# Hamiltonian assembly
# --------------------------------------------------------------------------

def _assemble(coords: np.ndarray, opa: int, b: int, cutoff: float,
              rng: np.random.Generator, dirs: Sequence[str]):
    n_atoms = coords.shape[0]
    n = n_atoms * opa
    nocc_a = opa // 2
    eps_occ = rng.uniform(-1.0, -0.5, size=(n_atoms, nocc_a))
    eps_vir = rng.uniform(0.2, 0.8, size=(n_atoms, opa - nocc_a))

    pairs = cKDTree(coords).query_pairs(cutoff, output_type="ndarray")
    if pairs.size == 0:
        pairs = np.zeros((0, 2), dtype=np.int64)
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))].astype(np.int64)
    r = np.linalg.norm(coords[pairs[:, 0]] - coords[pairs[:, 1]], axis=1)
    hop = rng.standard_normal((pairs.shape[0], opa, opa))
    hop *= (HOP_SCALE * np.exp(-r / HOP_DECAY))[:, None, None]

    s_blocks = {}
    for d in DIRS:
        g = rng.standard_normal((n_atoms, opa, opa)) * SIGMA_H1
        up = np.triu(g)
        s_blocks[d] = up + np.transpose(np.triu(g, 1), (0, 2, 1))

    diag0 = np.zeros((n_atoms, opa, opa))
    idx = np.arange(nocc_a)
    diag0[:, idx, idx] = eps_occ
    idx_v = np.arange(nocc_a, opa)
    diag0[:, idx_v, idx_v] = eps_vir

    # atom-level block list: diagonal, (I,J) and (J,I)
    ai = np.concatenate([np.arange(n_atoms), pairs[:, 0], pairs[:, 1]])
    aj = np.concatenate([np.arange(n_atoms), pairs[:, 1], pairs[:, 0]])
    ablk = np.concatenate([diag0, hop, np.transpose(hop, (0, 2, 1))])
    h0 = _atom_blocks_to_bsr(ai, aj, ablk, n_atoms, opa, b)

    h1 = []
    for d in dirs:
        k = DIRS.index(d)
        blk = s_blocks[d].copy()
        ii = np.arange(opa)
        blk[:, ii, ii] += coords[:, k][:, None]
        h1.append(_atom_blocks_to_bsr(np.arange(n_atoms), np.arange(n_atoms), blk, n_atoms, opa, b))
    return h0, h1, pairs.shape[0]


def _atom_blocks_to_bsr(ai, aj, ablk, n_atoms, opa, b) -> Bsr:
    n = n_atoms * opa
    nb = -(-n // b)
    if b % opa == 0:
        g = b // opa
        bi = ai // g
        bj = aj // g
        key = bi.astype(np.int64) * nb + bj
        ukey, inv = np.unique(key, return_inverse=True)
        rows = (ukey // nb).astype(np.int64)
        cols = (ukey % nb).astype(np.int32)
        # every diagonal block must exist (padding rows included)
        diag_missing = np.setdiff1d(np.arange(nb, dtype=np.int64) * nb + np.arange(nb), ukey)
        if diag_missing.size:
            ukey2 = np.union1d(ukey, diag_missing)
            pos = np.searchsorted(ukey2, ukey)
            inv = pos[inv]
            ukey = ukey2
            rows = (ukey // nb).astype(np.int64)
            cols = (ukey % nb).astype(np.int32)
        vals = np.zeros((ukey.shape[0], b, b))
        oi = (ai % g) * opa
        oj = (aj % g) * opa
        r_idx = oi[:, None, None] + np.arange(opa)[None, :, None]
        c_idx = oj[:, None, None] + np.arange(opa)[None, None, :]
        vals[inv[:, None, None], r_idx, c_idx] = ablk
        row_ptr = np.zeros(nb + 1, dtype=np.int64)
        np.add.at(row_ptr, rows + 1, 1)
        row_ptr = np.cumsum(row_ptr).astype(np.int32)
        return Bsr(nb, b, n, row_ptr, cols, vals)
    # general block sizes (b not a multiple of the atom block): go through dense
    dense = np.zeros((n, n))
    for t in range(ai.shape[0]):
        I, J = ai[t], aj[t]
        dense[I * opa:(I + 1) * opa, J * opa:(J + 1) * opa] = ablk[t]
    return Bsr.from_dense(dense, b)


# --------------------------------------------------------------------------
# public constructors
# --------------------------------------------------------------------------

def _finish(name, kind, coords, opa, b, cutoff, rng, seed, dirs, meta) -> System:
    coords = coords - coords.mean(axis=0)
    h0, h1, npairs = _assemble(coords, opa, b, cutoff, rng, dirs)
    meta = dict(meta)
    meta["n_hop_pairs"] = int(npairs)
    return System(name, kind, coords, opa, coords.shape[0] * opa // 2, b, h0, h1,
                  tuple(dirs), cutoff, seed, meta)


def make_chain(n_atoms: int, opa: int = 4, b: int = 4, spacing: float = 2.8,
               cutoff: float = 8.0, seed: int = 0, dirs: Sequence[str] = ("x",),
               name: str = "chain") -> System:
    """1-D chain along x with uniform spacing (no random positions)."""
    rng = np.random.default_rng(seed)
    coords = np.zeros((n_atoms, 3))
    coords[:, 0] = spacing * np.arange(n_atoms)
    return _finish(name, "chain", coords, opa, b, cutoff, rng, seed, dirs,
                   {"spacing": spacing})


def make_cluster(n_atoms: int, opa: int = 8, b: int = 32, cutoff: float = 10.0,
                 density: float = WATER_DENSITY, seed: int = 1,
                 dirs: Sequence[str] = DIRS, name: str = "cluster") -> System:
    """Random-packed cube at liquid-water atom density, Morton ordered."""
    rng = np.random.default_rng(seed)
    side = (n_atoms / density) ** (1.0 / 3.0)
    pos = _rsa(rng, n_atoms, np.array([side, side, side]), MIN_DIST)
    pos = pos[morton_order(pos)]
    return _finish(name, "cluster", pos, opa, b, cutoff, rng, seed, dirs, {"side": side})


def make_slab(n_atoms: int, thickness: float = 30.0, opa: int = 8, b: int = 32,
              cutoff: float = 10.0, density: float = WATER_DENSITY, seed: int = 4,
              dirs: Sequence[str] = DIRS, name: str = "slab") -> System:
    """Non-periodic slab of fixed thickness along z, square in x-y."""
    rng = np.random.default_rng(seed)
    side = (n_atoms / (density * thickness)) ** 0.5
    pos = _rsa(rng, n_atoms, np.array([side, side, thickness]), MIN_DIST)
    pos = pos[morton_order(pos)]
    return _finish(name, "slab", pos, opa, b, cutoff, rng, seed, dirs,
                   {"side": side, "thickness": thickness})


def carve_sphere(sys_: System, n_keep: int, b: int | None = None, name: str | None = None) -> System:
    """Sub-system of the n_keep atoms nearest the centroid, with the same
    matrix elements (a carve-out for the dense oracle).  Atoms keep their
    Morton order; coordinates keep their original origin."""
    b = sys_.b if b is None else b
    d = np.linalg.norm(sys_.coords, axis=1)
    keep = np.sort(np.argsort(d, kind="stable")[:n_keep])
    opa = sys_.opa
    orb = (keep[:, None] * opa + np.arange(opa)[None, :]).reshape(-1)
    h0 = Bsr.from_dense(sys_.h0.submatrix_dense(orb), b)
    h1 = [Bsr.from_dense(m.submatrix_dense(orb), b) for m in sys_.h1]
    return System(name or f"{sys_.name}-carve{n_keep}", sys_.kind, sys_.coords[keep], opa,
                  n_keep * opa // 2, b, h0, h1, sys_.dirs, sys_.cutoff, sys_.seed,
                  {"parent": sys_.name, "n_keep": n_keep})


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

CONFIGS = {
    1: "chain 64 atoms x 4 orbitals (N=256), b=4, H1 = D_x, tau=0, FP64, seed 0",
    2: "cluster 2,000 atoms x 8 orbitals (N=16,000), b=32, tau=1e-6, H1 = D_x, D_y, D_z, seed 1",
    3: "cluster 20,000 atoms x 8 orbitals (N=160,000), b=32, tau 1e-5 -> 1e-7, seed 2",
    4: "batch of 24 chains/clusters, 300-8,000 atoms x 8 orbitals, seed 3 (system s: 1000+s)",
    5: "slabs 30 bohr thick, 5k/20k/50k/100k atoms x 8 orbitals, tau=1e-6, seed 4",
}


def make_config(cfg: int, n_atoms: int | None = None, b: int | None = None,
                dirs: Sequence[str] | None = None) -> System:
    """Build workload ``cfg`` (1, 2, 3 or 5).  ``n_atoms`` overrides the size
    (used for scaled-down test cases and the slab sweep)."""
    if cfg == 1:
        return make_chain(n_atoms or 64, opa=4, b=b or 4, spacing=2.8, cutoff=8.0, seed=0,
                          dirs=dirs or ("x",), name="cfg1-chain")
    if cfg == 2:
        return make_cluster(n_atoms or 2000, opa=8, b=b or 32, cutoff=10.0, seed=1,
                            dirs=dirs or DIRS, name="cfg2-cluster")
    if cfg == 3:
        return make_cluster(n_atoms or 20000, opa=8, b=b or 32, cutoff=10.0, seed=2,
                            dirs=dirs or DIRS, name="cfg3-cluster")
    if cfg == 5:
        return make_slab(n_atoms or 5000, opa=8, b=b or 32, cutoff=10.0, seed=4,
                         dirs=dirs or DIRS, name=f"cfg5-slab{n_atoms or 5000}")
    raise ValueError(f"unknown workload {cfg}")


def make_batch_config(n_systems: int = 24, lo: int = 300, hi: int = 8000, b: int = 32,
                      seed: int = 3, dirs: Sequence[str] = DIRS) -> List[System]:
    """Workload 4: uneven sizes U{lo..hi} atoms, type Bernoulli(1/2) chain or
    cluster.  The size/type draws use ``seed``; system s uses seed 1000+s."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=n_systems)
    kinds = rng.integers(0, 2, size=n_systems)
    out = []
    for s in range(n_systems):
        if kinds[s] == 0:
            out.append(make_chain(int(sizes[s]), opa=8, b=b, spacing=2.8, cutoff=8.0,
                                  seed=1000 + s, dirs=dirs, name=f"batch{s}-chain"))
        else:
            out.append(make_cluster(int(sizes[s]), opa=8, b=b, cutoff=10.0, seed=1000 + s,
                                    dirs=dirs, name=f"batch{s}-cluster"))
    return out


# --------------------------------------------------------------------------
# non-orthogonal basis: an overlap matrix for a system
# --------------------------------------------------------------------------

OVL_SCALE = 0.04            # overlap between orbitals of neighbouring atoms
OVL_DECAY = 2.0             # bohr


def make_overlap(sys_: System, seed_offset: int = 7777) -> Bsr:
    """A synthetic overlap matrix S for the atoms of `sys_`, in its block layout:
    identity inside every atom, and for every pair of atoms closer than the
    system's cutoff a block of iid N(0,1) * OVL_SCALE * exp(-r / OVL_DECAY)
    (S[J,I] = S[I,J]^T).  Drawn from default_rng(seed + seed_offset), pairs in
    lexicographic order, so the system's own matrices do not change.  S is
    checked positive definite through a Gershgorin lower bound > 0.1."""
    rng = np.random.default_rng(sys_.seed + seed_offset)
    coords, opa, n_atoms = sys_.coords, sys_.opa, sys_.coords.shape[0]
    pairs = cKDTree(coords).query_pairs(sys_.cutoff, output_type="ndarray")
    if pairs.size == 0:
        pairs = np.zeros((0, 2), dtype=np.int64)
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))].astype(np.int64)
    r = np.linalg.norm(coords[pairs[:, 0]] - coords[pairs[:, 1]], axis=1)
    blk = rng.standard_normal((pairs.shape[0], opa, opa)) * (OVL_SCALE * np.exp(-r / OVL_DECAY))[:, None, None]
    eye = np.broadcast_to(np.eye(opa), (n_atoms, opa, opa)).copy()
    ai = np.concatenate([np.arange(n_atoms), pairs[:, 0], pairs[:, 1]])
    aj = np.concatenate([np.arange(n_atoms), pairs[:, 1], pairs[:, 0]])
    s = _atom_blocks_to_bsr(ai, aj, np.concatenate([eye, blk, np.transpose(blk, (0, 2, 1))]), n_atoms, opa,
                            sys_.b)
    # Gershgorin: 1 - sum of the off-diagonal magnitudes in every row
    rows = np.zeros(sys_.n)
    for t in range(pairs.shape[0]):
        I, J = pairs[t]
        a = np.abs(blk[t])
        rows[I * opa:(I + 1) * opa] += a.sum(axis=1)
        rows[J * opa:(J + 1) * opa] += a.sum(axis=0)
    if rows.size and 1.0 - rows.max() <= 0.1:
        raise ValueError("synthetic overlap not safely positive definite")
    return s
