"""Seeded synthetic structures and model inputs.

This module makes inputs only: atomic structures (positions, species, cells),
random draws (coefficients alpha, species-mixing weights, sparse-point
indices) and the hyperparameter sets of the five workloads.  It holds none of
the GAP arithmetic (no descriptor, kernel or derivative), so both the FP64
oracle under ``oracle/`` and the CUDA path read the same inputs from here.

Random numbers come from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with the seed
``0x231003921 ^ (workload << 40) ^ (cell << 20) ^ stream``; normal deviates use
the Box-Muller transform.  The datasets of the paper (Si GAP-18, HEA, SiC,
QM9-GW) are not available; these generators stand in for them with
structures of the same shape: near-crystalline diamond Si cells (Sec. 4.1
uses a silicon database) and random multi-species packings at fixed density.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 0x231003921
STREAMS = {
    "displacement": 1, "strain": 2, "alpha": 3, "sparse": 4, "species": 5,
    "packing": 6, "mix": 7, "count": 8, "sigma": 9, "dims": 10, "teacher": 11,
    "alpha2": 12,
}
_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def seed_for(workload: int, cell: int, stream: str) -> int:
    return (SEED_BASE ^ (workload << 40) ^ (cell << 20) ^ STREAMS[stream]) & _MASK


class SplitMix64:
    """Counter-based splitmix64: output k is mix(seed + k * golden)."""

    def __init__(self, seed: int):
        self.seed = seed & _MASK
        self.count = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.count + 1, self.count + n + 1, dtype=np.uint64)
        self.count += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + k * np.uint64(_GOLDEN)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, std: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([rad * np.cos(2 * np.pi * u2), rad * np.sin(2 * np.pi * u2)])
        return std * z[:n]

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi]."""
        span = hi - lo + 1
        return lo + (self.u64(n) % np.uint64(span)).astype(np.int64)

    def choice(self, n_pool: int, k: int) -> np.ndarray:
        """k distinct indices from range(n_pool) (partial Fisher-Yates)."""
        idx = np.arange(n_pool, dtype=np.int64)
        r = self.u64(k)
        for t in range(k):
            s = t + int(r[t] % np.uint64(n_pool - t))
            idx[t], idx[s] = idx[s], idx[t]
        return idx[:k].copy()


@dataclasses.dataclass
class Structure:
    pos: np.ndarray       # [N][3] f64, Angstrom
    species: np.ndarray   # [N] i32, species index 0..S-1
    cell: np.ndarray      # [3][3] f64, rows are lattice vectors
    pbc: np.ndarray       # [3] i32

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclasses.dataclass
class Batch:
    pos: np.ndarray             # [N][3]
    species: np.ndarray         # [N]
    cell: np.ndarray            # [C][3][3]
    pbc: np.ndarray             # [C][3]
    config_offsets: np.ndarray  # [C+1] i32

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_configs(self) -> int:
        return int(self.cell.shape[0])

    def structure(self, c: int) -> Structure:
        a, b = int(self.config_offsets[c]), int(self.config_offsets[c + 1])
        return Structure(self.pos[a:b].copy(), self.species[a:b].copy(),
                         self.cell[c].copy(), self.pbc[c].copy())


def make_batch(structs: list[Structure]) -> Batch:
    offs = np.zeros(len(structs) + 1, dtype=np.int32)
    offs[1:] = np.cumsum([s.n for s in structs])
    return Batch(
        pos=np.ascontiguousarray(np.concatenate([s.pos for s in structs]), dtype=np.float64),
        species=np.ascontiguousarray(np.concatenate([s.species for s in structs]), dtype=np.int32),
        cell=np.ascontiguousarray(np.stack([s.cell for s in structs]), dtype=np.float64),
        pbc=np.ascontiguousarray(np.stack([s.pbc for s in structs]), dtype=np.int32),
        config_offsets=offs,
    )


# ---------------------------------------------------------------- lattices

_DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


def diamond(reps=(2, 2, 2), a: float = 5.431) -> Structure:
    """Conventional 8-atom diamond-cubic cell repeated reps times, periodic."""
    nx, ny, nz = reps
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 1, 3)
    frac = ((g + _DIAMOND_BASIS[None]) / np.array(reps, dtype=np.float64)).reshape(-1, 3)
    cell = np.diag(np.array(reps, dtype=np.float64) * a)
    return Structure(frac @ cell, np.zeros(frac.shape[0], np.int32), cell, np.ones(3, np.int32))


def displaced_diamond(workload: int, cell_id: int, reps=(2, 2, 2), sigma: float = 0.1,
                      strain: float = 0.0, a: float = 5.431) -> Structure:
    """Diamond supercell with iid N(0, sigma^2) displacements per component and,
    if strain > 0, a symmetric lattice strain with components uniform in [-strain, strain]."""
    s = diamond(reps, a)
    frac = s.pos @ np.linalg.inv(s.cell)
    cell = s.cell
    if strain > 0.0:
        e = SplitMix64(seed_for(workload, cell_id, "strain")).uniform(6, -strain, strain)
        eps = np.array([[e[0], e[3], e[4]], [e[3], e[1], e[5]], [e[4], e[5], e[2]]])
        cell = cell @ (np.eye(3) + eps)
    pos = frac @ cell + SplitMix64(seed_for(workload, cell_id, "displacement")).normal(3 * s.n, sigma).reshape(-1, 3)
    return Structure(pos, s.species, cell, s.pbc)


def random_packing(workload: int, cell_id: int, n: int, density: float, d_min: float,
                   n_species: int = 1, batch: int = 384) -> Structure:
    """Random sequential addition of n points in a periodic cubic box of volume
    n / density, rejecting any point closer than d_min (minimum image) to an
    accepted one.  Species are drawn uniformly from 0..n_species-1."""
    L = (n / density) ** (1.0 / 3.0)
    rng = SplitMix64(seed_for(workload, cell_id, "packing"))
    nc = max(1, int(math.floor(L / d_min)))
    use_grid = nc >= 3
    cap = 8
    grid = np.full((nc, nc, nc, cap), -1, dtype=np.int64)
    gcount = np.zeros((nc, nc, nc), dtype=np.int64)
    pos = np.zeros((n, 3))
    got = 0
    d2min = d_min * d_min
    offs = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)])
    tries = 0
    while got < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("random packing did not converge")
        b = min(batch, max(16, 2 * (n - got)))
        cand = rng.uniform(3 * b, 0.0, L).reshape(b, 3)
        ok = np.ones(b, dtype=bool)
        if got:
            if use_grid:
                ci = np.minimum((cand / L * nc).astype(np.int64), nc - 1)
                nb = (ci[:, None, :] + offs[None]) % nc                     # [b][27][3]
                ids = grid[nb[..., 0], nb[..., 1], nb[..., 2]].reshape(b, -1)   # [b][27*cap]
                row, col = np.nonzero(ids >= 0)
                dv = pos[ids[row, col]] - cand[row]
                dv -= L * np.round(dv / L)
                close = np.einsum("kx,kx->k", dv, dv) < d2min
                ok[row[close]] = False
            else:
                dv = pos[None, :got, :] - cand[:, None, :]
                dv -= L * np.round(dv / L)
                ok &= ~((np.einsum("bkx,bkx->bk", dv, dv) < d2min).any(axis=1))
        dv = cand[None, :, :] - cand[:, None, :]
        dv -= L * np.round(dv / L)
        ea, eb = np.nonzero(np.triu(np.einsum("abx,abx->ab", dv, dv) < d2min, 1))
        # greedy in proposal order: a candidate conflicting with an earlier
        # accepted one of the same batch is rejected (pairs sorted by the later index)
        for t in np.argsort(eb, kind="stable"):
            if ok[ea[t]] and ok[eb[t]]:
                ok[eb[t]] = False
        take = np.nonzero(ok)[0][: n - got]
        for k in take:
            pos[got] = cand[k]
            if use_grid:
                c = np.minimum((cand[k] / L * nc).astype(np.int64), nc - 1)
                slot = gcount[c[0], c[1], c[2]]
                if slot >= cap:
                    raise RuntimeError("packing grid capacity exceeded")
                grid[c[0], c[1], c[2], slot] = got
                gcount[c[0], c[1], c[2]] += 1
            got += 1
    species = SplitMix64(seed_for(workload, cell_id, "species")).integers(n, 0, n_species - 1).astype(np.int32)
    return Structure(pos, species, np.eye(3) * L, np.ones(3, np.int32))


# ------------------------------------------------------------- model draws

def alpha_draw(workload: int, species: int, m: int, std: float = 0.1) -> np.ndarray:
    """Sparse-GP coefficients alpha ~ N(0, 0.01), read as variance 0.01."""
    return SplitMix64(seed_for(workload, species, "alpha")).normal(m, std)


def mixing_weights(workload: int, K: int, n_species: int) -> np.ndarray:
    """Element-embedding weights w^k_alpha ~ N(0, 1) (Sec. 3.3.3: normally
    distributed random weights, not optimised).  Shape [K][n_species]."""
    return SplitMix64(seed_for(workload, 0, "mix")).normal(K * n_species).reshape(K, n_species)


def sparse_indices(workload: int, species: int, n_pool: int, m: int) -> np.ndarray:
    """'random' sparse-point selection: m distinct candidate indices."""
    return SplitMix64(seed_for(workload, species, "sparse")).choice(n_pool, m)


# ----------------------------------------------------------- the workloads

@dataclasses.dataclass
class SoapSpec:
    n_max: int
    l_max: int
    rc: float
    sigma: float
    d: float = 1.0
    central_weight: float = 1.0
    n_species: int = 1
    mix_K: int = 0
    mix_w: np.ndarray | None = None


@dataclasses.dataclass
class TwoBodySpec:
    rc: float
    d: float
    theta: float
    delta: float
    x: np.ndarray       # [M2] sparse distances
    alpha: np.ndarray   # [M2]


@dataclasses.dataclass
class Workload:
    name: str
    index: int
    soap: SoapSpec
    M: int               # sparse points per central species
    zeta: int
    delta: float
    two_body: TwoBodySpec | None = None


def two_body_spec(workload: int, rc: float, m: int = 50) -> TwoBodySpec:
    """distance_2b with the SE kernel: theta = 1.0 A and delta = 10 eV as in
    the HEA example (Sec. 4.3); sparse distances by the 'uniform' method, one
    per bin centre on [1.4, rc]; alpha_2 ~ N(0, 0.01)."""
    lo, hi = 1.4, rc
    x = lo + (hi - lo) * (np.arange(m) + 0.5) / m
    a2 = SplitMix64(seed_for(workload, 0, "alpha2")).normal(m, 0.1)
    return TwoBodySpec(rc=rc, d=1.0, theta=1.0, delta=10.0, x=x, alpha=a2)


def workload(index: int) -> Workload:
    """Hyperparameters of the five workloads (single source for tests and bench)."""
    if index == 0:
        return Workload("diamond-Si-64 predict", 0, SoapSpec(6, 4, 5.0, 0.5), M=100, zeta=4, delta=1.0)
    if index == 1:
        return Workload("diamond-Si K_NM 200 cells", 1, SoapSpec(8, 6, 5.0, 0.5), M=2000, zeta=4, delta=1.0)
    if index == 2:
        return Workload("diamond-Si-32768 MD predict", 2, SoapSpec(8, 8, 5.0, 0.5), M=4000, zeta=4, delta=1.0)
    if index == 3:
        sp = SoapSpec(8, 6, 5.0, 0.5, n_species=4, mix_K=4, mix_w=mixing_weights(3, 4, 4))
        return Workload("4-species packing 512 configs", 3, sp, M=3000, zeta=4, delta=1.0)
    if index == 4:
        return Workload("amorphous-110592 predict", 4, SoapSpec(10, 8, 4.5, 0.5), M=9000, zeta=4, delta=1.0,
                        two_body=two_body_spec(4, 4.5))
    raise ValueError(index)


def structures(index: int, n_cells: int | None = None) -> list[Structure]:
    """The structures of a workload (n_cells truncates multi-cell workloads)."""
    if index == 0:
        return [displaced_diamond(0, 0, (2, 2, 2), 0.1)]
    if index == 1:
        n = 200 if n_cells is None else n_cells
        out = []
        for c in range(n):
            dims = tuple(int(v) for v in SplitMix64(seed_for(1, c, "dims")).integers(3, 2, 3))
            sig = float(SplitMix64(seed_for(1, c, "sigma")).uniform(1, 0.05, 0.2)[0])
            out.append(displaced_diamond(1, c, dims, sig, strain=0.03))
        return out
    if index == 2:
        return [displaced_diamond(2, 0, (16, 16, 16), 0.1)]
    if index == 3:
        n = 512 if n_cells is None else n_cells
        out = []
        for c in range(n):
            na = int(SplitMix64(seed_for(3, c, "count")).integers(1, 8, 256)[0])
            out.append(random_packing(3, c, na, 0.05, 1.8, n_species=4))
        return out
    if index == 4:
        return [random_packing(4, 0, 110592, 0.1, 1.4)]
    raise ValueError(index)


def sparse_candidate_structures(index: int) -> list[Structure]:
    """Seeded cells (distinct from the workload's own cells) whose descriptors
    form the candidate pool for 'random' sparse-point selection; the pool
    holds at least M candidates per central species."""
    base = 1000
    if index == 0:
        return [displaced_diamond(0, base + c, (2, 2, 2), 0.1) for c in range(5)]
    if index == 1:
        return [displaced_diamond(1, base + c, (3, 3, 3), 0.05 + 0.03 * (c % 5), strain=0.03)
                for c in range(12)]
    if index == 2:
        return [displaced_diamond(2, base + c, (3, 3, 3), 0.1) for c in range(20)]
    if index == 3:
        return [random_packing(3, base + c, 256, 0.05, 1.8, n_species=4) for c in range(64)]
    if index == 4:
        return [random_packing(4, base + c, 2048, 0.1, 1.4) for c in range(5)]
    raise ValueError(index)
