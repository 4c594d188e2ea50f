"""Seeded synthetic protein-like atom sets (the workloads' inputs).

The paper's inputs (PDB structures processed to centres and van der Waals
radii, §4) are not available, so every workload is generated here.  This
module holds only the input recipe -- no surface arithmetic -- and serves both
the CUDA path and the CPU oracle.

Recipe:

* a C-alpha random walk with 3.8 A steps, each new C-alpha at least 3.0 A from
  every earlier one (100 tries per step, then the chain restarts);
* three side atoms per C-alpha at a distance uniform in [1.5, 2.5] A in a
  direction uniform on the sphere;
* every atom's element drawn independently with P(C, N, O, S) =
  (.62, .17, .19, .02) and radius (1.7, 1.55, 1.52, 1.8) A;
* a count that is not a multiple of 4 truncates the last residue;
* "compacted" walks reject C-alpha steps that leave the sphere of radius
  (3N / (4 pi rho))^(1/3) - 2.5 A, giving a globule of density rho atoms/A^3;
* random numbers from numpy's PCG64, seeded per workload and molecule.

Paper-density variant (``paper_density``): the appendix table of the paper
implies about 0.1 atoms per cubic Angstrom of enclosed volume, eight times the
globules above.  A 3.0 A self-avoiding C-alpha walk with three side atoms per
residue cannot reach that density (the walk traps itself), so the variant
keeps the walk and fills the rest with side atoms: eight atoms per residue
(the C-alpha and seven side atoms at 1.5-2.5 A, about the heavy-atom count of
a real residue), the C-alpha walk confined to the sphere for rho = 0.1, and a
trapped step backs the walk up four residues instead of restarting the chain.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

RADII = np.array([1.7, 1.55, 1.52, 1.8])
FREQS = np.array([0.62, 0.17, 0.19, 0.02])
STEP = 3.8
MIN_CA = 3.0
SIDE_MIN, SIDE_MAX = 1.5, 2.5
PROTEIN_DENSITY = 0.0125  # atoms / A^3 of the compacted globules
PAPER_DENSITY = 0.1       # atoms / A^3 of the paper-density variant
DENSE_RESIDUE_ATOMS = 8   # C-alpha + 7 side atoms per residue in that variant
DENSE_BACKTRACK = 4       # residues a trapped walk backs up


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _ca_walk(rng: np.random.Generator, n_res: int, confine: float | None) -> np.ndarray:
    """Self-avoiding C-alpha walk (min spacing 3.0 A), optionally confined to a sphere."""
    cell = MIN_CA
    while True:
        pts = np.zeros((n_res, 3))
        grid: dict[tuple[int, int, int], list[int]] = {}
        grid.setdefault((0, 0, 0), []).append(0)
        ok = True
        for k in range(1, n_res):
            placed = False
            dirs = _unit_vectors(rng, 100)
            for t in range(100):
                cand = pts[k - 1] + STEP * dirs[t]
                if confine is not None and float(cand @ cand) > confine * confine:
                    continue
                key = (int(math.floor(cand[0] / cell)), int(math.floor(cand[1] / cell)), int(math.floor(cand[2] / cell)))
                clash = False
                for dx in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dz in (-1, 0, 1):
                            lst = grid.get((key[0] + dx, key[1] + dy, key[2] + dz))
                            if not lst:
                                continue
                            d = pts[lst] - cand
                            if np.any(np.einsum("ij,ij->i", d, d) < MIN_CA * MIN_CA):
                                clash = True
                                break
                        if clash:
                            break
                    if clash:
                        break
                if clash:
                    continue
                pts[k] = cand
                grid.setdefault(key, []).append(k)
                placed = True
                break
            if not placed:
                ok = False
                break
        if ok:
            return pts


def _ca_walk_backtrack(rng: np.random.Generator, n_res: int, confine: float, back: int = DENSE_BACKTRACK,
                       max_traps: int = 1_000_000) -> np.ndarray:
    """Self-avoiding C-alpha walk (min spacing 3.0 A) confined to a sphere; a
    step whose 100 tries all fail backs the walk up `back` residues."""
    pts = np.zeros((n_res, 3))
    k, traps = 1, 0
    while k < n_res:
        cand = pts[k - 1] + STEP * _unit_vectors(rng, 100)
        ok = np.einsum("ij,ij->i", cand, cand) <= confine * confine
        d = cand[:, None, :] - pts[None, :k, :]
        ok &= (np.einsum("ijk,ijk->ij", d, d) >= MIN_CA * MIN_CA).all(axis=1)
        hit = np.flatnonzero(ok)
        if len(hit):
            pts[k] = cand[hit[0]]
            k += 1
        else:
            traps += 1
            if traps > max_traps:
                raise RuntimeError("confined walk did not finish")
            k = max(1, k - back)
    return pts


def paper_density(n_atoms: int, seed: int, density: float = PAPER_DENSITY):
    """Return (xyz, radii) of a globule at the paper's packing density: eight
    atoms per residue, a confined C-alpha walk that backtracks when trapped
    (recipe in the module docstring)."""
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    side = DENSE_RESIDUE_ATOMS - 1
    n_res = (n_atoms + DENSE_RESIDUE_ATOMS - 1) // DENSE_RESIDUE_ATOMS
    confine = max((3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0) - 2.5, STEP)
    ca = _ca_walk_backtrack(rng, n_res, confine)
    side_dir = _unit_vectors(rng, side * n_res).reshape(n_res, side, 3)
    side_len = rng.uniform(SIDE_MIN, SIDE_MAX, size=(n_res, side, 1))
    xyz = np.concatenate([ca[:, None, :], ca[:, None, :] + side_dir * side_len], axis=1).reshape(-1, 3)[:n_atoms]
    types = rng.choice(4, size=xyz.shape[0], p=FREQS)
    xyz = xyz - xyz.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(RADII[types])


def protein_like(n_atoms: int, seed: int, density: float | None = None):
    """Return (xyz float64 (n,3), radii float64 (n,)) for a protein-like chain.

    density=None gives a free walk; otherwise the walk is confined so that the
    globule has about `density` atoms per cubic Angstrom.
    """
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    n_res = (n_atoms + 3) // 4
    confine = None
    if density is not None:
        confine = (3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0) - 2.5
        confine = max(confine, STEP)
    ca = _ca_walk(rng, n_res, confine)
    side_dir = _unit_vectors(rng, 3 * n_res).reshape(n_res, 3, 3)
    side_len = rng.uniform(SIDE_MIN, SIDE_MAX, size=(n_res, 3, 1))
    side = ca[:, None, :] + side_dir * side_len
    xyz = np.concatenate([ca[:, None, :], side], axis=1).reshape(-1, 3)[:n_atoms]
    types = rng.choice(4, size=xyz.shape[0], p=FREQS)
    radii = RADII[types]
    # centre the molecule (translation only)
    xyz = xyz - xyz.mean(axis=0, keepdims=True)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(radii)


def hollow_shell(shell_radius: float = 8.0, spacing: float = 2.4, radius: float = 1.7, seed: int = 77,
                 jitter: float = 0.05):
    """A closed shell of atoms around an empty core: centres on a Fibonacci
    sphere of the given radius, about `spacing` A apart, each moved by a seeded
    uniform offset of at most `jitter` A per axis; all radii `radius`.  With
    spacing < 2 (radius + r_p) sin 60 deg no probe passes between the atoms,
    so the free space inside is a cavity.  Returns (xyz (n,3), radii (n,))."""
    n = max(4, int(round(4.0 * math.pi * shell_radius ** 2 / (spacing ** 2 * math.sqrt(3.0) / 2.0))))
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * k
    rr = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    xyz = shell_radius * np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = xyz + rng.uniform(-jitter, jitter, size=xyz.shape)
    return np.ascontiguousarray(xyz), np.full(n, float(radius))


def icosahedral_rotations() -> np.ndarray:
    """The 60 rotations of the icosahedral group, by closure of two generators."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0

    def rot(axis, ang):
        axis = np.asarray(axis, float)
        axis = axis / np.linalg.norm(axis)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)

    g5 = rot([0.0, 1.0, phi], 2 * math.pi / 5)   # through a vertex of the icosahedron
    g3 = rot([1.0, 1.0, 1.0], 2 * math.pi / 3)   # through a face centre
    group = [np.eye(3)]
    frontier = [np.eye(3)]
    while frontier:
        nxt = []
        for m in frontier:
            for g in (g5, g3):
                c = g @ m
                if not any(np.abs(c - e).max() < 1e-9 for e in group):
                    group.append(c)
                    nxt.append(c)
        frontier = nxt
    if len(group) != 60:
        raise RuntimeError(f"icosahedral closure gave {len(group)} elements")
    return np.stack(group)


@dataclass(frozen=True)
class Workload:
    name: str
    r_p: float
    h: float
    margin: float
    block_pts: int


# The five workloads (sizes and parameters); margin 0.8 A is the paper's
# "grid extension" (§4) where a workload does not name one.
WORKLOADS = {
    1: Workload("plain-200", 1.4, 0.5, 4.0, 0),
    2: Workload("globule-5000", 1.4, 0.25, 0.8, 64),
    3: Workload("batch-256", 1.4, 0.5, 0.8, 64),
    4: Workload("globule-50000", 1.4, 0.2, 0.8, 64),
    5: Workload("assembly-1M", 1.4, 0.3, 0.8, 64),
}


def workload_atoms(config: int, molecule: int = 0, n_atoms: int | None = None):
    """Atoms of a workload (seed = 1000 * config + molecule)."""
    seed = 1000 * config + molecule
    if config == 1:
        return protein_like(n_atoms or 200, seed, None)
    if config == 2:
        return protein_like(n_atoms or 5000, seed, PROTEIN_DENSITY)
    if config == 3:
        return protein_like(n_atoms or batch_sizes()[molecule], seed, PROTEIN_DENSITY)
    if config == 4:
        return protein_like(n_atoms or 50000, seed, PROTEIN_DENSITY)
    if config == 5:
        return assembly(n_atoms or 16667)
    raise ValueError(f"unknown workload {config}")


def batch_sizes(n_mol: int = 256, lo: int = 300, hi: int = 20000, seed: int = 3999) -> np.ndarray:
    """Atom counts log-uniform in [lo, hi] for the batched workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_mol))).astype(np.int64)


def assembly(copy_atoms: int = 16667, shell_radius: float = 300.0, seed: int = 5000):
    """60 rotated copies of one globule on an icosahedral shell."""
    xyz0, r0 = protein_like(copy_atoms, seed, PROTEIN_DENSITY)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    p = _unit_vectors(rng, 1)[0] * shell_radius
    rots = icosahedral_rotations()
    xyz = np.concatenate([xyz0 @ g.T + g @ p for g in rots], axis=0)
    radii = np.tile(r0, len(rots))
    return np.ascontiguousarray(xyz), np.ascontiguousarray(radii)
