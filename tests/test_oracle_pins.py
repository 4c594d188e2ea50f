"""Pins of the FP64 oracle against closed forms, brute force and invariants.

Each test checks the oracle against something other than itself:

* one atom: labels are exactly |x - c| <= r; intersections are the roots of
  the sphere quadratic; normals are radial; area and volume converge to
  4 pi r^2 and 4/3 pi r^3;
* two atoms: distances from the sampled meridian free boundary; area and
  volume by Pappus on the exact profile (non-spindle and spindle);
* 3-10 atoms: dense sampling of free probe centres bounds the distance from
  above within the sample spacing, and from below exactly (every sample is a
  free point);
* invariants: 1-Lipschitz distance, block-size invariance (§2.2, §4), no
  inside point on the domain faces (§2.5), cell-list queries equal brute force;
* the appendix table's block counts (tests/golden/tabA_blocks.txt).
"""
import math
import os

import numpy as np
import pytest

import oracle
from tests.exact_geometry import SampledFree, TwoAtoms, circle_of_spheres, sphere_first_root, trilaterate
from paper_1809_04352_gb300 import inputs

RP = 1.4
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _grid_points(res, idx):
    dims = res.dims
    i = idx // (dims[1] * dims[2])
    j = (idx // dims[2]) % dims[1]
    k = idx % dims[2]
    return res.lo[None, :] + res.h * np.stack([i, j, k], 1).astype(np.float64)


def _all_points(res):
    return _grid_points(res, np.arange(int(np.prod(res.dims)), dtype=np.int64))


# ---------------------------------------------------------------- one atom
def test_single_atom_labels_roots_normals():
    c = np.array([[0.3, -0.2, 0.11]])
    r = np.array([1.7])
    res = oracle.run(c, r, RP, 0.25, 1.0)
    pts = _all_points(res)
    expect = (np.linalg.norm(pts - c, axis=1) <= 1.7).astype(np.int8)
    assert np.array_equal(res.labels.reshape(-1), expect)
    assert res.slow_edges == 0
    for a in range(3):
        assert len(res.idx[a]) > 0
        s = _grid_points(res, res.idx[a])
        for e in range(len(s)):
            t = sphere_first_root(s[e], a, res.h, c[0], 1.7)
            assert t is not None
            assert abs(t - res.tau[a][e]) * res.h < 1e-9
            p = s[e].copy()
            p[a] += res.tau[a][e] * res.h
            n_exp = (p - c[0]) / 1.7
            assert np.abs(res.normal[a][e] - n_exp).max() < 1e-8
        assert np.all(res.ptype[a] == oracle.TYPE_F)


def test_single_atom_tangent_edges():
    """Grid lines tangent to the sphere at a grid point (centre and radius on
    the grid, all values exact in binary): the distance to the surface is
    quadratic in tau there, and the root must still be the closed-form one."""
    c = np.array([[0.0, 0.0, 0.0]])
    res = oracle.run(c, np.array([1.5]), RP, 0.25, 0.75)
    assert np.allclose(res.lo, -2.25)
    tangent = 0
    for a in range(3):
        s = _grid_points(res, res.idx[a])
        for e in range(len(s)):
            d = s[e] - c[0]
            if abs(d[a] ** 2 - (d @ d - 2.25)) < 1e-12:  # discriminant zero
                tangent += 1
            t = sphere_first_root(s[e], a, res.h, c[0], 1.5)
            assert t is not None
            assert abs(t - res.tau[a][e]) * res.h < 1e-9
    assert tangent >= 8


def test_two_atom_torus_tangent_edge():
    """Two atoms (r = 1, centres +-1.5 on z, r_p = 1.5): their expanded
    spheres meet in the circle rho = 2 in z = 0 and the saddle surface passes
    through (0.5, 0, 0), a grid point, at the middle of its arc.  Along y
    the distance to the circle is sqrt(0.25 + y^2) - 2 in magnitude, r_p only
    at y = 0: the grid line touches the surface there from the solvent side,
    so the edge ending at the point has its (double) root at tau = 1, the
    point is inside (the tie of C5) and the edge leaving it crosses at
    tau = 0.  A double root is fixed by FP64 only to about sqrt(eps) of the
    length scale: 1e-7 A here."""
    res = oracle.run(np.array([[0.0, 0, -1.5], [0, 0, 1.5]]), np.array([1.0, 1.0]), 1.5, 0.25, 1.0)
    assert np.allclose(res.lo, [-2.0, -2.0, -3.5])
    d = res.dims
    assert res.labels[10, 8, 14] == 1 and res.labels[10, 7, 14] == 0 and res.labels[10, 9, 14] == 0
    for j, tau in ((7, 1.0), (8, 0.0)):
        p = (10 * d[1] + j) * d[2] + 14
        e = int(np.searchsorted(res.idx[1], p))
        assert res.idx[1][e] == p and res.ptype[1][e] == oracle.TYPE_E
        assert abs(res.tau[1][e] - tau) * 0.25 < 1e-7
        assert np.abs(res.normal[1][e] - [1.0, 0.0, 0.0]).max() < 1e-6  # towards the circle point (2, 0, 0)


@pytest.mark.parametrize("h,tol", [(0.2, 6e-3), (0.1, 2e-3)])
def test_single_atom_area_volume_converge(h, tol):
    r = 1.8
    res = oracle.run(np.array([[0.05, 0.0, -0.07]]), np.array([r]), RP, h, 1.0)
    assert abs(res.area / (4 * math.pi * r * r) - 1) < tol
    assert abs(res.volume / (4 / 3 * math.pi * r ** 3) - 1) < tol


# ---------------------------------------------------------------- two atoms
TWO = [
    ((0.0, 0.0, 0.0), (2.1, 2.4, 0.9), 1.7, 1.55),   # D ~ 3.31, non-spindle saddle
    ((0.1, 0.0, 0.0), (4.0, 3.9, 1.3), 1.52, 1.8),   # D ~ 5.6, spindle (rho < r_p)
]


@pytest.mark.parametrize("c1,c2,r1,r2", TWO)
def test_two_atoms_distance_matches_meridian_boundary(c1, c2, r1, r2):
    ta = TwoAtoms(c1, c2, r1, r2, RP)
    xyz = np.array([c1, c2], float)
    rad = np.array([r1, r2])
    rng = np.random.default_rng(7)
    lo = xyz.min(0) - 3.5
    hi = xyz.max(0) + 3.5
    pts = rng.uniform(lo, hi, size=(4000, 3))
    cap = 6.0
    d, q, t, _ = oracle.distance(xyz, rad, RP, pts, cap)
    dref = np.minimum(ta.distance(pts), cap)
    # the sampled boundary is made of free points: it never undershoots; it
    # overshoots by at most the chord sagitta, spacing^2 / (8 d) for d >> spacing
    assert np.all(d <= dref + 1e-9)
    assert np.all(dref - d <= 1e-9 + ta.spacing ** 2 / (4 * np.maximum(d, 1e-6)))
    # both convex (F) and saddle (E) witnesses occur
    assert (t == oracle.TYPE_F).sum() > 100 and (t == oracle.TYPE_E).sum() > 20
    lab = oracle.label_points(xyz, rad, RP, pts)
    clear = np.abs(dref - RP) > 1e-6
    assert np.array_equal(lab[clear], (dref[clear] >= RP).astype(np.int8))


@pytest.mark.parametrize("c1,c2,r1,r2", TWO)
def test_two_atoms_area_volume_pappus(c1, c2, r1, r2):
    ta = TwoAtoms(c1, c2, r1, r2, RP, n_samples=2000)
    A, V = ta.area_volume()
    res = oracle.run(np.array([c1, c2], float), np.array([r1, r2]), RP, 0.1, 1.0)
    assert abs(res.area / A - 1) < 4e-3
    assert abs(res.volume / V - 1) < 2e-3
    # every intersection lies on the SES: distance r_p from the free boundary
    for a in range(3):
        s = _grid_points(res, res.idx[a])
        p = s.copy()
        p[:, a] += res.tau[a] * res.h
        dd = ta.distance(p)
        assert np.abs(dd - RP).max() < 5e-6


# ---------------------------------------------------------------- few atoms
def _cluster(n, seed):
    rng = np.random.default_rng(seed)
    xyz = [np.zeros(3)]
    while len(xyz) < n:
        base = xyz[rng.integers(len(xyz))]
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        cand = base + v * rng.uniform(2.2, 3.4)
        if min(np.linalg.norm(cand - p) for p in xyz) > 1.8:
            xyz.append(cand)
    rad = inputs.RADII[rng.choice(4, size=n, p=inputs.FREQS)]
    return np.array(xyz), rad


@pytest.mark.parametrize("n,seed", [(3, 1), (4, 2), (6, 3), (10, 4)])
def test_few_atoms_distance_bracketed_by_sampling(n, seed):
    xyz, rad = _cluster(n, seed)
    sf = SampledFree(xyz, rad, RP, n_per_sphere=120000)
    rng = np.random.default_rng(seed + 100)
    lo, hi = xyz.min(0) - 3.0, xyz.max(0) + 3.0
    pts = rng.uniform(lo, hi, size=(3000, 3))
    cap = 5.0
    d, q, t, _ = oracle.distance(xyz, rad, RP, pts, cap)
    ds = np.minimum(sf.distance(pts), cap)
    # every sample is a free point: the exact distance never exceeds it
    assert np.all(d <= ds + 1e-9)
    # and the samples come within a few spacings of the exact distance
    assert np.all(ds - d <= 4 * sf.spacing)
    # labels agree wherever the sampled distance is clear of r_p
    lab = oracle.label_points(xyz, rad, RP, pts)
    clear = (np.abs(ds - RP) > 4 * sf.spacing) & (np.abs(d - RP) > 4 * sf.spacing)
    assert np.array_equal(lab[clear], (d[clear] >= RP).astype(np.int8))
    assert np.array_equal(lab[clear], (ds[clear] >= RP).astype(np.int8))
    # witnesses are free points at the reported distance
    has = t >= 0
    assert np.abs(np.linalg.norm(q[has] - pts[has], axis=1) - d[has]).max() < 1e-9
    d2 = ((q[has][:, None, :] - xyz[None]) ** 2).sum(-1)
    assert np.all(d2 >= (rad + RP)[None, :] ** 2 - 1e-9)
    if n >= 4:
        assert (t == oracle.TYPE_V).sum() > 0


def test_free_vertices_lie_on_three_spheres_and_are_free():
    xyz, rad = _cluster(10, 4)
    npairs, nv, verts, _ = oracle.model_stats(xyz, rad, RP, max_vertices=10000)
    assert nv > 0 and npairs > 0
    R = rad + RP
    dd = np.linalg.norm(verts[:, None, :] - xyz[None], axis=2) - R[None]
    on = (np.abs(dd) < 1e-9).sum(1)
    assert np.all(on >= 3)
    assert np.all(dd > -1e-9)


@pytest.mark.parametrize("seed", [5, 6])
def test_few_atoms_intersections_on_surface_and_first(seed):
    xyz, rad = _cluster(6, seed)
    sf = SampledFree(xyz, rad, RP, n_per_sphere=120000)
    res = oracle.run(xyz, rad, RP, 0.3, 1.0)
    assert res.slow_edges == 0
    tol = 4 * sf.spacing
    for a in range(3):
        s = _grid_points(res, res.idx[a])
        p = s.copy()
        p[:, a] += res.tau[a] * res.h
        d, q, t, _ = oracle.distance(xyz, rad, RP, p, RP + 1.0)
        assert np.abs(d - RP).max() < 1e-9
        ds = sf.distance(p)
        assert np.all(ds - d <= tol) and np.all(d <= ds + 1e-9)
        # normal = unit vector from the root to its witness
        nn = (q - p) / np.linalg.norm(q - p, axis=1, keepdims=True)
        assert np.abs(nn - res.normal[a]).max() < 1e-7
        # first root: no clear label change on [s, p) before the root
        lab_s = res.labels.reshape(-1)[res.idx[a]]
        for f in (0.25, 0.5, 0.75):
            m = s.copy()
            m[:, a] += f * res.tau[a] * res.h
            dm = sf.distance(m)
            wrong = np.where(lab_s == 1, dm < RP - tol, dm > RP + tol)
            assert not wrong.any()


# ---------------------------------------------------------------- invariants
def test_distance_is_1_lipschitz():
    xyz, rad = _cluster(8, 9)
    rng = np.random.default_rng(3)
    lo, hi = xyz.min(0) - 2.0, xyz.max(0) + 2.0
    a = rng.uniform(lo, hi, size=(5000, 3))
    b = a + rng.normal(scale=0.3, size=a.shape)
    cap = 8.0
    da, *_ = oracle.distance(xyz, rad, RP, a, cap)
    db, *_ = oracle.distance(xyz, rad, RP, b, cap)
    assert np.all(np.abs(da - db) <= np.linalg.norm(a - b, axis=1) + 1e-12)


def test_cell_lists_equal_brute_force():
    xyz, rad = inputs.protein_like(60, 11)
    rng = np.random.default_rng(1)
    pts = rng.uniform(xyz.min(0) - 2, xyz.max(0) + 2, size=(3000, 3))
    d1, q1, t1, i1 = oracle.distance(xyz, rad, RP, pts, 4.0, brute=False)
    d2, q2, t2, i2 = oracle.distance(xyz, rad, RP, pts, 4.0, brute=True)
    assert np.array_equal(d1, d2)
    assert np.array_equal(t1, t2)


def test_block_decomposition_invariance():
    xyz, rad = inputs.protein_like(80, 12)
    whole = oracle.run(xyz, rad, RP, 0.5, 2.0, block_pts=0)
    for B in (9, 16, 33):
        blk = oracle.run(xyz, rad, RP, 0.5, 2.0, block_pts=B)
        assert np.array_equal(whole.labels, blk.labels)
        for a in range(3):
            assert np.array_equal(whole.idx[a], blk.idx[a])
            assert np.array_equal(whole.tau[a], blk.tau[a])
            assert np.array_equal(whole.normal[a], blk.normal[a])
        assert abs(whole.area - blk.area) < 1e-9 * whole.area
        assert abs(whole.volume - blk.volume) < 1e-9 * whole.volume


def test_domain_faces_hold_no_inside_point():
    xyz, rad = inputs.protein_like(40, 13)
    res = oracle.run(xyz, rad, RP, 0.4, 0.8, block_pts=16)
    L = res.labels
    assert (L >= 0).all()
    for face in (L[0], L[-1], L[:, 0], L[:, -1], L[:, :, 0], L[:, :, -1]):
        assert not face.any()
    assert res.near_ties == 0


# ---------------------------------------------------------------- appendix table
def test_appendix_block_counts():
    rows = []
    with open(os.path.join(GOLDEN, "tabA_blocks.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            g = [int(v) for v in line.split()]
            rows.append(g)
    assert len(rows) == 290
    for g in rows:
        for a in range(3):
            assert oracle.block_count(g[a], 64) == g[3 + a], g


def test_flop_model_counts_single_atom_brute_force():
    """The flop model's counters (the roofline's algorithmic work) on one
    atom, against brute force over the grid: reach = points within r + 2 r_p,
    shell = points in r <= |x - c| < r + r_p (one face candidate each, no arc
    or vertex), and every crossing edge meets exactly the van der Waals
    sphere (no probe sphere, no torus)."""
    c = np.array([[0.13, -0.21, 0.07]])
    r = np.array([1.7])
    h, margin = 0.25, 0.8
    fc = oracle.flop_counts(c, r, RP, h, margin)
    res = oracle.run(c, r, RP, h, margin)
    d = np.linalg.norm(_all_points(res) - c[0], axis=1)
    reach = int(np.count_nonzero(d < r[0] + 2 * RP))
    shell = int(np.count_nonzero((d >= r[0]) & (d < r[0] + RP)))
    assert fc["points"] == int(np.prod(res.dims))
    assert fc["sum_reach"] == reach
    assert fc["shell_points"] == shell and fc["sum_face"] == shell and fc["sum_face_x_reach"] == shell
    assert fc["sum_arc"] == 0 and fc["sum_vert"] == 0
    assert fc["model_flops"] == 8 * reach + 12 * shell + 8 * shell
    ec = oracle.edge_flop_counts(c, r, RP, h, margin, res.idx)
    ne = sum(int(a.shape[0]) for a in res.idx)
    assert ne > 0 and ec["edges"] == ne and ec["vdw_spheres"] == ne
    assert ec["probe_spheres"] == 0 and ec["tori"] == 0 and ec["model_flops"] == 20 * ne


def test_flop_model_edge_tori_two_atoms():
    """Two overlapping atoms: the edges that cross the saddle (torus) part of
    the surface count the pair's torus; brute force over 257 points of each
    edge segment decides which edges come within r_p of the circle."""
    c = np.array([[0.0, 0.0, 0.0], [2.6, 0.3, -0.2]])
    r = np.array([1.7, 1.52])
    h, margin = 0.25, 0.8
    res = oracle.run(c, r, RP, h, margin)
    ec = oracle.edge_flop_counts(c, r, RP, h, margin, res.idx)
    R = r + RP
    D = np.linalg.norm(c[1] - c[0])
    u = (c[1] - c[0]) / D
    aa = (D * D + R[0] ** 2 - R[1] ** 2) / (2 * D)
    o = c[0] + aa * u
    rho = math.sqrt(R[0] ** 2 - aa * aa)
    sure = maybe = 0
    for ax in range(3):
        p0 = _grid_points(res, res.idx[ax])
        t = np.linspace(0.0, h, 257)
        y = p0[:, None, :] + t[None, :, None] * np.eye(3)[ax][None, None, :] - o
        z = y @ u
        w = np.sqrt(np.maximum((y * y).sum(-1) - z * z, 0.0))
        dist = np.sqrt((w - rho) ** 2 + z * z)
        lo, hi = dist.min(1), dist.max(1)
        # the counter's sampled meet test with its Lipschitz slack lies
        # between the edges that surely meet the tube and those that may
        sure += int(np.count_nonzero((lo <= RP) & (hi >= RP)))
        maybe += int(np.count_nonzero((lo - h / 64 <= RP) & (hi + h / 64 >= RP)))
    assert sure > 0
    assert sure <= ec["tori"] <= maybe
    assert ec["model_flops"] == 20 * (ec["vdw_spheres"] + ec["probe_spheres"]) + 150 * ec["tori"]


def test_sparse_block_run_equals_dense_run():
    """The sparse oracle run (labels of the listed blocks only, for grids too
    large to hold on the host) gives the dense run's labels and edges."""
    xyz, rad = inputs.protein_like(120, 77, inputs.PROTEIN_DENSITY)
    full = oracle.run(xyz, rad, RP, 0.3, 0.8, block_pts=16)
    ids = [3, 17, 40]
    dims, lo, blocks, idx, tau, nrm = oracle.run_blocks(xyz, rad, RP, 0.3, 0.8, 16, ids)
    part = oracle.run(xyz, rad, RP, 0.3, 0.8, block_pts=16, block_ids=ids)
    assert np.array_equal(dims, full.dims) and np.array_equal(lo, full.lo)
    for blo, bhi, lab in blocks:
        assert np.array_equal(lab, full.labels[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]])
    for a in range(3):
        assert np.array_equal(idx[a], part.idx[a]) and np.array_equal(tau[a], part.tau[a])
        assert np.array_equal(nrm[a], part.normal[a])


def test_coincident_atoms_are_one_ball():
    """Repeating an atom (same centre and radius) leaves the union of balls,
    hence the labels, intersections and area/volume, unchanged."""
    xyz = np.array([[0.1, 0.2, 0.3], [2.9, 0.4, -0.6], [0.7, 2.3, 0.2]])
    rad = np.array([1.7, 1.55, 1.52])
    one = oracle.run(xyz, rad, RP, 0.25, 1.0)
    rep = oracle.run(np.vstack([xyz, xyz[:1], xyz[2:3]]), np.concatenate([rad, rad[:1], rad[2:3]]), RP, 0.25, 1.0)
    assert np.array_equal(one.labels, rep.labels)
    for a in range(3):
        assert np.array_equal(one.idx[a], rep.idx[a]) and np.array_equal(one.tau[a], rep.tau[a])
    assert one.area == rep.area and one.volume == rep.volume


# ------------------------------------------------- patch atoms of each root
def test_intersection_patch_atoms_generate_the_surface_point():
    """Every intersection's reported patch atoms (§4.1's nearby atoms) carry
    the surface there, checked by closed forms that do not use the oracle:
    a convex patch's point lies on the atom's van der Waals sphere; a saddle
    patch's point lies at distance r_p from the intersection circle of the
    pair's expanded spheres; a concave patch's point at distance r_p from one
    of the two points where the triple's expanded spheres meet.  A wrong atom
    index, or a type that does not match the ids, fails."""
    xyz, rad = inputs.protein_like(80, 17, inputs.PROTEIN_DENSITY)
    res = oracle.run(xyz, rad, RP, 0.35, 0.8)
    R = rad + RP
    seen = set()
    for a in range(3):
        s = _grid_points(res, res.idx[a])
        for e in range(len(s)):
            p = s[e].copy()
            p[a] += res.tau[a][e] * res.h
            t, ids = int(res.ptype[a][e]), res.atoms[a][e]
            n_ids = int((ids >= 0).sum())
            assert n_ids == t + 1 and np.all(ids[:n_ids] >= 0) and np.all(ids[n_ids:] == -1), (t, ids)
            seen.add(t)
            if t == 0:
                i = ids[0]
                assert abs(np.linalg.norm(p - xyz[i]) - rad[i]) < 1e-7
            elif t == 1:
                i, j = ids[0], ids[1]
                o, u, rho = circle_of_spheres(xyz[i], R[i], xyz[j], R[j])
                w = p - o
                z = w @ u
                dist = math.hypot(math.sqrt(max(w @ w - z * z, 0.0)) - rho, z)
                assert abs(dist - RP) < 1e-7
            else:
                q1, q2 = trilaterate(xyz[ids], R[ids])
                off = min(abs(np.linalg.norm(p - q1) - RP), abs(np.linalg.norm(p - q2) - RP))
                assert off < 1e-7
    assert seen == {0, 1, 2}
