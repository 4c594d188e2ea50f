"""Triangle mesh of the surface (reading M1, cube by cube).

CPU: the library's case table (a host function, no device) equals the
oracle's, written separately; the rule's own properties (each case uses
exactly its cut edges, the loop boundaries run along cube faces); the
oracle's meshes are closed and face the solvent, a sphere's has Euler
characteristic 2 and its area and volume approach 4 pi r^2 and 4/3 pi r^3,
and a closed shell of atoms gives two surfaces (characteristic 4), one once
its cavity is filled.  GPU: the library's mesh equals the oracle's (the same
triangles with the same orientation; vertices within 1e-6 A).
"""
import collections

import numpy as np
import pytest

import oracle
from oracle import mesh_oracle as mo
from paper_1809_04352_gb300 import inputs

RP = 1.4


def closed_and_chi(keys):
    """(every directed edge has its reverse exactly once, V - E + F)."""
    de = collections.Counter()
    for t in keys.tolist():
        for k in range(3):
            de[(t[k], t[(k + 1) % 3])] += 1
    closed = all(v == 1 for v in de.values()) and all(de.get((b, a), 0) == 1 for (a, b) in de)
    v = len(set(keys.reshape(-1).tolist()))
    return closed, v - len(de) // 2 + len(keys)


def area_volume(xyz):
    n = np.cross(xyz[:, 1] - xyz[:, 0], xyz[:, 2] - xyz[:, 0])
    vol = np.einsum("ij,ij->i", xyz[:, 0], np.cross(xyz[:, 1], xyz[:, 2])).sum() / 6.0
    return 0.5 * np.linalg.norm(n, axis=1).sum(), vol


def test_library_table_equals_oracle_table():
    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses
    libbuild.build()
    tri, n = eses.eses_mesh_table()
    for c in range(256):
        t = mo.TABLE[c]
        assert int(n[c]) == len(t)
        assert [tuple(int(v) for v in tri[c, k]) for k in range(len(t))] == t
        assert np.all(tri[c, len(t):] == -1)


def test_table_rule_properties():
    faces = [set(f) for f in mo.FACES]
    for c in range(256):
        ins = [(c >> i) & 1 for i in range(8)]
        cut = {e for e, (_, lo, hi) in enumerate(mo.EDGES) if ins[lo] != ins[hi]}
        t = mo.TABLE[c]
        assert {e for tri in t for e in tri} == cut
        de = collections.Counter()
        for tri in t:
            for k in range(3):
                de[(tri[k], tri[(k + 1) % 3])] += 1
        for (a, b), m in de.items():
            if de.get((b, a), 0) == 0:  # a loop edge: the two cut edges share a face
                assert m == 1 and any(a in f and b in f for f in faces), (c, a, b)
    assert max(len(t) for t in mo.TABLE) <= 5 and mo.TABLE[0] == [] and mo.TABLE[255] == []


def test_oracle_mesh_of_one_atom():
    c, r = np.array([[0.3, -0.2, 0.11]]), 1.7
    res = oracle.run(c, np.array([r]), RP, 0.2, 1.0)
    keys, xyz = mo.mesh(res.labels, res.lo, res.h, res.idx, res.tau)
    closed, chi = closed_and_chi(keys)
    assert closed and chi == 2
    n = np.cross(xyz[:, 1] - xyz[:, 0], xyz[:, 2] - xyz[:, 0])
    assert np.all(np.einsum("ij,ij->i", n, xyz.mean(1) - c[0]) > 0)  # towards the solvent
    # every vertex lies on the sphere (the intersections are exact)
    assert np.abs(np.linalg.norm(xyz - c[0], axis=2) - r).max() < 1e-9
    area, vol = area_volume(xyz)
    assert abs(area / (4 * np.pi * r * r) - 1) < 0.01
    assert abs(vol / (4 / 3 * np.pi * r ** 3) - 1) < 0.01


def test_oracle_mesh_of_a_closed_shell():
    xyz, rad = inputs.hollow_shell(shell_radius=6.5)
    res = oracle.run(xyz, rad, RP, 0.5, 1.0)
    keys, pts = mo.mesh(res.labels, res.lo, res.h, res.idx, res.tau)
    closed, chi = closed_and_chi(keys)
    assert closed and chi == 4  # outer surface and the cavity's
    ext, _ = oracle.exterior_labels(res.labels)
    keys2, pts2 = mo.mesh(ext, res.lo, res.h, res.idx, res.tau)
    closed2, chi2 = closed_and_chi(keys2)
    assert closed2 and chi2 == 2
    a1, v1 = area_volume(pts)
    a2, v2 = area_volume(pts2)
    assert a2 < a1 and v2 > v1 > 0


# ------------------------------------------------------------------- GPU
def canonical(keys, xyz):
    """Each triangle rotated to start at its smallest key (orientation kept),
    rows sorted: (keys, xyz) in that order."""
    k = np.asarray(keys)
    r = np.argmin(k, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    k2 = np.take_along_axis(k, idx, axis=1)
    x2 = np.take_along_axis(np.asarray(xyz), idx[:, :, None], axis=1)
    order = np.lexsort((k2[:, 2], k2[:, 1], k2[:, 0]))
    return k2[order], x2[order]


def _gpu_mesh(xyz, rad, h, margin, exterior=0, precision=None):
    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses
    libbuild.build()
    ctx = eses.eses_create(xyz, rad, RP, h, margin)
    try:
        if precision is not None:
            eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, precision)
        eses.eses_set_option(ctx, eses.ESES_OPT_EXTERIOR, exterior)
        with pytest.raises(eses.EsesError):
            eses.eses_mesh_count(ctx)  # no results yet
        eses.eses_run(ctx)
        n = eses.eses_mesh_count(ctx)
        keys, pts = eses.eses_mesh(ctx)
        assert keys.shape == (n, 3)
        return keys, pts
    finally:
        eses.eses_destroy(ctx)


CASES = {
    "one-atom": (np.array([[0.3, -0.2, 0.11]]), np.array([1.7]), 0.25, 1.0),
    "plain-40": inputs.protein_like(40, 11) + (0.3, 1.0),
    "globule-300": inputs.protein_like(300, 4242, inputs.PROTEIN_DENSITY) + (0.35, 0.8),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(CASES))
def test_gpu_mesh_equals_oracle_mesh(name):
    xyz, rad, h, margin = CASES[name]
    res = oracle.run(xyz, rad, RP, h, margin)
    ok, ox = canonical(*mo.mesh(res.labels, res.lo, res.h, res.idx, res.tau))
    gk, gx = canonical(*_gpu_mesh(xyz, rad, h, margin))
    assert np.array_equal(gk, ok)
    assert np.abs(gx - ox).max() < 1e-6
    closed, chi = closed_and_chi(gk)
    assert closed and chi % 2 == 0


@pytest.mark.gpu
def test_gpu_mesh_of_the_shell_with_and_without_cavity():
    xyz, rad = inputs.hollow_shell(shell_radius=6.5)
    res = oracle.run(xyz, rad, RP, 0.5, 1.0)
    ext, _ = oracle.exterior_labels(res.labels)
    for lab, mode, chi_exp in ((res.labels, 0, 4), (ext, 1, 2)):
        ok, ox = canonical(*mo.mesh(lab, res.lo, res.h, res.idx, res.tau))
        gk, gx = canonical(*_gpu_mesh(xyz, rad, 0.5, 1.0, exterior=mode))
        assert np.array_equal(gk, ok)
        assert np.abs(gx - ox).max() < 1e-6
        assert closed_and_chi(gk) == (True, chi_exp)


@pytest.mark.gpu
def test_gpu_mesh_refuses_a_batch():
    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses
    libbuild.build()
    ctx = eses.eses_create_batch([inputs.protein_like(30, 1), inputs.protein_like(20, 2)], RP, 0.5, 1.0)
    try:
        eses.eses_run(ctx)
        with pytest.raises(eses.EsesError):
            eses.eses_mesh_count(ctx)
    finally:
        eses.eses_destroy(ctx)
