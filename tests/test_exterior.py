"""Exterior-only surface (reading X1: cavities filled).

CPU pins of the oracle: its flood fill equals the connected components of
the outside points found by scipy (components that touch the domain boundary
stay outside, the others become inside), and on a closed shell of atoms the
centre is a cavity point that the exterior-only run fills, with the edges and
area/volume changed only where the cavity was.  GPU parity: labels bit-exact,
edges identical, roots within 1e-6 A, area/volume to summation order, for a
single molecule, both precisions, a batch, and with the CUDA graph on.
"""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import inputs

RP = 1.4
SHELL = dict(shell_radius=6.5)


def components_fill(lab):
    """Independent form of the fill: scipy's 6-connected components."""
    ndimage = pytest.importorskip("scipy.ndimage")
    comp, n = ndimage.label(lab == 0, structure=ndimage.generate_binary_structure(3, 1))
    border = np.zeros(n + 1, bool)
    for face in (comp[0], comp[-1], comp[:, 0], comp[:, -1], comp[:, :, 0], comp[:, :, -1]):
        border[np.unique(face)] = True
    border[0] = True  # label 0 of `comp` is the inside points
    out = lab.copy()
    out[~border[comp]] = 1
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_flood_fill_matches_connected_components(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rng.integers(6, 24, size=3))
    lab = (rng.random(shape) < 0.45).astype(np.int8)  # 1 inside, about 55 % outside
    # a walled box with an empty core: a certain cavity
    lab[1:5, 1:5, 1:5] = 1
    lab[2:4, 2:4, 2:4] = 0
    lab[0], lab[-1], lab[:, 0], lab[:, -1], lab[:, :, 0], lab[:, :, -1] = 0, 0, 0, 0, 0, 0
    got, n = oracle.exterior_labels(lab)
    exp = components_fill(lab)
    assert np.array_equal(got, exp)
    assert n == int((got != lab).sum()) and n >= 8
    assert np.all(got >= lab)


@pytest.fixture(scope="module")
def shell_runs():
    xyz, rad = inputs.hollow_shell(**SHELL)
    full = oracle.run(xyz, rad, RP, 0.5, 1.0)
    ext = oracle.run(xyz, rad, RP, 0.5, 1.0, exterior=True)
    return xyz, rad, full, ext


def test_exterior_only_hollow_shell_oracle(shell_runs):
    xyz, rad, full, ext = shell_runs
    c = tuple(int(v) // 2 for v in full.dims)
    # the centre is a free probe position (every centre is 6.5 A away, R = 3.1 A)
    # enclosed by the shell: outside on the full surface, filled here
    assert np.min(np.linalg.norm(xyz - (full.lo + 0.5 * np.array(c)), axis=1)) > rad[0] + RP
    assert full.labels[c] == 0 and ext.labels[c] == 1
    assert np.array_equal(ext.labels, components_fill(full.labels))
    filled = int((ext.labels != full.labels).sum())
    assert filled > 100
    assert abs((ext.volume_count - full.volume_count) - filled * 0.5 ** 3) < 1e-9
    # the outer surface is kept: its edges are the full run's edges that avoid the cavity
    stride = [full.dims[1] * full.dims[2], full.dims[2], 1]
    for a in range(3):
        keep = ext.labels.reshape(-1)[full.idx[a]] != ext.labels.reshape(-1)[full.idx[a] + stride[a]]
        assert np.array_equal(ext.idx[a], full.idx[a][keep])
        assert np.array_equal(ext.tau[a], full.tau[a][keep])
        assert np.array_equal(ext.normal[a], full.normal[a][keep])
        assert len(ext.idx[a]) < len(full.idx[a])
    assert ext.area < full.area and ext.volume > full.volume


# ------------------------------------------------------------------- GPU
def _gpu_modules():
    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses
    libbuild.build()
    return eses


def _check(eses, g, o, h, xyz, rad):
    from tests.test_gpu_parity import TAU_TOL_A, normal_error
    assert np.array_equal(g["dims"], o.dims)
    assert np.array_equal(g["labels"], o.labels)
    for a in range(3):
        ga = g["axes"][a]
        order = np.argsort(ga["idx"], kind="stable")
        assert np.array_equal(ga["idx"][order], o.idx[a])
        if len(order):
            assert np.abs(ga["tau"][order] - o.tau[a]).max() * h < TAU_TOL_A
            en, _ = normal_error(xyz, rad, RP, ga["idx"][order], ga["tau"][order], ga["normal"][order], o.normal[a],
                              o.dims, o.lo, h, a)
            assert en.max() < 1e-6
    assert abs(g["area"] - o.area) <= 1e-9 * max(o.area, 1.0)
    assert abs(g["volume"] - o.volume) <= 1e-9 * max(o.volume, 1.0)


def _single(eses, xyz, rad, h, margin, precision, exterior=1, graph=0, runs=1):
    ctx = eses.eses_create(xyz, rad, RP, h, margin)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, precision)
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, graph)
        eses.eses_set_option(ctx, eses.ESES_OPT_EXTERIOR, exterior)
        for _ in range(runs):
            eses.eses_run(ctx)
        dims, lo = eses.eses_grid(ctx)
        out = dict(dims=dims, lo=lo, labels=eses.eses_labels(ctx), stats=eses.eses_stats(ctx))
        out["area"], out["volume"] = eses.eses_area_volume(ctx)
        out["axes"] = [eses.eses_intersections(ctx, a) for a in range(3)]
        return out
    finally:
        eses.eses_destroy(ctx)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exterior_hollow_shell_matches_oracle(shell_runs, precision):
    eses = _gpu_modules()
    xyz, rad, full, ext = shell_runs
    prec = eses.ESES_PREC_FP64 if precision == "fp64" else eses.ESES_PREC_FP32_FILTERED
    g = _single(eses, xyz, rad, 0.5, 1.0, prec)
    _check(eses, g, ext, 0.5, xyz, rad)
    assert g["stats"]["cavity_points"] == int((ext.labels != full.labels).sum())
    assert g["stats"]["exterior_sweeps"] >= 2
    assert g["stats"]["root_failures"] == 0


@pytest.mark.gpu
def test_exterior_globule_matches_oracle():
    eses = _gpu_modules()
    xyz, rad = inputs.protein_like(300, 4242, inputs.PROTEIN_DENSITY)
    h = 0.3
    o = oracle.run(xyz, rad, RP, h, 0.8, exterior=True)
    g = _single(eses, xyz, rad, h, 0.8, eses.ESES_PREC_FP32_FILTERED)
    _check(eses, g, o, h, xyz, rad)


@pytest.mark.gpu
def test_exterior_with_graph_option_and_toggling(shell_runs):
    """The graph option leaves the exterior-only run eager (and correct);
    switching the option off again gives the full surface."""
    eses = _gpu_modules()
    xyz, rad, full, ext = shell_runs
    ctx = eses.eses_create(xyz, rad, RP, 0.5, 1.0)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 1)
        for mode, o in ((0, full), (1, ext), (1, ext), (0, full), (0, full)):
            eses.eses_set_option(ctx, eses.ESES_OPT_EXTERIOR, mode)
            assert eses.eses_get_option(ctx, eses.ESES_OPT_EXTERIOR) == mode
            eses.eses_run(ctx)
            assert np.array_equal(eses.eses_labels(ctx), o.labels)
            for a in range(3):
                idx = np.sort(eses.eses_intersections(ctx, a)["idx"])
                assert np.array_equal(idx, o.idx[a])
    finally:
        eses.eses_destroy(ctx)


@pytest.mark.gpu
def test_exterior_batch_matches_single_runs(shell_runs):
    eses = _gpu_modules()
    from tests.test_batch import mol_result, same_result
    xyz, rad, full, ext = shell_runs
    mols = [(xyz, rad), inputs.protein_like(200, 77, inputs.PROTEIN_DENSITY), (xyz + 3.0, rad)]
    ctx = eses.eses_create_batch(mols, RP, 0.5, 1.0)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_EXTERIOR, 1)
        eses.eses_run(ctx)
        for m, (x, r) in enumerate(mols):
            same_result(mol_result(ctx, m), _single(eses, x, r, 0.5, 1.0, eses.ESES_PREC_FP32_FILTERED), 0.5)
        assert np.array_equal(mol_result(ctx, 0)["labels"], ext.labels)
    finally:
        eses.eses_destroy(ctx)
