"""Block selections of the library (eses_create_on_grid + eses_set_blocks):
the parts of a molecule split by blocks, each run on its halo atoms only,
merge to the whole run.

Labels, crossing edges, intersections and normals must equal the whole-grid
run bit for bit (the selections compute the same tiles in the same tile
frames); area and volume to 1e-12 relative (partial sums added in another
order).  Slabs along axis 0 (the partition of ``shard.partition``) and a
2 x 2 x 2 split (every axis' ownership rule) are both checked, in both
precisions, and a selection's device label buffer is bounded by its blocks.
"""
import numpy as np
import pytest

from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs, shard

pytestmark = pytest.mark.gpu

RP, H = 1.4, 0.3


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return eses.load()


def whole(xyz, rad, precision):
    ctx = eses.eses_create(xyz, rad, RP, H, 0.8)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, precision)
        eses.eses_run(ctx)
        dims, origin = eses.eses_grid(ctx)
        axes = [eses.eses_intersections(ctx, a, fp32=False) for a in range(3)]
        out = dict(dims=dims, origin=origin, labels=eses.eses_labels(ctx), axes=axes,
                   av=eses.eses_area_volume(ctx), points=eses.eses_stats(ctx)["points"])
    finally:
        eses.eses_destroy(ctx)
    return out


def parts_of(xyz, rad, w, boxes, B, precision):
    parts = []
    for lo, hi in boxes:
        sel = shard.halo_atoms(xyz, rad, RP, H, w["origin"], w["dims"], B, lo, hi)
        ctx = eses.eses_create_on_grid(xyz[sel], rad[sel], RP, H, w["origin"], w["dims"])
        try:
            eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, precision)
            eses.eses_set_option(ctx, eses.ESES_OPT_BLOCK_PTS, B)
            eses.eses_set_blocks(ctx, lo, hi)
            eses.eses_run(ctx)
            blo, ext = eses.eses_owned_box(ctx)
            assert np.array_equal(blo, np.asarray(lo) * B)
            assert eses.eses_stats(ctx)["points"] == int(np.prod(ext))
            p = shard.Part(lo=blo, dims=ext, labels=eses.eses_labels(ctx).reshape(-1))
            axes = [eses.eses_intersections(ctx, a, fp32=False) for a in range(3)]
            p.idx = [x["idx"] for x in axes]
            p.tau = [x["tau"] for x in axes]
            p.normal = [x["normal"] for x in axes]
            p.area, p.volume = eses.eses_area_volume(ctx)
            parts.append(p)
        finally:
            eses.eses_destroy(ctx)
    return parts


def check(w, merged):
    lab, idx, tau, nrm, area, vol = merged
    assert np.array_equal(lab, w["labels"])
    for a in range(3):
        o = np.argsort(w["axes"][a]["idx"], kind="stable")
        assert np.array_equal(idx[a], w["axes"][a]["idx"][o])
        assert np.array_equal(tau[a], w["axes"][a]["tau"][o])
        assert np.array_equal(nrm[a], w["axes"][a]["normal"][o])
    assert abs(area - w["av"][0]) <= 1e-12 * w["av"][0]
    assert abs(vol - w["av"][1]) <= 1e-12 * w["av"][1]


@pytest.mark.parametrize("precision", [eses.ESES_PREC_FP64, eses.ESES_PREC_FP32_FILTERED])
def test_slabs_on_halo_atoms_merge_to_the_whole_run(precision):
    xyz, rad = inputs.protein_like(900, 71, inputs.PROTEIN_DENSITY)
    w = whole(xyz, rad, precision)
    B = 24
    costs = shard.block_costs(xyz, rad, RP, H, w["origin"], w["dims"], B)
    boxes = [s for s in shard.partition(costs, 3) if s is not None]
    assert len(boxes) == 3
    check(w, shard.combine(parts_of(xyz, rad, w, boxes, B, precision), w["dims"]))


def test_octants_merge_to_the_whole_run():
    xyz, rad = inputs.protein_like(600, 72, inputs.PROTEIN_DENSITY)
    w = whole(xyz, rad, eses.ESES_PREC_FP32_FILTERED)
    B = 40
    nb = shard.n_blocks(w["dims"], B)
    assert np.all(nb >= 2)
    cut = nb // 2
    boxes = []
    for i in range(8):
        c = [(i >> 2) & 1, (i >> 1) & 1, i & 1]
        lo = np.array([0 if c[a] == 0 else cut[a] for a in range(3)])
        hi = np.array([cut[a] if c[a] == 0 else nb[a] for a in range(3)])
        boxes.append((lo, hi))
    check(w, shard.combine(parts_of(xyz, rad, w, boxes, B, eses.ESES_PREC_FP32_FILTERED), w["dims"]))


def test_selection_rules():
    xyz, rad = inputs.protein_like(300, 73, inputs.PROTEIN_DENSITY)
    ctx = eses.eses_create(xyz, rad, RP, H, 0.8)
    try:
        for bad in (12, 0, 7):  # not a multiple of 8 in [8, 2^20]
            with pytest.raises(eses.EsesError):
                eses.eses_set_option(ctx, eses.ESES_OPT_BLOCK_PTS, bad)
        eses.eses_set_option(ctx, eses.ESES_OPT_BLOCK_PTS, 16)
        nb = eses.eses_num_blocks(ctx)
        with pytest.raises(eses.EsesError):
            eses.eses_set_blocks(ctx, [0, 0, 0], [nb[0] + 1, nb[1], nb[2]])
        eses.eses_set_blocks(ctx, [0, 0, 0], [1, nb[1], nb[2]])
        with pytest.raises(eses.EsesError):
            eses.eses_set_option(ctx, eses.ESES_OPT_EXTERIOR, 1)
        eses.eses_run(ctx)
        with pytest.raises(eses.EsesError) as ei:
            eses.eses_mesh_count(ctx)
        assert ei.value.code == eses.ESES_ESTATE
        lo, ext = eses.eses_owned_box(ctx)
        assert list(lo) == [0, 0, 0] and ext[0] == 16
        eses.eses_set_blocks(ctx)  # whole grid again
        eses.eses_run(ctx)
        dims, _ = eses.eses_grid(ctx)
        assert np.array_equal(eses.eses_owned_box(ctx)[1], dims)
        eses.eses_mesh_count(ctx)
    finally:
        eses.eses_destroy(ctx)
