"""The remaining workloads against the oracle, and the paper-density variant.

* globule-50000 (50,000 atoms, h 0.2, the trained proposer on): six seeded
  64-point blocks that hold surface, labels bit-exact, crossing edges equal,
  intersections within 1e-6 A, normals within 1e-6;
* the paper-density globule (0.1 atoms/A^3, eight atoms per residue; the
  density the paper's appendix implies) with 5,000 atoms at h 0.25 and at the
  paper's h 0.4 (margin 0.8): FP32-filtered labels equal the FP64 form's
  everywhere, and twelve 32-point surface blocks match the oracle; a 700-atom globule at
  the same density is compared with the oracle on the whole grid in both
  precisions.
"""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs
from paper_1809_04352_gb300 import proposer as prop
from tests.test_gpu_parity import NRM_TOL, TAU_TOL_A, compare, gpu_run, normal_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return eses.load()


def surface_blocks(labels, n, seed, bp=64):
    """n seeded bp-point blocks (shared faces, bp - 1 cells) holding surface:
    between 2 % and 90 % of their points inside."""
    nb = [oracle.block_count(int(d), bp) for d in labels.shape]
    rng = np.random.default_rng(seed)
    ids = []
    for _ in range(200000):
        b = [int(rng.integers(k)) for k in nb]
        bid = (b[0] * nb[1] + b[1]) * nb[2] + b[2]
        lo = np.array(b) * (bp - 1)
        sl = labels[lo[0]:lo[0] + bp - 1, lo[1]:lo[1] + bp - 1, lo[2]:lo[2] + bp - 1]
        if 0.02 < sl.mean() < 0.9 and bid not in ids:
            ids.append(bid)
            if len(ids) == n:
                break
    assert len(ids) == n
    return sorted(ids)


def check_blocks(g, xyz, rad, rp, h, margin, ids, bp=64):
    o = oracle.run(xyz, rad, rp, h, margin, block_pts=bp, block_ids=ids)
    m = o.labels >= 0
    assert m.sum() > len(ids) * (bp - 14) ** 3
    assert np.array_equal(g["labels"][m], o.labels[m])
    n_edges = 0
    for a in range(3):
        gi = g["axes"][a]["idx"]
        sel = m.reshape(-1)[gi]
        order = np.argsort(gi[sel], kind="stable")
        assert np.array_equal(gi[sel][order], o.idx[a])
        n_edges += len(order)
        if len(order):
            gt = g["axes"][a]["tau"][sel][order]
            assert np.abs(gt - o.tau[a]).max() * h < TAU_TOL_A
            en, crease = normal_error(xyz, rad, rp, gi[sel][order], gt, g["axes"][a]["normal"][sel][order],
                                      o.normal[a], o.dims, o.lo, h, a)
            assert en.max() < NRM_TOL
            assert crease <= 2 + len(order) // 1000
    assert n_edges > 1000


def test_globule_50000_with_proposer_sampled_blocks_match_oracle():
    wl = inputs.WORKLOADS[4]
    xyz, rad = inputs.workload_atoms(4)
    ctx = eses.eses_create(xyz, rad, wl.r_p, wl.h, wl.margin)
    try:
        eses.eses_set_proposer(ctx, eses.ESES_PROPOSER_MLP, prop.load_params(), 0.5)
        eses.eses_run(ctx)
        st = eses.eses_stats(ctx)
        assert st["root_failures"] == 0
        assert st["tiles_certified"] > st["tiles"] // 2  # the proposer did skip work
        dims, lo = eses.eses_grid(ctx)
        g = dict(dims=dims, lo=lo, labels=eses.eses_labels(ctx),
                 axes=[eses.eses_intersections(ctx, a) for a in range(3)])
    finally:
        eses.eses_destroy(ctx)
    assert int(np.prod(dims)) > 9e8
    check_blocks(g, xyz, rad, wl.r_p, wl.h, wl.margin, surface_blocks(g["labels"], 6, 4004))


@pytest.mark.parametrize("h", [0.25, 0.4])
def test_paper_density_5000_fp32_equals_fp64_and_sampled_blocks_match_oracle(h):
    xyz, rad = inputs.paper_density(5000, 2200)
    g32 = gpu_run(xyz, rad, 1.4, h, 0.8, eses.ESES_PREC_FP32_FILTERED)
    g64 = gpu_run(xyz, rad, 1.4, h, 0.8, eses.ESES_PREC_FP64)
    assert g32["stats"]["root_failures"] == 0
    assert np.array_equal(g32["labels"], g64["labels"])
    for a in range(3):
        o32 = np.argsort(g32["axes"][a]["idx"], kind="stable")
        o64 = np.argsort(g64["axes"][a]["idx"], kind="stable")
        assert np.array_equal(g32["axes"][a]["idx"][o32], g64["axes"][a]["idx"][o64])
        assert np.abs(g32["axes"][a]["tau"][o32] - g64["axes"][a]["tau"][o64]).max() * h < TAU_TOL_A
    # 32-point blocks: the oracle's cost per point grows with the density
    check_blocks(g32, xyz, rad, 1.4, h, 0.8, surface_blocks(g32["labels"], 12, 2201, bp=32), bp=32)


@pytest.fixture(scope="module")
def dense_700():
    xyz, rad = inputs.paper_density(700, 2300)
    return xyz, rad, oracle.run(xyz, rad, 1.4, 0.4, 0.8, block_pts=16)


@pytest.mark.parametrize("precision", [eses.ESES_PREC_FP64, eses.ESES_PREC_FP32_FILTERED])
def test_paper_density_700_whole_grid_matches_oracle(precision, dense_700):
    xyz, rad, o = dense_700
    g = gpu_run(xyz, rad, 1.4, 0.4, 0.8, precision)
    compare(g, o, 0.4, atoms=(xyz, rad, 1.4))


@pytest.fixture(scope="module")
def dense_cluster():
    """400 atoms at 0.3 atoms/A^3 (three times a protein's packing): every
    tile near the middle stages more than the 320 atoms the shared-memory
    lists hold, so those tiles take the global-memory tier."""
    rng = np.random.default_rng(9)
    n, dens = 400, 0.3
    side = (n / dens) ** (1 / 3)
    xyz = rng.uniform(0, side, (n, 3))
    rad = inputs.RADII[rng.choice(4, n, p=inputs.FREQS)]
    return xyz, rad, oracle.run(xyz, rad, 1.4, 0.4, 0.8, block_pts=16)


@pytest.mark.parametrize("precision", [eses.ESES_PREC_FP64, eses.ESES_PREC_FP32_FILTERED])
def test_overflowing_tiles_take_the_global_memory_tier_and_match_oracle(precision, dense_cluster):
    xyz, rad, o = dense_cluster
    g = gpu_run(xyz, rad, 1.4, 0.4, 0.8, precision)
    assert g["stats"]["big_tier_tiles"] > 0
    compare(g, o, 0.4, atoms=(xyz, rad, 1.4))


@pytest.mark.parametrize("precision", [eses.ESES_PREC_FP64, eses.ESES_PREC_FP32_FILTERED])
def test_buried_patch_culling_changes_nothing_but_the_work(precision):
    """Without the pre-culling every circle and every face carries witnesses
    into the tiles; the witnesses of buried patches are never free, so the
    labels, edges and intersections must be identical, bit for bit.  (A
    globule at 0.0125 atoms/A^3: at the paper's density the unculled circles
    overflow even the global-memory staging, which the next test checks.)"""
    xyz, rad = inputs.protein_like(1500, 2301, inputs.PROTEIN_DENSITY)
    out = {}
    for cull in (1, 0):
        ctx = eses.eses_create(xyz, rad, 1.4, 0.4, 0.8)
        try:
            eses.eses_set_option(ctx, eses.ESES_OPT_PRECISION, precision)
            eses.eses_set_option(ctx, eses.ESES_OPT_CULL, cull)
            eses.eses_run(ctx)
            out[cull] = (eses.eses_labels(ctx), [eses.eses_intersections(ctx, a, fp32=False) for a in range(3)],
                         eses.eses_patch_counts(ctx))
        finally:
            eses.eses_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0])
    for a in range(3):
        x, y = out[0][1][a], out[1][1][a]
        assert np.array_equal(x["idx"], y["idx"])
        assert np.array_equal(x["tau"], y["tau"])
        assert np.array_equal(x["normal"], y["normal"])
    n_pairs, n_free, _ = out[1][2]
    assert n_free < n_pairs  # the culling does remove buried circles here


def test_without_culling_the_paper_density_overflows_and_reports_it():
    """At 0.1 atoms/A^3 a tile meets thousands of circles, most of them buried:
    without the pre-culling its staging overflows even the global-memory tier,
    and the run reports ESES_ECAPACITY (with every output written, so the
    context stays usable); with the culling the same molecule runs."""
    xyz, rad = inputs.paper_density(700, 2300)
    ctx = eses.eses_create(xyz, rad, 1.4, 0.4, 0.8)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_CULL, 0)
        with pytest.raises(eses.EsesError) as ei:
            eses.eses_run(ctx)
        assert ei.value.code == eses.ESES_ECAPACITY
        eses.eses_set_option(ctx, eses.ESES_OPT_CULL, 1)
        eses.eses_run(ctx)
        assert eses.eses_stats(ctx)["root_failures"] == 0
    finally:
        eses.eses_destroy(ctx)
