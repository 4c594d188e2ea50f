"""Batched path: many molecules in one context, persistent tile kernels with a
device work queue, CUDA-graph replay and the launch-shape autotuner.

Every molecule of a batch must give exactly what a context of that molecule
alone gives (labels and crossing edges identical, roots and normals equal,
area/volume to summation order), and small batches are checked against the
oracle directly.  The full 256-molecule batch (log-uniform 300-20,000 atoms,
h = 0.5) is checked on sampled molecules and blocks against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs
from tests.test_gpu_parity import TAU_TOL_A, gpu_run, normal_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return eses.load()


def mol_result(ctx, m):
    dims, lo = eses.eses_mol_grid(ctx, m)
    out = dict(dims=dims, lo=lo, labels=eses.eses_mol_labels(ctx, m))
    out["area"], out["volume"] = eses.eses_mol_area_volume(ctx, m)
    out["axes"] = [eses.eses_mol_intersections(ctx, m, a) for a in range(3)]
    return out


def same_result(b, s, h, tau_tol=1e-12):
    assert np.array_equal(b["dims"], s["dims"])
    assert np.array_equal(b["lo"], s["lo"])
    assert np.array_equal(b["labels"], s["labels"])
    for a in range(3):
        assert np.array_equal(b["axes"][a]["idx"], s["axes"][a]["idx"])
        if len(b["axes"][a]["idx"]):
            assert np.abs(b["axes"][a]["tau"] - s["axes"][a]["tau"]).max() * h <= tau_tol
            assert np.abs(b["axes"][a]["normal"] - s["axes"][a]["normal"]).max() <= 1e-9
    assert abs(b["area"] - s["area"]) <= 1e-9 * max(s["area"], 1.0)
    assert abs(b["volume"] - s["volume"]) <= 1e-9 * max(s["volume"], 1.0)


def small_batch():
    return [inputs.protein_like(n, 300 + k, inputs.PROTEIN_DENSITY) for k, n in enumerate([1, 40, 300, 90, 700, 2])]


def test_batch_equals_single_molecule_runs():
    mols = small_batch()
    h = 0.4
    ctx = eses.eses_create_batch(mols, 1.4, h, 0.8)
    try:
        assert eses.eses_num_molecules(ctx) == len(mols)
        eses.eses_run(ctx)
        st = eses.eses_stats(ctx)
        assert st["root_failures"] == 0
        for m, (xyz, rad) in enumerate(mols):
            same_result(mol_result(ctx, m), gpu_run(xyz, rad, 1.4, h, 0.8), h)
        # the single-molecule accessors refuse a batch
        with pytest.raises(eses.EsesError):
            eses.eses_labels(ctx)
        with pytest.raises(eses.EsesError):
            eses.eses_mol_labels(ctx, len(mols))
    finally:
        eses.eses_destroy(ctx)


def test_small_batch_matches_oracle():
    mols = [inputs.protein_like(n, 900 + n, inputs.PROTEIN_DENSITY) for n in (25, 60, 11)]
    h = 0.3
    ctx = eses.eses_run_batch(mols, 1.4, h, 0.9)
    try:
        for m, (xyz, rad) in enumerate(mols):
            o = oracle.run(xyz, rad, 1.4, h, 0.9)
            g = mol_result(ctx, m)
            assert np.array_equal(g["dims"], o.dims)
            assert np.array_equal(g["labels"], o.labels)
            for a in range(3):
                ga = g["axes"][a]
                order = np.argsort(ga["idx"], kind="stable")
                assert np.array_equal(ga["idx"][order], o.idx[a])
                if len(order):
                    assert np.abs(ga["tau"][order] - o.tau[a]).max() * h < TAU_TOL_A
                    en, _ = normal_error(xyz, rad, 1.4, ga["idx"][order], ga["tau"][order], ga["normal"][order],
                                      o.normal[a], o.dims, o.lo, h, a)
                    assert en.max() < 1e-6
            assert abs(g["area"] - o.area) <= 1e-9 * o.area
            assert abs(g["volume"] - o.volume) <= 1e-9 * o.volume
    finally:
        eses.eses_destroy(ctx)


def test_graph_replay_and_queue_modes_give_identical_results():
    mols = small_batch()[1:5]
    h = 0.35
    ref = eses.eses_create_batch(mols, 1.4, h, 0.8)
    ctx = eses.eses_create_batch(mols, 1.4, h, 0.8)
    try:
        eses.eses_run(ref)
        base = [mol_result(ref, m) for m in range(len(mols))]
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 1)
        assert eses.eses_get_option(ctx, eses.ESES_OPT_GRAPH) == 1
        for _ in range(3):  # plan, capture, replay
            eses.eses_run(ctx)
            for m in range(len(mols)):
                same_result(mol_result(ctx, m), base[m], h, tau_tol=0.0)
        assert eses.eses_stats(ctx)["kernel_launches"] > 20
        # grid-stride tile order and other launch shapes: same results
        eses.eses_set_option(ctx, eses.ESES_OPT_QUEUE, 0)
        eses.eses_set_option(ctx, eses.ESES_OPT_CLS_CTAS, 1)
        eses.eses_set_option(ctx, eses.ESES_OPT_EDGE_TILES, 3)
        eses.eses_set_option(ctx, eses.ESES_OPT_ROOT_THREADS, 128)
        eses.eses_run(ctx)
        eses.eses_run(ctx)
        for m in range(len(mols)):
            same_result(mol_result(ctx, m), base[m], h, tau_tol=0.0)
    finally:
        eses.eses_destroy(ctx)
        eses.eses_destroy(ref)


def test_graph_replay_with_stage_timing():
    xyz, rad = inputs.protein_like(400, 41, inputs.PROTEIN_DENSITY)
    ctx = eses.eses_create(xyz, rad, 1.4, 0.3, 0.8)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 1)
        eses.eses_set_option(ctx, eses.ESES_OPT_PROFILE, 1)
        for _ in range(3):
            eses.eses_run(ctx)
            st = eses.eses_stage_times(ctx)
            assert all(v >= 0.0 for v in st.values()) and st["classify"] > 0.0
    finally:
        eses.eses_destroy(ctx)


def test_autotune_picks_a_shape_and_keeps_results():
    mols = small_batch()[2:5]
    h = 0.4
    ctx = eses.eses_create_batch(mols, 1.4, h, 0.8)
    try:
        eses.eses_run(ctx)
        base = [mol_result(ctx, m) for m in range(len(mols))]
        ms = eses.eses_autotune(ctx, 2)
        assert ms[0] > 0.0 and ms[1] > 0.0
        assert eses.eses_get_option(ctx, eses.ESES_OPT_CLS_CTAS) >= 1
        assert eses.eses_get_option(ctx, eses.ESES_OPT_EDGE_CTAS) >= 1
        assert eses.eses_get_option(ctx, eses.ESES_OPT_ROOT_THREADS) in (128, 256)
        for m in range(len(mols)):
            same_result(mol_result(ctx, m), base[m], h, tau_tol=0.0)
    finally:
        eses.eses_destroy(ctx)


def test_batch_256_sampled_against_oracle():
    """The 256-molecule workload (atom counts log-uniform in [300, 20000],
    h = 0.5) in one context; three molecules (the smallest, a median one and
    the largest) are checked against the oracle on seeded 64-point blocks."""
    wl = inputs.WORKLOADS[3]
    sizes = inputs.batch_sizes()
    mols = [inputs.workload_atoms(3, molecule=m) for m in range(len(sizes))]
    ctx = eses.eses_create_batch(mols, wl.r_p, wl.h, wl.margin)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_GRAPH, 1)
        eses.eses_run(ctx)
        eses.eses_run(ctx)
        st = eses.eses_stats(ctx)
        assert st["root_failures"] == 0
        order = np.argsort(sizes)
        rng = np.random.default_rng(33)
        for m in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
            xyz, rad = mols[m]
            g = mol_result(ctx, m)
            a_, v_ = g["area"], g["volume"]
            assert a_ > 0 and v_ > 0
            dims = g["dims"]
            nb = [oracle.block_count(int(d), 64) for d in dims]
            # two seeded blocks that hold surface (between 2 % and 90 % of their
            # points inside; a molecule of one or two blocks gives all of them)
            surf = []
            for bid in range(nb[0] * nb[1] * nb[2]):
                b = (bid // (nb[1] * nb[2]), (bid // nb[2]) % nb[1], bid % nb[2])
                lo = np.array(b) * 63
                sl = g["labels"][lo[0]:lo[0] + 64, lo[1]:lo[1] + 64, lo[2]:lo[2] + 64]
                if 0.02 < sl.mean() < 0.9:
                    surf.append(bid)
            assert surf
            ids = sorted(int(v) for v in rng.choice(surf, size=min(2, len(surf)), replace=False))
            o = oracle.run(xyz, rad, wl.r_p, wl.h, wl.margin, block_pts=64, block_ids=ids)
            msk = o.labels >= 0
            assert np.array_equal(g["labels"][msk], o.labels[msk])
            for a in range(3):
                gi = g["axes"][a]["idx"]
                sel = msk.reshape(-1)[gi]
                srt = np.argsort(gi[sel], kind="stable")
                assert np.array_equal(gi[sel][srt], o.idx[a])
                if len(srt):
                    assert np.abs(g["axes"][a]["tau"][sel][srt] - o.tau[a]).max() * wl.h < TAU_TOL_A
    finally:
        eses.eses_destroy(ctx)
