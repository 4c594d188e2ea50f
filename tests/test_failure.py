"""Failure detection without a GPU fault.

* The proposer's tensor-core waits are bounded.  With ESES_OPT_TC_WAIT = 0
  every scoring wait gives up at once: eses_run must return ESES_ETIMEOUT,
  the tiles must go to the exact classification (labels and intersections
  equal to the oracle's), and the context must stay usable (the next run with
  the default limit succeeds with the same results).  The teardown wait keeps
  its full limit, so no tensor memory is freed under a multiply in flight.
* Device allocation failure is injected on the host (ESES_OPT_FAIL_ALLOC): the
  N-th allocation fails before cudaMalloc is called.  eses_run must return
  ESES_ENOMEM, a later run must succeed with exact results, and eses_destroy
  must give back every byte the context took.
"""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs
from paper_1809_04352_gb300 import proposer as prop

pytestmark = pytest.mark.gpu

RP, H, MARGIN = 1.4, 0.35, 0.8


@pytest.fixture(scope="module")
def case():
    libbuild.build()
    eses.load()
    xyz, rad = inputs.protein_like(700, 9101, inputs.PROTEIN_DENSITY)
    return xyz, rad, oracle.run(xyz, rad, RP, H, MARGIN, block_pts=16)


def _check_exact(ctx, ref):
    assert np.array_equal(eses.eses_labels(ctx), ref.labels)
    for a in range(3):
        got = eses.eses_intersections(ctx, a)
        order = np.argsort(got["idx"], kind="stable")
        assert np.array_equal(got["idx"][order], ref.idx[a])
        if len(order):
            assert np.abs(got["tau"][order] - ref.tau[a]).max() * H < 1e-6


def test_tensor_core_wait_timeout_falls_back_to_exact_path(case):
    xyz, rad, ref = case
    ctx = eses.eses_create(xyz, rad, RP, H, MARGIN)
    try:
        eses.eses_set_proposer(ctx, eses.ESES_PROPOSER_MLP, prop.load_params(), 0.5)
        eses.eses_set_option(ctx, eses.ESES_OPT_TC_WAIT, 0)
        with pytest.raises(eses.EsesError) as ei:
            eses.eses_run(ctx)
        assert ei.value.code == eses.ESES_ETIMEOUT
        _check_exact(ctx, ref)
        st = eses.eses_stats(ctx)
        assert st["tiles_proposed_far"] == 0  # no tile was scored: all went to the exact path
        eses.eses_set_option(ctx, eses.ESES_OPT_TC_WAIT, -1)
        eses.eses_run(ctx)
        _check_exact(ctx, ref)
        assert eses.eses_stats(ctx)["tiles_proposed_far"] > 0
    finally:
        eses.eses_destroy(ctx)


def test_allocation_failure_reports_enomem_and_destroy_releases_everything(case):
    import torch

    xyz, rad, ref = case
    torch.cuda.synchronize()
    # warm-up: kernels load lazily on first launch and keep their memory
    w = eses.eses_create(xyz, rad, RP, H, MARGIN)
    eses.eses_set_proposer(w, eses.ESES_PROPOSER_MLP, prop.load_params(), 0.5)
    eses.eses_run(w)
    eses.eses_mesh_count(w)
    eses.eses_destroy(w)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for n in (1, 2, 7, 20, 45):
        ctx = eses.eses_create(xyz, rad, RP, H, MARGIN)
        try:
            eses.eses_set_proposer(ctx, eses.ESES_PROPOSER_MLP, prop.load_params(), 0.5)
            eses.eses_set_option(ctx, eses.ESES_OPT_FAIL_ALLOC, n)
            with pytest.raises(eses.EsesError) as ei:
                eses.eses_run(ctx)
            assert ei.value.code == eses.ESES_ENOMEM, n
            assert eses.eses_get_option(ctx, eses.ESES_OPT_FAIL_ALLOC) == 0
            with pytest.raises(eses.EsesError) as ei:  # no results after a failed run
                eses.eses_labels(ctx)
            assert ei.value.code == eses.ESES_ESTATE
            eses.eses_run(ctx)  # the countdown has fired: the context recovers
            _check_exact(ctx, ref)
        finally:
            eses.eses_destroy(ctx)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert abs(free1 - free0) <= 1 << 20, (n, free0, free1)
