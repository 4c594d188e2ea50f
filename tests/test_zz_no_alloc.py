"""The allocation-free crossing-edge entry point against the regular path.

eses_crossing_edges_noalloc serves callers that cannot call cudaMalloc (device
memory owned by a framework allocator or a fixed budget, or work issued where
allocation is not allowed): it takes a device label grid and caller-allocated
outputs, and keeps its own working memory in a fixed device array.  This test
runs the full path once through eses_run, then calls the entry point twice in
a row on the same device labels and requires the crossing-edge lists of both
calls to equal eses_intersections' exactly (same edges, same order).
"""
import numpy as np
import pytest

from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs

pytestmark = pytest.mark.gpu


def test_noalloc_crossing_edges_match_regular_path_twice():
    import torch

    libbuild.build()
    eses.load()
    xyz, rad = inputs.protein_like(400, 31, inputs.PROTEIN_DENSITY)
    ctx = eses.eses_create(xyz, rad, 1.4, 0.3, 0.8)
    try:
        eses.eses_run(ctx)
        dims, _ = eses.eses_grid(ctx)
        ref = [eses.eses_intersections(ctx, a)["idx"] for a in range(3)]
        labels_ptr = eses.eses_labels_device(ctx)
        cap = [len(r) + 64 for r in ref]
        for call in range(2):
            outs = [torch.full((c,), -1, dtype=torch.int64, device="cuda") for c in cap]
            counts = eses.eses_crossing_edges_noalloc(labels_ptr, dims, outs[0], outs[1], outs[2], cap)
            for a in range(3):
                assert counts[a] == len(ref[a]), (call, a)
                got = outs[a][: counts[a]].cpu().numpy()
                assert np.array_equal(got, ref[a]), (call, a)
                assert bool((outs[a][counts[a]:] == -1).all())
    finally:
        eses.eses_destroy(ctx)


def test_noalloc_rejects_oversized_grid_and_small_capacity():
    import torch

    libbuild.build()
    eses.load()
    dummy = torch.zeros(8, dtype=torch.int8, device="cuda")
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(eses.EsesError) as ei:
        eses.eses_crossing_edges_noalloc(dummy, [4096, 4096, 4096], out, out, out, [4, 4, 4])
    assert ei.value.code == eses.ESES_EINVAL
    lab = torch.zeros((10, 10, 10), dtype=torch.int8, device="cuda")
    lab[3:7, 3:7, 3:7] = 1
    with pytest.raises(eses.EsesError) as ei:
        eses.eses_crossing_edges_noalloc(lab, [10, 10, 10], out, out, out, [1, 1, 1])
    assert ei.value.code == eses.ESES_ECAPACITY
