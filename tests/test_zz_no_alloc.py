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


def _reference_edges(lab):
    """Crossing edges of a host label grid in the library's order: 8x8x8 tiles
    in C order, then C order of the lower point inside its tile."""
    dims = lab.shape
    out = []
    for a in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, dims[a] - 1)
        hi[a] = slice(1, dims[a])
        g = np.argwhere(lab[tuple(lo)] != lab[tuple(hi)]).astype(np.int64)
        t = g // 8
        l = g % 8
        tile = (t[:, 0] * ((dims[1] + 7) // 8) + t[:, 1]) * ((dims[2] + 7) // 8) + t[:, 2]
        loc = (l[:, 0] * 8 + l[:, 1]) * 8 + l[:, 2]
        order = np.lexsort((loc, tile))
        idx = (g[:, 0] * dims[1] + g[:, 1]) * dims[2] + g[:, 2]
        out.append(idx[order])
    return out


def test_noalloc_on_a_user_stream_at_the_largest_grid():
    """A grid of exactly 131,072 tiles (the largest accepted: 256 x 512 x 512
    points) on a stream the caller created, twice in a row, against the
    crossing edges numpy finds in the same labels."""
    import torch

    libbuild.build()
    eses.load()
    dims = (256, 512, 512)
    rng = np.random.default_rng(77)
    lab = np.zeros(dims, np.int8)
    for _ in range(24):
        c = rng.uniform([0, 0, 0], dims)
        r = rng.uniform(10, 60)
        lo = [max(0, int(c[a] - r) - 1) for a in range(3)]
        hi = [min(dims[a], int(c[a] + r) + 2) for a in range(3)]
        z, y, x = np.ogrid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
        ball = ((z - c[0]) ** 2 + (y - c[1]) ** 2 + (x - c[2]) ** 2) <= r * r
        lab[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] |= ball.astype(np.int8)
    ref = _reference_edges(lab)
    dlab = torch.from_numpy(lab).cuda()
    cap = [len(r) + 16 for r in ref]
    st = torch.cuda.Stream()
    for call in range(2):
        outs = [torch.full((c,), -1, dtype=torch.int64, device="cuda") for c in cap]
        torch.cuda.synchronize()
        counts = eses.eses_crossing_edges_noalloc(dlab, dims, outs[0], outs[1], outs[2], cap, stream=st.cuda_stream)
        for a in range(3):
            assert counts[a] == len(ref[a]), (call, a)
            assert np.array_equal(outs[a][: counts[a]].cpu().numpy(), ref[a]), (call, a)
            assert bool((outs[a][counts[a]:] == -1).all())


def test_noalloc_short_capacity_writes_the_leading_edges():
    """Under ESES_ECAPACITY the first capacity[a] edges of each axis are
    written, in order, and nothing past them."""
    import torch

    libbuild.build()
    eses.load()
    dims = (20, 17, 33)
    rng = np.random.default_rng(5)
    lab = (rng.random(dims) < 0.3).astype(np.int8)
    ref = _reference_edges(lab)
    dlab = torch.from_numpy(lab).cuda()
    cap = [len(ref[0]) // 3, 7, len(ref[2])]
    outs = [torch.full((c + 8,), -1, dtype=torch.int64, device="cuda") for c in cap]
    import ctypes
    lib = eses.load()
    d = np.asarray(dims, np.int64)
    c = np.asarray(cap, np.int64)
    counts = np.zeros(3, np.int64)
    rc = lib.eses_crossing_edges_noalloc(ctypes.c_void_p(dlab.data_ptr()), d.ctypes.data,
                                         *[ctypes.c_void_p(o.data_ptr()) for o in outs], c.ctypes.data,
                                         counts.ctypes.data, None)
    assert rc == eses.ESES_ECAPACITY
    for a in range(3):
        assert counts[a] == len(ref[a])
        assert np.array_equal(outs[a][: cap[a]].cpu().numpy(), ref[a][: cap[a]]), a
        assert bool((outs[a][cap[a]:] == -1).all()), a
