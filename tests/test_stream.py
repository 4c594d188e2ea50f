"""Grids run slab by slab (stream.py: block selections on two contexts and
two streams, results copied to the host per slab).

* A globule streamed in small slabs merges to the whole-grid run bit for bit.
* The 1,000,000-atom assembly at h = 0.1 A: 3.1e11 grid points, 312 GB of
  labels alone -- more than the device holds -- streamed in slabs; eight
  seeded 64-point blocks around surface atoms are kept by the sink and
  compared with the oracle (labels bit-exact, crossing edges equal,
  intersections within 1e-6 A).
"""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs, shard, stream
from paper_1809_04352_gb300 import proposer as prop

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    libbuild.build()
    return eses.load()


def test_streamed_slabs_merge_to_the_whole_run():
    xyz, rad = inputs.protein_like(2000, 81, inputs.PROTEIN_DENSITY)
    ctx = eses.eses_create(xyz, rad, 1.4, 0.3, 0.8)
    try:
        eses.eses_run(ctx)
        dims, _ = eses.eses_grid(ctx)
        whole = dict(labels=eses.eses_labels(ctx), axes=[eses.eses_intersections(ctx, a, fp32=False)
                                                         for a in range(3)], av=eses.eses_area_volume(ctx))
    finally:
        eses.eses_destroy(ctx)
    parts = {}

    def sink(k, p):
        p.labels = p.labels.copy().reshape(-1)  # the pinned buffer is reused
        parts[k] = p

    tot = stream.stream(xyz, rad, 1.4, 0.3, 0.8, sink, max_points=int(np.prod(dims)) // 5, block_pts=16)
    assert tot["slabs"] >= 5 and tot["points"] == int(np.prod(dims))
    lab, idx, tau, nrm, area, vol = shard.combine([parts[k] for k in sorted(parts)], dims)
    assert np.array_equal(lab, whole["labels"])
    for a in range(3):
        o = np.argsort(whole["axes"][a]["idx"], kind="stable")
        assert np.array_equal(idx[a], whole["axes"][a]["idx"][o])
        assert np.array_equal(tau[a], whole["axes"][a]["tau"][o])
        assert np.array_equal(nrm[a], whole["axes"][a]["normal"][o])
    assert abs(area - whole["av"][0]) <= 1e-12 * whole["av"][0]
    assert abs(vol - whole["av"][1]) <= 1e-12 * whole["av"][1]


def test_assembly_beyond_device_memory_streamed_sampled_blocks_match_oracle():
    import torch

    xyz, rad = inputs.workload_atoms(5)
    h, rp, margin = 0.1, 1.4, 0.8
    dims, lo = oracle.grid(xyz, rad, h, margin)
    npts = int(np.prod(dims))
    assert npts > torch.cuda.get_device_properties(0).total_memory  # labels alone exceed the device
    # eight seeded 64-point blocks (63 cells, shared faces) around atoms far
    # from their copy's centre, i.e. near the surface
    ncopy = 60
    per = len(xyz) // ncopy
    rng = np.random.default_rng(505)
    nb = [oracle.block_count(int(d), 64) for d in dims]
    ids = []
    while len(ids) < 8:
        c = int(rng.integers(ncopy))
        x = xyz[c * per:(c + 1) * per]
        d = np.linalg.norm(x - x.mean(0), axis=1)
        cand = np.flatnonzero(d > 0.92 * d.max())
        p = x[int(rng.choice(cand))]
        b = np.minimum(((p - lo) / (63 * h)).astype(np.int64), np.array(nb) - 1)
        bid = int((b[0] * nb[1] + b[1]) * nb[2] + b[2])
        if bid not in ids:
            ids.append(bid)
    ids.sort()
    odims, olo, oblocks, oidx, otau, _ = oracle.run_blocks(xyz, rad, rp, h, margin, 64, ids)
    assert np.array_equal(odims, dims)
    kept_lab = [np.full(tuple(int(v) for v in bhi - blo), -1, np.int8) for blo, bhi, _ in oblocks]
    kept = [[[], []] for _ in range(3)]  # per axis: idx, tau

    def in_blocks(idx):
        g = np.stack([idx // (dims[1] * dims[2]), (idx // dims[2]) % dims[1], idx % dims[2]], 1)
        m = np.zeros(len(idx), bool)
        for blo, bhi, _ in oblocks:
            m |= np.all((g >= blo) & (g < bhi), axis=1)
        return m

    def sink(k, part):
        plo, phi = part.lo, part.lo + part.dims
        for t, (blo, bhi, _) in enumerate(oblocks):
            a0, a1 = np.maximum(plo, blo), np.minimum(phi, bhi)
            if np.any(a1 <= a0):
                continue
            kept_lab[t][a0[0] - blo[0]:a1[0] - blo[0], a0[1] - blo[1]:a1[1] - blo[1], a0[2] - blo[2]:a1[2] - blo[2]] = \
                part.labels[a0[0] - plo[0]:a1[0] - plo[0], a0[1] - plo[1]:a1[1] - plo[1], a0[2] - plo[2]:a1[2] - plo[2]]
        for a in range(3):
            m = in_blocks(part.idx[a])
            kept[a][0].append(part.idx[a][m])
            kept[a][1].append(part.tau[a][m])

    tot = stream.stream(xyz, rad, rp, h, margin, sink, max_points=6 << 30, block_pts=128,
                        proposer_params=prop.load_params())
    assert tot["points"] == npts
    assert tot["crossing_edges"] > 1e9 and tot["area"] > 0 and tot["volume"] > 0
    for t, (blo, bhi, olab) in enumerate(oblocks):
        assert np.array_equal(kept_lab[t], olab), t
    for a in range(3):
        gi = np.concatenate(kept[a][0])
        gt = np.concatenate(kept[a][1])
        order = np.argsort(gi, kind="stable")
        assert np.array_equal(gi[order], oidx[a])
        assert np.abs(gt[order] - otau[a]).max() * h < 1e-6
