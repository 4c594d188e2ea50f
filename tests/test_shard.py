"""One molecule split over ranks (§2.2-2.5: blocks are independent) and merged.

CPU tests (gloo, world sizes 2 and 3): every rank takes a slab of the block
partition, keeps only its halo atoms, computes its part with the oracle on
the molecule's own grid (the compute is injected: the library does this on a
GPU), and the parts are merged with the collectives of ``shard.merge``.  The
merged labels, crossing edges, intersections and normals must equal the
single oracle run bit for bit; area and volume (sums in another order) to
1e-12 relative.  A rank missing an atom it needs, a partition with a gap or
an overlap, or a merge that drops or repeats records fails.
"""
import math
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import inputs, shard

RP, H, B = 1.4, 0.4, 16


def _molecule():
    return inputs.protein_like(160, 61, inputs.PROTEIN_DENSITY)


def oracle_part(xyz, rad, origin, dims, blo, bhi):
    """A rank's part from the oracle: its halo atoms only, on the molecule's
    grid; the owned box, the owned edges (lower point owned) and their C9
    area and volume terms."""
    sel = shard.halo_atoms(xyz, rad, RP, H, origin, dims, B, blo, bhi)
    res = oracle.run_on_grid(xyz[sel], rad[sel], RP, H, origin, dims, ids=sel, block_pts=16)
    lo = np.asarray(blo) * B
    hi = np.minimum(np.asarray(bhi) * B, dims)
    lab = res.labels[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
    part = shard.Part(lo=lo, dims=hi - lo, labels=lab.reshape(-1).copy())
    idx, tau, nrm = [], [], []
    area = 0.0
    lines = 0.0
    full = res.labels
    for a in range(3):
        i = res.idx[a]
        g = np.stack([i // (dims[1] * dims[2]), (i // dims[2]) % dims[1], i % dims[2]], 1)
        own = np.all((g >= lo) & (g < hi), axis=1)
        idx.append(i[own]); tau.append(res.tau[a][own]); nrm.append(res.normal[a][own])
        area += H * H * float(np.abs(res.normal[a][own][:, a]).sum())
        ls = full.reshape(-1)[i[own]]
        lines += float(np.where(ls == 1, tau[-1] * H, (1.0 - tau[-1]) * H).sum())
        # edges with both ends inside and the lower point owned
        sl = [slice(lo[0], hi[0]), slice(lo[1], hi[1]), slice(lo[2], hi[2])]
        nx = list(sl)
        nx[a] = slice(lo[a] + 1, min(hi[a] + 1, dims[a]))
        cut = list(sl)
        cut[a] = slice(lo[a], min(hi[a], dims[a] - 1))
        lines += H * float(((full[tuple(cut)] == 1) & (full[tuple(nx)] == 1)).sum())
    part.idx, part.tau, part.normal = idx, tau, nrm
    part.area = area
    part.volume = H * H * lines / 3.0
    return part


def test_partition_covers_every_block_once_and_balances():
    rng = np.random.default_rng(3)
    for trial in range(20):
        nb = rng.integers(1, 12, size=3)
        costs = rng.random(tuple(nb)) * rng.integers(1, 100)
        for P in range(1, 6):
            slabs = shard.partition(costs, P)
            assert len(slabs) == P
            seen = np.zeros(tuple(nb), np.int64)
            loads = []
            for s in slabs:
                if s is None:
                    continue
                lo, hi = s
                seen[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += 1
                loads.append(costs[lo[0]:hi[0]].sum())
            assert np.all(seen == 1)
            layer_max = costs.sum(axis=(1, 2)).max()
            assert max(loads) <= costs.sum() / P + layer_max + 1e-9


def test_halo_atoms_keep_every_atom_that_reaches_the_box():
    xyz, rad = _molecule()
    dims, origin = oracle.grid(xyz, rad, H, 0.8)
    nb = shard.n_blocks(dims, B)
    blo, bhi = np.array([1, 0, 1]), np.array([2, nb[1], 2])
    sel = set(shard.halo_atoms(xyz, rad, RP, H, origin, dims, B, blo, bhi).tolist())
    lo, hi = shard.computed_box(dims, B, blo, bhi)
    # brute force over the box's points
    g = np.stack(np.meshgrid(*[np.arange(lo[a], hi[a]) for a in range(3)], indexing="ij"), -1).reshape(-1, 3)
    pts = origin + H * g
    for i in range(len(xyz)):
        near = np.min(np.linalg.norm(pts - xyz[i], axis=1)) < rad[i] + 2 * RP
        if near:
            assert i in sel


def test_single_process_merge_equals_the_whole_run():
    xyz, rad = _molecule()
    full = oracle.run(xyz, rad, RP, H, 0.8, block_pts=16)
    dims, origin = full.dims, full.lo
    costs = shard.block_costs(xyz, rad, RP, H, origin, dims, B)
    parts = [oracle_part(xyz, rad, origin, dims, lo, hi) for lo, hi in
             (s for s in shard.partition(costs, 3) if s is not None)]
    lab, idx, tau, nrm, area, vol = shard.combine(parts, dims)
    _same(full, lab, idx, tau, nrm, area, vol)


def _same(full, lab, idx, tau, nrm, area, vol):
    assert np.array_equal(lab, full.labels)
    for a in range(3):
        assert np.array_equal(idx[a], full.idx[a])
        assert np.array_equal(tau[a], full.tau[a])  # bit for bit
        assert np.array_equal(nrm[a], full.normal[a])
    assert abs(area - full.area) <= 1e-12 * full.area
    assert abs(vol - full.volume) <= 1e-12 * full.volume


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        xyz, rad = _molecule()
        dims, origin = oracle.grid(xyz, rad, H, 0.8)
        costs = shard.block_costs(xyz, rad, RP, H, origin, dims, B)
        slab = shard.partition(costs, world)[rank]
        part = None if slab is None else oracle_part(xyz, rad, origin, dims, slab[0], slab[1])
        lab, idx, tau, nrm, area, vol, offs = shard.merge(part, dims)
        if rank == 0:
            np.savez(os.path.join(out_dir, "merged.npz"), lab=lab, area=area, vol=vol, offs=offs,
                     **{f"idx{a}": idx[a] for a in range(3)}, **{f"tau{a}": tau[a] for a in range(3)},
                     **{f"nrm{a}": nrm[a] for a in range(3)})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_merge_to_the_whole_run(world, tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    m = np.load(tmp_path / "merged.npz")
    xyz, rad = _molecule()
    full = oracle.run(xyz, rad, RP, H, 0.8, block_pts=16)
    _same(full, m["lab"], [m[f"idx{a}"] for a in range(3)], [m[f"tau{a}"] for a in range(3)],
          [m[f"nrm{a}"] for a in range(3)], float(m["area"]), float(m["vol"]))
    offs = m["offs"]
    assert offs.shape == (3, world) and np.all(offs[:, 0] == 0)
