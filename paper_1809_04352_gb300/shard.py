"""One molecule's grid split over ranks by blocks, and the merge of the parts.

The paper computes its blocks independently, each from the atoms near it
(§2.2-2.5, Algorithm 1), and concatenates their outputs in one ordered step.
Here the same independence splits one molecule over P processes:

* ``block_costs``: an estimate of each block's work from the atoms whose
  reach (r + 2 r_p) meets it -- empty blocks cost their points, blocks near
  atoms cost in proportion to those atoms (a cheap host count, no surface
  arithmetic);
* ``partition``: P slabs of whole block layers along axis 0 with about equal
  summed cost (prefix sums of the layer costs);
* ``halo_atoms``: the atoms a slab needs -- every atom within r + 2 r_p of
  the box its run computes (the owned blocks and one 8-point layer beyond
  them), by the locality of §2.2 (nothing farther changes a point);
* ``combine`` and ``merge``: the parts' owned labels placed in the grid,
  intersections concatenated in rank order and then put in lower-index
  order, area and volume summed.  ``merge`` does it across ranks with
  collectives: an all-reduce of (area, volume) as two float64, an all-gather
  of the per-axis intersection counts, their exclusive scan for each rank's
  offsets, and an all-gatherv (padded all-gather) of the intersections; the
  owned label boxes go to every rank the same way when asked for.

This module holds no surface arithmetic: each rank's part comes from the
library (``eses_create_on_grid`` on the halo atoms, ``eses_set_blocks`` on
its slab), or from any function with the same outputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Part:
    """One rank's results: the owned box and its labels, the owned edges'
    intersections (full-grid lower indices), and the owned area and volume."""
    lo: np.ndarray                      # first owned point (3,)
    dims: np.ndarray                    # owned extent (3,)
    labels: np.ndarray                  # int8 owned box, C order
    idx: list = field(default_factory=lambda: [np.zeros(0, np.int64)] * 3)
    tau: list = field(default_factory=lambda: [np.zeros(0)] * 3)
    normal: list = field(default_factory=lambda: [np.zeros((0, 3))] * 3)
    area: float = 0.0
    volume: float = 0.0


def n_blocks(dims, block_pts: int) -> np.ndarray:
    return np.array([-(-int(d) // block_pts) for d in dims], np.int64)


def block_costs(xyz, radii, r_p: float, h: float, origin, dims, block_pts: int, atom_weight: float = 64.0):
    """Cost estimate per block (nb0, nb1, nb2): points owned + atom_weight *
    (atoms whose reach r + 2 r_p meets the block) * points / block_pts^3."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    radii = np.asarray(radii, np.float64).reshape(-1)
    origin = np.asarray(origin, np.float64)
    dims = np.asarray(dims, np.int64)
    nb = n_blocks(dims, block_pts)
    edge = block_pts * h
    touch = np.zeros(tuple(nb), np.float64)
    reach = radii + 2.0 * r_p
    lo = np.floor((xyz - reach[:, None] - origin) / edge).astype(np.int64)
    hi = np.floor((xyz + reach[:, None] - origin) / edge).astype(np.int64)
    lo = np.clip(lo, 0, nb - 1)
    hi = np.clip(hi, 0, nb - 1)
    for i in range(xyz.shape[0]):  # each atom adds one to the blocks its reach box meets
        touch[lo[i, 0]:hi[i, 0] + 1, lo[i, 1]:hi[i, 1] + 1, lo[i, 2]:hi[i, 2] + 1] += 1.0
    pts = np.ones(tuple(nb), np.float64)
    for a in range(3):
        ext = np.full(nb[a], float(block_pts))
        ext[-1] = float(dims[a] - block_pts * (nb[a] - 1))
        shape = [1, 1, 1]
        shape[a] = nb[a]
        pts = pts * ext.reshape(shape)
    return pts * (1.0 + atom_weight * touch / float(block_pts) ** 3)


def partition(costs: np.ndarray, n_ranks: int):
    """Slabs of whole block layers along axis 0, one per rank, cutting the
    prefix sums of the layer costs at equal fractions.  Returns a list of
    (block_lo (3,), block_hi (3,)) or None for a rank left without layers."""
    nb = np.array(costs.shape, np.int64)
    layer = costs.sum(axis=(1, 2))
    cum = np.concatenate([[0.0], np.cumsum(layer)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, n_ranks):
        target = total * r / n_ranks
        k = int(np.searchsorted(cum, target, side="left"))
        # the nearer of the two layer boundaries around the target
        if k > 0 and abs(cum[k - 1] - target) <= abs(cum[min(k, nb[0])] - target):
            k -= 1
        cuts.append(int(min(max(k, cuts[-1]), nb[0])))
    cuts.append(int(nb[0]))
    out = []
    for r in range(n_ranks):
        a, b = cuts[r], cuts[r + 1]
        out.append(None if b <= a else (np.array([a, 0, 0], np.int64), np.array([b, nb[1], nb[2]], np.int64)))
    return out


def computed_box(dims, block_pts: int, block_lo, block_hi):
    """Points [lo, hi) that a run of the blocks [block_lo, block_hi) labels:
    the owned points plus one 8-point tile layer beyond them, clipped."""
    dims = np.asarray(dims, np.int64)
    lo = np.asarray(block_lo, np.int64) * block_pts
    own_hi = np.minimum(np.asarray(block_hi, np.int64) * block_pts, dims)
    hi = np.minimum(-(-own_hi // 8) * 8 + 8, dims)
    return lo, hi


def halo_atoms(xyz, radii, r_p: float, h: float, origin, dims, block_pts: int, block_lo, block_hi,
               slack: float = 1e-3) -> np.ndarray:
    """Indices of the atoms within r + 2 r_p (+ slack) of the computed box of
    the blocks [block_lo, block_hi)."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    radii = np.asarray(radii, np.float64).reshape(-1)
    origin = np.asarray(origin, np.float64)
    lo, hi = computed_box(dims, block_pts, block_lo, block_hi)
    b0 = origin + h * lo
    b1 = origin + h * (hi - 1)
    e = np.maximum(0.0, np.maximum(b0 - xyz, xyz - b1))
    d2 = np.einsum("ij,ij->i", e, e)
    reach = radii + 2.0 * r_p + slack
    return np.flatnonzero(d2 < reach * reach)


def combine(parts, dims, labels: bool = True):
    """Merge parts in rank order: (labels of the whole grid or None, idx, tau,
    normal per axis in lower-index order, area, volume).  Area and volume are
    summed in rank order."""
    dims = np.asarray(dims, np.int64)
    lab = None
    if labels:
        lab = np.full(tuple(int(d) for d in dims), -1, np.int8)
        for p in parts:
            lo, ext = p.lo, p.dims
            lab[lo[0]:lo[0] + ext[0], lo[1]:lo[1] + ext[1], lo[2]:lo[2] + ext[2]] = p.labels.reshape(tuple(ext))
    idx, tau, nrm = [], [], []
    for a in range(3):
        i = np.concatenate([p.idx[a] for p in parts]) if parts else np.zeros(0, np.int64)
        t = np.concatenate([p.tau[a] for p in parts]) if parts else np.zeros(0)
        n = np.concatenate([p.normal[a].reshape(-1, 3) for p in parts]) if parts else np.zeros((0, 3))
        order = np.argsort(i, kind="stable")
        idx.append(i[order]); tau.append(t[order]); nrm.append(n[order])
    area = math.fsum(p.area for p in parts)
    volume = math.fsum(p.volume for p in parts)
    return lab, idx, tau, nrm, area, volume


def _gatherv(dist, arr: np.ndarray, torch):
    """All-gatherv of a 1-D array by a padded all-gather: every rank's array,
    in rank order."""
    world = dist.get_world_size()
    n = torch.tensor([arr.shape[0]], dtype=torch.int64)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, n)
    counts = [int(c.item()) for c in counts]
    width = max(max(counts), 1)
    buf = torch.zeros(width, dtype=torch.from_numpy(arr[:0]).dtype)
    if arr.shape[0]:
        buf[: arr.shape[0]] = torch.from_numpy(np.ascontiguousarray(arr))
    outs = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf)
    return [o[:c].numpy() for o, c in zip(outs, counts)], counts


def merge(part: Part | None, dims, gather_labels: bool = True):
    """Merge every rank's part over torch.distributed (call on every rank; a
    rank without blocks passes None).  Returns, on every rank: (labels of the
    whole grid or None, idx, tau, normal per axis in lower-index order, area,
    volume, offsets) where offsets[a][r] is rank r's first record in axis a's
    rank-order concatenation (the exclusive scan of the gathered counts)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size()
    if part is None:
        part = Part(lo=np.zeros(3, np.int64), dims=np.zeros(3, np.int64), labels=np.zeros(0, np.int8))
    av = torch.tensor([part.area, part.volume], dtype=torch.float64)
    dist.all_reduce(av)  # (area, volume): 2 x f64
    cnt = torch.tensor([len(part.idx[a]) for a in range(3)], dtype=torch.int64)
    allc = [torch.zeros(3, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allc, cnt)
    counts = np.stack([c.numpy() for c in allc])            # (world, 3)
    offsets = np.vstack([np.zeros((1, 3), np.int64), np.cumsum(counts, axis=0)])[:-1].T  # exclusive scan
    parts = [Part(lo=np.zeros(3, np.int64), dims=np.zeros(3, np.int64), labels=np.zeros(0, np.int8))
             for _ in range(world)]
    for a in range(3):
        gi, _ = _gatherv(dist, np.asarray(part.idx[a], np.int64), torch)
        gt, _ = _gatherv(dist, np.asarray(part.tau[a], np.float64), torch)
        gn, _ = _gatherv(dist, np.asarray(part.normal[a], np.float64).reshape(-1), torch)
        for r in range(world):
            assert gi[r].shape[0] == counts[r, a]
            parts[r].idx = parts[r].idx[:a] + [gi[r]] + parts[r].idx[a + 1:]
            parts[r].tau = parts[r].tau[:a] + [gt[r]] + parts[r].tau[a + 1:]
            parts[r].normal = parts[r].normal[:a] + [gn[r].reshape(-1, 3)] + parts[r].normal[a + 1:]
    if gather_labels:
        box = torch.from_numpy(np.concatenate([np.asarray(part.lo, np.int64), np.asarray(part.dims, np.int64)]))
        boxes = [torch.zeros(6, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(boxes, box)
        gl, _ = _gatherv(dist, np.asarray(part.labels, np.int8).reshape(-1), torch)
        for r in range(world):
            b = boxes[r].numpy()
            parts[r].lo, parts[r].dims, parts[r].labels = b[:3], b[3:], gl[r]
        keep = [p for p in parts if int(np.prod(p.dims)) > 0]
    else:
        keep = parts
    lab, idx, tau, nrm, _, _ = combine(keep, dims, labels=gather_labels)
    return lab, idx, tau, nrm, float(av[0]), float(av[1]), offsets


def run_part(eses, xyz, radii, r_p: float, h: float, origin, dims, block_pts: int, block_lo, block_hi) -> Part:
    """One rank's part on its GPU: the halo atoms of its blocks on the
    molecule's grid, run on the blocks, results copied to the host."""
    sel = halo_atoms(xyz, radii, r_p, h, origin, dims, block_pts, block_lo, block_hi)
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    radii = np.asarray(radii, np.float64).reshape(-1)
    ctx = eses.eses_create_on_grid(xyz[sel], radii[sel], r_p, h, origin, dims)
    try:
        eses.eses_set_option(ctx, eses.ESES_OPT_BLOCK_PTS, block_pts)
        eses.eses_set_blocks(ctx, block_lo, block_hi)
        eses.eses_run(ctx)
        lo, ext = eses.eses_owned_box(ctx)
        part = Part(lo=lo, dims=ext, labels=eses.eses_labels(ctx).reshape(-1))
        axes = [eses.eses_intersections(ctx, a, fp32=False) for a in range(3)]
        part.idx = [x["idx"] for x in axes]
        part.tau = [x["tau"] for x in axes]
        part.normal = [x["normal"] for x in axes]
        part.area, part.volume = eses.eses_area_volume(ctx)
    finally:
        eses.eses_destroy(ctx)
    return part
