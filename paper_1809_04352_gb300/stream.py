"""Grids larger than the device, run slab by slab (the paper's out-of-core
blocks, §2.3 and §3: memory bounded by the block, not by the grid).

``stream`` splits the molecule's grid into slabs of whole block layers along
axis 0 (at most ``max_points`` points each, ESES_OPT_BLOCK_PTS-point blocks)
and runs them with ``n_buffers`` contexts that hold the same atoms and the
same grid, each on its own CUDA stream and driven by its own host thread:
while one context computes a slab, the others copy their last slab's labels
and intersections to host memory and hand them to the caller's sink.  Device
memory is the model of the atoms plus ``n_buffers`` slabs, whatever the
grid's size; host memory is one pinned label buffer and the intersections of
a slab per context, unless the sink keeps more.

The sink is called as sink(slab_index, part) with a ``shard.Part`` (owned box,
its labels -- a view into a reused pinned buffer, valid during the call --,
the owned intersections with full-grid lower indices, area and volume); calls
may come from several threads and out of slab order, and are serialised by a
lock.  This module only drives the library; it holds no surface arithmetic.
"""
from __future__ import annotations

import threading

import numpy as np

from . import eses
from .shard import Part


def slabs(dims, block_pts: int, max_points: int):
    """Block ranges [(lo, hi), ...] of slabs of whole block layers along axis 0,
    each owning at most max_points points (at least one layer)."""
    dims = np.asarray(dims, np.int64)
    nb = [-(-int(d) // block_pts) for d in dims]
    layer_pts = block_pts * int(dims[1]) * int(dims[2])
    per = max(1, int(max_points) // max(layer_pts, 1))
    out = []
    for b0 in range(0, nb[0], per):
        b1 = min(nb[0], b0 + per)
        out.append((np.array([b0, 0, 0], np.int64), np.array([b1, nb[1], nb[2]], np.int64)))
    return out


def stream(xyz, radii, r_p: float, h: float, margin: float, sink, max_points: int = 1 << 31,
           block_pts: int = 64, n_buffers: int = 2, proposer_params=None, precision=None):
    """Run every slab of the molecule's grid and pass each to sink(k, part).
    Returns a dict with the grid (dims, origin), the slab count and the
    summed points, crossing edges, area and volume."""
    import torch

    ctxs = []
    try:
        for _ in range(n_buffers):
            c = eses.eses_create(xyz, radii, r_p, h, margin)
            ctxs.append(c)
            eses.eses_set_option(c, eses.ESES_OPT_BLOCK_PTS, block_pts)
            if precision is not None:
                eses.eses_set_option(c, eses.ESES_OPT_PRECISION, precision)
            if proposer_params is not None:
                eses.eses_set_proposer(c, eses.ESES_PROPOSER_MLP, proposer_params, 0.5)
        dims, origin = eses.eses_grid(ctxs[0])
        work = slabs(dims, block_pts, max_points)
        lab_cap = max(int(np.prod(np.minimum(hi * block_pts, dims) - lo * block_pts)) for lo, hi in work)
        lock = threading.Lock()
        errors = []
        totals = {"points": 0, "crossing_edges": 0, "area": 0.0, "volume": 0.0}

        def worker(t):
            ctx = ctxs[t]
            buf = torch.empty(lab_cap, dtype=torch.int8).pin_memory()
            try:
                for k in range(t, len(work), n_buffers):
                    lo, hi = work[k]
                    eses.eses_set_blocks(ctx, lo, hi)
                    eses.eses_run(ctx)
                    blo, ext = eses.eses_owned_box(ctx)
                    n = int(np.prod(ext))
                    lab = buf.numpy()[:n].reshape(tuple(int(v) for v in ext))
                    eses.eses_labels(ctx, lab)
                    part = Part(lo=blo, dims=ext, labels=lab)
                    axes = [eses.eses_intersections(ctx, a, fp32=False) for a in range(3)]
                    part.idx = [x["idx"] for x in axes]
                    part.tau = [x["tau"] for x in axes]
                    part.normal = [x["normal"] for x in axes]
                    part.area, part.volume = eses.eses_area_volume(ctx)
                    with lock:
                        totals["points"] += n
                        totals["crossing_edges"] += sum(len(x) for x in part.idx)
                        totals["area"] += part.area
                        totals["volume"] += part.volume
                        sink(k, part)
            except Exception as e:  # re-raised on the calling thread
                with lock:
                    errors.append(e)

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(n_buffers)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errors:
            raise errors[0]
        totals.update(dims=dims, origin=origin, slabs=len(work), block_pts=block_pts, max_points=int(max_points))
        return totals
    finally:
        for c in ctxs:
            eses.eses_destroy(c)
