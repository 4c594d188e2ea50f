"""The 1,000,000-atom assembly (60 rotated copies of a 16,667-atom globule on
an icosahedral shell of radius 300 A, h = 0.3 A, ~1.3e10 grid points) in one
context on one GPU -- its 13 GB of labels fit in HBM, so no block streaming
-- checked against the oracle on 64 seeded 64-point blocks: 32 around seeded
atoms (surface-rich) and 32 anywhere in the grid."""
import numpy as np
import pytest

import oracle
from paper_1809_04352_gb300 import build as libbuild
from paper_1809_04352_gb300 import eses, inputs, proposer
from tests.test_gpu_parity import TAU_TOL_A

pytestmark = pytest.mark.gpu


class _DevView:
    """A device array (pointer, element count, dtype) for torch.as_tensor."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _dev(ptr, n, typestr):
    import torch
    return torch.as_tensor(_DevView(ptr, n, typestr), device="cuda")


def test_assembly_1M_sampled_blocks_match_oracle():
    libbuild.build()
    wl = inputs.WORKLOADS[5]
    xyz, rad = inputs.workload_atoms(5)
    assert xyz.shape[0] == 60 * 16667
    ctx = eses.eses_create(xyz, rad, wl.r_p, wl.h, wl.margin)
    try:
        eses.eses_set_proposer(ctx, eses.ESES_PROPOSER_MLP, proposer.load_params(), 0.5)
        eses.eses_run(ctx)
        st = eses.eses_stats(ctx)
        assert st["root_failures"] == 0
        dims, lo = eses.eses_grid(ctx)
        npts = int(np.prod(dims))
        assert npts > 1e10
        lab = _dev(eses.eses_labels_device(ctx), npts, "|i1").view(*[int(d) for d in dims])
        edges = []
        for a in range(3):
            n = eses.eses_num_intersections(ctx, a)
            pi, pt, _, _, _ = eses.eses_intersections_device(ctx, a)
            edges.append((_dev(pi, n, "<i8"), _dev(pt, n, "<f8")))
        nb = [oracle.block_count(int(d), 64) for d in dims]
        rng = np.random.default_rng(5050)
        ids = set()
        for k in rng.choice(xyz.shape[0], size=32, replace=False):
            g = np.floor((xyz[k] - lo) / wl.h).astype(np.int64)
            b = np.minimum(g // 63, np.array(nb) - 1)
            ids.add(int((b[0] * nb[1] + b[1]) * nb[2] + b[2]))
        while len(ids) < 64:
            ids.add(int(rng.integers(nb[0] * nb[1] * nb[2])))
        ids = sorted(ids)
        odims, olo, blocks, oidx, otau, _ = oracle.run_blocks(xyz, rad, wl.r_p, wl.h, wl.margin, 64, ids)
        assert np.array_equal(odims, dims) and np.array_equal(olo, lo)
        inside = 0
        for blo, bhi, blab in blocks:
            g = lab[blo[0]:bhi[0], blo[1]:bhi[1], blo[2]:bhi[2]].cpu().numpy()
            assert np.array_equal(g, blab)
            inside += int(blab.sum())
        assert inside > 0
        s0, s1 = int(dims[1] * dims[2]), int(dims[2])
        for a in range(3):
            gi, gt = edges[a]
            i0, i1, i2 = gi // s0, (gi // s1) % int(dims[1]), gi % s1
            sel = None
            for blo, bhi, _ in blocks:
                m = ((i0 >= int(blo[0])) & (i0 < int(bhi[0])) & (i1 >= int(blo[1])) & (i1 < int(bhi[1])) &
                     (i2 >= int(blo[2])) & (i2 < int(bhi[2])))
                sel = m if sel is None else (sel | m)
            gsel = gi[sel].cpu().numpy()
            tsel = gt[sel].cpu().numpy()
            order = np.argsort(gsel, kind="stable")
            assert np.array_equal(gsel[order], oidx[a])
            if len(order):
                assert np.abs(tsel[order] - otau[a]).max() * wl.h < TAU_TOL_A
    finally:
        eses.eses_destroy(ctx)
