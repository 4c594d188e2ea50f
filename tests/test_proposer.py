"""The learned tile proposer: MLP kernels against the FP64 oracle of the MLP,
the oracle's gradient against finite differences, tile data, and exactness
of every proposer mode (the labels and intersections never depend on the
network: far calls are certified, everything else is classified exactly).
"""
import numpy as np
import pytest

import oracle.mlp_oracle as mo

RNG = np.random.default_rng


def _data(n, seed):
    rng = RNG(seed)
    X = rng.normal(0.0, 1.0, (n, 32))
    y = (rng.random(n) < 0.3).astype(np.float64)
    w = rng.random(n) / n
    p = rng.normal(0.0, 0.25, mo.N_PARAM)
    return p, X, y, w


def test_mlp_oracle_gradient_matches_finite_differences():
    """Central differences of the loss (fp64) on a sample of parameters of
    every block: a dropped term, wrong index or transposed weight in the
    analytic chain rule fails this."""
    p, X, y, w = _data(40, 1)
    g = mo.grad(p, X, y, w)
    rng = RNG(2)
    starts = np.cumsum([0] + [n for _, n in mo.SIZES])
    idx = np.concatenate([rng.integers(starts[k], starts[k + 1], size=min(12, starts[k + 1] - starts[k]))
                          for k in range(len(mo.SIZES))])
    eps = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = eps
        fd = (mo.loss(p + d, X, y, w) - mo.loss(p - d, X, y, w)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_mlp_oracle_single_path_closed_form():
    """One active path (x0 -> h1_0 -> h2_0 -> z): z = w3_0 * relu(W2_00 * relu(W1_00 x0 + b1_0) + b2_0) + b3."""
    p = np.zeros(mo.N_PARAM)
    q = mo.unpack(p)
    off = dict(zip([n for n, _ in mo.SIZES], np.cumsum([0] + [n for _, n in mo.SIZES])[:-1]))
    p[off["W1"] + 0] = 1.5
    p[off["b1"] + 0] = -0.25
    p[off["W2"] + 0] = -2.0
    p[off["b2"] + 0] = 3.0
    p[off["w3"] + 0] = 0.5
    p[off["b3"]] = 0.125
    X = np.zeros((3, 32))
    X[:, 0] = [0.0, 1.0, 2.0]
    z, _ = mo.forward(p, X)
    h1 = np.maximum(1.5 * X[:, 0] - 0.25, 0)
    h2 = np.maximum(-2.0 * h1 + 3.0, 0)
    assert np.allclose(z, 0.5 * h2 + 0.125)
    assert q["W1"].shape == (32, 64)


gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1809_04352_gb300 import build as libbuild
    from paper_1809_04352_gb300 import eses
    libbuild.build()
    return eses.load()


@gpu
def test_mlp_forward_and_gradient_kernels_match_oracle(lib):
    import torch
    from paper_1809_04352_gb300 import eses
    n = 1000  # not a multiple of the kernel's 64-sample blocks
    p, X, y, w = _data(n, 3)
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    Pd = torch.from_numpy(p.astype(np.float32)).to(dev)
    z = torch.empty(n, dtype=torch.float32, device=dev)
    eses.eses_mlp_forward(Xd, n, Pd, z)
    torch.cuda.synchronize()
    z_ref, _ = mo.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    assert np.abs(z.cpu().numpy() - z_ref).max() <= 1e-4 * max(1.0, np.abs(z_ref).max())
    g = torch.empty(mo.N_PARAM, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    scratch = torch.empty(eses.eses_mlp_grad_scratch(n), dtype=torch.float32, device=dev)
    yd = torch.from_numpy(y.astype(np.float32)).to(dev)
    wd = torch.from_numpy(w.astype(np.float32)).to(dev)
    eses.eses_mlp_grad(Xd, yd, wd, n, Pd, g, loss, scratch)
    torch.cuda.synchronize()
    args = (p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64), y,
            w.astype(np.float32).astype(np.float64))
    g_ref = mo.grad(*args)
    gg = g.cpu().numpy()
    assert np.abs(gg - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    assert abs(float(loss.item()) - mo.loss(*args)) <= 1e-5 * abs(mo.loss(*args))
    # deterministic
    g2 = torch.empty_like(g)
    eses.eses_mlp_grad(Xd, yd, wd, n, Pd, g2, loss, scratch)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


@gpu
def test_adam_kernel_step(lib):
    import torch
    from paper_1809_04352_gb300 import eses
    rng = RNG(5)
    p = rng.normal(0, 1, mo.N_PARAM).astype(np.float32)
    g = rng.normal(0, 1, mo.N_PARAM).astype(np.float32)
    m = rng.normal(0, 0.1, mo.N_PARAM).astype(np.float32)
    v = rng.random(mo.N_PARAM).astype(np.float32)
    step, lr = 7, 1e-3
    t = [torch.from_numpy(a.copy()).cuda() for a in (p, g, m, v)]
    eses.eses_mlp_adam(t[0], t[1], t[2], t[3], step, lr)
    torch.cuda.synchronize()
    m1 = 0.9 * m.astype(np.float64) + 0.1 * g
    v1 = 0.999 * v.astype(np.float64) + 0.001 * g.astype(np.float64) ** 2
    p1 = p - lr * (m1 / (1 - 0.9 ** step)) / (np.sqrt(v1 / (1 - 0.999 ** step)) + 1e-8)
    assert np.abs(t[0].cpu().numpy() - p1).max() < 1e-5
    assert np.abs(t[2].cpu().numpy() - m1).max() < 1e-6


def _run(mols, h, mode=0, params=None, p_far=0.5):
    from paper_1809_04352_gb300 import eses
    ctx = eses.eses_create_batch(mols, 1.4, h, 0.8)
    try:
        if mode:
            eses.eses_set_proposer(ctx, mode, params, p_far)
        eses.eses_run(ctx)
        out = []
        for m in range(len(mols)):
            out.append((eses.eses_mol_labels(ctx, m), [eses.eses_mol_intersections(ctx, m, a) for a in range(3)],
                        eses.eses_mol_area_volume(ctx, m)))
        return out, eses.eses_stats(ctx)
    finally:
        eses.eses_destroy(ctx)


def _same(a, b):
    for (la, ea, ava), (lb, eb, avb) in zip(a, b):
        assert np.array_equal(la, lb)
        for x, y in zip(ea, eb):
            assert np.array_equal(x["idx"], y["idx"])
            assert np.array_equal(x["tau"], y["tau"])
        assert ava == avb


@gpu
def test_tile_targets_are_the_tiles_holding_surface(lib):
    import torch
    from paper_1809_04352_gb300 import eses, inputs
    xyz, rad = inputs.protein_like(300, 12, inputs.PROTEIN_DENSITY)
    ctx = eses.eses_create(xyz, rad, 1.4, 0.3, 0.8)
    try:
        eses.eses_run(ctx)
        lab = eses.eses_labels(ctx)
        nt = eses.eses_num_tiles(ctx)
        feat = torch.empty((nt, 32), dtype=torch.float32, device="cuda")
        tgt = torch.empty(nt, dtype=torch.uint8, device="cuda")
        eses.eses_tile_data(ctx, feat, tgt)
        t = tgt.cpu().numpy()
        f = feat.cpu().numpy()
    finally:
        eses.eses_destroy(ctx)
    d = lab.shape
    tiles = [-(-n // 8) for n in d]
    ref = np.zeros(tiles, np.uint8)
    for i in range(tiles[0]):
        for j in range(tiles[1]):
            for k in range(tiles[2]):
                blk = lab[8 * i:8 * i + 8, 8 * j:8 * j + 8, 8 * k:8 * k + 8]
                ref[i, j, k] = blk.min() != blk.max()
    assert np.array_equal(t, ref.reshape(-1))
    assert np.isfinite(f).all()
    assert np.allclose(f[:, 30], np.log1p(np.expm1(f[:, :27]).sum(1)), rtol=1e-5, atol=1e-5)


@gpu
def test_every_proposer_mode_gives_the_exact_results(lib):
    from paper_1809_04352_gb300 import eses, inputs
    mols = [inputs.protein_like(n, 70 + n, inputs.PROTEIN_DENSITY) for n in (600, 45, 1500)]
    h = 0.3
    base, st0 = _run(mols, h)
    cert, stc = _run(mols, h, eses.ESES_PROPOSER_CERTIFY)
    _same(cert, base)
    assert stc["tiles_certified"] > 0.3 * st0["tiles"]
    rnd = RNG(9).normal(0, 0.3, mo.N_PARAM).astype(np.float32)
    for p_far in (0.2, 0.9):
        r, st = _run(mols, h, eses.ESES_PROPOSER_MLP, rnd, p_far)
        _same(r, base)
        assert st["tiles_certified"] <= st["tiles_proposed_far"]


@gpu
def test_gpu_training_learns_far_tiles_and_stays_exact(lib):
    """Train on tiles of 12 seeded globules with the library's kernels; the
    loss falls, the network calls most far tiles of held-out molecules far,
    and with it the results equal the exact path's."""
    from paper_1809_04352_gb300 import eses, inputs, proposer
    train_mols = [inputs.protein_like(int(n), 500 + k, inputs.PROTEIN_DENSITY)
                  for k, n in enumerate(RNG(4).integers(300, 1500, size=12))]
    X, y = proposer.collect(train_mols, 1.4, 0.3, 0.8, seed=1)
    assert 0 < y.sum() < len(y)
    params, losses = proposer.train(X, y, steps=400, batch=2048, lr=3e-3, seed=3)
    assert np.mean(losses[-50:]) < 0.7 * np.mean(losses[:20])
    test_mols = [inputs.protein_like(n, 900 + n, inputs.PROTEIN_DENSITY) for n in (800, 2000)]
    Xt, yt = proposer.collect(test_mols, 1.4, 0.3, 0.8, seed=2, max_far_ratio=1e9)
    c = proposer.evaluate(params, Xt, yt)
    assert c["far_called_far"] > 0.6 * (c["far_called_far"] + c["far_called_near"])
    base, _ = _run(test_mols, 0.3)
    r, st = _run(test_mols, 0.3, eses.ESES_PROPOSER_MLP, params, 0.5)
    _same(r, base)
    assert st["tiles_certified"] > 0.3 * st["tiles"]


@gpu
def test_tensor_core_mlp_matches_the_bf16_oracle(lib):
    """The proposer's tcgen05 path (BF16 operands, FP32 accumulation) against
    the FP64 oracle evaluated on the same BF16-rounded weights and inputs
    (hidden activations rounded to BF16 too): agreement to FP32 summation
    order; against the FP32 forward kernel to BF16 rounding."""
    import torch
    from paper_1809_04352_gb300 import eses
    n = 1000  # several 128-row groups and a ragged last one
    p, X, _, _ = _data(n, 11)
    p = p.astype(np.float32)
    X = X.astype(np.float32)

    def bf16(a):
        b = np.asarray(a, np.float32).view(np.uint32)
        r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
        return r.view(np.float32).astype(np.float64)

    q = mo.unpack(p.astype(np.float64))
    W1, W2 = bf16(q["W1"].astype(np.float32)), bf16(q["W2"].astype(np.float32))
    h1 = bf16(np.maximum(bf16(X) @ W1 + q["b1"], 0.0).astype(np.float32))
    h2 = np.maximum(h1 @ W2 + q["b2"], 0.0)
    z_ref = h2 @ q["w3"] + q["b3"]
    dev = torch.device("cuda")
    Xd = torch.from_numpy(X).to(dev)
    Pd = torch.from_numpy(p).to(dev)
    z = torch.empty(n, dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    eses.eses_mlp_forward_tc(Xd, n, Pd, z, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    zt = z.cpu().numpy().astype(np.float64)
    scale = max(1.0, np.abs(z_ref).max())
    assert np.abs(zt - z_ref).max() <= 2e-3 * scale
    z32, _ = mo.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.abs(zt - z32).max() <= 0.05 * max(1.0, np.abs(z32).max())
