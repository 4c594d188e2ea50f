"""Training of the learned tile proposer on the GPU, with the library's own
kernels (eses_mlp_grad, eses_mlp_adam) and data labelled by the exact path.

Data: synthetic globules from the input generator, run through a batched
context with the proposer off; every tile gives its 32 features and the
target "labels not all equal" (eses_tile_data).  Far tiles vastly outnumber
the others, so each chunk keeps every near tile and an equal number of far
ones, drawn with a seeded generator; the loss weights the classes equally.

Run ``python -m paper_1809_04352_gb300.proposer`` on a GPU to train on 2,000
molecules and write the parameters next to this file (proposer_params.npy);
``load_params`` reads them.
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

from . import eses, inputs

PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposer_params.npy")
N_PARAM = eses.ESES_MLP_NPARAM


def load_params() -> np.ndarray:
    """The trained parameters shipped with the package (float32[6337])."""
    p = np.load(PARAMS_FILE).astype(np.float32)
    if p.shape != (N_PARAM,):
        raise ValueError(f"{PARAMS_FILE}: expected {N_PARAM} parameters")
    return p


def init_params(seed: int) -> np.ndarray:
    """He-uniform initial weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w1 = rng.uniform(-1, 1, (32, 64)) * math.sqrt(6.0 / 32)
    w2 = rng.uniform(-1, 1, (64, 64)) * math.sqrt(6.0 / 64)
    w3 = rng.uniform(-1, 1, 64) * math.sqrt(6.0 / 64)
    return np.concatenate([w1.reshape(-1), np.zeros(64), w2.reshape(-1), np.zeros(64), w3, [0.0]]).astype(np.float32)


def collect(mols, r_p: float, h: float, margin: float, seed: int, max_far_ratio: float = 1.0):
    """Features and targets of the tiles of `mols` (one batched context, exact
    labels); keeps every near tile and up to max_far_ratio times as many far
    ones.  Returns host arrays (float32 [n, 32], uint8 [n])."""
    import torch

    ctx = eses.eses_create_batch(mols, r_p, h, margin)
    try:
        eses.eses_run(ctx)
        nt = eses.eses_num_tiles(ctx)
        feat = torch.empty((nt, 32), dtype=torch.float32, device="cuda")
        tgt = torch.empty(nt, dtype=torch.uint8, device="cuda")
        eses.eses_tile_data(ctx, feat, tgt)
        t = tgt.cpu().numpy()
        rng = np.random.Generator(np.random.PCG64(seed))
        near = np.nonzero(t)[0]
        far = np.nonzero(t == 0)[0]
        k = min(len(far), int(max_far_ratio * max(len(near), 1)))
        pick = np.sort(np.concatenate([near, rng.choice(far, size=k, replace=False)]))
        idx = torch.from_numpy(pick).cuda()
        return feat.index_select(0, idx).cpu().numpy(), t[pick]
    finally:
        eses.eses_destroy(ctx)


def train(X: np.ndarray, y: np.ndarray, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
          params: np.ndarray | None = None, log_every: int = 0):
    """Adam on the class-balanced BCE loss, minibatches drawn with a seeded
    permutation; every step runs the library's gradient and Adam kernels.
    Returns (params float32[6337], losses per step)."""
    import torch

    n = X.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = max(int(y.sum()), 1)
    neg = max(n - pos, 1)
    wcls = np.where(y > 0, 0.5 / pos, 0.5 / neg)  # balanced, sums to 1 over the data
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    yd = torch.from_numpy(y.astype(np.float32)).to(dev)
    wd = torch.from_numpy((wcls * n / batch).astype(np.float32)).to(dev)  # a batch's weights sum to ~1
    P = torch.from_numpy(init_params(seed) if params is None else params.astype(np.float32)).to(dev)
    g = torch.zeros(N_PARAM, dtype=torch.float32, device=dev)
    m = torch.zeros_like(g)
    v = torch.zeros_like(g)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    scratch = torch.empty(eses.eses_mlp_grad_scratch(batch), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    hist = torch.empty(steps, dtype=torch.float32, device=dev)
    perm = rng.permutation(n)
    at = 0
    order = torch.empty(batch, dtype=torch.int64, device=dev)
    for step in range(1, steps + 1):
        if at + batch > n:
            perm = rng.permutation(n)
            at = 0
        order.copy_(torch.from_numpy(perm[at:at + batch]))
        at += batch
        xb = Xd.index_select(0, order)
        yb = yd.index_select(0, order)
        wb = wd.index_select(0, order)
        eses.eses_mlp_grad(xb, yb, wb, batch, P, g, loss, scratch, stream)
        eses.eses_mlp_adam(P, g, m, v, step, lr, stream)
        hist[step - 1:step].copy_(loss)
        if log_every and step % log_every == 0:
            print(f"step {step} loss {float(loss.item()):.4f}", flush=True)
    torch.cuda.synchronize()
    losses = hist.cpu().numpy().astype(np.float64).tolist()
    return P.cpu().numpy(), losses


def evaluate(params: np.ndarray, X: np.ndarray, y: np.ndarray, p_far: float = 0.5) -> dict:
    """Confusion counts of the proposer's far call on (X, y), scored by the
    library's forward kernel."""
    import torch

    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    z = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    Pd = torch.from_numpy(params.astype(np.float32)).cuda()
    eses.eses_mlp_forward(Xd, X.shape[0], Pd, z, torch.cuda.current_stream().cuda_stream)
    far = (1.0 / (1.0 + np.exp(-z.cpu().numpy().astype(np.float64)))) < p_far
    return {"far_called_far": int(np.sum(far & (y == 0))), "near_called_far": int(np.sum(far & (y > 0))),
            "far_called_near": int(np.sum(~far & (y == 0))), "near_called_near": int(np.sum(~far & (y > 0)))}


def training_molecules(n_mol: int = 2000, lo: int = 300, hi: int = 3000, seed: int = 4000):
    """Seeded globules, atom counts log-uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_mol))).astype(np.int64)
    for k, n in enumerate(sizes):
        yield inputs.protein_like(int(n), seed + 1 + k, inputs.PROTEIN_DENSITY)


def main(argv=None):
    import argparse

    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--molecules", type=int, default=2000)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--h", type=float, default=0.2)
    ap.add_argument("--out", default=PARAMS_FILE)
    args = ap.parse_args(argv)
    from . import build as libbuild

    libbuild.build()
    t0 = time.time()
    Xs, ys, chunk = [], [], []
    for k, mol in enumerate(training_molecules(args.molecules)):
        chunk.append(mol)
        if len(chunk) == args.chunk or k == args.molecules - 1:
            X, y = collect(chunk, 1.4, args.h, 0.8, seed=k)
            Xs.append(X)
            ys.append(y)
            chunk = []
            print(f"{k + 1} molecules, {sum(len(v) for v in ys)} tiles, {time.time() - t0:.0f} s", flush=True)
    X = np.concatenate(Xs)
    y = np.concatenate(ys)
    params, _ = train(X, y, steps=args.steps, log_every=500)
    print("train confusion", evaluate(params, X, y), flush=True)
    np.save(args.out, params.astype(np.float32))
    print(f"wrote {args.out} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    sys.exit(main())
