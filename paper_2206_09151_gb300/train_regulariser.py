"""Trains the learned regulariser (RECON_FILTER_MLP) on seeded phantoms, on the GPU.

The training set is simulated by the package's own forward model (``phantoms.training_set``):
128^3 phantoms, alternately Gaussian pseudo-atoms and uniform balls, four random views each,
multislice images with Poisson noise, and the true projection of each depth layer as the
target, at each physics' own dose (or, with ``--dose lo hi``, one dose per mini-batch,
log-uniform in that range).  The network learns a per-view eps: the noise-to-signal power
of the Wiener reading of Eq. 11's bracket.  A tomogram of D views averages each voxel over
D independent images, so it is reconstructed with that eps divided by D (the plan option
``mlp_views``).  ``recon_mlp_train`` (the library's forward and backward kernels) takes Adam steps
on mini-batches of phantoms in successive calls that carry Adam's moments, over several
epochs; a held-out set of phantoms gives the validation loss after each epoch.

    python -m paper_2206_09151_gb300.train_regulariser            # writes data/regulariser.npz

The result holds the weights (RECON_MLP_PARAMS float32), the training configuration and
the loss curves.  Sec. 3 chose eps = 0.1 "ad hoc"; the network replaces that constant by
a per-(direction, layer, radial frequency) eps learned from these pairs."""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import phantoms as ph
from .recon import train_mlp

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "data", "regulariser.npz")


def load_weights(path: str = DEFAULT_OUT) -> np.ndarray:
    """The trained network's parameters (float32, RECON_MLP_PARAMS)."""
    with np.load(path) as f:
        return f["weights"].astype(np.float32)


def _fit(w, adam, step, data, sel, steps, lr):
    d = data
    w, loss, _ = train_mlp(w, d["images"][sel].contiguous(), d["targets"][sel].contiguous(), d["rot"][sel.cpu().numpy()],
                           d["defocus"][sel.cpu().numpy()], d["grid"], nz_layers=d["nz_layers"], lam=d["lam"],
                           delta=d["delta"], sigma=d["sigma"], cs=d["cs"], nsr=d["nsr"], steps=steps, lr=lr,
                           adam_state=adam, adam_step=step)
    return w, [float(x) for x in loss]


def _loss(w, data, chunk=400):
    tot, n = 0.0, data["images"].shape[0]
    for a in range(0, n, chunk):
        sel = torch.arange(a, min(n, a + chunk), device=data["images"].device)
        _, loss = _fit(w, None, 0, data, sel, 0, 1e-3)
        tot += loss[0] * sel.numel()
    return tot / n


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--phantoms-c3", type=int, default=5000, help="training phantoms at the 512^3 scan's physics")
    ap.add_argument("--phantoms-c5", type=int, default=1000, help="training phantoms at the slab's physics")
    ap.add_argument("--held-out", type=int, default=50, help="validation phantoms per physics")
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--views", type=int, default=4)
    ap.add_argument("--nz", type=int, default=16)
    ap.add_argument("--batch", type=int, default=100, help="phantoms per mini-batch")
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--steps", type=int, default=4, help="Adam steps per mini-batch")
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--dose", type=float, nargs=2, default=None,
                    help="electrons per pixel, log-uniform per mini-batch (default: each physics' own dose)")
    ap.add_argument("--init-seed", type=int, default=7)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()
    dev = torch.device("cuda")
    t0 = time.time()
    rng = np.random.default_rng(args.init_seed)
    batches = []  # (physics, data) per mini-batch of phantoms, one dose each
    for phys, count in (("c3", args.phantoms_c3), ("c5", args.phantoms_c5)):
        for a in range(0, count, args.batch):
            dose = math.exp(rng.uniform(math.log(args.dose[0]), math.log(args.dose[1]))) if args.dose else None
            batches.append((phys, ph.training_set(a, min(args.batch, count - a), phys, n=args.n, views=args.views,
                                                  nz_layers=args.nz, device=dev, photons=dose)))
    sets = {phys: None for phys, _ in batches}
    doses = (args.dose[0], math.sqrt(args.dose[0] * args.dose[1]), args.dose[1]) if args.dose else (None,)
    held = {(phys, dose): ph.training_set(1_000_000, args.held_out, phys, n=args.n, views=args.views,
                                          nz_layers=args.nz, device=dev, photons=dose)
            for phys in sets for dose in doses}
    t_data = time.time() - t0
    w = ph.mlp_init(args.init_seed).astype(np.float32)
    adam = np.zeros(2 * w.size, np.float32)
    step = 0
    history, val = [], []

    def validate():
        return {(f"{p}@{d:.0f}e/px" if d else p): _loss(w, h) for (p, d), h in held.items()}

    val.append(validate())
    for ep in range(args.epochs):
        for q in rng.permutation(len(batches)):
            data = batches[q][1]
            sel = torch.arange(data["images"].shape[0], device=dev)
            w, loss = _fit(w, adam, step, data, sel, args.steps, args.lr)
            step += args.steps
            history.append(loss[0])
        val.append(validate())
        print(json.dumps({"epoch": ep + 1, "steps": step, "train_loss_last_batch": history[-1], "held_out": val[-1]}),
              flush=True)
    cfg = dict(vars(args), images=sum(d["images"].shape[0] for _, d in batches), adam_steps=step,
               data_seconds=t_data, seconds=time.time() - t0)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez(args.out, weights=w, train_loss=np.asarray(history, np.float32),
             held_out=json.dumps(val), config=json.dumps(cfg))
    print(json.dumps({"out": args.out, **cfg}))


if __name__ == "__main__":
    main()
