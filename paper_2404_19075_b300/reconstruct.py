"""Reconstruction driver: train a DINR on one of the seeded workloads and
report the reconstruction error against the phantom as training proceeds.

    python -m paper_2404_19075_b300.reconstruct --workload 2 --steps 2000 \
        --eval-every 250 [--prec bf16] [--lr-decay 0.95] [--poisson I0]

Each evaluation queries mu0 * M on a 64^3 grid of cell centres inside the
field of view at 8 view times and prints one JSON line with the loss, the
relative L2 error and the PSNR (peak = the phantom's maximum). The learning
rate is multiplied by --lr-decay after every epoch (App. C). --poisson I0
replaces the exact projections by Poisson transmission data with I0 incident
photons per ray, p = -log(max(N, 1) / I0) with N ~ Poisson(I0 exp(-p))
(the noise model of the paper's simulated data), drawn from a seeded stream.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from dataclasses import replace

import numpy as np
import torch

from . import Dinr, phantom_project


def poisson_transmission(proj: torch.Tensor, i0: float, seed: int) -> torch.Tensor:
    """Noisy line integrals from Poisson photon counts (Beer-Lambert)."""
    g = torch.Generator(device=proj.device)
    g.manual_seed(seed)
    counts = torch.poisson(i0 * torch.exp(-proj), generator=g)
    return -torch.log(torch.clamp(counts, min=1.0) / i0)


def main(argv=None) -> int:
    from synthetic import truth, workloads as wl

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--prec", default="bf16", choices=["bf16", "fp32", "fp8"])
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--eval-every", type=int, default=250)
    ap.add_argument("--lr", type=float, default=0.0, help="0: the workload's")
    ap.add_argument("--lr-decay", type=float, default=1.0, help="per epoch (App. C: 0.95)")
    ap.add_argument("--rays", type=int, default=0, help="rays per step (0: the workload's)")
    ap.add_argument("--poisson", type=float, default=0.0, help="incident photons per ray")
    ap.add_argument("--grid", type=int, default=64)
    args = ap.parse_args(argv)

    w = wl.workload(args.workload)
    train = w.train
    if args.rays:
        train = replace(train, batch_rays=args.rays)
    if args.lr:
        train = replace(train, lr=args.lr)
    train = replace(train, lr_decay_per_epoch=args.lr_decay)
    g, net = w.geom, w.net
    ph = wl.phantom(w)
    proj = phantom_project(g, ph)
    if args.poisson > 0:
        proj = poisson_transmission(proj, args.poisson, w.seeds["noise"])
    theta = wl.he_init(net, w.seeds["weights"]).astype(np.float32)
    m = Dinr(g, net, train, proj, prec=args.prec, init_params=theta,
             sampler_seed=w.seeds["sampler"])
    times = [(k + 0.5) / 8 for k in range(8)]
    n = args.grid
    mask = truth.fov_mask(n)
    gt = [truth.attenuation_grid(ph, t, n) for t in times]
    steps_per_epoch = math.ceil(g.n_proj / train.batch_rays)
    t0 = time.perf_counter()
    for k in range(1, args.steps + 1):
        m.train_step(None, n=train.batch_rays, sync=False)
        if k % args.eval_every == 0 or k == args.steps:
            loss = m.loss()
            sc = [truth.scores(m.query_grid(t, (-1, -1, -1), (1, 1, 1), (n, n, n)).cpu().numpy(),
                               gt_t, mask) for t, gt_t in zip(times, gt)]
            print(json.dumps({"step": k, "epoch": k / steps_per_epoch, "loss": loss,
                              "rel_l2": float(np.mean([x["rel_l2"] for x in sc])),
                              "psnr_db": float(np.mean([x["psnr_db"] for x in sc])),
                              "wall_s": time.perf_counter() - t0}), flush=True)
    m.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
