"""Train the learned-guess MLP and write its weight file.

    python -m paper_1708_00033_gb300.train_guess [--n-train 2000] [--steps 4000] [--out FILE]

The training set is the learned-guess workload: seeded clusters of U{2..8}
waters (seeds (5, m)), each converged by the plain FP64 SCF (Schwarz 1e-10,
the benchmark primitive threshold); per atom pair the features of
hf_guess_features and the density block of hf_guess_targets.  Training is
hf_guess_train (minibatches of 2,048 pairs, Adam, cosine decay from 1e-3).
The weight file (numpy .npz) holds the float32 weights and a JSON record of
how they were made; guess.load_weights reads it.
"""
from __future__ import annotations

import argparse
import sys
import time

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description="Train the learned-guess MLP on plain-SCF densities.")
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=2048)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--workers", type=int, default=8, help="host threads generating the SCF densities")
    ap.add_argument("--out", default=None, help="weight file (default: the package's guess_weights.npz)")
    a = ap.parse_args(argv)
    from . import guess, hf, inputs
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731
    ctx = hf.Context(0)
    data = guess.make_dataset(ctx, a.n_train, prim_tau=inputs.BENCH_PRIM_TAU, log=log, workers=a.workers)
    log(f"dataset: {data['X'].shape[0]} atom pairs from {a.n_train} clusters in {data['seconds']:.1f} s")
    model = hf.Model(ctx, inputs.guess_init_weights(a.seed))
    t0 = time.perf_counter()
    losses = guess.train(model, data, steps=a.steps, batch=a.batch, lr=a.lr, seed=a.seed, log=log)
    train_s = time.perf_counter() - t0
    meta = {"n_train": a.n_train, "train_config": inputs.CONFIG_GUESS_TRAIN, "waters": [2, 8], "steps": a.steps,
            "batch": a.batch, "lr": a.lr, "seed": a.seed, "schwarz_tau": 1e-10, "prim_tau": inputs.BENCH_PRIM_TAU,
            "atom_pairs": int(data["X"].shape[0]), "dataset_s": round(data["seconds"], 1),
            "train_s": round(train_s, 2), "loss_first10": float(np.mean(losses[:10])),
            "loss_last100": float(np.mean(losses[-100:])),
            "mean_scf_iterations": float(np.mean(data["scf_iterations"]))}
    out = a.out or guess.WEIGHTS_PATH
    guess.save_weights(out, model.weights(), meta)
    log(f"wrote {out}: {meta}")
    print(out)


if __name__ == "__main__":
    main()
