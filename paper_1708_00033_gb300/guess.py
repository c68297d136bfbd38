"""Learned initial guess around the library's MLP kernels.

* make_dataset: seeded water clusters, converged densities from the plain
  FP64 SCF (hf_scf_run), per-atom-pair features (hf_guess_features) and the
  matching density blocks as targets (hf_guess_targets);
* train: hf_guess_train (minibatch draws, cosine learning-rate decay and Adam
  steps run in the library);
* predict: hf_guess_predict (device), with the core-Hamiltonian guess as the
  fallback when the prediction is unusable;
* evaluate: SCF iterations and time from the learned vs the core guess,
  and the difference of the converged energies.
The seeded initial weights are drawn by inputs.guess_init_weights.
"""
from __future__ import annotations

import json
import os
import threading
import time

import numpy as np

from . import hf, inputs

init_weights = inputs.guess_init_weights

# Trained weights shipped with the package (written by train_guess.py from plain-SCF densities).
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "guess_weights.npz")


def load_weights(path: str = WEIGHTS_PATH):
    """(float32 weight vector, metadata dict) of a weight file written by train_guess.py."""
    with np.load(path) as z:
        return z["weights"].astype(np.float32), json.loads(str(z["meta"]))


def save_weights(path: str, weights: np.ndarray, meta: dict):
    np.savez_compressed(path, weights=np.asarray(weights, dtype=np.float32), meta=json.dumps(meta))


def _cluster_sample(ctx, config, m, lo, hi, tau, prim_tau):
    geom = inputs.batch_cluster(config, m, lo, hi)
    basis = inputs.synthetic_basis(geom)
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
    try:
        r = hf.scf(s, e_tol=1e-9, d_tol=1e-6)
        X, _ = hf.guess_features(s)
        T, M = hf.guess_targets(s, r["P"])
    finally:
        s.close()
    return X, T, M, r["iterations"]


def make_dataset(ctx: hf.Context, n_clusters: int, config: int = inputs.CONFIG_GUESS_TRAIN, lo: int = 2, hi: int = 8,
                 tau: float = inputs.BENCH_SCHWARZ_TAU, prim_tau: float = inputs.BENCH_PRIM_TAU, log=None,
                 workers: int = 1):
    """Features and plain-SCF density targets of clusters m = 0..n_clusters-1 (seeds (config, m)).  With
    workers > 1, that many host threads each drive their own context and CUDA stream, so that the small
    clusters' SCFs overlap on the GPU; the result does not depend on the number of workers."""
    t0 = time.perf_counter()
    out = [None] * n_clusters
    if workers <= 1:
        for m in range(n_clusters):
            out[m] = _cluster_sample(ctx, config, m, lo, hi, tau, prim_tau)
            if log and (m + 1) % 100 == 0:
                log(f"dataset: {m + 1}/{n_clusters} clusters, {time.perf_counter() - t0:.1f} s")
    else:
        import torch
        dev = ctx.device
        lock = threading.Lock()
        nxt = [0]
        errors = []

        def run():
            try:
                stream = torch.cuda.Stream(device=dev)
                wctx = hf.Context(dev, stream)
                while True:
                    with lock:
                        m = nxt[0]
                        nxt[0] += 1
                    if m >= n_clusters:
                        break
                    out[m] = _cluster_sample(wctx, config, m, lo, hi, tau, prim_tau)
                    if log and (m + 1) % 100 == 0:
                        log(f"dataset: {m + 1}/{n_clusters} clusters, {time.perf_counter() - t0:.1f} s")
                wctx.close()
            except Exception as e:  # reported after the join
                errors.append(e)

        threads = [threading.Thread(target=run) for _ in range(workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
    return {"X": np.concatenate([o[0] for o in out]), "T": np.concatenate([o[1] for o in out]),
            "M": np.concatenate([o[2] for o in out]), "seconds": time.perf_counter() - t0, "clusters": n_clusters,
            "scf_iterations": [o[3] for o in out]}


def train(model: hf.Model, data: dict, steps: int = 3000, batch: int = 2048, lr: float = 1e-3, seed: int = 0,
          log=None) -> list:
    """hf_guess_train over the whole dataset (moved to the device once); returns the minibatch losses."""
    import torch
    dev = torch.device("cuda", model.ctx.device)
    X = torch.from_numpy(data["X"]).to(dev)
    T = torch.from_numpy(data["T"]).to(dev)
    M = torch.from_numpy(data["M"]).to(dev)
    losses = hf.guess_train(model, X, T, M, steps=steps, batch=batch, lr=lr, seed=seed)
    if log:
        log(f"train: {steps} steps, loss {float(losses[:10].mean()):.5f} -> {float(losses[-100:].mean()):.5f}")
    return [float(x) for x in losses]


def predict_or_none(model: hf.Model, system: hf.System):
    """The learned density, or None when it is unusable (the caller keeps the core guess)."""
    try:
        P = hf.guess_predict(model, system)
    except hf.HFError:
        return None
    if not np.all(np.isfinite(P)):
        return None
    return P


def evaluate(ctx: hf.Context, model: hf.Model, n_eval: int = 32, waters: int = 32,
             config: int = inputs.CONFIG_GUESS_EVAL, tau: float = inputs.BENCH_SCHWARZ_TAU,
             prim_tau: float = inputs.BENCH_PRIM_TAU,
             fp32_cutoff: float = 1e-4, log=None) -> dict:
    """Per held-out cluster, three SCFs to the same convergence test (|dE| < 1e-9, RMS dP < 1e-6):
    plain FP64 from the core-Hamiltonian guess, FP64 from the learned guess, and mixed precision
    (FP32 for Q_ij Q_kl < fp32_cutoff until |dE| < 1e-5, then FP64) from the learned guess.
    SCF times exclude system setup, which is reported separately."""
    import torch
    rows = []
    for m in range(n_eval):
        geom = inputs.water_cluster(waters, config, m)
        basis = inputs.synthetic_basis(geom)
        t0 = time.perf_counter()
        s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
        setup64 = time.perf_counter() - t0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        core = hf.scf(s, e_tol=1e-9, d_tol=1e-6)
        t_core = time.perf_counter() - t0
        t0 = time.perf_counter()
        Pg = predict_or_none(model, s)
        t_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        learned = hf.scf(s, e_tol=1e-9, d_tol=1e-6, P_guess=Pg) if Pg is not None else core
        t_learn = time.perf_counter() - t0 + t_pred
        s.close()
        t0 = time.perf_counter()
        sm = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau, fp32_cutoff=fp32_cutoff)
        setup_mixed = time.perf_counter() - t0
        t0 = time.perf_counter()
        mixed = hf.scf(sm, e_tol=1e-9, d_tol=1e-6, P_guess=Pg)
        t_mixed = time.perf_counter() - t0 + t_pred
        sm.close()
        rows.append({"cluster": m, "core_iterations": core["iterations"], "core_s": t_core,
                     "learned_iterations": learned["iterations"], "learned_s": t_learn,
                     "mixed_learned_iterations": mixed["iterations"], "mixed_learned_s": t_mixed,
                     "mixed_learned_mixed_iterations": mixed["mixed_iterations"],
                     "predict_s": t_pred, "setup_fp64_s": setup64, "setup_mixed_s": setup_mixed,
                     "fallback": Pg is None, "core_energy": core["energy"], "learned_energy": learned["energy"],
                     "mixed_learned_energy": mixed["energy"],
                     "abs_dE": abs(core["energy"] - learned["energy"]),
                     "abs_dE_mixed": abs(core["energy"] - mixed["energy"])})
        if log:
            log(f"eval {m}: core {core['iterations']} it {t_core:.2f} s | learned {learned['iterations']} it "
                f"{t_learn:.2f} s | mixed+learned {mixed['iterations']} it {t_mixed:.2f} s | "
                f"|dE| {rows[-1]['abs_dE']:.1e} {rows[-1]['abs_dE_mixed']:.1e}")
    mean = lambda k: float(np.mean([r[k] for r in rows]))  # noqa: E731
    return {"rows": rows,
            "mean_core_iterations": mean("core_iterations"), "mean_learned_iterations": mean("learned_iterations"),
            "mean_mixed_learned_iterations": mean("mixed_learned_iterations"),
            "mean_core_s": mean("core_s"), "mean_learned_s": mean("learned_s"),
            "mean_mixed_learned_s": mean("mixed_learned_s"),
            "max_abs_dE": float(max(r["abs_dE"] for r in rows)),
            "max_abs_dE_mixed": float(max(r["abs_dE_mixed"] for r in rows)),
            "fallbacks": int(sum(r["fallback"] for r in rows))}
