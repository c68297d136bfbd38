"""Learned initial guess around the library's MLP kernels.

* make_dataset: seeded water clusters, converged densities from the plain
  FP64 SCF (hf_scf_run), per-atom-pair features from hf_guess_features and
  the matching density blocks as targets;
* train: minibatch Adam steps, each one hf_model_train_step;
* predict: hf_guess_predict (device), with the core-Hamiltonian guess as the
  fallback when the prediction is unusable;
* evaluate: SCF iterations and time from the learned guess vs the core guess,
  and the difference of the converged energies.
Weight initialisation is drawn here (seeded numpy) and passed to the library.
"""
from __future__ import annotations

import time

import numpy as np

from . import hf, inputs

HEAD_OFF = (0, 225, 300)
HEAD_SHAPE = ((15, 15), (15, 5), (5, 5))


def init_weights(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases (float32 vector in the library's layout)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((16, 256), (256, 256), (256, 325)):
        lim = np.sqrt(6.0 / fan_in) * (1.0 if fan_out != 325 else 0.1)
        parts.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, dtype=np.float32))
    return np.concatenate(parts)


def pair_targets(P: np.ndarray, meta: np.ndarray):
    """Target blocks and 0/1 masks for each pair's head."""
    n = meta.shape[0]
    T = np.zeros((n, 325), dtype=np.float32)
    M = np.zeros((n, 325), dtype=np.float32)
    for t in range(n):
        r0, c0, h, _ = (int(x) for x in meta[t])
        nr, nc = HEAD_SHAPE[h]
        T[t, HEAD_OFF[h]:HEAD_OFF[h] + nr * nc] = P[r0:r0 + nr, c0:c0 + nc].ravel()
        M[t, HEAD_OFF[h]:HEAD_OFF[h] + nr * nc] = 1.0
    return T, M


def make_dataset(ctx: hf.Context, n_clusters: int, config: int = inputs.CONFIG_GUESS_TRAIN, lo: int = 2, hi: int = 8,
                 tau: float = 1e-10, prim_tau: float = 1e-14, log=None):
    Xs, Ts, Ms = [], [], []
    t0 = time.perf_counter()
    iters = []
    for m in range(n_clusters):
        geom = inputs.batch_cluster(config, m, lo, hi)
        basis = inputs.synthetic_basis(geom)
        s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
        r = hf.scf(s, e_tol=1e-9, d_tol=1e-6)
        X, meta = hf.guess_features(s)
        T, M = pair_targets(r["P"], meta)
        Xs.append(X)
        Ts.append(T)
        Ms.append(M)
        iters.append(r["iterations"])
        s.close()
        if log and (m + 1) % 100 == 0:
            log(f"dataset: {m + 1}/{n_clusters} clusters, {time.perf_counter() - t0:.1f} s")
    return {"X": np.concatenate(Xs), "T": np.concatenate(Ts), "M": np.concatenate(Ms),
            "seconds": time.perf_counter() - t0, "clusters": n_clusters, "scf_iterations": iters}


def train(model: hf.Model, data: dict, steps: int = 3000, batch: int = 2048, lr: float = 1e-3, seed: int = 0,
          log=None) -> list:
    import torch
    dev = torch.device("cuda", model.ctx.device)
    X = torch.from_numpy(data["X"]).to(dev)
    T = torch.from_numpy(data["T"]).to(dev)
    M = torch.from_numpy(data["M"]).to(dev)
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for k in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=g).to(dev)
        xb, tb, mb = X[idx].contiguous(), T[idx].contiguous(), M[idx].contiguous()
        lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / steps))  # cosine decay
        losses.append(model.train_step(xb, tb, mb, lr_k))
        if log and (k + 1) % 500 == 0:
            log(f"train: step {k + 1}/{steps} loss {np.mean(losses[-100:]):.5f}")
    return losses


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
             config: int = inputs.CONFIG_GUESS_EVAL, tau: float = 1e-10, prim_tau: float = 1e-14,
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
