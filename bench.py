#!/usr/bin/env python
"""Fock builds/s of the GB300 direct-SCF Fock build (one JSON line on stdout).

Workload (default): the 64-water cluster of the SCF configuration (seed
(2, rank)), 1,600 Cartesian basis functions, Schwarz screening at 1e-10,
plain FP64 integrals; one step = one full Fock build (density in, J and K of
all 21 angular classes, F = H + J - K/2 and the energy out).  With N ranks
each rank builds its own cluster (independent problems, weak scaling, no
collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The default line also carries the SCF half of the metric (plain FP64, mixed
precision, and mixed precision from the learned guess on held-out 32-water
clusters), the roofline of the dominant ERI kernel, and the CPU oracle's
baseline.  --impl reference times the CPU oracle (as it stands) on the host
cores over stratified random samples of the same Fock build and reports the
same metric.  --mode shard shards one molecule's build over the ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DFMA_PEAK_GFLOPS = 152 * 2 * 2 * 2.070  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (nominal, derived)

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the dominant kernel, from one
# ncu capture of the default workload, with the SHA-256 of the sources that kernel is compiled from at that
# time; the bench reports it only while those sources are unchanged (else the counters describe another
# kernel and traffic is null).  Capture: the 64-water FP64 build at the bench's thresholds (`--mode case
# --case fock --waters 64`), one pass, both launches of k_eri_1110<double>: 3.79 GB + 630.90 MB and
# 3.80 GB + 632.54 MB; their mean.
NCU_TRAFFIC = {"kernel": "k_eri_1110", "bytes_per_launch": 4.4267e9,
               "sources_sha256": "18cdc26cad87ad9d767e774a67808fd25df6ef1a68ef13699d23cc8cda1164c0"}
TRAFFIC_SOURCES = ("paper_1708_00033_gb300/csrc/gen_eri.py", "paper_1708_00033_gb300/csrc/eri_common.cuh",
                   "paper_1708_00033_gb300/csrc/hf_internal.h")


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    root = os.path.dirname(os.path.abspath(__file__))
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(root, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel: str):
    if NCU_TRAFFIC["kernel"] != kernel or NCU_TRAFFIC["bytes_per_launch"] is None:
        return None
    return NCU_TRAFFIC["bytes_per_launch"] if kernel_sources_sha256() == NCU_TRAFFIC["sources_sha256"] else None
L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--waters", type=int, default=64)
    ap.add_argument("--config-id", type=int, default=2)
    ap.add_argument("--tau", type=float, default=1e-10)
    ap.add_argument("--fp32-cutoff", type=float, default=0.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--prim-tau", type=float, default=None, help="default: the benchmark primitive threshold")
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="oracle time budget of --impl reference over all its steps")
    ap.add_argument("--mode", default="fock",
                    choices=["fock", "scf", "mixed", "batch", "guess", "copies", "peaks", "shard", "rys", "case"])
    ap.add_argument("--case", default="fock", choices=["fock", "scf", "train"], help="workload of --mode case")
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-eval", type=int, default=32)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--n-mol", type=int, default=512)
    ap.add_argument("--scf-variants", default="fp64,mixed,fp64_incremental,mixed_incremental")
    ap.add_argument("--copies", default="1,8,152,608", help="accumulator copies compared by --mode copies")
    ap.add_argument("--copies-workloads", default="4:0,16:1e-10,64:1e-10", help="waters:schwarz_tau list")
    ap.add_argument("--scf-clusters", type=int, default=4,
                    help="held-out 32-water clusters of the SCF comparison in the default line (0: none)")
    ap.add_argument("--scf-waters", type=int, default=32)
    a = ap.parse_args()
    if a.prim_tau is None:
        from paper_1708_00033_gb300 import inputs
        a.prim_tau = inputs.BENCH_PRIM_TAU
    if a.mode == "mixed" and "--waters" not in sys.argv:
        a.waters, a.config_id = 256, 3
    if a.mode == "mixed" and "--fp32-cutoff" not in sys.argv:
        a.fp32_cutoff = 1e-4
    return a


def workload_name(a):
    prec = "FP64" if a.fp32_cutoff <= 0 else f"mixed FP32<{a.fp32_cutoff:g}"
    return (f"{a.waters}-water cluster, {25 * a.waters} Cartesian BF, synthetic 3-primitive basis, "
            f"Schwarz tau={a.tau:g}, primitive tau={a.prim_tau:g}, {prec} Fock build (J+K)")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, dist, device) -> float:
    """Largest value of x over all ranks (the bench's max-over-ranks timing)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def random_density(S, n_occ, cfg, idx):
    """P = 2 C C^T with C = G L^-T, L L^T = G^T S G (input preparation, untimed)."""
    import numpy as np
    from paper_1708_00033_gb300 import inputs
    G = inputs.random_orbitals(S.shape[0], n_occ, cfg, idx)
    L = np.linalg.cholesky(G.T @ S @ G)
    C = np.linalg.solve(L, G.T).T
    return 2.0 * C @ C.T


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9 and f[1].replace(".", "").isdigit():
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return out
        out["sm_mhz"] = statistics.median(float(r[1]) for r in rows)
        out["sm_max_mhz"] = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(n)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1708_00033_gb300 import hf, inputs

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    geom = inputs.water_cluster(a.waters, a.config_id, rank)
    basis = inputs.synthetic_basis(geom)
    ctx = hf.Context(local)
    sysm = hf.System(ctx, geom, basis, schwarz_tau=a.tau, fp32_cutoff=a.fp32_cutoff, prim_tau=a.prim_tau)
    N = sysm.n_bf
    S, _ = sysm.one_electron()
    n_occ = inputs.n_electrons(geom) // 2
    P = random_density(S, n_occ, a.config_id, rank)
    Pd = torch.from_numpy(P).to(dev)
    Fd = torch.empty_like(Pd)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(a.warmup):
        sysm.fock_build(Pd, F=Fd)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, stats = [], []
    torch.cuda.synchronize()
    for _ in range(a.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = sysm.fock_build(Pd, F=Fd, timing=True)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        stats.append(out["stats"])
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = reduce_max(total_ms, dist, dev)
        dist.barrier()
    value = world * a.steps / (total_ms / 1e3)

    # end to end through the C-ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not a.no_e2e:
        Ph = torch.from_numpy(P).pin_memory()
        Fh = torch.empty((N, N), dtype=torch.float64).pin_memory()
        sysm.fock_build(Ph.numpy(), F=Fh.numpy())
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            sysm.fock_build(Ph.numpy(), F=Fh.numpy())
        dt = time.perf_counter() - t0
        if world > 1:
            dt = reduce_max(dt, dist, dev)
        e2e = {"value": world * a.steps / dt, "unit": "Fock builds/s", "h2d_bytes_per_step": N * N * 8,
               "d2h_bytes_per_step": N * N * 8 + 8}

    # roofline of the dominant kernel (the class kernel with the largest device time)
    ms_cls = np.mean([s["ms_class_fp64"] for s in stats], axis=0) + np.mean([s["ms_class_fp32"] for s in stats], axis=0)
    c = int(np.argmax(ms_cls))
    fl = stats[0]["class_flops_fp64"][c] + stats[0]["class_flops_fp32"][c]
    achieved = fl / (ms_cls[c] / 1e3) / 1e9
    eri_ms = float(np.mean([s["ms_eri"] for s in stats]))
    eri_gflops = (stats[0]["flops_fp64"] + stats[0]["flops_fp32"]) / (eri_ms / 1e3) / 1e9
    line = {
        "metric": "Fock builds/s",
        "value": value,
        "unit": "Fock builds/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if a.fp32_cutoff <= 0 else "f64+f32",
        "data": "synthetic",
        "config": {"workload": workload_name(a), "waters": a.waters, "n_bf": N, "schwarz_tau": a.tau,
                   "prim_tau": a.prim_tau, "fp32_cutoff": a.fp32_cutoff,
                   "density": "random S-orthonormal C, n_occ=%d" % n_occ,
                   "quartets_evaluated": stats[0]["quartets_fp64"] + stats[0]["quartets_fp32"],
                   "quartets_fp32": stats[0]["quartets_fp32"],
                   "primitive_quartets": stats[0]["prim_quartets_fp64"] + stats[0]["prim_quartets_fp32"],
                   "quartets_unscreened": stats[0]["quartets_unscreened"],
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "gpu_launches": int(sum(s["kernels_launched"] for s in stats)),
        "clocks": clk,
        "roofline": {"bound": "alu", "kernel": hf.CLASS_KERNELS[c], "class": hf.CLASS_NAMES[c], "achieved": achieved,
                     "peak": DFMA_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / DFMA_PEAK_GFLOPS,
                     "traffic": measured_traffic(hf.CLASS_KERNELS[c]),
                     "peak_kind": "FP64 FMA pipe, derived from unit counts and max clock (hf_measure_peaks: 1,252)",
                     "all_eri_kernels": {"ms": eri_ms, "achieved": eri_gflops,
                                         "frac": eri_gflops / DFMA_PEAK_GFLOPS}},
        "class_ms": {hf.CLASS_NAMES[i]: round(float(ms_cls[i]), 3) for i in range(len(ms_cls))},
    }
    if e2e:
        line["e2e"] = e2e
    if a.scf_clusters > 0:
        line["scf"] = scf_comparison(a, ctx, hf, inputs, rank)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, geom, basis, P, a.cpu_sample_seconds, hf=hf, ctx=ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def screened_row_counts(Qp, tau: float, block: int = 8192):
    """Exact number of quartets Algorithm 1 evaluates in each row ij (kets kl <= ij with Q_ij Q_kl >= tau),
    from the pair bounds Qp in canonical pair order; blocked so that memory stays O(block^2)."""
    import numpy as np
    n = Qp.size
    if tau <= 0:
        return np.arange(1, n + 1, dtype=np.int64)
    counts = np.empty(n, dtype=np.int64)
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        thr = tau / np.maximum(Qp[b0:b1], 1e-300)
        prefix = np.sort(Qp[:b0])
        c = prefix.size - np.searchsorted(prefix, thr, side="left")
        M = np.tril(Qp[b0:b1][None, :] >= thr[:, None])
        counts[b0:b1] = c + M.sum(axis=1)
    return counts


class OracleEstimator:
    """Time of one full oracle Fock build of a large system, estimated from timed random samples of rows
    (bra pairs ij of Algorithm 1's outer loop).  Rows are stratified by the bra's pair class (ss, ps, pp,
    ds, dp, dd); within a class the sampled rows' work is scaled by the ratio of the class's exact screened
    quartet count (from the Schwarz bounds) to the sampled rows' count.  The work of a row is the time a
    thread spends in it (the oracle sums it over its threads), so that a sample too small to keep every
    thread busy still measures its rows; the full build's wall time is that work divided by the thread
    count and by the parallel efficiency the oracle reaches on a full build of a small system
    (calibrate())."""

    def __init__(self, mol, P, tau):
        import numpy as np
        import oracle
        self.mol, self.P, self.tau = mol, P, tau
        self.threads = oracle.num_threads()
        self.efficiency = 1.0
        Q = mol.schwarz()
        n = mol.n_shells
        i, j = np.tril_indices(n)  # canonical order: ij = i (i + 1) / 2 + j, j <= i
        order = np.lexsort((j, i))
        i, j = i[order], j[order]
        self.Qp = Q[i, j]
        lsh = np.asarray([0 if c == 1 else (1 if c == 3 else 2) for c in mol.ncomp])
        la, lb = np.maximum(lsh[i], lsh[j]), np.minimum(lsh[i], lsh[j])
        self.cls = np.array([{(0, 0): 0, (1, 0): 1, (1, 1): 2, (2, 0): 3, (2, 1): 4, (2, 2): 5}[(a, b)]
                             for a, b in zip(la, lb)])
        self.counts = screened_row_counts(self.Qp, tau)
        self.total = int(self.counts.sum())
        self.strata = [c for c in range(6) if self.counts[self.cls == c].sum() > 0]

    def calibrate(self, mol, P, tau):
        """Parallel efficiency of a full build of a small system: (thread-seconds / threads) / wall seconds."""
        import numpy as np
        rows = np.arange(mol.n_shells * (mol.n_shells + 1) // 2)
        t0 = time.perf_counter()
        _, busy = mol.jk_unique_rows(P, tau, rows)
        wall = time.perf_counter() - t0
        self.efficiency = min(1.0, busy / self.threads / wall)
        return {"wall_s": wall, "thread_s": busy, "efficiency": self.efficiency}

    def estimate(self, seconds: float, rng):
        """One estimate of the full build's wall seconds from about `seconds` of sampled rows' work."""
        import numpy as np
        per = seconds / len(self.strata)
        work, sampled = 0.0, 0
        for c in self.strata:
            rows = np.flatnonzero((self.cls == c) & (self.counts > 0))
            perm = rng.permutation(rows)
            # pilot: a few rows give this class's work per quartet, then the rest of its budget
            k, acc = 0, 0
            while k < perm.size and acc < 2000:
                acc += int(self.counts[perm[k]])
                k += 1
            _, w_pilot = self.mol.jk_unique_rows(self.P, self.tau, perm[:k])
            rate = acc / max(w_pilot, 1e-6)
            want = int(rate * max(per - w_pilot, 0.0))
            k2, acc2 = k, 0
            while k2 < perm.size and acc2 < want:
                acc2 += int(self.counts[perm[k2]])
                k2 += 1
            w_main = self.mol.jk_unique_rows(self.P, self.tau, perm[k:k2])[1] if k2 > k else 0.0
            q_s = acc + acc2
            work += (w_pilot + w_main) * (int(self.counts[rows].sum()) / q_s)
            sampled += q_s
        return work / (self.threads * self.efficiency), sampled


def _time_oracle_full(mol, P, tau):
    t0 = time.perf_counter()
    mol.jk_unique(P, tau)
    return time.perf_counter() - t0, mol.last_quartets


def _gpu_build_ms(hf, ctx, geom, basis, P, tau, prim_tau, reps=3):
    import torch
    s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=prim_tau)
    Pd = torch.from_numpy(P).cuda()
    F = torch.empty_like(Pd)
    s.fock_build(Pd, F=F)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.fock_build(Pd, F=F)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    s.close()
    return min(ms)


def cpu_baseline(a, geom, basis, P, seconds, hf=None, ctx=None):
    """The oracle on the host cores: a stratified-sample estimate of one build of the benchmarked workload
    (the line's value), and full, unextrapolated builds of the 4-water cluster (100 BF, no screening) and of
    the first 16 waters of the 256-water cluster (400 BF, Schwarz 1e-10), each beside the GPU's time for
    the same build."""
    import numpy as np
    import oracle
    from paper_1708_00033_gb300 import inputs
    mol = oracle.Molecule(geom, basis)
    t0 = time.perf_counter()
    est = OracleEstimator(mol, P, a.tau)
    setup_s = time.perf_counter() - t0
    calib = est.calibrate(*_calibration_system(inputs))
    build_s, q = est.estimate(seconds, np.random.default_rng(12345))
    full = {}
    for name, g, tau, cfg in (("C1_4_waters_tau0", inputs.water_cluster(4, inputs.CONFIG_SINGLE_BUILD), 0.0, 1),
                              ("subset_16_waters_tau1e-10",
                               inputs.subset_waters(inputs.water_cluster(256, inputs.CONFIG_MIXED), 16), 1e-10, 3)):
        b = inputs.synthetic_basis(g)
        m = oracle.Molecule(g, b)
        S, _ = m.core_hamiltonian()
        Pm = random_density(S, inputs.n_electrons(g) // 2, cfg, 0)
        if tau > 0:
            m.schwarz()
        osec, nq = _time_oracle_full(m, Pm, tau)
        row = {"n_bf": m.n_bf, "schwarz_tau": tau, "oracle_s": osec, "oracle_quartets": nq}
        if hf is not None:
            gms = _gpu_build_ms(hf, ctx, g, b, Pm, tau, a.prim_tau)
            row.update(gpu_ms=gms, gpu_over_oracle=osec / (gms / 1e3))
        full[name] = row
    return {"value": 1.0 / build_s, "unit": "Fock builds/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"stratified random sample of bra-pair rows (6 pair classes, {q} of {est.total} screened "
                       f"quartets, ~{seconds:.0f} s), each class scaled by its exact screened quartet count: "
                       f"{build_s:.0f} s per build"),
            "estimate_s_per_build": build_s, "setup_s": setup_s, "calibration": calib, "full_builds": full}


def _calibration_system(inputs):
    """The 4-water cluster without screening: the full build whose parallel efficiency calibrates the
    sampled estimates."""
    import oracle
    g = inputs.water_cluster(4, inputs.CONFIG_SINGLE_BUILD)
    m = oracle.Molecule(g, inputs.synthetic_basis(g))
    S, _ = m.core_hamiltonian()
    return m, random_density(S, inputs.n_electrons(g) // 2, 1, 0), 0.0


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1708_00033_gb300 import inputs
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    mol = oracle.Molecule(geom, basis)
    S, _ = mol.core_hamiltonian()
    P = random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)
    est = OracleEstimator(mol, P, a.tau)
    calib = est.calibrate(*_calibration_system(inputs))
    per_step = max(1.0, a.reference_seconds / max(1, a.steps + a.warmup))
    rng = np.random.default_rng(777)
    for _ in range(a.warmup):
        est.estimate(per_step, rng)
    runs = [est.estimate(per_step, rng)[0] for _ in range(a.steps)]
    build_s = float(np.mean(runs))
    spread = float(np.std(runs, ddof=1)) if len(runs) > 1 else 0.0
    value = 1.0 / build_s
    line = {"metric": "Fock builds/s", "value": value, "unit": "Fock builds/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": build_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(a), "waters": a.waters, "schwarz_tau": a.tau},
            "cpu_baseline": {"value": value, "unit": "Fock builds/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": (f"{a.steps} independent stratified random samples of bra-pair rows "
                                        f"(~{per_step:.0f} s each), each scaled to one build by the exact screened "
                                        f"quartet counts: {build_s:.0f} +- {spread:.0f} s per build")},
            "estimate_spread_s": spread, "estimates_s": [round(x, 1) for x in runs], "calibration": calib,
            "e2e": {"value": value, "unit": "Fock builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def scf_comparison(a, ctx, hf, inputs, rank=0):
    """The SCF half of the metric: time to a converged energy (|dE| < 1e-9, RMS dP < 1e-6; the energy then
    agrees with the plain FP64 SCF's to 1e-8 Eh) on held-out 32-water clusters (seeds (6, m), never trained
    on), for three arms: plain FP64 builds from the core-Hamiltonian guess; mixed precision (FP32 for
    Q_ij Q_kl < 1e-4 until |dE| < 1e-5, then FP64) from the core guess; and mixed precision from the learned
    guess of the shipped network.  Wall times of the SCF call (plus the prediction for the learned arm);
    system setup is reported separately.  Each rank takes its own clusters."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import guess
    w, meta = guess.load_weights()
    model = hf.Model(ctx, w)
    rows = []
    for m in range(a.scf_clusters):
        idx = rank * a.scf_clusters + m
        geom = inputs.water_cluster(a.scf_waters, inputs.CONFIG_GUESS_EVAL, idx)
        basis = inputs.synthetic_basis(geom)
        row = {"cluster": idx}
        for arm, cut, learned in (("fp64", 0.0, False), ("mixed", 1e-4, False), ("mixed_learned", 1e-4, True)):
            t0 = time.perf_counter()
            s = hf.System(ctx, geom, basis, schwarz_tau=a.tau, prim_tau=a.prim_tau, fp32_cutoff=cut)
            torch.cuda.synchronize()
            setup = time.perf_counter() - t0
            t0 = time.perf_counter()
            Pg = guess.predict_or_none(model, s) if learned else None
            r = hf.scf(s, e_tol=1e-9, d_tol=1e-6, P_guess=Pg, raise_on_noconv=False)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            s.close()
            row[arm] = {"s": dt, "iterations": r["iterations"], "mixed_iterations": r["mixed_iterations"],
                        "converged": bool(r["converged"]), "energy": r["energy"], "setup_s": setup,
                        "fock_s": r["seconds_fock"], "diag_s": r["seconds_diag"],
                        "fallback_to_core": bool(learned and Pg is None)}
            print(f"scf cluster {idx} {arm}: {r['iterations']} it {dt:.2f} s E={r['energy']:.10f}", file=sys.stderr,
                  flush=True)
        for arm in ("mixed", "mixed_learned"):
            row[arm]["abs_dE_vs_fp64"] = abs(row[arm]["energy"] - row["fp64"]["energy"])
        rows.append(row)
    mean = lambda arm, k: float(np.mean([r[arm][k] for r in rows]))  # noqa: E731
    out = {"metric": "SCF time to converged energy (|dE|<1e-9, RMS dP<1e-6)", "unit": "s",
           "workload": f"{len(rows)} held-out {a.scf_waters}-water clusters (seeds (6, m)), "
                       f"{25 * a.scf_waters} BF, Schwarz tau={a.tau:g}, primitive tau={a.prim_tau:g}",
           "guess_network": meta,
           "mean_s": {arm: mean(arm, "s") for arm in ("fp64", "mixed", "mixed_learned")},
           "mean_iterations": {arm: mean(arm, "iterations") for arm in ("fp64", "mixed", "mixed_learned")},
           "max_abs_dE_vs_fp64": {arm: float(max(r[arm]["abs_dE_vs_fp64"] for r in rows))
                                  for arm in ("mixed", "mixed_learned")},
           "all_converged": all(r[arm]["converged"] for r in rows for arm in ("fp64", "mixed", "mixed_learned")),
           "rows": rows}
    out["speedup_vs_fp64"] = {arm: out["mean_s"]["fp64"] / out["mean_s"][arm] for arm in ("mixed", "mixed_learned")}
    return out


def run_shard(a):
    """One molecule's Fock build sharded over the ranks (strong scaling): every rank builds the quartet
    shard `rank` of every angular class (hf_fock_build_partial), J and K are summed over the ranks with one
    NCCL allreduce each as device tensors (the paper's ddi_gsumf), and the library assembles F.  At N = 1
    the line also reports the largest difference from hf_fock_build."""
    import torch
    import torch.distributed as dist
    from paper_1708_00033_gb300 import hf, inputs
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    ctx = hf.Context(local)
    sysm = hf.System(ctx, geom, basis, schwarz_tau=a.tau, fp32_cutoff=a.fp32_cutoff, prim_tau=a.prim_tau)
    S, _ = sysm.one_electron()
    P = random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)
    Pd = torch.from_numpy(P).to(dev)

    def allsum(t):
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t

    for _ in range(a.warmup):
        hf.sharded_fock_build(sysm, Pd, rank, world, allsum)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        F, J, K, E = hf.sharded_fock_build(sysm, Pd, rank, world, allsum)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = e0.elapsed_time(e1)
    if world > 1:
        total_ms = reduce_max(total_ms, dist, dev)
        dist.barrier()
    line = {"metric": "Fock builds/s", "value": a.steps / (total_ms / 1e3), "unit": "Fock builds/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a) + ", sharded over the ranks (J, K allreduce)",
                       "parallelism": f"quartet shards x{world}, NCCL allreduce of J and K"},
            "clocks": clk, "E_elec": E}
    if world == 1:
        ref = sysm.fock_build(Pd)
        line["max_abs_dF_vs_fock_build"] = float((F - ref["F"]).abs().max())
        line["abs_dE_vs_fock_build"] = abs(E - ref["E_elec"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_rys(a):
    """Rys quadrature vs Obara-Saika for the classes of total angular momentum L >= 6: per-class device time
    of the same FP64 Fock build (best of `steps` after `warmup`), with the largest difference of F; and the
    build with the library's per-class default choice."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import hf, inputs
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    ctx = hf.Context(0)
    s = hf.System(ctx, geom, basis, schwarz_tau=a.tau, prim_tau=a.prim_tau)
    S, _ = s.one_electron()
    Pd = torch.from_numpy(random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)).cuda()
    res = {}
    for name, rys in (("obara_saika", False), ("rys", True), ("default", None)):
        F = torch.empty_like(Pd)
        for _ in range(max(1, a.warmup)):
            s.fock_build(Pd, F=F, rys=rys)
        best = None
        for _ in range(max(1, a.steps)):
            st = s.fock_build(Pd, F=F, rys=rys, timing=True)["stats"]
            if best is None or st["ms_eri"] < best["ms_eri"]:
                best = st
        res[name] = {"F": F, "stats": best}
    L6 = [c for c in range(hf.NUM_CLASSES) if sum(int(x) for x in hf.CLASS_KERNELS[c][-4:]) >= 6]
    rows = {}
    for c in L6:
        o, r = res["obara_saika"]["stats"], res["rys"]["stats"]
        rows[hf.CLASS_NAMES[c]] = {"quartets": o["class_quartets_fp64"][c], "ms_os": o["ms_class_fp64"][c],
                                   "ms_rys": r["ms_class_fp64"][c],
                                   "gflops_os": o["class_flops_fp64"][c] / max(o["ms_class_fp64"][c], 1e-9) / 1e6,
                                   "gflops_rys": r["class_flops_fp64"][c] / max(r["ms_class_fp64"][c], 1e-9) / 1e6}
    tot_os = sum(v["ms_os"] for v in rows.values())
    tot_rys = sum(v["ms_rys"] for v in rows.values())
    line = {"metric": "ERI class kernel time, Rys quadrature vs Obara-Saika (L >= 6 classes)", "unit": "ms",
            "value": tot_rys, "higher_is_better": False, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "dtype": "f64", "data": "synthetic", "config": {"workload": workload_name(a)},
            "classes": rows, "total_ms_os": tot_os, "total_ms_rys": tot_rys, "speedup_rys": tot_os / tot_rys,
            "build_ms_os": res["obara_saika"]["stats"]["ms_total"], "build_ms_rys": res["rys"]["stats"]["ms_total"],
            "build_ms_default": res["default"]["stats"]["ms_total"],
            "max_abs_dF": float((res["rys"]["F"] - res["obara_saika"]["F"]).abs().max()),
            "max_abs_dF_default": float((res["default"]["F"] - res["obara_saika"]["F"]).abs().max())}
    print(json.dumps(line), flush=True)


def run_case(a):
    """Small fixed workloads for profiler captures (no timing, no JSON line): --case fock (two builds of the
    --waters cluster with --fp32-cutoff), scf (two SCF iterations of the --waters cluster), train (20
    learned-guess training steps of 2,048 random samples)."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import hf, inputs
    ctx = hf.Context(0)
    if a.case == "fock":
        geom = inputs.water_cluster(a.waters, a.config_id, 0)
        s = hf.System(ctx, geom, inputs.synthetic_basis(geom), schwarz_tau=a.tau, prim_tau=a.prim_tau,
                      fp32_cutoff=a.fp32_cutoff)
        S, _ = s.one_electron()
        P = torch.from_numpy(random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)).cuda()
        for _ in range(2):
            out = s.fock_build(P, stats=True)
        torch.cuda.synchronize()
        print("quartets", out["stats"]["quartets_fp64"], out["stats"]["quartets_fp32"], file=sys.stderr)
    elif a.case == "scf":
        geom = inputs.water_cluster(a.waters, a.config_id, 0)
        s = hf.System(ctx, geom, inputs.synthetic_basis(geom), schwarz_tau=a.tau, prim_tau=a.prim_tau)
        r = hf.scf(s, max_iter=2, raise_on_noconv=False)
        print("scf", r["iterations"], r["energy"], file=sys.stderr)
    else:
        rng = np.random.default_rng(0)
        X = torch.from_numpy(rng.standard_normal((4096, 16)).astype(np.float32)).cuda()
        T = torch.from_numpy(rng.standard_normal((4096, 325)).astype(np.float32)).cuda()
        m = hf.Model(ctx, inputs.guess_init_weights(0))
        hf.guess_train(m, X, T, torch.ones_like(T), steps=20, batch=2048)
        print("train done", file=sys.stderr)


def _scf_run(hf, sysm, **kw):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = hf.scf(sysm, **kw)
    torch.cuda.synchronize()
    r["wall_s"] = time.perf_counter() - t0
    return r


def run_scf(a):
    """SCF time to a converged energy (one step = one SCF).  Variants: plain FP64 builds, mixed-then-FP64
    builds, and both with incremental builds (J, K accumulated from density-screened builds of the density
    change, a full rebuild every 8 iterations and before convergence is declared)."""
    from paper_1708_00033_gb300 import hf, inputs
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    ctx = hf.Context(0)
    out = {}
    variants = {"fp64": (0.0, False), "mixed": (1e-4, False), "fp64_incremental": (0.0, True),
                "mixed_incremental": (1e-4, True)}
    for name in a.scf_variants.split(","):
        cut, inc = variants[name]
        t0 = time.perf_counter()
        sysm = hf.System(ctx, geom, basis, schwarz_tau=a.tau, prim_tau=a.prim_tau, fp32_cutoff=cut)
        setup = time.perf_counter() - t0
        r = _scf_run(hf, sysm, e_tol=1e-9, d_tol=1e-6, incremental=inc, raise_on_noconv=False)
        print(f"{name}: converged={r['converged']} it={r['iterations']} full={r['full_builds']} "
              f"{r['wall_s']:.1f} s E={r['energy']:.10f}", file=sys.stderr, flush=True)
        out[name] = {"converged": bool(r["converged"]), "energy": r["energy"], "iterations": r["iterations"],
                     "mixed_iterations": r["mixed_iterations"],
                     "full_builds": r["full_builds"],
                     "scf_s": r["wall_s"], "setup_s": setup, "total_s": r["wall_s"] + setup,
                     "fock_s": r["seconds_fock"], "diag_s": r["seconds_diag"], "jacobi_sweeps": r["jacobi_sweeps"],
                     "energies": [float(x) for x in r["energies"]]}
        del sysm
    base = out[next(iter(out))]
    line = {"metric": "SCF time to converged energy (|dE|<1e-9, RMS dP<1e-6)", "value": base["total_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": 1, "warmup": 0,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{a.waters}-water cluster SCF, core-Hamiltonian guess", "schwarz_tau": a.tau,
                       "prim_tau": a.prim_tau},
            "variants": out,
            "energy_diff_vs_first": {k: abs(v["energy"] - base["energy"]) for k, v in out.items()},
            "speedup_vs_first": {k: base["total_s"] / v["total_s"] for k, v in out.items()}}
    print(json.dumps(line), flush=True)


def run_mixed(a):
    """One mixed-precision build vs one FP64 build of the same cluster."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import hf, inputs
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    ctx = hf.Context(0)
    res = {}
    Pd = None
    for name, cut in (("mixed", a.fp32_cutoff), ("fp64", 0.0)):
        t0 = time.perf_counter()
        sysm = hf.System(ctx, geom, basis, schwarz_tau=a.tau, prim_tau=a.prim_tau, fp32_cutoff=cut)
        setup = time.perf_counter() - t0
        if Pd is None:
            S, _ = sysm.one_electron()
            P = random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)
            Pd = torch.from_numpy(P).cuda()
            del S
        Fd = torch.empty_like(Pd)
        if name == "mixed":
            sysm.fock_build(Pd, F=Fd)  # warm-up (the FP64 build runs for minutes and needs none)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = sysm.fock_build(Pd, F=Fd, timing=True)
        e1.record()
        torch.cuda.synchronize()
        res[name] = {"ms": e0.elapsed_time(e1), "E_elec": out["E_elec"], "stats": out["stats"], "setup_s": setup,
                     "F": Fd.clone()}
        del sysm
    st = res["mixed"]["stats"]
    dF = float((res["mixed"]["F"] - res["fp64"]["F"]).abs().max())
    n32 = st["quartets_fp32"]
    line = {"metric": "Fock builds/s", "value": 1e3 / res["mixed"]["ms"], "unit": "Fock builds/s",
            "higher_is_better": True, "n_gpus": 1, "steps": 1, "warmup": 1, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "fp32_cutoff": a.fp32_cutoff},
            "fp64_builds_per_s": 1e3 / res["fp64"]["ms"], "speedup_vs_fp64": res["fp64"]["ms"] / res["mixed"]["ms"],
            "abs_dE_vs_fp64_gpu": abs(res["mixed"]["E_elec"] - res["fp64"]["E_elec"]), "max_abs_dF_vs_fp64_gpu": dF,
            "fp32_quartet_fraction": n32 / max(1, n32 + st["quartets_fp64"]),
            "ms": {k: v["ms"] for k, v in res.items()}, "setup_s": {k: v["setup_s"] for k, v in res.items()},
            "flops": {"fp64": st["flops_fp64"], "fp32": st["flops_fp32"]},
            "class_ms_fp32": [round(x, 2) for x in st["ms_class_fp32"]],
            "class_ms_fp64": [round(x, 2) for x in st["ms_class_fp64"]]}
    print(json.dumps(line), flush=True)


def run_batch(a):
    """512 independent clusters of 1..16 waters: graph-captured batched builds vs per-molecule launches."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import hf, inputs
    ctx = hf.Context(0)
    geoms = [inputs.batch_cluster(inputs.CONFIG_BATCH, m) for m in range(a.n_mol)]
    bases = [inputs.synthetic_basis(g) for g in geoms]
    t0 = time.perf_counter()
    batch = hf.Batch(ctx, geoms, bases, schwarz_tau=a.tau, prim_tau=a.prim_tau)
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    batch.tune(os.path.join(tempfile.gettempdir(), "hf_batch_tune.txt"), sample_quartets=500000)
    tune_s = time.perf_counter() - t0
    rng = np.random.default_rng(4)
    P = np.zeros(int(batch.offsets[-1]))
    for m, n in enumerate(batch.n_bf):
        G = rng.standard_normal((n, max(1, n // 5)))
        P[batch.offsets[m]:batch.offsets[m + 1]] = (0.2 * G @ G.T).ravel()
    Pd = torch.from_numpy(P).cuda()
    F = torch.empty_like(Pd)
    for _ in range(a.warmup):
        batch.fock_build(Pd, F)
    ms_graph = [batch.fock_build(Pd, F)[0] for _ in range(a.steps)]
    Fs = torch.empty_like(Pd)
    batch.fock_build(Pd, Fs, sequential=True)
    ms_seq = [batch.fock_build(Pd, Fs, sequential=True)[0] for _ in range(max(1, a.steps // 2))]
    dF = float((F - Fs).abs().max())
    info = batch.info()
    g = sum(ms_graph) / len(ms_graph)
    s = sum(ms_seq) / len(ms_seq)
    line = {"metric": "Fock builds/s", "value": a.n_mol / (g / 1e3), "unit": "molecule Fock builds/s",
            "higher_is_better": True, "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{a.n_mol} clusters of U{{1..16}} waters (seeds (4,m)), Schwarz tau={a.tau:g}, "
                                   f"primitive tau={a.prim_tau:g}", "n_bf_total": info["n_bf_total"],
                       "quartets": info["quartets"]},
            "graph_ms": g, "sequential_ms": s, "sequential_builds_per_s": a.n_mol / (s / 1e3),
            "speedup_vs_per_molecule_launches": s / g, "max_abs_dF_graph_vs_sequential": dF,
            "setup_s": setup, "tune_s": tune_s,
            "tuned": {"block": info["block"], "chunk": info["chunk"], "blocks_per_sm": info["blocks_per_sm"]}}
    print(json.dumps(line), flush=True)


def run_guess(a):
    """Learned initial guess: train on plain-SCF densities of U{2..8}-water clusters (seeds (5,m)), then
    compare SCF iterations/time from the learned vs the core-Hamiltonian guess on 32-water clusters (seeds (6,m))."""
    import numpy as np
    from paper_1708_00033_gb300 import guess, hf
    ctx = hf.Context(0)
    logs = []
    log = lambda s: (logs.append(s), print(s, file=sys.stderr, flush=True))  # noqa: E731
    if a.n_train > 0:
        data = guess.make_dataset(ctx, a.n_train, log=log, workers=8)
        model = hf.Model(ctx, guess.init_weights(0))
        t0 = time.perf_counter()
        losses = guess.train(model, data, steps=a.train_steps, batch=2048, lr=1e-3, log=log)
        train_s = time.perf_counter() - t0
        np.save(os.path.join(tempfile.gettempdir(), "hf_guess_weights.npy"), model.weights())
        dataset_s, samples = data["seconds"], int(data["X"].shape[0])
        loss0, loss1 = float(np.mean(losses[:10])), float(np.mean(losses[-100:]))
    else:  # the shipped network
        w, meta = guess.load_weights()
        model = hf.Model(ctx, w)
        train_s, dataset_s, samples = meta["train_s"], meta["dataset_s"], meta["atom_pairs"]
        loss0, loss1 = meta["loss_first10"], meta["loss_last100"]
    ev = guess.evaluate(ctx, model, n_eval=a.n_eval, waters=32, log=log)
    line = {"metric": "SCF time to converged energy, learned vs core-Hamiltonian guess", "value": ev["mean_mixed_learned_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": a.n_eval, "warmup": 0, "dtype": "bf16+f32 (MLP), f64 (SCF)",
            "data": "synthetic",
            "config": {"workload": f"train {a.n_train or 2000} clusters U{{2..8}} waters seeds (5,m); eval {a.n_eval} 32-water clusters seeds (6,m)",
                       "schwarz_tau": a.tau, "prim_tau": a.prim_tau, "train_steps": a.train_steps},
            "dataset_s": dataset_s, "train_samples": samples, "train_s": train_s,
            "final_loss": loss1, "initial_loss": loss0, "network": "shipped" if a.n_train <= 0 else "trained here",
            "mean_core_iterations": ev["mean_core_iterations"], "mean_learned_iterations": ev["mean_learned_iterations"],
            "mean_mixed_learned_iterations": ev["mean_mixed_learned_iterations"],
            "mean_core_s": ev["mean_core_s"], "mean_learned_s": ev["mean_learned_s"],
            "mean_mixed_learned_s": ev["mean_mixed_learned_s"],
            "speedup_learned": ev["mean_core_s"] / ev["mean_learned_s"],
            "speedup_mixed_learned": ev["mean_core_s"] / ev["mean_mixed_learned_s"],
            "max_abs_dE": ev["max_abs_dE"], "max_abs_dE_mixed": ev["max_abs_dE_mixed"],
            "fallbacks": ev["fallbacks"], "rows": ev["rows"]}
    print(json.dumps(line), flush=True)


def run_copies(a):
    """Shared vs private Fock accumulators (the paper's Table 3 comparison on GPU thread blocks): FP64 build
    time per accumulator-copy count, per workload, with the device memory the copies take."""
    import numpy as np
    import torch
    from paper_1708_00033_gb300 import hf, inputs
    ctx = hf.Context(0)
    copies = [int(c) for c in a.copies.split(",")]
    rows = []
    for item in a.copies_workloads.split(","):
        nw, tau = item.split(":")
        nw, tau = int(nw), float(tau)
        cfg = inputs.CONFIG_SINGLE_BUILD if nw == 4 else a.config_id
        geom = inputs.water_cluster(nw, cfg, 0)
        basis = inputs.synthetic_basis(geom)
        s = hf.System(ctx, geom, basis, schwarz_tau=tau, prim_tau=a.prim_tau)
        S, _ = s.one_electron()
        Pd = torch.from_numpy(random_density(S, inputs.n_electrons(geom) // 2, cfg, 0)).cuda()
        Fd = torch.empty_like(Pd)
        ref = None
        steps = max(1, a.steps)
        for c in copies:
            s.set_fock_copies(c)
            s.fock_build(Pd, F=Fd)  # warm-up
            torch.cuda.synchronize()
            ms = []
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.fock_build(Pd, F=Fd)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            F = Fd.cpu().numpy()
            if ref is None:
                ref = F
            rows.append({"waters": nw, "n_bf": s.n_bf, "schwarz_tau": tau, "copies": c,
                         "ms_median": float(np.median(ms)), "ms": ms,
                         "copy_bytes": 0 if c == 1 else 2 * c * s.n_bf * s.n_bf * 8,
                         "max_abs_dF_vs_shared": float(np.abs(F - ref).max())})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        s.close()
    line = {"metric": "FP64 Fock build time, shared vs private accumulators", "unit": "ms", "value": None,
            "higher_is_better": False, "n_gpus": 1, "steps": a.steps, "warmup": 1, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "water clusters, random S-orthonormal density",
                                            "prim_tau": a.prim_tau},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_peaks(a):
    """The roofline denominators measured by the library's own microbenchmarks, with clocks sampled."""
    from paper_1708_00033_gb300 import hf
    ctx = hf.Context(0)
    hf.measure_peaks(ctx)  # warm-up
    clk = ClockSampler(0)
    clk.start()
    runs = [hf.measure_peaks(ctx) for _ in range(max(1, a.steps))]
    clocks = clk.stop()
    best = {k: max(r[k] for r in runs) for k in runs[0]}
    derived = best["num_sms"] * 2 * 2 * best["sm_max_mhz"] * 1e-3
    line = {"metric": "device peaks (microbenchmarks)", "unit": "GFLOP/s | Gop/s", "value": best["fp64_fma_gflops"],
            "higher_is_better": True, "n_gpus": 1, "steps": len(runs), "warmup": 1, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "FMA chains on every SM; FP64 atomic adds into 8 MB"},
            "best": best, "runs": runs, "fp64_fma_derived_gflops": derived,
            "fp32_to_fp64_ratio": best["fp32_fma_gflops"] / best["fp64_fma_gflops"], "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "scf":
        run_scf(a)
    elif a.mode == "mixed":
        run_mixed(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "guess":
        run_guess(a)
    elif a.mode == "copies":
        run_copies(a)
    elif a.mode == "peaks":
        run_peaks(a)
    elif a.mode == "shard":
        run_shard(a)
    elif a.mode == "rys":
        run_rys(a)
    elif a.mode == "case":
        run_case(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
