#!/usr/bin/env python
"""Fock builds/s of the GB300 direct-SCF Fock build (one JSON line on stdout).

Workload (default): the 64-water cluster of the SCF configuration (seed
(2, rank)), 1,600 Cartesian basis functions, Schwarz screening at 1e-10,
plain FP64 integrals; one step = one full Fock build (density in, J and K of
all 21 angular classes, F = H + J - K/2 and the energy out).  With N ranks
each rank builds its own cluster (independent problems, weak scaling, no
collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (as it stands) on the host cores over
strided samples of the same Fock build and reports the same metric.
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
# kernel and traffic is null).
NCU_TRAFFIC = {"kernel": "k_eri_1000", "bytes_per_launch": None, "sources_sha256": None}
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
    ap.add_argument("--prim-tau", type=float, default=1e-14)
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="oracle time budget of --impl reference over all its steps")
    ap.add_argument("--mode", default="fock", choices=["fock", "scf", "mixed", "batch", "guess", "copies", "peaks"])
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-eval", type=int, default=32)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--n-mol", type=int, default=512)
    ap.add_argument("--scf-variants", default="fp64,mixed,fp64_incremental,mixed_incremental")
    ap.add_argument("--copies", default="1,8,152,608", help="accumulator copies compared by --mode copies")
    ap.add_argument("--copies-workloads", default="4:0,16:1e-10,64:1e-10", help="waters:schwarz_tau list")
    a = ap.parse_args()
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
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, geom, basis, P, a.cpu_sample_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _oracle_sample(a, geom, basis, P, seconds, offset=0, mol=None):
    """Time the oracle on every stride-th bra pair; extrapolate to one build."""
    import oracle
    if mol is None:
        mol = oracle.Molecule(geom, basis)
    mol.schwarz()  # setup, untimed
    n_sh = mol.n_shells
    n_p = n_sh * (n_sh + 1) // 2
    total_unscreened = n_p * (n_p + 1) // 2
    # calibrate the stride on a tiny sample
    stride = max(1, n_p // 8)
    t0 = time.perf_counter()
    _, u0 = mol.jk_unique_sample(P, a.tau, stride, offset)
    dt0 = max(time.perf_counter() - t0, 1e-3)
    rate = u0 / dt0
    stride = max(1, int(stride * (dt0 / seconds)) if dt0 < seconds else stride)
    t0 = time.perf_counter()
    nq, u = mol.jk_unique_sample(P, a.tau, stride, offset)
    dt = time.perf_counter() - t0
    build_s = dt * total_unscreened / max(u, 1)
    return mol, {"seconds": dt, "stride": stride, "quartets": nq, "unscreened_rows": u,
                 "est_build_s": build_s, "value": 1.0 / build_s, "rate_hint": rate}


def cpu_baseline(a, geom, basis, P, seconds):
    import oracle
    _, r = _oracle_sample(a, geom, basis, P, seconds)
    return {"value": r["value"], "unit": "Fock builds/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"oracle unique-quartet digestion over every {r['stride']}-th bra shell pair "
                       f"({r['quartets']} screened quartets, {r['seconds']:.1f} s), scaled by the unscreened "
                       f"quartets the sampled rows span to one full build ({r['est_build_s']:.0f} s)")}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1708_00033_gb300 import inputs
    geom = inputs.water_cluster(a.waters, a.config_id, 0)
    basis = inputs.synthetic_basis(geom)
    mol = oracle.Molecule(geom, basis)
    S, _ = mol.core_hamiltonian()
    P = random_density(S, inputs.n_electrons(geom) // 2, a.config_id, 0)
    per_step = max(1.0, a.reference_seconds / max(1, a.steps + a.warmup))
    for w in range(a.warmup):
        _oracle_sample(a, geom, basis, P, per_step / 4, offset=w, mol=mol)
    est = []
    for k in range(a.steps):
        _, r = _oracle_sample(a, geom, basis, P, per_step, offset=a.warmup + k, mol=mol)
        est.append(r)
    build_s = sum(r["est_build_s"] for r in est) / len(est)
    value = 1.0 / build_s
    line = {"metric": "Fock builds/s", "value": value, "unit": "Fock builds/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": build_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(a), "waters": a.waters, "schwarz_tau": a.tau},
            "cpu_baseline": {"value": value, "unit": "Fock builds/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{a.steps} strided bra-pair samples of ~{per_step:.0f} s each, scaled to one build"},
            "e2e": {"value": value, "unit": "Fock builds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    data = guess.make_dataset(ctx, a.n_train, log=log)
    model = hf.Model(ctx, guess.init_weights(0))
    t0 = time.perf_counter()
    losses = guess.train(model, data, steps=a.train_steps, batch=2048, lr=1e-3, log=log)
    train_s = time.perf_counter() - t0
    np.save(os.path.join(tempfile.gettempdir(), "hf_guess_weights.npy"), model.weights())
    ev = guess.evaluate(ctx, model, n_eval=a.n_eval, waters=32, log=log)
    line = {"metric": "SCF time to converged energy, learned vs core-Hamiltonian guess", "value": ev["mean_mixed_learned_s"],
            "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": a.n_eval, "warmup": 0, "dtype": "bf16+f32 (MLP), f64 (SCF)",
            "data": "synthetic",
            "config": {"workload": f"train {a.n_train} clusters U{{2..8}} waters seeds (5,m); eval {a.n_eval} 32-water clusters seeds (6,m)",
                       "schwarz_tau": 1e-10, "prim_tau": 1e-14, "train_steps": a.train_steps},
            "dataset_s": data["seconds"], "train_samples": int(data["X"].shape[0]), "train_s": train_s,
            "final_loss": float(np.mean(losses[-100:])), "initial_loss": float(np.mean(losses[:10])),
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
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
