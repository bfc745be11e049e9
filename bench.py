"""Benchmark of the ROKS plane-wave hot path on GB300.

A step is one PCG iteration (every row of the hot path: density, Hartree and
Slater potentials, class potentials, F^n|n> and S|n> for all bands,
subspace matrices, gradient, TPA preconditioner, Fletcher-Reeves direction,
trial and final rotation + Cholesky orthonormalisation with their density
and energy passes).  The metric counts the band applications F^n|psi_n>
per second (one per band per step) and also reports seconds per PCG
iteration and seconds to converge (|dE| < 1e-6 Ha twice), mixed precision
against the plain FP64 GPU path.

Default workload: the MgO-vacancy-shaped supercell (3x3x3 rocksalt cell,
a = 7.96 Bohr, one O removed: 215 atoms, 1288 projectors; 120^3 grid, Ecut
15 Ha, 37705 plane waves; 428 closed + 2 open bands), synthetic seeded
inputs, mixed precision.  The time-to-convergence legs (mixed vs plain FP64,
TPA with and without the learned correction, DIIS) run on the organic-molecule
box (20 Bohr, 96^3, 34265 plane waves, 172 projectors, 40 + 2 bands), where
the FP64 leg converges within a minute.  Multi-GPU (torchrun): independent
replicas, one per rank (seed = rank), no collective on the data path.

--impl reference times the FP64 CPU oracle (the only reference there is) on
a bounded sample of the same workload on all host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ROKS band-H|ψ> applies/s; s/PCG-to-1e-6 Ha, chosen vs plain FP64 on 1 GB300"
UNIT = "band-applies/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="mgo-120")
    ap.add_argument("--converge-workload", default="organic-96",
                    help="workload of the time-to-convergence legs")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--converge-iters", type=int, default=2000,
                    help="iteration cap of the time-to-convergence runs (0 skips them)")
    ap.add_argument("--converge-seconds", type=float, default=60.0,
                    help="wall-clock cap of each time-to-convergence run")
    ap.add_argument("--g-tol", type=float, default=2e-4,
                    help="gradient-norm criterion of the convergence legs (beside |dE| < 1e-6 Ha twice)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU work per host core of the oracle sample")
    ap.add_argument("--hybrid-applies", type=int, default=3,
                    help="timed roks_apply_h calls on the hybrid-exchange workload (hybrid-72); 0 skips them")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--force-calls", type=int, default=10,
                    help="timed roks_forces calls on the final orbitals; 0 skips them")
    ap.add_argument("--n-closed", type=int, default=0,
                    help="override the workload's closed-shell band count (profiler captures of a "
                         "smaller context with the same block shapes); 0: the workload's own")
    ap.add_argument("--gamma-steps", type=int, default=20,
                    help="PCG steps of the Gamma-point leg (real orbitals, half sphere; 0: skip)")
    ap.add_argument("--autotune", type=int, default=1, choices=(0, 1),
                    help="1: the library times its launch shapes on each context's buffers at setup; "
                         "0: the default shapes (for profiler runs, whose timing the autotuner should not read)")
    ap.add_argument("--gga-steps", type=int, default=10,
                    help="PCG steps of the PBE-exchange leg (roks_options.xc = ROKS_XC_PBE_X; 0: skip)")
    ap.add_argument("--diis-steps", type=int, default=50,
                    help="timed DIIS steps (roks_diis_step) after the PCG legs; 0 skips them")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Largest value of x over the ranks (all-reduce MAX on `device`); x itself
    when one process runs.  Timings are reported as the slowest rank's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_config(workload: str, rank: int) -> dict:
    """Each replica steps its own seeded system (seed = rank): the path does not
    shard, so N GPUs run N independent problems (weak scaling)."""
    from paper_2605_28637_gb300 import synthetic as syn
    return syn.make_config(workload, rank)


def syn_with(cfg: dict, **kw) -> dict:
    from paper_2605_28637_gb300 import synthetic as syn
    return syn.with_changes(cfg, **kw)


def aggregate_value(nb: int, steps: int, world: int, ms_max: float) -> float:
    """Band-applies per second of the whole job: all ranks' bands over the slowest rank's time."""
    return nb * steps * world / (ms_max / 1000.0)


# FP32 FMA rate from the unit counts and the maximum SM clock (no measured
# FP32 peak is provided): 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_TFLOPS_NOMINAL = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_TFLOPS_NOMINAL = 1.25
# FP32 (SIMT) and FP64 throughput measured on this GPU by measure_alu_peaks
# (cuBLAS SGEMM with TF32 off, DGEMM), when the bench has run it
MEASURED_ALU = {}


def measure_alu_peaks(torch):
    """Dense GEMM throughput of the library cuBLAS in FP32 (TF32 disabled)
    and FP64, timed with CUDA events after a warm-up: the denominators of the
    SIMT-FP32 and FP64 rooflines (MEASURED_PEAKS.json holds the HBM copy and
    BF16 rates only)."""
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n, reps in (("fp32", torch.float32, 8192, 5), ("fp64", torch.float64, 4096, 3)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            c = a @ b
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                c = a @ b
            e1.record()
            torch.cuda.synchronize()
            out[name] = 2.0 * n ** 3 * reps / (e0.elapsed_time(e1) / 1000.0) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    MEASURED_ALU.update(out)
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=None):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                if gpu_index is not None and parts[0] != str(gpu_index):
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- algorithmic bytes per launch
def algorithmic_bytes(ctx, cfg, family: str, csize: int, rsize: int):
    """Compulsory DRAM bytes of one launch of a kernel family (all bands)."""
    N = cfg["grid"]
    nb, npw = ctx.nb, ctx.npw
    geo = _geometry(ctx.miller)
    npl, ncol = geo["np"], geo["ncol"]
    planes = nb * npl * N * N * csize
    cols = nb * ncol * N * csize
    band = nb * npw * csize
    return {
        "fft_x_apply": 2 * planes + 3 * N ** 3 * rsize,
        "fft_x_density": planes + 3 * N ** 3 * 8,
        "fft_y_inv": cols + planes,
        "fft_y_fwd": planes + cols,
        "fft_z_inv": band + cols,
        "fft_z_fwd": cols + 2 * band,
    }.get(family)


def family_work(ctx, cfg, family: str, csize: int, rsize: int, precision: str, tensor=frozenset()):
    """(bound, algorithmic work per launch) of a kernel family: compulsory
    DRAM bytes for the band-transform stages, flops (8 per complex
    multiply-add) for the contractions; None for other families."""
    b = algorithmic_bytes(ctx, cfg, family, csize, rsize)
    if b is not None:
        return "hbm", float(b)
    npw, nb, npj = float(ctx.npw), float(ctx.nb), float(ctx.nproj)
    flops = {
        "proj_PhPsi": 8 * npw * npj * nb,          # B = P^H Psi
        "proj_PX": 8 * npw * npj * nb,             # F += P (D B) or S = Psi + P (Q B)
        "orth_overlap": 8 * npw * nb * nb,         # O = Psi^H Psi
        "orth_apply": 8 * npw * nb * nb,           # Psi L^{-H}
        "subspace_theta": 8 * npw * nb * nb,       # Theta = Psi^H F Psi
        "subspace_project": 16 * npw * nb * nb,    # (S Psi)^H x, then x - Psi M
        "gradient_precond": 16 * npw * nb * nb,    # F - S Gam, F - S Theta
    }.get(family)
    if flops is None or flops == 0:
        return None
    return ("tensor" if family in tensor else "alu"), flops


def tensor_families(ctx, precision: str, tc_launches: int):
    """Kernel families whose products the library puts on the tcgen05 tensor
    cores at this workload (the shape rule of k_tcgemm.cu: A^H B with
    M >= 128, N >= 64, K >= 1024; tall products with M >= 4096, N >= 64,
    K >= 64), provided tensor-core launches were counted."""
    if precision != "mixed" or not tc_launches:
        return frozenset()
    nb, npj, npw = ctx.nb, ctx.nproj, ctx.npw

    def cn(M, N, K):
        return M >= 128 and N >= 64 and K >= 1024

    def nn(M, N, K):
        return M >= 4096 and N >= 64 and K >= 64
    fams = set()
    if cn(npj, nb, npw):
        fams.add("proj_PhPsi")
    if nn(npw, nb, npj):
        fams.add("proj_PX")
    if cn(nb, nb, npw):
        fams |= {"orth_overlap", "subspace_theta"}
    if nn(npw, nb, nb):
        fams |= {"orth_apply", "gradient_precond"}
    if cn(nb, nb, npw) and nn(npw, nb, nb):
        fams.add("subspace_project")
    return frozenset(fams)


def bf16_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def alu_peak(precision: str, bound: str = "alu"):
    """Peak of a contraction family.  Tensor cores: the TF32 rate (measured
    bf16 peak x the nominal TF32/BF16 ratio 1.1/2.25) over the three TF32
    products each FP32 product takes.  SIMT: FP32 FMA from the unit counts
    and clock (no measured FP32 peak is provided), or the FP64 rate."""
    if bound == "tensor":
        b, kind = bf16_peak()
        return b * (1.1 / 2.25) / 3.0, (f"{kind} bf16 peak x 1.1/2.25 (TF32) / 3 TF32 products per FP32 product")
    if precision == "fp64":
        if "fp64" in MEASURED_ALU:
            return MEASURED_ALU["fp64"], "measured FP64 (cuBLAS DGEMM on this GPU)"
        return FP64_TFLOPS_NOMINAL, "nominal FP64: 1.25 TFLOP/s (GB300 dense FP64)"
    if "fp32" in MEASURED_ALU:
        return MEASURED_ALU["fp32"], "measured FP32 SIMT (cuBLAS SGEMM, TF32 off, on this GPU)"
    return FP32_TFLOPS_NOMINAL, "nominal FP32: 152 SMs x 128 lanes x 2 flops x 2.07 GHz"


def _geometry(miller):
    ij = {(int(a), int(b)) for a, b, _ in miller}
    i = {int(a) for a, _, _ in miller}
    return {"ncol": len(ij), "np": len(i)}


def traffic_record(family, workload=None, alg_bytes=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (one hash over every file listed).  A
    capture on a smaller workload (the capture size rule keeps full-size
    multi-pass captures off the GPU) is scaled to this launch by the ratio of
    algorithmic bytes (the stage streams its planes once per band, so its
    traffic grows in proportion); returns (bytes, note)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None, None
    with open(p) as f:
        rec = json.load(f)
    ent = rec.get("kernels", {}).get(family)
    if not ent:
        return None, None
    h = hashlib.sha256()
    for rel_path in ent.get("sources", []):
        src = os.path.join(ROOT, rel_path)
        if not os.path.exists(src):
            return None, None
        with open(src, "rb") as f:
            h.update(f.read())
    if not ent.get("sources") or h.hexdigest()[:16] != ent.get("source_sha"):
        return None, None
    if workload is None or workload == ent.get("workload"):
        return float(ent["bytes_per_launch"]), f"ncu on {ent.get('workload')}"
    if alg_bytes and ent.get("algorithmic_bytes_per_launch"):
        scaled = float(ent["bytes_per_launch"]) * alg_bytes / float(ent["algorithmic_bytes_per_launch"])
        return scaled, f"ncu on {ent.get('workload')}, scaled by algorithmic bytes"
    return None, None


# ---------------------------------------------------------------- CPU oracle sample
def host_cores() -> int:
    """Host cores this process may run on (the affinity mask; os.cpu_count()
    where the mask is not available)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _mem_available_bytes() -> float:
    """Memory the oracle workers may use: MemAvailable, capped by a cgroup limit."""
    avail = float("inf")
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = float(line.split()[1]) * 1024
    except Exception:
        pass
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            with open(path) as f:
                v = f.read().strip()
            if v.isdigit():
                avail = min(avail, float(v))
        except Exception:
            pass
    return avail


def _oracle_worker(name, seed, band, mode, amount, warmup, barrier, out):
    """One host core: the oracle's F^n|n> (kinetic + local + non-local, FP64)
    of one band of the seeded start, at the potential of the start's first
    two bands, repeated `amount` times (mode "steps", after `warmup` untimed
    repeats) or for `amount` seconds (mode "seconds").  The timed loops of all
    workers start together (barrier)."""
    try:
        from oracle import roks as R
        from paper_2605_28637_gb300 import synthetic as syn
        cfg = syn.make_config(name, seed)
        s = R.System(cfg)

        def band_coeffs(b0, nb):
            u = syn.orbital_uniforms(cfg, s.npw, b0, nb)
            return (u[..., 0] + 1j * u[..., 1]).T / (1.0 + s.g2)[:, None]

        rho = np.zeros((3, s.N ** 3))
        c2 = band_coeffs(0, min(2, s.nb))
        for n in range(c2.shape[1]):
            psi = s.to_real(c2[:, n])
            rho[0] += (psi.conj() * psi).real
        pot = s.potentials(rho)
        b = band % s.nb
        X = band_coeffs(b, 1)
        cls = s.cls[b:b + 1]
        for _ in range(warmup):
            s.apply(X, pot, classes=cls)
        barrier.wait(timeout=600)
        t0 = time.perf_counter()
        reps = 0
        while (mode == "steps" and reps < amount) or (mode == "seconds" and (reps == 0 or
                                                                              time.perf_counter() - t0 < amount)):
            s.apply(X, pot, classes=cls)
            reps += 1
        out.put((reps, time.perf_counter() - t0, s.npw, s.nproj))
    except Exception as e:   # reported by the parent
        try:
            barrier.abort()
        except Exception:
            pass
        out.put(("error", repr(e)))


def oracle_parallel(name: str, seed: int, mode: str, amount: float, warmup: int = 0, per_worker_gb: float = 2.5):
    """The oracle's band applies on all host cores at once: one spawned
    process per core (each with single-threaded BLAS), each applying F to its
    own band of the workload.  Returns band-applies/s over the slowest
    worker's timed loop, the cores used and the seconds."""
    import multiprocessing as mp
    cores = host_cores()
    mem_cap = int(0.6 * _mem_available_bytes() / (per_worker_gb * 2 ** 30))
    workers = max(1, min(cores, mem_cap))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(name, seed, w, mode, amount, warmup, barrier, out))
             for w in range(workers)]
    for p in procs:
        p.start()
    res = [out.get(timeout=1800) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    errs = [r[1] for r in res if r[0] == "error"]
    if errs:
        raise RuntimeError(f"oracle worker failed: {errs[0]}")
    applies = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return {"value": applies / dt, "cores": workers, "seconds": dt, "applies": applies,
            "npw": res[0][2], "nproj": res[0][3], "host_cores": cores}


def cpp_oracle_rate(name: str, seed: int, mode: str, amount: float, warmup: int = 0):
    """The C++ FP64 oracle's band applies on all host cores (OpenMP, one band
    per thread): F^n|n> of `cores` bands of the seeded start at the potential
    of its first two bands, repeated `amount` times (mode "steps", after
    `warmup` untimed rounds) or for `amount` seconds."""
    from oracle import cpp_oracle as CO
    from paper_2605_28637_gb300 import synthetic as syn
    cfg = syn.make_config(name, seed)
    cores = host_cores()
    c = CO.CppSystem(cfg, threads=cores)
    g2 = (np.asarray(c.miller, dtype=np.float64) ** 2).sum(axis=1) * (2.0 * np.pi / cfg["L"]) ** 2

    def coeffs(b0, nb):
        u = syn.orbital_uniforms(cfg, c.npw, b0, nb)
        return (u[..., 0] + 1j * u[..., 1]).T / (1.0 + g2)[:, None]

    Vk, _ = c.potentials(c.class_densities(coeffs(0, min(2, c.nb))))
    nb = min(cores, c.nb)
    X = coeffs(0, nb)
    cls = c.cls[:nb]
    for _ in range(warmup):
        c.apply(X, Vk, classes=cls)
    t0 = time.perf_counter()
    rounds = 0
    while (mode == "steps" and rounds < amount) or (mode == "seconds" and (rounds == 0 or
                                                                            time.perf_counter() - t0 < amount)):
        c.apply(X, Vk, classes=cls)
        rounds += 1
    dt = time.perf_counter() - t0
    out = {"value": rounds * nb / dt, "cores": cores, "seconds": dt, "applies": rounds * nb, "npw": c.npw,
           "nproj": c.nproj, "host_cores": cores, "kind": "C++ oracle (OpenMP)"}
    c.close()
    return out


def cpu_baseline_leg(name: str, seconds: float):
    """The FP64 C++ oracle on all host cores; the NumPy oracle (one process
    per core) if the C++ one cannot be built on this host."""
    try:
        r = cpp_oracle_rate(name, 0, "seconds", seconds)
        impl = "FP64 C++ oracle, OpenMP"
    except Exception:
        r = oracle_parallel(name, 0, "seconds", seconds)
        impl = "FP64 numpy oracle, one process per core"
    desc = (f"F^n|n> (kinetic + local + non-local, {impl}) of one band per core of {name} "
            f"({r['npw']} plane waves, {r['nproj']} projectors) at the potential of the seeded start's first two "
            f"bands, repeated for about {seconds:.0f} s on {r['cores']} host cores at once "
            f"({r['applies']} band applies); scaled to band-applies/s")
    return {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": desc,
            "seconds": r["seconds"], "host_cores": r["host_cores"]}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2605_28637_gb300 import synthetic as syn
    cfg = syn.make_config(args.workload, 0)
    # each step: every host core applies F to one band of the workload
    try:
        r = cpp_oracle_rate(args.workload, 0, "steps", args.steps, warmup=args.warmup)
        impl = "FP64 C++ oracle (OpenMP)"
    except Exception:
        r = oracle_parallel(args.workload, 0, "steps", args.steps, warmup=args.warmup)
        impl = "FP64 numpy oracle (one process per core)"
    value = r["value"]
    sample = (f"each step: F^n|n> (kinetic + local + non-local) of one band per host core of {cfg['name']} "
              f"({cfg['grid']}^3, {r['npw']} plane waves, {r['nproj']} projectors), {impl}, "
              f"{r['cores']} cores at once, fixed potential")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * r["seconds"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": cfg["name"], "grid": cfg["grid"], "bands": syn.n_bands(cfg),
                       "plane_waves": r["npw"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def time_pcg(ctx, psi, steps, torch, profile=False):
    from paper_2605_28637_gb300 import roks
    st = ctx.stream
    if profile:
        roks.roks_profile_enable(ctx.ctx, 1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    infos = []
    for _ in range(steps):
        infos.append(ctx.pcg_step(psi))
    e1.record(st)
    torch.cuda.synchronize()
    prof = None
    if profile:
        prof = roks.roks_profile_read(ctx.ctx)
        roks.roks_profile_enable(ctx.ctx, 0)
    return e0.elapsed_time(e1), infos, prof


def converge(cfg, precision, cap, torch, max_seconds, g_tol, params=None, keep=False):
    """Seconds and iterations of PCG from the seeded start to |dE| < 1e-6 Ha
    twice with |g| < g_tol, stopped after cap iterations or max_seconds of
    wall clock; with params, the TPA step is corrected by the trained network
    (TPA judges the last steps).  keep: also return the final orbitals."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    ctx = roks.Context(cfg, precision, e_tol=1e-6, g_tol=g_tol)
    if params is not None:
        ctx.set_preconditioner(params)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, info = 0, None
    for it in range(1, cap + 1):
        info = ctx.pcg_step(psi)
        if info["converged"] or time.perf_counter() - t0 > max_seconds:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"seconds": dt, "iterations": it, "converged": bool(info and info["converged"]),
           "E_final": info["E_new"] if info else None, "grad_norm_final": info["grad_norm"] if info else None,
           "s_per_iter": dt / max(it, 1)}
    psi64 = None
    if info is not None:
        # the final orbitals re-evaluated in FP64 (orthonormalised there first):
        # a mixed leg's energy must be that of its own state, not an FP32 artefact
        c64 = roks.Context(cfg, "fp64")
        psi64 = c64.new_bands()
        psi64[:, :ctx.npw] = psi[:, :ctx.npw].to(psi64.dtype)
        torch.cuda.synchronize()
        roks.roks_orthonormalize(c64.ctx, psi64, c64.ld)
        c64.density(psi64)
        out["E_final_fp64_eval"] = c64.potential()["E_total"]
        out["dE_vs_fp64_eval"] = out["E_final"] - out["E_final_fp64_eval"]
        c64.close()
    ctx.close()
    return (out, psi64) if keep else out


def open_overlap(cfg, psi_a, psi_b, torch):
    """min over the open orbitals x = a, b of |<x_A|S|x_B>| (FP64 orbitals of
    two legs; S applied by the library): the same-state test of two runs."""
    from paper_2605_28637_gb300 import roks
    c64 = roks.Context(cfg, "fp64")
    sb = c64.new_bands()
    fb = c64.new_bands()
    c64.density(psi_b)
    c64.potential()
    roks.roks_apply_h(c64.ctx, psi_b, c64.ld, fb, sb, None)
    nb = c64.nb
    vals = []
    for col in (nb - 2, nb - 1):
        vals.append(float(torch.abs(torch.vdot(psi_a[col, :c64.npw], sb[col, :c64.npw])).item()))
    c64.close()
    return min(vals)


def converge_diis(cfg, precision, cap, torch, max_seconds, g_tol, history=6):
    """DIIS (roks_diis_step, lambda = 1/2) from the seeded start to |dE| < 1e-6 Ha
    twice with residual norm below g_tol, capped like converge()."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    ctx = roks.Context(cfg, precision, e_tol=1e-6, g_tol=g_tol)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    it, info = 0, None
    for it in range(1, cap + 1):
        info = ctx.diis_step(psi, history=history)
        if info["converged"] or time.perf_counter() - t0 > max_seconds:
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"seconds": dt, "iterations": it, "converged": bool(info and info["converged"]),
           "E_final": info["E_new"] if info else None, "res_norm_final": info["res_norm"] if info else None,
           "s_per_iter": dt / max(it, 1), "history": history}
    ctx.close()
    return out


def hybrid_leg(args, torch):
    """roks_apply_h on the hybrid-exchange workload (2x2x2 rocksalt cell minus
    one O, 72^3, 128 bands, exact-exchange fraction 1/3): the exchange apply
    makes 8256 pair transforms (both directions) per call.  Its HBM roofline
    counts 12.1 MB per pair (read psi_j, psi_n, one grid round trip of the
    pair density, the field update: 4 x 8 N^3 + the pair's sphere data)."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    cfg = syn.make_config("hybrid-72", 0)
    ctx = roks.Context(cfg, "mixed")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    ctx.density(psi)
    e = ctx.potential()
    f = ctx.new_bands()
    sp = ctx.new_bands()
    roks.roks_apply_h(ctx.ctx, psi, ctx.ld, f, sp, None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(args.hybrid_applies):
        roks.roks_apply_h(ctx.ctx, psi, ctx.ld, f, sp, None)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.hybrid_applies
    roks.roks_profile_enable(ctx.ctx, 1)
    roks.roks_apply_h(ctx.ctx, psi, ctx.ld, f, sp, None)
    prof = {x["name"]: x for x in roks.roks_profile_read(ctx.ctx)}
    roks.roks_profile_enable(ctx.ctx, 0)
    N = cfg["grid"]
    npairs = ctx.nb * (ctx.nb + 1) // 2
    alg = npairs * (4 * 8 * N ** 3 + 16 * ctx.npw)
    ex = prof.get("exchange")
    roof = None
    if ex:
        hbm, kind = peaks()
        ach = alg / (ex["ms"] / ex["launches"] / 1000.0) / 1e9
        roof = {"bound": "hbm", "kernel": "exchange (pair densities, batched grid transforms, kernel multiply, "
                                          "field accumulation)", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "peak_kind": f"{kind} (copy bandwidth)", "algorithmic_bytes_per_call": alg,
                "ms_per_call": ex["ms"] / ex["launches"]}
    out = {"workload": cfg["name"], "bands": ctx.nb, "pairs": npairs, "ms_per_apply": ms,
           "value": ctx.nb / (ms / 1000.0), "unit": UNIT, "E_total": e["E_total"], "E_hf_M": e["E_hf_M"],
           "roofline_exchange": roof}
    ctx.close()
    return out


def gamma_leg(args, cfg, torch, complex_ms_per_step):
    """The benchmark's workload with real orbitals at the Gamma point
    (roks_options.gamma): half-sphere coefficients, two orbitals per complex
    transform.  Same seeded start drawn on the half sphere, graph-replayed
    PCG steps timed with CUDA events on the context's stream."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    ctx = roks.Context(cfg, args.precision, autotune=args.autotune, gamma=1)
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    for _ in range(max(3, args.warmup)):
        ctx.pcg_step(psi)
    ms, infos, _ = time_pcg(ctx, psi, args.gamma_steps, torch)
    _, _, prof = time_pcg(ctx, psi, min(args.gamma_steps, 10), torch, profile=True)
    prof = [e for e in prof if e["name"] not in ("kernel_launches", "tensor_core_launches")]
    per = ms / args.gamma_steps
    out = {"workload": cfg["name"], "plane_waves_half_sphere": ctx.npw, "bands": ctx.nb,
           "steps": args.gamma_steps, "ms_per_step": per, "value": ctx.nb / (per / 1000.0), "unit": UNIT,
           "speedup_per_step_vs_complex": complex_ms_per_step / per, "tuning": ctx.tuning(),
           "E_last": infos[-1]["E_new"],
           "profile": {e["name"]: {"launches": e["launches"], "ms": e["ms"]} for e in prof},
           "launch": "one CUDA graph per PCG iteration"}
    ctx.close()
    return out


def gga_leg(args, cfg, torch, slater_ms_per_step):
    """The benchmark's workload with PBE exchange (the GGA) in place of the
    Slater exchange: graph-replayed PCG steps timed with CUDA events, and the
    potential family's time per call from a profiled eager pass (its grid
    gradient and divergence transforms)."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    c = syn.with_changes(cfg, xc="pbe_x")
    ctx = roks.Context(c, args.precision, autotune=args.autotune)
    psi = ctx.init_orbitals(syn.orbital_uniforms(c, ctx.npw))
    for _ in range(max(3, args.warmup)):
        ctx.pcg_step(psi)
    ms, infos, _ = time_pcg(ctx, psi, args.gga_steps, torch)
    _, _, prof = time_pcg(ctx, psi, min(args.gga_steps, 5), torch, profile=True)
    pot = [e for e in prof if e["name"] == "potential"]
    per = ms / args.gga_steps
    out = {"workload": cfg["name"], "xc": "pbe_x", "steps": args.gga_steps, "ms_per_step": per,
           "value": ctx.nb / (per / 1000.0), "unit": UNIT, "ms_per_step_slater": slater_ms_per_step,
           "potential_ms_per_call": pot[0]["ms"] / pot[0]["launches"] if pot else None,
           "E_last": infos[-1]["E_new"], "launch": "one CUDA graph per PCG iteration"}
    ctx.close()
    return out


def fp64_leg(cfg, torch, steps=5):
    """The plain FP64 path on the convergence workload: seconds per PCG step
    (graph replays) and the rooflines of its kernel families from a profiled
    eager pass, against the measured FP64 rate (contractions) and the HBM
    copy bandwidth (transform stages)."""
    from paper_2605_28637_gb300 import roks, synthetic as syn
    ctx = roks.Context(cfg, "fp64")
    psi = ctx.init_orbitals(syn.orbital_uniforms(cfg, ctx.npw))
    for _ in range(3):
        ctx.pcg_step(psi)
    ms, _, _ = time_pcg(ctx, psi, steps, torch)
    _, _, prof = time_pcg(ctx, psi, steps, torch, profile=True)
    prof = [e for e in prof if e["name"] not in ("kernel_launches", "tensor_core_launches")]
    total = sum(e["ms"] for e in prof) or 1.0
    hbm, peak_kind = peaks()
    rows = []
    for e in sorted(prof, key=lambda e: -e["ms"]):
        work = family_work(ctx, cfg, e["name"], 16, 8, "fp64")
        if work is None:
            continue
        bound, amount = work
        per = e["ms"] / e["launches"]
        if bound == "hbm":
            ach = amount / (per / 1000.0) / 1e9
            rows.append({"bound": "hbm", "kernel": e["name"], "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "peak_kind": f"{peak_kind} (copy bandwidth)", "ms_per_launch": per,
                         "share_of_step": e["ms"] / total})
        else:
            pk, kind = alu_peak("fp64", bound)
            ach = amount / (per / 1000.0) / 1e12
            rows.append({"bound": "alu", "kernel": e["name"], "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                         "frac": ach / pk, "peak_kind": kind, "ms_per_launch": per, "share_of_step": e["ms"] / total})
    out = {"workload": cfg["name"], "ms_per_step": ms / steps, "rooflines": rows,
           "profile": {e["name"]: {"launches": e["launches"], "ms": e["ms"]} for e in prof}}
    ctx.close()
    return out


def csize_of(precision):
    """Bytes of one complex coefficient on the path."""
    return 16 if precision == "fp64" else 8


def train_network(torch):
    """The preconditioner network trained on seeded tiny systems (singlet and
    closed shell, seeds 1-8), on the GPU; returns (device params, seconds, losses)."""
    import numpy as np
    from paper_2605_28637_gb300 import learned, synthetic as syn
    t0 = time.perf_counter()
    Us, ts, ws = [], [], []
    for seed in range(1, 9):
        c = syn.make_config("tiny-16", seed)
        for cfg in (c, syn.with_changes(c, mode=0, n_closed=5)):
            U, t, w = learned.make_pairs(cfg)
            Us.append(U); ts.append(t); ws.append(w)
    params, losses = learned.train(np.concatenate(Us), np.concatenate(ts), np.concatenate(ws), steps=1500, lr=2e-3)
    torch.cuda.synchronize()
    return params, time.perf_counter() - t0, losses


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2605_28637_gb300 import roks, synthetic as syn
    cfg = replica_config(args.workload, rank)
    if args.n_closed > 0:
        cfg = syn_with(cfg, n_closed=args.n_closed)
    # the autotuner picks the density's band grouping and the tensor-core
    # schedule on this context's own buffers (roks_options.autotune)
    ctx = roks.Context(cfg, args.precision, autotune=args.autotune)
    tuning = ctx.tuning()
    u = syn.orbital_uniforms(cfg, ctx.npw)
    psi = ctx.init_orbitals(u)
    for _ in range(args.warmup):
        ctx.pcg_step(psi)
    roks.roks_profile_read(ctx.ctx)   # restart the launch count
    # ---- timed region: K PCG steps (graph replays), inputs resident in HBM
    clocks = ClockSampler()
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms, infos, _ = time_pcg(ctx, psi, args.steps, torch, profile=False)
    if world > 1:
        torch.distributed.barrier()
    ck = clocks.stop(gpu_index=None if world == 1 else local)
    timed_launches = [e for e in roks.roks_profile_read(ctx.ctx) if e["name"] == "kernel_launches"]
    # ---- per-family device times: CUDA events around each kernel family on
    # the launching stream, over a profiled pass of the same steps (eager launches)
    prof_steps = min(args.steps, 20)
    prof_ms, _, prof = time_pcg(ctx, psi, prof_steps, torch, profile=True)
    ms_max = max_over_ranks(ms, world)
    value = aggregate_value(ctx.nb, args.steps, world, ms_max)
    # ---- apply-only throughput (roks_apply_h over all bands)
    f = ctx.new_bands()
    sp = ctx.new_bands()
    for _ in range(3):
        roks.roks_apply_h(ctx.ctx, psi, ctx.ld, f, sp, None)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    n_apply = 20
    for _ in range(n_apply):
        roks.roks_apply_h(ctx.ctx, psi, ctx.ld, f, sp, None)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    apply_ms = e0.elapsed_time(e1) / n_apply
    # ---- end to end: host orbitals in pinned memory, copied in and out each step
    host = torch.empty_like(psi, device="cpu").pin_memory()
    host.copy_(psi)
    e2e_steps = max(3, args.steps // 4)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    for _ in range(e2e_steps):
        psi.copy_(host, non_blocking=True)
        ctx.pcg_step(psi)
        host.copy_(psi, non_blocking=True)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_value = aggregate_value(ctx.nb, e2e_steps, world, max_over_ranks(e2e_ms, world))
    bytes_psi = psi.numel() * psi.element_size()
    # ---- DIIS steps (roks_diis_step: eager launches, one host read per step)
    # on a copy of the orbitals; its history builds during the warm-up
    diis = None
    if args.diis_steps > 0:
        pd = psi.clone()
        for _ in range(max(3, args.warmup)):
            ctx.diis_step(pd)
        roks.roks_profile_read(ctx.ctx)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        dinfo = [ctx.diis_step(pd) for _ in range(args.diis_steps)]
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        d_ms = e0.elapsed_time(e1)
        d_launch = [e for e in roks.roks_profile_read(ctx.ctx) if e["name"] == "kernel_launches"]
        d_ms = max_over_ranks(d_ms, world)
        # per-family device times of the same steps (eager, CUDA events per family)
        # and the HBM roofline of the extrapolation kernel: it reads 2h band
        # blocks (h pairs of the window) and writes one
        roks.roks_profile_enable(ctx.ctx, 1)
        pinfo = [ctx.diis_step(pd) for _ in range(10)]
        dprof = [e for e in roks.roks_profile_read(ctx.ctx) if e["name"] not in ("kernel_launches", "tensor_core_launches")]
        roks.roks_profile_enable(ctx.ctx, 0)
        comb = next((e for e in dprof if e["name"] == "diis_combine"), None)
        comb_roof = None
        if comb is not None:
            blk = ctx.nb * ctx.npw * csize_of(args.precision)
            alg = sum((2 * i["window"] + 1) * blk for i in pinfo)
            achieved = alg / (comb["ms"] / 1000.0) / 1e9
            hbm, peak_kind = peaks()
            comb_roof = {"bound": "hbm", "kernel": "k_diis_combine", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "peak_kind": f"{peak_kind} (copy bandwidth)",
                         "algorithmic_bytes_per_launch": alg / len(pinfo),
                         "ms_per_launch": comb["ms"] / comb["launches"]}
        diis = {"value": aggregate_value(ctx.nb, args.diis_steps, world, d_ms), "unit": UNIT,
                "roofline_combine": comb_roof,
                "profile": {e["name"]: {"launches": e["launches"], "ms": e["ms"]} for e in dprof},
                "ms_per_step": d_ms / args.diis_steps, "steps": args.diis_steps, "history": 6, "tau": 0.5,
                "launches_per_step": d_launch[0]["launches"] / args.diis_steps if d_launch else None,
                "launch": "eager (the ring slot changes every step), host read of the step's scalars",
                "E_last": dinfo[-1]["E_new"], "window_last": dinfo[-1]["window"]}
    # ---- forces on the atoms (roks_forces: density, potentials, apply, the
    # projector derivatives and the local term; one host read per call)
    forces_leg = None
    if args.force_calls > 0:
        for _ in range(2):
            ctx.forces(psi)
        roks.roks_profile_read(ctx.ctx)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        for _ in range(args.force_calls):
            Fa = ctx.forces(psi)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        f_ms = e0.elapsed_time(e1) / args.force_calls
        f_launch = [e for e in roks.roks_profile_read(ctx.ctx) if e["name"] == "kernel_launches"]
        forces_leg = {"ms_per_call": f_ms, "calls": args.force_calls, "natoms": ctx.natoms,
                      "launches_per_call": f_launch[0]["launches"] / args.force_calls if f_launch else None,
                      "max_abs_force_ha_per_bohr": float(abs(Fa).max()),
                      "launch": "eager, one host read per call"}
    # ---- measured FP32 (SIMT) and FP64 rates for the ALU rooflines
    alu_measured = measure_alu_peaks(torch)
    # ---- rooflines of the kernel families with known algorithmic work; the
    # family with the most device time is the line's "roofline"
    csize = 16 if args.precision == "fp64" else 8
    rsize = 8 if args.precision == "fp64" else 4
    tc_launches = next((e["launches"] for e in prof if e["name"] == "tensor_core_launches"), 0)
    tensor = tensor_families(ctx, args.precision, tc_launches)
    prof = [e for e in prof if e["name"] not in ("kernel_launches", "tensor_core_launches")]
    total_prof = sum(e["ms"] for e in prof) or 1.0
    hbm, peak_kind = peaks()
    rooflines = []
    for e in sorted(prof, key=lambda e: -e["ms"]):
        work = family_work(ctx, cfg, e["name"], csize, rsize, args.precision, tensor)
        if work is None:
            continue
        bound, amount = work
        per_launch_ms = e["ms"] / e["launches"]
        if bound == "hbm":
            achieved = amount / (per_launch_ms / 1000.0) / 1e9
            traffic, tnote = traffic_record(e["name"], cfg["name"], amount)
            ent = {"bound": "hbm", "kernel": e["name"], "achieved": achieved, "peak": hbm, "unit": "GB/s",
                   "frac": achieved / hbm, "peak_kind": f"{peak_kind} (copy bandwidth)",
                   "traffic": traffic, "traffic_source": tnote, "algorithmic_bytes_per_launch": amount}
        else:
            peak, pk = alu_peak(args.precision, bound)
            achieved = amount / (per_launch_ms / 1000.0) / 1e12
            ent = {"bound": bound, "kernel": e["name"], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                   "frac": achieved / peak, "peak_kind": pk, "traffic": None, "flops_per_launch": amount}
        ent["ms_per_launch"] = per_launch_ms
        ent["share_of_step"] = e["ms"] / total_prof
        rooflines.append(ent)
    roofline = rooflines[0] if rooflines else None
    roofline_hbm = next((r for r in rooflines if r["bound"] == "hbm"), None)
    launches = sum(e["launches"] for e in prof)
    # ---- time to convergence: chosen (mixed) vs plain FP64, on the
    # convergence workload, judged in the same state.  The closed-shell
    # ground state (one minimum) carries the time-to-solution comparison;
    # the singlet, whose minimisation has several stationary states, is
    # reported with the state each leg reached.
    pcg = None
    if args.converge_iters > 0 and rank == 0:
        base = replica_config(args.converge_workload, 0)
        params, t_train, losses = train_network(torch)
        ground = syn_with(base, mode=0, n_closed=base["n_closed"] + 1)
        g64 = converge(ground, "fp64", args.converge_iters, torch, args.converge_seconds, args.g_tol)
        gl = {}
        for key, prm in (("mixed_tpa", None), ("mixed_tpa_network", params)):
            leg = converge(ground, "mixed", args.converge_iters, torch, args.converge_seconds, args.g_tol, params=prm)
            leg["dE_vs_fp64_final"] = leg["E_final"] - g64["E_final"]
            leg["dE_fp64_eval_vs_fp64_final"] = leg["E_final_fp64_eval"] - g64["E_final"]
            leg["same_state_as_fp64"] = abs(leg["dE_fp64_eval_vs_fp64_final"]) < 1e-5
            ok = leg["converged"] and g64["converged"] and leg["same_state_as_fp64"]
            leg["time_to_solution_speedup_vs_fp64"] = g64["seconds"] / leg["seconds"] if ok else None
            gl[key] = leg
        singlet = {}
        s64, p64 = converge(base, "fp64", args.converge_iters, torch, min(args.converge_seconds, 20.0), args.g_tol,
                            keep=True)
        sm, pm = converge(base, "mixed", args.converge_iters, torch, min(args.converge_seconds, 20.0), args.g_tol,
                          keep=True)
        sm["open_overlap_with_fp64"] = open_overlap(base, pm, p64, torch)
        sm["same_state_as_fp64"] = sm["open_overlap_with_fp64"] > 0.99
        sm["dE_vs_fp64_final"] = sm["E_final"] - s64["E_final"]
        singlet = {"fp64_tpa": s64, "mixed_tpa": sm}
        del p64, pm
        pcg = {"workload": base["name"],
               "criterion": f"|E_i+1 - E_i| < 1e-6 Ha on two consecutive iterations and |g| < {args.g_tol:g}",
               "ground_state": {"fp64_tpa": g64, **gl,
                                "same_state": "energies of the final orbitals, re-evaluated in FP64, within 1e-5 Ha"},
               "singlet": {**singlet, "same_state": "open orbitals a, b: |<x|S|x_fp64>| > 0.99"},
               "network": {"trained_on": "tiny-16 seeds 1-8, singlet and closed shell", "train_seconds": t_train,
                           "loss_first": losses[0], "loss_last": losses[-1]},
               "speedup_s_per_iter_mixed_vs_fp64": g64["s_per_iter"] / gl["mixed_tpa"]["s_per_iter"],
               "mixed_diis_singlet": converge_diis(base, "mixed", args.converge_iters, torch,
                                                   min(args.converge_seconds, 20.0), args.g_tol),
               "note": "time-to-solution ratios only between converged legs in the FP64 leg's state",
               "fp64_path": fp64_leg(ground, torch)}
    gamma = None
    if args.gamma_steps > 0 and rank == 0:
        gamma = gamma_leg(args, cfg, torch, ms_max / args.steps)
    gga = None
    if args.gga_steps > 0 and rank == 0:
        gga = gga_leg(args, cfg, torch, ms_max / args.steps)
    hybrid = None
    if args.hybrid_applies > 0 and rank == 0:
        hybrid = hybrid_leg(args, torch)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(cfg["name"], args.cpu_seconds)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": cfg["grid"], "ecut_ha": cfg["ecut"], "bands": ctx.nb,
                       "plane_waves": ctx.npw, "atoms": len(cfg["atoms"]),
                       "precision": args.precision, "parallelism": f"replicas{world}",
                       "tuning": tuning,
                       "l2": "per-step working set above the 129 MB L2 (plane buffers, projectors, band blocks)"},
            "roofline": roofline,
            "roofline_hbm": roofline_hbm,
            "rooflines": rooflines,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_psi,
                    "d2h_bytes_per_step": bytes_psi},
            "gpu_launches": None,
            "clocks": ck,
            "apply_only": {"value": ctx.nb / (apply_ms / 1000.0), "unit": UNIT, "ms_per_apply_all_bands": apply_ms},
            "pcg": pcg,
            "alu_peaks_measured_tflops": alu_measured,
            "diis": diis,
            "forces": forces_leg,
            "hybrid": hybrid,
            "gamma": gamma,
            "gga": gga,
            "profile": {e["name"]: {"launches": e["launches"], "ms": e["ms"]} for e in prof},
            "launch": "one CUDA graph per PCG iteration",
            "E_last": infos[-1]["E_new"] if infos else None,
        }
        line["gpu_launches"] = timed_launches[0]["launches"] if timed_launches else None
        line["profiled_pass"] = {"steps": prof_steps, "ms_per_step": prof_ms / prof_steps,
                                 "kernel_groups": launches, "launch": "eager, one CUDA event pair per family"}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
