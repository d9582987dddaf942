"""Benchmark: time-to-solve of the lowest 8 eigenpairs at residual 1e-8 on the
synthetic n = 2,000,000 Kronecker matrix (~300 nonzeros per row, ~6e8
nonzeros), block size 8.

One step = the whole hot path once: the bootstrapped pivot (truncated space
of the 20,000 lowest-diagonal rows, sub-solve on the GPU), the
mixed-precision block Lanczos stage (FP32 SpMM and FP32 blocks, FP64
coefficients / Gram / T) and the polish stage to residual 1e-8 (float-float
blocks and products, FP64 coefficients / Gram / T), Ritz vectors and FP64
residuals.  The matrix (4.8 GB FP32 SELL + 4.8 GB FP32
CSR) is resident before the timed region; inputs exceed the 129 MB L2.

Also reported: the plain FP64 random-pivot block Lanczos time-to-solve on the
same GPU (the comparison the metric names), SpMM GB/s, the roofline of the
dominant kernel phase, an end-to-end number through host buffers, and the CPU
oracle timed on a bounded sample.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time
import types

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kron_n2e6"
B = 8
NEV = 8
TOL = 1e-8
TRUNC = 20000
# DRAM bytes per stored nonzero of one FP32 CSR SpMM launch (b = 8, 32 lanes
# per row), from an ncu capture of the same kernel on the half-scale matrix
# of the same family (dram__bytes_read.sum + dram__bytes_write.sum =
# 1.185 GB for 139,708,000 nonzeros); traffic grows with the nonzeros.
SPMM_TRAFFIC_PER_NNZ = 1.185e9 / 139_708_000
# the same for the FP32 SELL-C-sigma SpMM (b = 8; sigma = 1024 in the
# capture, the window the autotuner picks): 1.2045 GB for 139,708,000 nonzeros
SELL_TRAFFIC_PER_NNZ = 1.2045e9 / 139_708_000
SELL_SIGMA = 256
# the sorting window the autotuner picks for this family (kernels mode)
KERNELS_SELL_SIGMA = 1024
# DRAM bytes per algorithmic byte of the first-pass Gram from the FP16 basis
# copy (gram_half_kernel on the tensor cores, n*m*2 + n*8*4), from an ncu
# capture at n = 500,000, m = 400 (451.9 MB for 416 MB); it reads the copy
# once, so traffic grows with n*m (None: not captured since the kernel last
# changed)
GRAM16_TRAFFIC_PER_BYTE = 451.919616e6 / 416e6
METRIC = "time-to-solve lowest 8 eigenpairs @resid 1e-8 (s)"
# the headline step's settings: truncated-space sub-solve tolerance (FP32
# storage at >= 1e-5), FP32 stage tolerance before the polish, FP16 copy of
# the basis for the first Gram-Schmidt pass of the FP32 stage
SUB_TOL = 1e-4
STAGE1_TOL = 3e-7
HALF_FIRST_PASS = 1
PIVOT_SEED = 20221028
# the FP64 oracle's eigenvalues of this workload (plain block Lanczos, b = 8,
# residual 1e-8 * ||H||_inf), stored by the script beside them
ORACLE_EVALS = os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_fp64_oracle_evals.json")


def headline_pivot(bbl, M, sub_tol=SUB_TOL):
    """The bootstrapped pivot of one step: the TRUNC rows of lowest diagonal."""
    return bbl.pivot_bootstrap(M, TRUNC, B, sub_tol=sub_tol, seed=PIVOT_SEED)


def headline_solve(bbl, M, P, evecs="device", **opts):
    """The block Lanczos solve of one step (FP32 stage + float-float polish
    on an FP32-stored matrix)."""
    kw = {"stage1_tol": STAGE1_TOL, "half_first_pass": HALF_FIRST_PASS}
    kw.update(opts)
    return bbl.solve(M, NEV, B, pivot=P, tol=TOL, evecs=evecs, max_vectors=2000, **kw)


def oracle_eval_error(evals, path=None):
    """Largest relative difference from the stored FP64 oracle eigenvalues
    (None when the file is absent)."""
    try:
        with open(path or ORACLE_EVALS) as f:
            ref = np.array(json.load(f)["evals"])
    except (OSError, KeyError, ValueError):
        return None
    ev = np.asarray(evals)[:len(ref)]
    return float(np.max(np.abs(ev - ref) / np.abs(ref)))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int = 0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_matrix():
    import synth
    t = time.time()
    A = synth.kron_matrix(WORKLOAD)
    return A, time.time() - t


# ---------------------------------------------------------------------------- reference arm: the oracle
def oracle_measured(scale: float = 0.2):
    """The oracle's whole block Lanczos run (random pivot, b = 8, nev = 8,
    residual 1e-8) on the same family at a reduced size, timed end to end,
    beside the composition of oracle_sample at that size and block count:
    the check of the composition used at full size."""
    import synth
    from oracle import lanczos as OL
    from oracle import rng as OR
    A = synth.kron_matrix(WORKLOAD, scale=scale)
    H = A.to_scipy()
    piv = OR.normal_block(PIVOT_SEED, A.n, B)
    t0 = time.perf_counter()
    r = OL.block_lanczos(H, NEV, B, piv, tol=TOL, max_vectors=2000)
    measured = time.perf_counter() - t0
    composed, _, _ = oracle_sample(A, r.iters)
    return {"n": A.n, "nnz": A.nnz, "blocks": r.iters, "converged": bool(r.converged), "measured_s": measured,
            "composed_s": composed, "measured_over_composed": measured / composed}


def oracle_blocks_full_size(default: int = 110) -> int:
    """The oracle's own block count on the full workload (random pivot), as
    stored beside its eigenvalues."""
    try:
        with open(ORACLE_EVALS) as f:
            return int(json.load(f)["blocks"])
    except (OSError, KeyError, ValueError):
        return default


def oracle_sample(A, iters_gpu: int, budget_blocks: int = 3, k1: int = 8, k2: int = 32):
    """Times the CPU oracle's own steps and composes the cost of a block
    Lanczos run of `iters_gpu` blocks.  Per block: one SpMM (Eq. 3); the
    stacking of the basis and the two classical Gram-Schmidt passes against
    (j+1)*b columns (cost linear in the columns, timed together at two basis
    sizes); the CholQR2 normaliser; the assembly of T (Eq. 12, quadratic in
    its order) and its dense eigensolve (cubic), timed at one order and
    scaled."""
    from oracle import lanczos as OL
    from oracle import rng as OR
    from oracle.spmm import spmm as ospmm
    t_start = time.perf_counter()
    H = A.to_scipy()
    V = OR.normal_block(20221028, A.n, B)

    def tm(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    t_spmm = tm(lambda: ospmm(H, V))
    Q = OR.normal_block(7, A.n, k2 * B) / np.sqrt(A.n)
    blocks = [Q[:, i * B:(i + 1) * B] for i in range(k2)]

    def gs(k):
        basis = np.hstack(blocks[:k])
        return OL.cgs_pass(OL.cgs_pass(V, basis), basis)

    t1 = tm(lambda: gs(k1))
    t2 = tm(lambda: gs(k2))
    del Q, blocks
    c_col = max((t2 - t1) / ((k2 - k1) * B), 0.0)
    a_gs = max(t1 - c_col * k1 * B, 0.0)
    t_norm = tm(lambda: OL.cholqr2(V, 0.0))
    ke = 32
    As = [np.eye(B) for _ in range(ke)]
    Bs = [np.eye(B) for _ in range(ke - 1)]
    me = ke * B
    t_asm = tm(lambda: OL.block_tridiagonal(As, Bs))
    Te = np.random.default_rng(0).standard_normal((me, me))
    Te = Te + Te.T
    t_eig = tm(lambda: np.linalg.eigh(Te))
    J = max(iters_gpu, 1)
    est = 0.0
    for j in range(J):
        m = (j + 1) * B
        est += t_spmm + a_gs + c_col * m + t_norm + t_asm * (m / me) ** 2 + t_eig * (m / me) ** 3
    return float(est), float(time.perf_counter() - t_start), 1


def workload_name(A) -> str:
    """The workload both arms report in config.workload."""
    return (f"{WORKLOAD}: Kronecker H=Hp(x)I+I(x)Hn+sum_12 Cp(x)Cn, n={A.n}, nnz={A.nnz}, b={B}, nev={NEV}, "
            f"tol={TOL}")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, tgen = build_matrix()
    # the oracle's own block count on this workload (random pivot, residual 1e-8)
    iters = oracle_blocks_full_size()
    vals = []
    wall = 0.0
    for _ in range(args.warmup + args.steps if args.steps > 0 else 1):
        # a lighter sample per step (basis sizes 4 and 12 blocks for the linear fit)
        est, w, blocks = oracle_sample(A, iters, budget_blocks=2, k1=4, k2=12)
        vals.append(est)
        wall += w
    v = float(np.mean(vals[args.warmup:])) if len(vals) > args.warmup else float(np.mean(vals))
    check = oracle_measured()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(A),
                   "method": "the oracle: numpy/scipy FP64 block Lanczos (CGS2, CholQR2, LAPACK Ritz solve)",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"the oracle's steps timed once each at full size (SpMM, Gram-Schmidt passes "
                                   f"at two basis sizes, CholQR2, dense eigensolve) and composed into a {iters}-block "
                                   f"run (the oracle's own block count on this workload); the composition checked by a "
                                   f"whole oracle run at n = {check['n']}: measured {check['measured_s']:.1f} s vs "
                                   f"composed {check['composed_s']:.1f} s",
                         "composition_check": check},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest of the ranks' values (one collective); x itself at N = 1."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import paper_2210_15763_gb300 as bbl
    from paper_2210_15763_gb300 import _lib

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lib = _lib.load()
    A, tgen = build_matrix()
    st = torch.cuda.current_stream()
    t0 = time.perf_counter()
    from paper_2210_15763_gb300 import autotune
    sched = autotune.tune(A, B, storage="fp32", reps=3)

    def make_matrix(csr=A):
        M = bbl.Matrix(csr, storage="fp32", fmt=sched["fmt"], sell_sigma=sched["sigma"])
        if sched["fmt"] == "csr":
            M.set_spmm_lanes(sched["lanes"])
        return M

    t0 = time.perf_counter()
    M32 = make_matrix()
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0

    stats_log = []
    boot_ev = []
    solve_opts = {} if args.ritz_overlap is None else {"ritz_overlap": args.ritz_overlap}
    solve_opts["stage1_tol"] = args.stage1_tol
    solve_opts["half_first_pass"] = args.half_first_pass
    solve_opts["fused_update_gram"] = args.fused_update_gram
    solve_opts["narrow_old_updates"] = args.narrow_old_updates

    def step():
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(st)
        P = headline_pivot(bbl, M32, args.sub_tol)
        b1.record(st)
        boot_ev.append((b0, b1))
        r = headline_solve(bbl, M32, P, **solve_opts)
        stats_log.append(r.stats)
        return r

    for _ in range(args.warmup):
        r = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    stats_log.clear()
    boot_ev.clear()
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = lib.bbl_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed region
    results = [step() for _ in range(args.steps)]
    torch.cuda.nvtx.range_pop()
    e1.record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = lib.bbl_kernel_launches() - launches0
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / max(args.steps, 1), world, "cuda")
    r = results[-1]
    ok = all(x.converged for x in results)
    nrm = M32.norm_inf
    resid_rel = float(np.max(r.resid) / nrm)

    # phase rooflines over the timed region (CUDA events inside the solver, on this stream)
    tot = {k: sum(s[k] for s in stats_log) for k in stats_log[0]}
    hbm, peak_kind = peaks()
    reorth_gbs = tot["reorth_bytes_total"] / (tot["t_reorth_ms"] * 1e-3) / 1e9
    spmm_gbs = tot["spmm_bytes_total"] / (tot["t_spmm_ms"] * 1e-3) / 1e9
    phases = {"spmm_ms": tot["t_spmm_ms"] / args.steps, "reorth_ms": tot["t_reorth_ms"] / args.steps,
              "cholqr2_ms": tot["t_cholqr_ms"] / args.steps, "ritz_ms": tot["t_ritz_ms"] / args.steps,
              "assembly_ms": tot["t_other_ms"] / args.steps,
              "bootstrap_pivot_ms": sum(a.elapsed_time(b) for a, b in boot_ev) / args.steps,
              "solve_total_ms": tot["t_total_ms"] / args.steps}
    # per-kernel rooflines from the solver's own CUDA events (main stage, FP32):
    # the SpMM phase of an iteration is exactly one SpMM launch; the timed
    # first-pass Gram is the split-K Gram kernel plus its partial reduction
    spmm_calls = sum(s["spmm_calls"] for s in stats_log)
    spmm_total_ms = sum(s["spmm_bytes"] * s["spmm_calls"] / (s["spmm_gbs"] * 1e9) * 1e3 for s in stats_log)
    spmm_kernel_gbs = stats_log[-1]["spmm_bytes"] * spmm_calls / (spmm_total_ms * 1e-3) / 1e9
    gram_calls = tot["gram_calls"]
    gram_gbs = tot["gram_bytes_total"] / (tot["t_gram_ms"] * 1e-3) / 1e9
    kernels = {
        "spmm": {"kernel": f"spmm_csr_kernel<float,float,8,{sched['lanes'] or 32}>" if sched["fmt"] == "csr"
                 else "spmm_sell_kernel<float,float,8>", "launches": spmm_calls,
                 "total_ms": spmm_total_ms, "achieved": spmm_kernel_gbs,
                 "bytes_per_launch": stats_log[-1]["spmm_bytes"],
                 "traffic": (SPMM_TRAFFIC_PER_NNZ * A.nnz if sched["fmt"] == "csr" and (sched["lanes"] or 32) == 32
                             else SELL_TRAFFIC_PER_NNZ * A.nnz if sched["fmt"] == "sell" else None)},
        "gram": {"kernel": "gram_half_kernel + reduce_partials_kernel (first Gram-Schmidt pass of the FP32 "
                 "stage, from the FP16 copy of the basis, mma.sync on the tensor cores)", "launches": gram_calls, "total_ms": tot["t_gram_ms"],
                 "achieved": gram_gbs, "bytes_per_launch": tot["gram_bytes_total"] / max(gram_calls, 1),
                 "traffic": GRAM16_TRAFFIC_PER_BYTE * tot["gram_bytes_total"] / max(gram_calls, 1)
                 if GRAM16_TRAFFIC_PER_BYTE else None},
    }
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"])
    kd = kernels[dom]
    roofline = {"bound": "hbm", "achieved": round(kd["achieved"], 1), "peak": hbm, "unit": "GB/s",
                "frac": round(kd["achieved"] / hbm, 4), "traffic": kd["traffic"], "kernel": kd["kernel"],
                "peak_kind": peak_kind,
                "per_kernel": {k: {kk: (round(vv, 3) if isinstance(vv, float) else vv) for kk, vv in v.items()}
                               for k, v in kernels.items()}}

    # overlap of the bootstrapped pivot with each converged eigenvector (Sec. II.B)
    P_last = headline_pivot(bbl, M32, args.sub_tol)
    overlaps = bbl.pivot_overlap(P_last, r.evecs)
    del P_last

    # plain FP64 random-pivot block Lanczos (the comparison named by the metric)
    plain = None
    if not args.skip_plain:
        M64 = bbl.Matrix(A, storage="fp64", fmt="csr")
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(st)
        rp = bbl.solve(M64, NEV, B, pivot=None, seed=20221028, tol=TOL, evecs="device", max_vectors=2000)
        p1.record(st)
        torch.cuda.synchronize()
        t_plain = p0.elapsed_time(p1) / 1e3
        # is the FP64 SpMM limited by FP64 arithmetic or by memory?  Its
        # flop rate against the measured FP64 FMA rate, its bytes against HBM
        f64_rate = bbl.probe_fma_rate("fp64")
        sp = rp.stats
        flop_rate = 2.0 * A.nnz * B * sp["spmm_calls"] / (sp["t_spmm_ms"] * 1e-3)
        plain = {"time_s": t_plain, "iters": sp["iters"], "converged": rp.converged,
                 "spmm_gbs": sp["spmm_gbs"], "spmm_tflops": flop_rate / 1e12,
                 "fp64_fma_tflops_measured": f64_rate / 1e12,
                 "spmm_frac_of_fp64_fma": flop_rate / f64_rate, "spmm_frac_of_hbm": sp["spmm_gbs"] / hbm,
                 "dfma_bound": bool(flop_rate / f64_rate > sp["spmm_gbs"] / hbm),
                 "max_abs_eval_diff_vs_mixed": float(np.max(np.abs(rp.evals - r.evals)))}
        del M64
        torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers: matrix from the host
    # CSR arrays (page-locked copies made before the timed region), bootstrap
    # + solve, eigenvectors back into a page-locked host buffer
    Ah = types.SimpleNamespace(n=A.n, row_ptr=torch.from_numpy(A.row_ptr).pin_memory(),
                               col=torch.from_numpy(A.col).pin_memory(), val=torch.from_numpy(A.val).pin_memory())
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    Me = make_matrix(Ah)
    Pe = headline_pivot(bbl, Me, args.sub_tol)
    re = headline_solve(bbl, Me, Pe, evecs="pinned", **solve_opts)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - h0
    del Ah
    h2d = A.row_ptr.nbytes + A.col.nbytes + A.val.nbytes
    d2h = re.evecs.nbytes + 2 * NEV * 8
    Me.close()

    cpu = None
    if rank == 0 and not args.skip_cpu:
        iters_o = oracle_blocks_full_size()
        est, wall, blocks = oracle_sample(A, iters_o, budget_blocks=2)
        check = oracle_measured()
        cpu = {"value": est, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the FP64 oracle's steps timed once each at full size ({wall:.1f} s wall: one SpMM, "
                         f"Gram-Schmidt passes at two basis sizes, CholQR2, a dense eigensolve) and composed into a "
                         f"{iters_o}-block run, the oracle's own block count on this workload (random pivot); the "
                         f"composition checked by a whole oracle run at n = {check['n']} ({check['blocks']} blocks): "
                         f"measured {check['measured_s']:.1f} s vs composed {check['composed_s']:.1f} s; numpy BLAS "
                         "on all cores, scipy SpMM single-threaded",
               "composition_check": check}

    line = {
        "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        # FP32 storage, SpMM and Gram-Schmidt; FP16 products (FP32 sums) in
        # the first Gram pass when it reads the FP16 copy of the basis; FP64
        # coefficients, T, Ritz quotients and residuals
        "dtype": "f32+f16+f64" if args.half_first_pass else "f32+f64", "data": "synthetic",
        "config": {"workload": workload_name(A),
                   "method": f"bootstrap trunc_dim={TRUNC} sub_tol={args.sub_tol:g}, FP32 stage "
                             f"({sched['fmt']}, lanes {sched['lanes']}, sigma {sched['sigma']}"
                             f"{'' if args.stage1_tol is None else f', to {args.stage1_tol:g}'}"
                             f"{', FP16 first-pass Gram' if args.half_first_pass else ''}"
                             f"{', older blocks of both updates from the narrower copy' if args.narrow_old_updates else ''}"
                             f") + float-float polish, FP64 residuals",
                   "parallelism": "replicas only" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (matrix 4.8 GB)"},
        "converged": ok, "max_resid_rel": resid_rel,
        "max_rel_err_vs_oracle": oracle_eval_error(r.evals),
        "pivot_overlap": [round(float(x), 4) for x in overlaps],
        "iters": r.stats["iters"], "polish_iters": r.stats["polish_iters"], "ritz_solves": r.stats["ritz_solves"],
        "vec_equiv_iters": r.stats["vec_equiv_iters"],
        "spmm_gbs": round(spmm_gbs, 1), "reorth_gbs": round(reorth_gbs, 1), "phases_ms": phases,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (plain["time_s"] / (ms / 1e3)) if plain else None,
        "roofline": roofline,
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "cpu_baseline": cpu,
        "setup": {"generate_s": tgen, "matrix_create_s": t_create},
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_kernels(args):
    """Each hot kernel alone on a smaller matrix of the same family (inputs
    still larger than L2): used for ncu captures and per-kernel bandwidths."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    A = synth.kron_matrix(WORKLOAD, scale=args.scale)
    n = A.n
    M = bbl.Matrix(A, storage="fp32", fmt="sell", sell_sigma=KERNELS_SELL_SIGMA)
    g = torch.Generator(device="cuda").manual_seed(1)
    V = torch.randn(n, B, device="cuda", dtype=torch.float32, generator=g)
    W = torch.empty_like(V)
    nb = args.blocks
    basis = torch.randn(nb, n, B, device="cuda", dtype=torch.float32, generator=g)
    Wr = torch.randn(n, B, device="cuda", dtype=torch.float32, generator=g)

    def timeit(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"n": n, "nnz": A.nnz, "b": B, "basis_blocks": nb,
           "fma_tflops": {"fp32": bbl.probe_fma_rate("fp32") / 1e12, "fp64": bbl.probe_fma_rate("fp64") / 1e12}}
    t = timeit(lambda: bbl.spmm(M, V, W), args.reps)
    by = A.nnz * 8 + (n + 1) * 8 + 2 * n * B * 4
    out["spmm_sell_fp32"] = {"ms": t, "GBs": by / t / 1e6}
    Mc = bbl.Matrix(A, storage="fp32", fmt="csr")
    t = timeit(lambda: bbl.spmm(Mc, V, W), args.reps)
    out["spmm_csr_fp32"] = {"ms": t, "GBs": by / t / 1e6}
    del Mc
    # the tiled format with tiles of nN rows (one proton row per row block,
    # one proton column per tile), and b = 16 (64-byte rows of V) beside b = 8
    nN = synth.kron_config(WORKLOAD, args.scale)["nN"]
    Mt = bbl.Matrix(A, storage="fp32", fmt="tiled", sell_sigma=nN)
    t = timeit(lambda: bbl.spmm(Mt, V, W), args.reps)
    out["spmm_tiled_fp32"] = {"ms": t, "GBs": by / t / 1e6, "tile": nN}
    V16 = torch.randn(n, 16, device="cuda", dtype=torch.float32, generator=g)
    W16 = torch.empty_like(V16)
    by16 = A.nnz * 8 + (n + 1) * 8 + 2 * n * 16 * 4
    t = timeit(lambda: bbl.spmm(Mt, V16, W16), args.reps)
    out["spmm_tiled_fp32_b16"] = {"ms": t, "GBs": by16 / t / 1e6}
    del Mt
    t = timeit(lambda: bbl.spmm(M, V16, W16), args.reps)
    out["spmm_sell_fp32_b16"] = {"ms": t, "GBs": by16 / t / 1e6}
    del V16, W16
    m = nb * B
    t = timeit(lambda: bbl.block_gram(basis, Wr), args.reps)
    out["gram_fp32"] = {"ms": t, "GBs": (n * m * 4 + n * B * 4) / t / 1e6}
    basis16 = basis.half()
    t = timeit(lambda: bbl.block_gram_f16(basis16, Wr), args.reps)
    out["gram_f16_first_pass"] = {"ms": t, "GBs": (n * m * 2 + n * B * 4) / t / 1e6}
    del basis16
    basis /= float(np.sqrt(n))  # keep repeated in-place updates bounded
    Wt = torch.empty_like(Wr)
    t = timeit(lambda: bbl.block_reorth(basis, Wt.copy_(Wr), passes=1), args.reps)
    out["gram_update_fp32"] = {"ms": t, "GBs": (2 * n * m * 4 + 3 * n * B * 4) / t / 1e6}
    # the first update with the blocks older than the two newest from the FP16 copy (tensor cores)
    basis16 = basis.to(torch.float16)
    C1h = bbl.block_gram(basis, Wr)
    Wh = torch.empty_like(Wr)
    t = timeit(lambda: bbl.block_update_f16old(basis16, basis, Wh.copy_(Wr), C1h), args.reps)
    out["update_f16old"] = {"ms": t, "GBs": (n * (m - 16) * 2 + n * 16 * 4 + 3 * n * B * 4) / t / 1e6}
    del basis16, Wh
    # the fused first update + second Gram (tensor cores): one read of the basis
    C1 = bbl.block_gram(basis, Wr)
    Wf = torch.empty_like(Wr)
    t = timeit(lambda: bbl.block_update_gram(basis, Wf.copy_(Wr), C1), args.reps)
    out["update_gram_fused"] = {"ms": t, "GBs": (n * m * 4 + 3 * n * B * 4) / t / 1e6}
    del Wf
    Wc = Wr.clone()
    t = timeit(lambda: bbl.cholqr2(Wc.copy_(Wr)), args.reps)
    out["cholqr2_fp32"] = {"ms": t, "GBs": 6 * n * B * 4 / t / 1e6}
    rng = np.random.default_rng(0)
    mT, p = args.ritz_m, B
    Tb = np.zeros((mT, p + 1))
    Tb[:, 0] = rng.standard_normal(mT)
    for d in range(1, p + 1):
        Tb[d:, d] = rng.standard_normal(mT - d)
    Td = torch.from_numpy(Tb).cuda()
    t = timeit(lambda: bbl.ritz_banded(Td, NEV), max(1, args.reps // 2))
    out["ritz_banded"] = {"ms": t, "m": mT, "p": p, "nev": NEV,
                          "matrix": "random N(0,1) band: a dense spectrum, a stress case for bisection and the "
                                    "cluster step (Lanczos T_j has separated lowest eigenvalues)"}
    print(json.dumps(out))


def run_batched(args):
    """The batched form: `count` independent Kronecker matrices with n
    log-uniform in [2e3, 2e5] and 50-150 nonzeros per row, b = 4, 4 lowest
    eigenpairs each, FP32 storage with FP64 coefficients / Gram / T / residual,
    residual 1e-7 * ||H_s||_inf.  One graph launch for the whole batch, the
    SpMM schedule chosen by the autotuner; compared with one bbl_solve call
    per matrix on the same GPU."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    from paper_2210_15763_gb300 import autotune
    t0 = time.time()
    specs = synth.batch_matrices(count=args.count)
    mats = [synth.assemble(synth.kron_factors(s["nP"], s["nN"], s["K"], s["c"], s["seed"]), fp32_values=True)
            for s in specs]
    tgen = time.time() - t0
    offsets, rp, col, val = bbl.stack_block_diagonal(mats)
    stacked = synth.CSR(int(offsets[-1]), rp, col, val)
    best = autotune.tune(stacked, 4, storage="fp32", reps=3)
    Bt = bbl.Batch(mats, storage="fp32", fmt=best["fmt"], sell_sigma=best["sigma"])
    if best["fmt"] == "csr":
        Bt.set_schedule(best["lanes"])
    opts = dict(tol=1e-7, max_vectors=args.batch_max_vectors, seed=20221034)
    graph = bool(args.batch_graph)
    Bt.solve(4, 4, use_graph=graph, **opts)  # warm-up (graph build, caches)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ev, rs, it, st, stats = Bt.solve(4, 4, use_graph=graph, **opts)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    # one launch sequence per matrix (skipped with --skip-plain)
    its1 = []
    conv1 = 0
    t_single = float("nan")
    if not args.skip_plain:
        Ms = [bbl.Matrix(m, storage="fp32", fmt=best["fmt"], sell_sigma=best["sigma"]) for m in mats]
        torch.cuda.synchronize()
        e0.record()
        for M in Ms:
            r = bbl.solve(M, 4, 4, pivot=None, tol=1e-7, polish=0, max_vectors=args.batch_max_vectors,
                          seed=20221034, evecs=None)
            its1.append(r.stats["iters"])
            conv1 += r.converged
        e1.record()
        torch.cuda.synchronize()
        t_single = e0.elapsed_time(e1) / 1e3
    nrm = np.array([float(np.abs(m.to_scipy()).sum(axis=1).max()) for m in mats])
    out = {"metric": "batched solves/s (256 Kronecker matrices, n in [2e3, 2e5], b=4, nev=4, tol 1e-7)",
           "value": args.count / t_batch, "unit": "solves/s", "higher_is_better": True,
           "batched_s": t_batch, "one_launch_per_matrix_s": t_single if its1 else None,
           "one_launch_per_matrix_solves_per_s": args.count / t_single if its1 else None,
           "speedup": t_single / t_batch if its1 else None,
           "converged": int(np.sum(st == 0)), "converged_single": conv1, "count": args.count,
           "n_total": int(offsets[-1]), "nnz_total": int(rp[-1]),
           "iters_max": int(it.max()), "iters_mean": float(it.mean()), "iters_single_mean": float(np.mean(its1)) if its1 else None,
           "max_resid_rel": float(np.max(rs.max(axis=1) / nrm)),
           "schedule": {k: best[k] for k in ("fmt", "lanes", "sigma", "ms", "class")},
           "polish_iters_max": stats["polish_iters"],
           "graph_kernels_per_iteration": stats["graph_kernels"], "graph": graph, "generate_s": tgen}
    print(json.dumps(out))


def run_learned(args):
    """The learned-pivot form on H(g) = H0 + g V (H0: the n = 1e6 Kronecker
    matrix, V: six more coupling terms), 64 values g ~ U(0,1): 48 training
    solves (bootstrapped pivot, FP32 stage + FP64 polish) build the stored
    basis U (64 eigenvectors at 8 training g) and the targets; the MLP
    (1 -> 128 -> 128 -> 64*8, GELU) is trained on the GPU; on the 16 held-out
    g the iterations and times to residual 1e-8 are compared for the learned
    (gated) pivot, the bootstrapped pivot and a random pivot."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    from paper_2210_15763_gb300 import learned
    b = nev = 8
    trunc = max(64, int(round(20000 * args.family_scale ** 2)))
    h0, v = synth.learned_family(scale=args.family_scale)
    gs = synth.family_g()
    make = lambda g: synth.family_matrix(h0, v, g, fp32_values=True)
    t0 = time.time()
    lp = learned.fit(make, gs[:48], nev=nev, b=b, trunc_dim=trunc, n_basis_g=8, hidden=128, epochs=args.epochs,
                     lr=1e-3, seed=0, tol=TOL, storage="fp32", fmt="csr", sub_tol=args.sub_tol)
    t_fit = time.time() - t0
    rows = []
    for g in gs[48:]:
        A = bbl.Matrix(make(g), storage="fp32", fmt="csr")
        ev = torch.cuda.Event(enable_timing=True)
        ee = torch.cuda.Event(enable_timing=True)
        out = {"g": float(g)}
        ev.record()
        r_l, info = learned.solve_with_learned_pivot(A, lp, g, b, trunc, tol=TOL, sub_tol=args.sub_tol)
        ee.record()
        torch.cuda.synchronize()
        out.update(learned_iters=r_l.stats["iters"] + r_l.stats["polish_iters"], learned_s=ev.elapsed_time(ee) / 1e3,
                   **info)
        ev.record()
        P = bbl.pivot_bootstrap(A, trunc, b, sub_tol=args.sub_tol)
        r_b = bbl.solve(A, nev, b, pivot=P, tol=TOL)
        ee.record()
        torch.cuda.synchronize()
        out.update(boot_iters=r_b.stats["iters"] + r_b.stats["polish_iters"], boot_s=ev.elapsed_time(ee) / 1e3)
        ev.record()
        r_r = bbl.solve(A, nev, b, pivot=None, seed=7, tol=TOL)
        ee.record()
        torch.cuda.synchronize()
        out.update(random_iters=r_r.stats["iters"] + r_r.stats["polish_iters"], random_s=ev.elapsed_time(ee) / 1e3,
                   max_eval_diff=float(np.max(np.abs(r_l.evals - r_r.evals))),
                   converged=bool(r_l.converged and r_b.converged and r_r.converged))
        A.close()
        # the in-box baseline the forms must beat: plain FP64, random pivot
        A64 = bbl.Matrix(make(g), storage="fp64", fmt="csr")
        ev.record()
        r_p = bbl.solve(A64, nev, b, pivot=None, seed=7, tol=TOL, evecs=None)
        ee.record()
        torch.cuda.synchronize()
        out.update(plain_fp64_iters=r_p.stats["iters"], plain_fp64_s=ev.elapsed_time(ee) / 1e3)
        A64.close()
        rows.append(out)
    mean = lambda k: float(np.mean([r[k] for r in rows]))
    res = {"mode": "learned", "n": int(h0.n), "held_out": len(rows), "fit_s": t_fit,
           "train_loss_first_last": [float(lp.loss[0]), float(lp.loss[-1])], "epochs": args.epochs,
           "mean_iters": {"learned": mean("learned_iters"), "bootstrap": mean("boot_iters"),
                          "random": mean("random_iters")},
           "mean_time_s": {"learned": mean("learned_s"), "bootstrap": mean("boot_s"), "random": mean("random_s"),
                           "plain_fp64_random": mean("plain_fp64_s")},
           "learned_used_fraction": mean("learned_used"), "bootstrap_built_fraction": mean("bootstrap_built"),
           "all_converged": all(r["converged"] for r in rows),
           "max_eval_diff_learned_vs_random": max(r["max_eval_diff"] for r in rows), "per_g": rows}
    print(json.dumps(res))


def run_c3(args):
    """The mixed-precision form at n = 20,000,000 (5000 x 4000 Kronecker
    construction, 12 coupling terms, ~200 nonzeros per row, ~4e9 nonzeros):
    FP32 values in SELL-C-sigma (C = 32), FP32 blocks with b = 8, FP64
    coefficients / Gram / T, FP64 residual SpMV.  Two runs from the
    bootstrapped pivot: the stated configuration, at most `--c3-vectors`
    stored vectors (300) with thick restart keeping the 16 lowest Ritz
    vectors (the time-to-solve reported), and without the cap or restarts
    (2000 vectors) for comparison.  Optionally (--c3-kron) the capped run on
    the factored operator, and (--c3-fp64) the plain FP64 random-pivot solve
    on the same GPU."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    t0 = time.time()
    A = synth.kron_matrix("kron_n2e7", fp32_values=True)
    tgen = time.time() - t0
    out = {"mode": "c3", "n": int(A.n), "nnz": int(A.nnz), "nnz_per_row": A.nnz / A.n, "generate_s": tgen,
           "half_first_pass": args.half_first_pass}
    st = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    t0 = time.time()
    M = bbl.Matrix(A, storage="fp32", fmt="sell", sell_sigma=SELL_SIGMA)
    torch.cuda.synchronize()
    out["matrix_create_s"] = time.time() - t0
    out["device_bytes"] = int(M.device_bytes)
    out["sell_padded_nnz"] = int(M.padded_nnz)
    P, t_boot = timed(lambda: bbl.pivot_bootstrap(M, TRUNC, B, sub_tol=args.sub_tol, seed=PIVOT_SEED))
    out["bootstrap_s"] = t_boot

    def solve_run(Mx, Px, mv, keep):
        r, t = timed(lambda: bbl.solve(Mx, NEV, B, pivot=Px, tol=TOL, evecs=None, max_vectors=mv, restart_keep=keep,
                                       stage1_tol=args.stage1_tol, half_first_pass=args.half_first_pass))
        torch.cuda.empty_cache()
        return {"max_vectors": mv, "restart_keep": keep, "time_s": t, "converged": bool(r.converged),
                "iters": r.stats["iters"], "polish_iters": r.stats["polish_iters"], "restarts": r.stats["restarts"],
                "max_resid_rel": float(np.max(r.resid) / Mx.norm_inf), "evals": [float(x) for x in r.evals],
                "spmm_gbs": r.stats["spmm_gbs"], "status": r.status}

    # the stated configuration: at most 300 stored vectors, thick restart
    # keeping the 16 lowest Ritz vectors (both stages)
    out["capped"] = solve_run(M, P, args.c3_vectors, 16)
    out["uncapped"] = solve_run(M, P, 2000, 0)
    out["time_to_solve_s"] = out["bootstrap_s"] + out["capped"]["time_s"]
    out["max_abs_eval_diff_capped_vs_uncapped"] = float(np.max(np.abs(np.array(out["capped"]["evals"]) -
                                                                     np.array(out["uncapped"]["evals"]))))
    del M, P
    torch.cuda.empty_cache()
    if args.c3_kron:
        # the same configuration on the factored operator: H (3.8e9 nonzeros)
        # is never stored, the factors take a few MB (exact Kronecker sum, so
        # its eigenvalues differ from the FP32-rounded stored matrix's by ~1e-7)
        Mk = bbl.KronMatrix(synth.named_factors("kron_n2e7"), storage="fp32")
        Pk, tb_k = timed(lambda: bbl.pivot_bootstrap(Mk, TRUNC, B, sub_tol=args.sub_tol, seed=PIVOT_SEED))
        out["factored"] = solve_run(Mk, Pk, args.c3_vectors, 16)
        out["factored"].update(bootstrap_s=tb_k, matrix_device_bytes=int(Mk.device_bytes),
                               time_to_solve_s=tb_k + out["factored"]["time_s"])
        del Mk, Pk
        torch.cuda.empty_cache()
    if args.c3_fp64:
        M64 = bbl.Matrix(A, storage="fp64", fmt="csr")
        r, t = timed(lambda: bbl.solve(M64, NEV, B, pivot=None, seed=20221028, tol=TOL, evecs=None, max_vectors=2000))
        out["plain_fp64"] = {"time_s": t, "converged": bool(r.converged), "iters": r.stats["iters"],
                             "max_abs_eval_diff_vs_mixed": float(np.max(np.abs(r.evals - np.array(out["capped"]["evals"])))),
                             "status": r.status}
    print(json.dumps(out))


def run_kron(args):
    """The same step on the Kronecker-factored operator: H is never stored;
    every SpMM rebuilds it from Hp, Hn, Cp_k, Cn_k (the paper's on-the-fly
    matrix elements, Sec. I, Sec. III.A, Appendix A).  The matrix is the exact
    Kronecker sum of the kron_n2e6 factors (entries not rounded to FP32), so
    the eigenvalues are compared with the oracle's for that matrix.  Reported
    beside it: the factored SpMM per launch (its own CUDA events inside the
    solver), the bytes it streams through L2 per launch, and the plain FP64
    random-pivot solve of the same exact matrix stored as FP64 CSR."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    st = torch.cuda.current_stream()
    f = synth.named_factors(WORKLOAD)
    t0 = time.perf_counter()
    M = bbl.KronMatrix(f, storage="fp32")
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    solve_opts = {"stage1_tol": args.stage1_tol, "half_first_pass": args.half_first_pass}
    stats_log = []

    def step():
        P = headline_pivot(bbl, M, args.sub_tol)
        r = headline_solve(bbl, M, P, **solve_opts)
        stats_log.append(r.stats)
        return r

    for _ in range(args.warmup):
        step()
    stats_log.clear()
    sampler = ClockSampler(0)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    results = [step() for _ in range(args.steps)]
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    r = results[-1]
    # SpMM of the FP32 stage: one launch per phase event
    calls = sum(s["spmm_calls"] for s in stats_log)
    spmm_ms = sum(s["spmm_bytes"] * s["spmm_calls"] / (s["spmm_gbs"] * 1e9) * 1e3 for s in stats_log) / calls
    # bytes a launch streams: every output slab p reads the slabs of row p of
    # Hp and of each Cp_k, and its own slab once (b = 8 FP32 columns)
    lens = np.diff(f.Hp.row_ptr) + 1 + sum(np.diff(c.row_ptr) for c in f.Cp)
    stream_bytes = float(lens.sum()) * f.Hn.n * B * 4
    plain = None
    if not args.skip_plain:
        Hx = synth.assemble(f, exact=True)
        M64 = bbl.Matrix(Hx, storage="fp64", fmt="csr")
        del Hx
        torch.cuda.synchronize()
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(st)
        rp = bbl.solve(M64, NEV, B, pivot=None, seed=PIVOT_SEED, tol=TOL, evecs=None, max_vectors=2000)
        p1.record(st)
        torch.cuda.synchronize()
        plain = {"time_s": p0.elapsed_time(p1) / 1e3, "iters": rp.stats["iters"], "converged": rp.converged,
                 "max_abs_eval_diff_vs_factored": float(np.max(np.abs(rp.evals - r.evals)))}
        del M64
        torch.cuda.empty_cache()
    exact = os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_exact_fp64_oracle_evals.json")
    out = {"mode": "kron", "metric": METRIC, "value": ms / 1e3, "unit": "s", "steps": args.steps,
           "warmup": args.warmup, "higher_is_better": False,
           "config": {"workload": f"{WORKLOAD} factored: Hp 2000x2000, Hn 1000x1000, 12 coupling terms, n={M.n}, "
                                  f"nnz of the expansion={M.nnz} (never stored), b={B}, nev={NEV}, tol={TOL}",
                      "method": "bootstrap + FP32 stage + float-float polish on the factored operator"},
           "converged": all(x.converged for x in results), "iters": r.stats["iters"],
           "polish_iters": r.stats["polish_iters"], "max_resid_rel": float(np.max(r.resid) / M.norm_inf),
           "max_rel_err_vs_oracle": oracle_eval_error(r.evals, exact),
           "kron_spmm_ms_per_launch": spmm_ms, "kron_spmm_launches": calls,
           "stream_bytes_per_launch": stream_bytes, "stream_gbs": stream_bytes / (spmm_ms * 1e-3) / 1e9,
           "hbm_alg_bytes_per_launch": r.stats["spmm_bytes"],
           "matrix_device_bytes": int(M.device_bytes), "create_s": t_create,
           "phases_ms": {k: sum(s[k] for s in stats_log) / args.steps
                         for k in ("t_spmm_ms", "t_reorth_ms", "t_cholqr_ms", "t_ritz_ms", "t_total_ms")},
           "plain_fp64_stored_exact": plain, "clocks": clocks}
    print(json.dumps(out))


def run_kron_spmm(args):
    """The factored SpMM alone on the kron_n2e6 factors (n = 2,000,000): FP32
    blocks of b = 8 and 16, FP64 blocks of b = 8, each timed with CUDA events
    over --reps launches after one warm-up; used for the ncu captures of the
    factored kernel."""
    import torch
    import synth
    import paper_2210_15763_gb300 as bbl
    f = synth.named_factors(WORKLOAD)
    M = bbl.KronMatrix(f, storage="fp32")
    lens = np.diff(f.Hp.row_ptr) + 1 + sum(np.diff(c.row_ptr) for c in f.Cp)
    out = {"mode": "kron-spmm", "n": M.n, "nnz_expansion": M.nnz, "factor_bytes": int(M.device_bytes)}
    for dt, b in (("fp32", 8), ("fp32", 16), ("fp64", 8)):
        V = torch.randn(M.n, b, device="cuda", dtype=torch.float32 if dt == "fp32" else torch.float64)
        W = torch.empty_like(V)
        fn = (lambda: bbl.spmm(M, V, W)) if dt == "fp32" else (lambda: bbl.spmm_f64(M, V, W))
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        s_el = 4 if dt == "fp32" else 8
        stream = float(lens.sum()) * f.Hn.n * b * s_el
        out[f"{dt}_b{b}"] = {"ms": ms, "stream_bytes": stream, "stream_gbs": stream / (ms * 1e-3) / 1e9,
                             "hbm_alg_bytes": 2.0 * M.n * b * s_el,
                             "gflops_expansion": 2.0 * M.nnz * b / (ms * 1e-3) / 1e9}
    print(json.dumps(out))


def run_c2(args):
    """The b sweep of the plain FP64 configuration at n = 2,000,000 (the
    paper's Tables I-II: time per operation and vector-equivalent iterations
    against the block size): b in {1, 4, 8, 16}, 8 lowest eigenpairs to
    residual 1e-8, FP64 CSR, random pivot vs the pivot bootstrapped from the
    20,000 lowest-diagonal rows (its FP64 sub-solve to sub_tol).  Per run:
    blocks, vector-equivalent iterations, time-to-solve (including the
    bootstrap), SpMM ms per call, ns per operation t_SpMM / (nnz * b), and
    the largest relative eigenvalue error against the stored oracle values."""
    import torch
    import paper_2210_15763_gb300 as bbl
    A, tgen = build_matrix()
    M = bbl.Matrix(A, storage="fp64", fmt="csr")
    del A
    st = torch.cuda.current_stream()
    rows = []
    for b in [int(x) for x in args.c2_blocks.split(",")]:
        for pivot in ("random", "bootstrap"):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            eb = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            P = None if pivot == "random" else bbl.pivot_bootstrap(M, TRUNC, b, sub_tol=args.sub_tol, seed=PIVOT_SEED)
            eb.record(st)
            r = bbl.solve(M, NEV, b, pivot=P, seed=PIVOT_SEED, tol=TOL, evecs=None, max_vectors=2000)
            e1.record(st)
            torch.cuda.synchronize()
            s = r.stats
            t_call = s["t_spmm_ms"] / max(s["spmm_calls"], 1)
            rows.append({"b": b, "pivot": pivot, "converged": r.converged, "blocks": s["iters"],
                         "vec_equiv_iters": s["iters"] * b, "time_s": e0.elapsed_time(e1) / 1e3,
                         "bootstrap_s": e0.elapsed_time(eb) / 1e3, "spmm_ms_per_call": t_call,
                         "ns_per_op": t_call * 1e6 / (M.nnz * b), "spmm_gbs": s["spmm_gbs"],
                         "reorth_ms": s["t_reorth_ms"], "ritz_ms": s["t_ritz_ms"],
                         "max_rel_err_vs_oracle": oracle_eval_error(r.evals)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    print(json.dumps({"mode": "c2", "workload": f"{WORKLOAD} (n={M.n}, nnz={M.nnz}), FP64 CSR, nev={NEV}, tol={TOL}",
                      "runs": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "kernels", "batched", "learned", "c3", "kron", "c2", "kron-spmm"])
    ap.add_argument("--c2-blocks", default="1,4,8,16")
    ap.add_argument("--c3-vectors", type=int, default=300)
    ap.add_argument("--c3-fp64", action="store_true")
    ap.add_argument("--c3-kron", action="store_true", help="c3 mode: also run the factored operator at n = 2e7")
    ap.add_argument("--ritz-overlap", type=int, default=None)
    ap.add_argument("--sub-tol", type=float, default=SUB_TOL)
    ap.add_argument("--half-first-pass", type=int, default=HALF_FIRST_PASS,
                    help="1: the FP32 stage's first Gram-Schmidt pass reads the FP16 basis copy (library default)")
    ap.add_argument("--fused-update-gram", type=int, default=0,
                    help="1: the first update and the second Gram in one tensor-core kernel; 0 (library default, "
                         "faster at n = 2e6): two FP32 kernels")
    ap.add_argument("--narrow-old-updates", type=int, default=1,
                    help="1 (library default): the FP32 stage's updates read the blocks older than the two "
                         "newest from the FP16 copy; 0: every block in FP32")
    ap.add_argument("--stage1-tol", type=float, default=STAGE1_TOL,
                    help="FP32 stage tolerance before the polish (the library's default is 2e-6; 3e-7 measured "
                         "fastest on kron_n2e6)")
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--family-scale", type=float, default=1.0)
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--batch-max-vectors", type=int, default=400)
    ap.add_argument("--batch-graph", type=int, default=1, help="batched mode: 1 = one graph launch, 0 = host-driven")
    ap.add_argument("--scale", type=float, default=0.5)
    ap.add_argument("--blocks", type=int, default=50)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--ritz-m", type=int, default=728)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    args = ap.parse_args()
    if args.mode == "kernels":
        run_kernels(args)
    elif args.mode == "batched":
        run_batched(args)
    elif args.mode == "learned":
        run_learned(args)
    elif args.mode == "c3":
        run_c3(args)
    elif args.mode == "kron":
        run_kron(args)
    elif args.mode == "c2":
        run_c2(args)
    elif args.mode == "kron-spmm":
        run_kron_spmm(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
