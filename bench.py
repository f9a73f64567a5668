#!/usr/bin/env python
"""Throughput of the block recursive inverse (blocks of M^-1 per second).

Workload (default): n = 4096, k = 8 (b = 512), M = uniform[-1, 1) + n I
(seed 0), every block N_ij computed by its own run of the recursion; a step
is ``--blocks-per-step`` consecutive blocks in row-major order (cycling
through all k^2 blocks over the steps), whose runs are executed together
level by level (``--together``, 0 = one run after the other).  M (134 MB FP64) is larger than L2 (129 MB)
and L2 is also flushed between timed steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain FP64 restatement of the paper's recursion) on the host cores on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "inverse blocks/sec & GEMM % of tensor peak, mixed vs FP64 at ≤1e-10 rel err"
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 (DFMA / FP64 tensor), nominal
# DRAM bytes per algorithmic flop of the FP64_TC panel factorisation, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of the first panel
# launch of `bench.py --inverses 300 --n 512`: 300 panels of 512 rows x 64
# columns read and wrote 99.4 MB for 1.258 GFLOP).  With 64 columns a panel's
# flops and its row traffic both grow with its rows.
PANEL_DRAM_BYTES_PER_FLOP = 99.43e6 / (300 * 2 * 512 * 64 * 64)
# The same for the FP64_TC pivot inverses' digit products (per FP64-equivalent
# flop), from the first four oz_gemm_kernel launches of the same command: the
# products of the first panel pair of 300 matrices of order 512 (two cross
# products, the second panel's done rows, the K = 128 trailing update) read
# and wrote 1.972 GB for the two panels' update work.
UPDATE_DRAM_BYTES_PER_FLOP = 1.971966464e9 / (300 * (2 * 2 * 512 * 64 * 448 + 2 * 64 ** 3))
# The same for the FP64_TC Schur products, from the product launch of
# `bench.py --products 200 --n 512`: one grouped launch of 200 independent
# products of order 512 (42 waves) read and wrote 2.539 GB - the algorithmic
# bytes of its operands; an upper bound for the recursion's launches, whose
# products share operands.
SCHUR_DRAM_BYTES_PER_FLOP = (2.136734720e9 + 0.402228224e9) / (200 * 2 * 512 ** 3)
FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.070  # SMs x FP32 lanes x 2 flop x max GHz
DIGIT_PAIRS = 36  # BF16 digit-pair products per FP64 product on the fp64_tc path


def dtype_name(args):
    return {"fp64": "f64", "fp32": "f32", "mixed": f"bf16x{args.slices}/f32",
            "fp64_tc": "f64 (Schur products: exact bf16 digit products, f32 accumulate)"}[args.precision]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp64_tc", choices=["fp64", "fp32", "mixed", "fp64_tc"])
    p.add_argument("--n", type=int, default=4096)
    p.add_argument("--k", type=int, default=8)
    p.add_argument("--blocks-per-step", type=int, default=64)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-check", action="store_true",
                   help="skip the plain FP64 arm (fp64_tc): its blocks/s on the same step and the distance of the "
                        "last step's first block to it")
    p.add_argument("--products", type=int, default=0,
                   help="time this many grouped FP64_TC products Cin - A B of order n <= 512 (the Schur products' "
                        "kernels alone, through the library's product test hook) in one launch per step")
    p.add_argument("--inverses", type=int, default=0,
                   help="time this many independent pivoted inverses of order n (k = 1) in one batch")
    p.add_argument("--cpu-sample-blocks", type=int, default=1)
    p.add_argument("--cpu-threads", type=int, default=0,
                   help="host threads of the CPU oracle (cpu_baseline and the reference arm); 0 = all cores")
    p.add_argument("--slices", type=int, default=3)
    p.add_argument("--refine", type=int, default=None,
                   help="two-sided refinement steps (0 or 1); default 1 on fp64_tc and fp64, where it meets the "
                        "1e-10 target at k = 8, else 0")
    p.add_argument("--together", type=int, default=64,
                   help="run each step's blocks as independent runs, this many executed together level by level "
                        "in grouped launches (0: one run after the other)")
    p.add_argument("--variant", default="paper", choices=["paper", "principal"],
                   help="paper: the paper's recursion; principal: the reformulation around M/A (principal pivots)")
    p.add_argument("--matrix", default="uniform", choices=["uniform", "haar", "spd"])
    p.add_argument("--kappa", type=float, default=1e4)
    p.add_argument("--batched", type=int, default=0,
                   help="batched workload: this many independent matrices of uneven n and k, one block each")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the tuning of the pivot inverses' panel clusters (mbinv_autotune) that runs, untimed, "
                        "before the warm-up for the inverse batch sizes of the step")
    p.add_argument("--peaks", action="store_true",
                   help="measure the FP64 and FP32 (no TF32) library GEMM rates that the FP64/FP32 rooflines "
                        "are read against: torch.matmul on 8192^3, best of 5, CUDA events")
    p.add_argument("--large", action="store_true",
                   help="memory-bounded workload: n x n Householder matrix in FP32 host memory under a device cap, "
                        "one block per step by the bounded schedule (use --n 65536 --k 16)")
    p.add_argument("--cap-gb", type=float, default=24.0)
    p.add_argument("--sing-tol", type=float, default=0.0,
                   help="relative singularity threshold of the pivots (0: b times the unit roundoff)")
    p.add_argument("--block", type=int, nargs=2, default=[0, 15])
    p.add_argument("--backward", action="store_true",
                   help="differentiation workload: one block forward and the adjoint backward per step")
    args = p.parse_args()
    if args.refine is None:
        args.refine = 1 if args.precision in ("fp64_tc", "fp64") else 0
    return args


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def roofline_of(args, agg, secs):
    """The roofline of each kernel family from the step aggregates (algorithmic
    work / device time against its peak, DRAM traffic per launch where an ncu
    capture gives bytes per flop); the dominant family (most device time)
    heads the result, the others are under "families"."""
    pk, pk_src = peaks()
    npairs = {1: 1, 2: 3, 3: 6}[args.slices] if args.precision == "mixed" else 1
    alu = {"fp64": (FP64_NOMINAL_GFLOPS / 1e3, "nominal FP64 1.25 TFLOP/s (DFMA)"),
           "fp32": (FP32_NOMINAL_GFLOPS / 1e3, "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"),
           "mixed": (FP64_NOMINAL_GFLOPS / 1e3, "nominal FP64 1.25 TFLOP/s (DFMA)"),
           "fp64_tc": (FP64_NOMINAL_GFLOPS / 1e3, "nominal FP64 1.25 TFLOP/s (DFMA)")}[args.precision]
    fams = {}
    tc_src = f"bf16_tflops_sustained ({pk_src})"
    if args.precision == "mixed":
        fams["tc_gemm_kernel"] = {"bound": "tensor", "work": agg["gemm_flops"] * npairs,
                                  "dsec": agg["gemm_device_seconds"], "launches": agg["gemm_launches"],
                                  "peak": pk["bf16_tflops_sustained"],
                                  "peak_source": f"{tc_src}, executed BF16 slice products"}
    elif args.precision == "fp64_tc":
        fams["oz_gemm_kernel"] = {"bound": "tensor", "work": agg["gemm_flops"] * DIGIT_PAIRS,
                                  "dsec": agg["gemm_device_seconds"], "launches": agg["gemm_launches"],
                                  "peak": pk["bf16_tflops_sustained"],
                                  "peak_source": f"{tc_src}, executed BF16 digit-pair products "
                                                 f"({DIGIT_PAIRS} per FP64 product); Schur products only"}
    else:
        fams["gemm_grouped_kernel"] = {"bound": "alu", "work": agg["gemm_flops"], "dsec": agg["gemm_device_seconds"],
                                       "launches": agg["gemm_launches"], "peak": alu[0], "peak_source": alu[1]}
    fp_peak = alu
    fams["gj_panel_kernel"] = {"bound": "alu", "work": agg["inv_panel_flops"],
                               "dsec": agg["inv_panel_device_seconds"], "launches": agg["inv_panel_launches"],
                               "peak": fp_peak[0], "peak_source": fp_peak[1] + "; panel factorisations, 2 b w^2 "
                                                                  "flop per panel of width w"}
    upd_dsec = agg["inv_device_seconds"] - agg["inv_panel_device_seconds"]
    if args.precision == "fp64_tc":
        fams["gj_trailing_update"] = {"bound": "tensor", "work": agg["inv_update_flops"] * DIGIT_PAIRS,
                                      "dsec": upd_dsec, "launches": agg["inv_panel_launches"],
                                      "peak": pk["bf16_tflops_sustained"],
                                      "peak_source": f"{tc_src}, executed digit-pair products of the trailing "
                                                     "updates; time includes their digit packs and the inverses' "
                                                     "init/finalize"}
    else:
        fams["gj_trailing_update"] = {"bound": "alu", "work": agg["inv_update_flops"], "dsec": upd_dsec,
                                      "launches": None, "peak": fp_peak[0],
                                      "peak_source": fp_peak[1] + "; gj_update_kernel, time includes the "
                                                                  "inverses' init/finalize"}
    kernels = {}
    for name, f in fams.items():
        ach = f["work"] / f["dsec"] / 1e12 if f["dsec"] > 0 else 0.0
        kernels[name] = {"bound": f["bound"], "achieved": ach, "peak": f["peak"], "unit": "TFLOP/s",
                         "frac": ach / f["peak"], "device_seconds": f["dsec"], "peak_source": f["peak_source"]}
        if f.get("launches"):
            kernels[name]["launches"] = f["launches"]
        if name == "gj_panel_kernel" and args.precision == "fp64_tc" and f.get("launches"):
            # DRAM bytes of an average launch (ncu bytes per flop x its flops)
            kernels[name]["traffic"] = PANEL_DRAM_BYTES_PER_FLOP * f["work"] / f["launches"]
            kernels[name]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, "
                                               "scaled by algorithmic flops to the average launch")
        if name == "oz_gemm_kernel" and f.get("launches"):
            kernels[name]["traffic"] = SCHUR_DRAM_BYTES_PER_FLOP * agg["gemm_flops"] / f["launches"]
            kernels[name]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one Schur-product "
                                               "launch, scaled by algorithmic flops to the average launch")
        if name == "gj_trailing_update" and args.precision == "fp64_tc" and f.get("launches"):
            # one trailing update per panel launch; FP64-equivalent flops
            kernels[name]["traffic"] = UPDATE_DRAM_BYTES_PER_FLOP * agg["inv_update_flops"] / f["launches"]
            kernels[name]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one trailing-"
                                               "update oz_gemm_kernel launch, scaled by algorithmic flops to the "
                                               "average update (its digit packs and done-rows products excluded)")
        if args.precision == "fp64_tc" and f["bound"] == "tensor":
            # the method's own work: FP64-equivalent flops, against the BF16
            # rate the kernel runs on and against GB300's nominal FP64 rate
            kernels[name]["fp64_equivalent_tflops"] = ach / DIGIT_PAIRS
            kernels[name]["frac_fp64_equivalent_of_bf16"] = ach / DIGIT_PAIRS / f["peak"]
            kernels[name]["x_nominal_fp64"] = ach / DIGIT_PAIRS / (FP64_NOMINAL_GFLOPS / 1e3)
    if agg["pack_device_seconds"] > 0:
        gbs = agg.get("pack_bytes", 0.0) / agg["pack_device_seconds"] / 1e9
        kernels["oz_pack_kernel" if args.precision == "fp64_tc" else "pack_kernel"] = {
            "bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": gbs / pk["hbm_gbs"],
            "device_seconds": agg["pack_device_seconds"],
            "peak_source": f"hbm_gbs ({pk_src}); algorithmic bytes: each operand entry read once, its digits "
                           "(or slices) written once, one exponent per row"}
    dom = max((k for k in kernels if "bound" in kernels[k] and kernels[k]["unit"] == "TFLOP/s"),
              key=lambda k: kernels[k]["device_seconds"])
    roofline = dict(kernels[dom])
    roofline.update({"kernel": dom, "traffic": kernels[dom].get("traffic"), "step_tflops": (agg["gemm_flops"] + agg["inv_flops"]) / secs / 1e12,
                     "families": kernels})
    return roofline


def fp64_path_arm(args, M, k, b, bps, rank, world, first_block, m_host):
    """The plain FP64 path (CUDA-core products and inverses) on the bench's
    step: one untimed step, then one step timed with CUDA events; its blocks/s,
    its error against the dense inverse, and how far the headline path's first
    block of the last step lies from the FP64 path's."""
    import numpy as np
    import torch

    import paper_1612_00001_gb300 as mb
    stream = torch.cuda.current_stream()
    outs = [torch.empty((b, b), dtype=torch.float64, device="cuda") for _ in range(bps)]
    last = args.warmup + args.steps - 1
    ij = rank_blocks(k, rank, world, last, bps)
    with mb.Context(M, k, precision="fp64", refine=args.refine, variant=args.variant) as c64:
        c64.blocks(ij, outs=outs, width=args.together or 1)  # untimed: plans and workspace
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        c64.blocks(ij, outs=outs, width=args.together or 1)
        e1.record(stream)
        torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    inv = np.linalg.inv(m_host)
    errs = []
    for q, (i, j) in enumerate(ij):
        r = inv[i * b:(i + 1) * b, j * b:(j + 1) * b]
        errs.append(float(np.linalg.norm(outs[q].double().cpu().numpy() - r) / np.linalg.norm(r)))
    ref64 = outs[0].double().cpu().numpy()
    diff = float(np.linalg.norm(first_block.double().cpu().numpy() - ref64) / np.linalg.norm(ref64))
    return {"value": bps / secs, "unit": "blocks/s", "ms_per_step": 1e3 * secs, "steps": 1,
            "max_rel_err_vs_dense_inverse": max(errs), "refine": args.refine,
            "rel_diff_of_headline_block": diff}


def householder_svd_device(n, kappa, seed, reflectors=64):
    """M = U diag(sigma) V^T (the Householder construction of bri_inputs, the
    same reflector vectors) built on the GPU in FP64 for sizes the host
    cannot handle; returns (M on the device, vu, vv, sigma)."""
    import torch

    import bri_inputs as bi
    vu = torch.tensor(bi.gaussian(seed, bi.STREAM_HOUSE, reflectors * n).reshape(reflectors, n), device="cuda")
    vv = torch.tensor(bi.gaussian(seed + 0x5151, bi.STREAM_HOUSE, reflectors * n).reshape(reflectors, n),
                      device="cuda")
    sig = torch.tensor(bi.log_spaced(n, kappa), device="cuda")
    m = torch.diag(sig)
    for v in reversed(vu):  # U X = H_1 (H_2 (... H_r X))
        m.addr_(v, v @ m, alpha=-2.0 / float(v @ v))
    for v in reversed(vv):  # X V^T = X H_r ... H_1
        m.addr_(m @ v, v, alpha=-2.0 / float(v @ v))
    return m, vu, vv, sig


def householder_inverse_columns(vu, vv, sig, j0, j1):
    """Columns j0..j1-1 of M^-1 = V diag(1/sigma) U^T in closed form (FP64)."""
    import torch
    n = sig.shape[0]
    y = torch.zeros((n, j1 - j0), dtype=torch.float64, device="cuda")
    y[j0:j1] = torch.eye(j1 - j0, dtype=torch.float64, device="cuda")
    for v in vu:  # U^T Y = H_r (... (H_1 Y))
        y.addr_(v, v @ y, alpha=-2.0 / float(v @ v))
    y.div_(sig[:, None])
    for v in reversed(vv):  # V Y = H_1 (... (H_r Y))
        y.addr_(v, v @ y, alpha=-2.0 / float(v @ v))
    return y


def stored_inverse_columns(m_stored, vu, vv, sig, j0, j1, iters=2):
    """Columns j0..j1-1 of the inverse of the stored matrix (FP32 entries
    taken exactly): the closed form for the unrounded matrix, corrected by
    iterative refinement against the stored one (FP64 products)."""
    import torch
    y = householder_inverse_columns(vu, vv, sig, j0, j1)
    n = m_stored.shape[0]
    for _ in range(iters):
        r = -(m_stored @ y)
        r[j0:j1] += torch.eye(j1 - j0, dtype=torch.float64, device="cuda")
        # apply M^-1 in closed form to the residual columns
        for v in vu:
            r.addr_(v, v @ r, alpha=-2.0 / float(v @ v))
        r.div_(sig[:, None])
        for v in reversed(vv):
            r.addr_(v, v @ r, alpha=-2.0 / float(v @ v))
        y += r
        del r
    return y


def make_matrix(args, n):
    import bri_inputs as bi
    if args.matrix == "haar":
        return bi.haar_svd(n, args.kappa, 0)
    if args.matrix == "spd":
        return bi.spd(n, args.kappa, 0)
    return bi.uniform_shift(n, 0)


def matrix_name(args):
    return {"uniform": "uniform[-1,1)+nI", "haar": f"U diag(sigma) V^T, Haar U V, cond {args.kappa:g}",
            "spd": f"SPD Q diag(mu) Q^T, cond {args.kappa:g}"}[args.matrix]


def block_list(k, start, count):
    return [((start + t) % (k * k) // k, (start + t) % (k * k) % k) for t in range(count)]


def rank_blocks(k, rank, world, step, bps):
    """The blocks a replica computes in one step: the step's world*bps
    consecutive blocks of the row-major sequence, split into contiguous shares."""
    return block_list(k, (step * world + rank) * bps, bps)


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None  # samples go to a temporary file, summarised by stop()

    def start(self):
        import tempfile
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"mbinv_clocks{self.idx}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            self._remove()
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        try:
            return self._summary()
        finally:
            self._remove()

    def _remove(self):
        try:
            if getattr(self, "f", None) is not None and not self.f.closed:
                self.f.close()
            if self.path:
                os.remove(self.path)
        except OSError:
            pass

    def _summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_time(m, k, blocks, threads=0):
    """Seconds per block of the oracle (memoized recursion; all host cores, or
    `threads` of them)."""
    import oracle
    oracle.build()
    if threads > 0:
        oracle.set_num_threads(threads)
    t0 = time.perf_counter()
    for (i, j) in blocks:
        _, st, _ = oracle.bri_block(m, k, i, j, memo=True)
        assert st == oracle.OK
    return (time.perf_counter() - t0) / len(blocks), oracle.num_threads()


def run_reference(args, rank):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    import bri_inputs as bi
    m = bi.uniform_shift(args.n, 0)
    k = args.k
    seq = block_list(k, 0, args.warmup + args.steps)
    for t in range(args.warmup):
        cpu_oracle_time(m, k, [seq[t]], args.cpu_threads)
    per = []
    for t in range(args.steps):
        s, cores = cpu_oracle_time(m, k, [seq[args.warmup + t]], args.cpu_threads)
        per.append(s)
    secs = sum(per)
    value = args.steps / secs
    sample = f"{args.steps} blocks of the n={args.n}, k={k} uniform+nI matrix, one per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"n={args.n} k={k} b={args.n // k} uniform[-1,1)+nI FP64, one block per step",
                       "blocks_per_step": 1, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _clock_region(local):
    c = Clocks(local)
    c.start()
    return c


def run_batched(args, rank, world, dist):
    """Independent matrices of uneven n in [256, 4096] (multiples of 64) and k in
    {2..8}, uniform[-1,1)+nI, one block (i, j) each; a step is the whole batch
    through mbinv_batched_blocks."""
    import numpy as np
    import torch

    import bri_inputs as bi
    import paper_1612_00001_gb300 as mb
    probs = bi.ragged_batch(args.batched, 0)
    dt = torch.float64 if args.precision in ("fp64", "fp64_tc") else torch.float32
    mats = [torch.tensor(bi.uniform_shift(p["n"], p["seed"]), dtype=dt, device="cuda") for p in probs]
    work = [(M, p["k"], p["i"], p["j"]) for M, p in zip(mats, probs)]
    flops = 0.0
    for s in range(args.warmup):
        outs, st, rep, rc = mb.batched_blocks(work, precision=args.precision)
        assert rc == mb.OK, st
    stream = torch.cuda.current_stream()
    clocks = _clock_region(0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    agg = {"gemm_flops": 0.0, "inv_flops": 0.0, "launches": 0}
    torch.cuda.synchronize()
    for s in range(args.steps):
        ev[s][0].record(stream)
        outs, st, rep, rc = mb.batched_blocks(work, precision=args.precision)
        ev[s][1].record(stream)
        for key in agg:
            agg[key] += rep[key]
    torch.cuda.synchronize()
    clk = clocks.stop()
    secs = sum(a.elapsed_time(z) for a, z in ev) / 1e3
    # accuracy on a sample of the batch against dense inverses
    errs = []
    for q in range(0, len(probs), max(1, len(probs) // 8)):
        p = probs[q]
        m = bi.uniform_shift(p["n"], p["seed"])
        inv = np.linalg.inv(m.astype(np.float32 if dt == torch.float32 else np.float64).astype(np.float64))
        bb = -(-p["n"] // p["k"])
        r = inv[p["i"] * bb:p["i"] * bb + outs[q].shape[0], p["j"] * bb:p["j"] * bb + outs[q].shape[1]]
        errs.append(float(np.linalg.norm(outs[q].double().cpu().numpy() - r) / np.linalg.norm(r)))
    line = {"metric": METRIC, "value": args.batched * args.steps / secs, "unit": "blocks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_name(args),
            "data": "synthetic",
            "config": {"workload": f"{args.batched} matrices, n ~ U[256,4096] step 64, k ~ U{{2..8}}, "
                                   f"uniform[-1,1)+nI, one block each, runs executed together ({args.precision})",
                       "max_rel_err_vs_dense_inverse_sample": max(errs)},
            "step_tflops": (agg["gemm_flops"] + agg["inv_flops"]) / secs / 1e12, "gpu_launches": agg["launches"],
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_inverses(args, rank, world, dist):
    """The leaf pivot inverse alone: args.inverses independent matrices of
    order n, uniform[-1,1) + (n/8) I, each inverted by the blocked pivoted
    Gauss-Jordan kernels (a k = 1 request) in one batch per step."""
    import numpy as np
    import torch

    import bri_inputs as bi
    import paper_1612_00001_gb300 as mb
    n = args.n
    dt = torch.float64 if args.precision in ("fp64", "fp64_tc") else torch.float32
    mats = [torch.tensor(bi.uniform_shift(n, s, shift=n / 8), dtype=dt, device="cuda") for s in range(args.inverses)]
    work = [(M, 1, 0, 0) for M in mats]
    for s in range(args.warmup):
        outs, st, rep, rc = mb.batched_blocks(work, precision=args.precision)
        assert rc == mb.OK, st
    stream = torch.cuda.current_stream()
    clocks = _clock_region(0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = 0
    for s in range(args.steps):
        ev[s][0].record(stream)
        outs, st, rep, rc = mb.batched_blocks(work, precision=args.precision)
        ev[s][1].record(stream)
        launches += rep["launches"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    secs = sum(a.elapsed_time(z) for a, z in ev) / 1e3
    inv = np.linalg.inv(bi.uniform_shift(n, 0, shift=n / 8))
    err = float(np.linalg.norm(outs[0].double().cpu().numpy() - inv) / np.linalg.norm(inv))
    line = {"metric": "pivoted b x b inverses/s", "value": args.inverses * args.steps / secs, "unit": "inverses/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(args),
            "data": "synthetic",
            "config": {"workload": f"{args.inverses} inverses of order {n}, uniform[-1,1)+(n/8)I ({args.precision})",
                       "tflops_fp64_equivalent": 2.0 * n ** 3 * args.inverses * args.steps / secs / 1e12,
                       "rel_err_vs_dense_inverse": err},
            "gpu_launches": launches, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_products(args, rank, world, dist):
    """The Schur products' digit-product kernel alone: args.products
    independent FP64 products out = Cin - A B of order n (A, B, Cin uniform
    [-1, 1)), one grouped launch per step (the operands' digit packs
    included), through the library's product test hook."""
    import ctypes

    import torch

    import paper_1612_00001_gb300 as mb
    n, cnt = args.n, args.products
    g = torch.Generator(device="cuda").manual_seed(11)
    A = torch.rand((cnt, n, n), dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    B = torch.rand((cnt, n, n), dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    C = torch.rand((cnt, n, n), dtype=torch.float64, device="cuda", generator=g) * 2 - 1
    out = torch.empty_like(C)
    L = mb.test_lib()
    L.mbinv_debug_oz_products_bytes.restype = ctypes.c_size_t
    L.mbinv_debug_oz_products_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    f = L.mbinv_debug_oz_products
    f.restype = ctypes.c_int
    f.argtypes = ([ctypes.c_void_p] * 4 + [ctypes.c_int] * 2 + [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                                                 ctypes.c_void_p])
    wsb = L.mbinv_debug_oz_products_bytes(n, cnt)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(pack):
        rc = f(A.data_ptr(), B.data_ptr(), C.data_ptr(), out.data_ptr(), n, cnt, ws.data_ptr(), wsb, pack,
               stream.cuda_stream)
        assert rc == 0, rc

    for _ in range(args.warmup):
        step(1)
    clocks = _clock_region(0)

    def timed(pack):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for s in range(args.steps):
            ev[s][0].record(stream)
            step(pack)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(z) for a, z in ev) / 1e3

    secs = timed(1)
    secs_gemm = timed(0)  # the product launch alone (operands > L2: 200 x 8 MB of digits)
    clk = clocks.stop()
    ref = C[0] - A[0] @ B[0]
    err = float(torch.linalg.norm(out[0] - ref) / torch.linalg.norm(ref))
    flops = 2.0 * n ** 3 * cnt * args.steps
    pk, pk_src = peaks()
    peak = pk["bf16_tflops_sustained"]
    executed = DIGIT_PAIRS * flops / secs_gemm / 1e12
    line = {"metric": "FP64 products/s (digit products on the BF16 tensor cores)", "value": cnt * args.steps / secs,
            "unit": "products/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (exact bf16 digit products, f32 accumulate)", "data": "synthetic",
            "config": {"workload": f"{cnt} products Cin - A B of order {n}, uniform[-1,1) (fp64_tc), packs included",
                       "tflops_fp64_equivalent": flops / secs / 1e12, "rel_err_vs_torch_fp64": err,
                       "product_launch_ms": 1e3 * secs_gemm / args.steps,
                       "l2": "operands larger than L2 (digits 8 MB per product)"},
            "roofline": {"bound": "tensor", "kernel": "oz_gemm_kernel", "achieved": executed, "peak": peak,
                         "unit": "TFLOP/s", "frac": executed / peak, "device_seconds": secs_gemm,
                         "traffic": SCHUR_DRAM_BYTES_PER_FLOP * 2.0 * n ** 3 * cnt,
                         "peak_source": f"bf16_tflops_sustained ({pk_src}), executed BF16 digit-pair products "
                                        "(36 per FP64 product), the product launch alone"},
            "gpu_launches": 5 * args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_peaks(args, rank):
    """FP64 and FP32 GEMM rates of the library (cuBLAS through torch.matmul,
    TF32 off) on 8192^3: the measured ceilings beside the nominal FP64 1.25
    TFLOP/s used for the CUDA-core kernels' rooflines."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    n = 8192
    out = {}
    for name, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        a = torch.rand((n, n), dtype=dt, device="cuda")
        b = torch.rand((n, n), dtype=dt, device="cuda")
        for _ in range(2):
            a @ b
        best = 1e9
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        out[name] = 2.0 * n ** 3 / best / 1e12
        del a, b
    if rank == 0:
        print(json.dumps({"metric": "library GEMM rate (torch.matmul, 8192^3, best of 5)", "unit": "TFLOP/s",
                          "fp64_tflops": out["fp64"], "fp32_tflops": out["fp32"], "tf32": False}), flush=True)


def run_large(args, rank, world, dist):
    """The memory-bounded workload: n = 65536, k = 16 (b = 4096), M = U diag(sigma)
    V^T with U, V each a product of 64 Householder reflectors, cond(M) = kappa,
    stored in FP32 (17.2 GB) in pinned host memory; a device cap (24 GB); one
    block N_ij per step through the C ABI with the bounded schedule (frames
    depth first in the slots the cap leaves, values needed later in pinned host
    memory, M read block by block), FP64_TC arithmetic, the block returned in
    FP64.  Its error is taken against the inverse of the stored FP32 matrix:
    the closed form V diag(1/sigma) U^T of the unrounded matrix, corrected by
    two steps of iterative refinement with FP64 products."""
    import numpy as np
    import torch

    import paper_1612_00001_gb300 as mb
    n, k = args.n, args.k
    b = n // k
    cap = int(args.cap_gb * 1e9)
    m64, vu, vv, sig = householder_svd_device(n, args.kappa, 0)
    m32 = m64.to(torch.float32)
    del m64
    torch.cuda.empty_cache()
    mh = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    mh.copy_(m32)
    i, j = args.block
    stream = torch.cuda.current_stream()
    out = torch.empty((b, b), dtype=torch.float64, device="cuda")
    ctx = mb.Context(mh, k, precision=args.precision, cap=cap, out_dtype=torch.float64, sing_tol=args.sing_tol,
                     pivot_cond=True)
    for _ in range(args.warmup):
        ctx.block(i, j, out=out)
    clocks = _clock_region(0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = []
    for s in range(args.steps):
        ev[s][0].record(stream)
        ctx.block(i, j, out=out)
        ev[s][1].record(stream)
        reps.append(ctx.last_report)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    secs = sum(a.elapsed_time(z) for a, z in ev) / 1e3
    rep = reps[-1]
    ctx.close()
    # the inverse of the stored matrix, block column j, rows of block i
    ms = m32.to(torch.float64)
    del m32
    y = stored_inverse_columns(ms, vu, vv, sig, j * b, (j + 1) * b)
    ref = y[i * b:(i + 1) * b].clone()
    del y, ms
    err = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
    closed = householder_inverse_columns(vu, vv, sig, j * b, (j + 1) * b)[i * b:(i + 1) * b]
    err_unrounded = float(torch.linalg.norm(out - closed) / torch.linalg.norm(closed))
    flops = rep["gemm_flops"] + rep["inv_flops"]
    line = {"metric": METRIC, "value": args.steps / secs, "unit": "blocks/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(args),
            "data": "synthetic",
            "config": {"workload": f"n={n} k={k} b={b} U diag(sigma) V^T (64 Householder reflectors each), "
                                   f"cond {args.kappa:g}, FP32 storage in pinned host memory, device cap "
                                   f"{args.cap_gb:g} GB, block ({i},{j}), bounded schedule ({args.precision})",
                       "device_cap_bytes": cap, "peak_device_bytes": rep["peak_device_bytes"],
                       "planned_device_bytes": rep["planned_device_bytes"],
                       "host_in_bytes": rep["host_in_bytes"], "host_out_bytes": rep["host_out_bytes"],
                       "host_spill_bytes": rep["host_spill_bytes"], "frames": rep["frames"],
                       "inversions": rep["inversions"], "launches": rep["launches"],
                       "max_pivot_cond": rep["max_pivot_cond"], "sing_tol": args.sing_tol,
                       "fp64_equivalent_tflops": flops / secs / 1e12,
                       "rel_err_vs_inverse_of_stored_matrix": err,
                       "rel_err_vs_inverse_of_unrounded_matrix": err_unrounded,
                       "wall_seconds": wall,
                       "launches_per_block": rep["launches"]},
            "gpu_launches": rep["launches"] * args.steps, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_backward(args, rank, world, dist):
    """Differentiation: L = sum(W * N_ij), W ~ N(0,1); a step is the forward
    block and dL/dM = -(X_i)^T W (Y_j)^T, the block row and column recomputed
    block by block."""
    import numpy as np
    import torch

    import bri_inputs as bi
    import paper_1612_00001_gb300 as mb
    n, k = args.n, args.k
    b = -(-n // k)
    m = bi.spd(n, args.kappa, 0) if args.matrix == "spd" else make_matrix(args, n)
    dt = torch.float64 if args.precision in ("fp64", "fp64_tc") else torch.float32
    M = torch.tensor(m, dtype=dt, device="cuda")
    W = torch.tensor(bi.gaussian_matrix(b, b, 0), dtype=dt, device="cuda")
    i, j = 1, k - 2
    ctx = mb.Context(M, k, precision=args.precision, slices=args.slices, refine=args.refine, variant=args.variant)
    dM = torch.zeros((n, n), dtype=dt, device="cuda")

    def step():
        nb = ctx.block(i, j)
        dM.zero_()
        ctx.backward(i, j, W, dM)
        return nb

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    clocks = _clock_region(0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for s in range(args.steps):
        ev[s][0].record(stream)
        nb = step()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    secs = sum(a.elapsed_time(z) for a, z in ev) / 1e3
    # FP64 reference gradient from a dense inverse on the host
    inv = np.linalg.inv(m)
    ref = -(inv[i * b:(i + 1) * b, :].T @ W.double().cpu().numpy() @ inv[:, j * b:(j + 1) * b].T)
    gerr = float(np.linalg.norm(dM.double().cpu().numpy() - ref) / np.linalg.norm(ref))
    ferr = float(np.linalg.norm(nb.double().cpu().numpy() - inv[i * b:(i + 1) * b, j * b:(j + 1) * b])
                 / np.linalg.norm(inv[i * b:(i + 1) * b, j * b:(j + 1) * b]))
    line = {"metric": METRIC, "value": args.steps / secs, "unit": "forward+backward/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_name(args),
            "data": "synthetic",
            "config": {"workload": f"n={n} k={k} b={b} {matrix_name(args)}, L = sum(W * N_{i}{j}), "
                                   f"forward + adjoint ({args.precision}, refine {args.refine}"
                                   + (", principal-Schur variant" if args.variant == "principal" else "") + ")",
                       "rel_err_forward_vs_dense": ferr, "rel_err_grad_vs_fp64_reference": gerr},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch

    import bri_inputs as bi
    import paper_1612_00001_gb300 as mb

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mb.build()
    if args.batched:
        return run_batched(args, rank, world, dist)
    if args.inverses:
        return run_inverses(args, rank, world, dist)
    if args.products:
        return run_products(args, rank, world, dist)
    if args.backward:
        return run_backward(args, rank, world, dist)
    if args.large:
        return run_large(args, rank, world, dist)
    if args.peaks:
        return run_peaks(args, rank)
    n, k = args.n, args.k
    b = -(-n // k)
    bps = args.blocks_per_step
    m_host = make_matrix(args, n)
    dt = torch.float64 if (args.precision in ("fp64", "fp64_tc") or args.refine) else torch.float32
    M = torch.tensor(m_host, dtype=dt, device="cuda")
    stream = torch.cuda.current_stream()
    ctx = mb.Context(M, k, precision=args.precision, profile=True, slices=args.slices, refine=args.refine,
                     variant=args.variant)
    outs = [torch.empty((b, b), dtype=dt, device="cuda") for _ in range(bps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # each rank takes its own share of the block sequence (replicas, no collective)

    def step(s, c=ctx, dst=outs):
        reps = []
        ij = rank_blocks(k, rank, world, s, bps)
        if args.together:
            c.blocks(ij, outs=dst, width=args.together)
            return [c.last_report]
        for q, (i, j) in enumerate(ij):
            c.block(i, j, out=dst[q])
            reps.append(c.last_report)
        return reps

    tuned = None
    if not args.no_autotune and args.precision in ("fp64", "fp64_tc"):
        # the step's inverse batches: the merged plan's pivots per level (powers
        # of two bucket the batch sizes)
        tuned = {}
        for cnt in (1, 4, 8, 64, 128, 512, 1024):
            tuned[cnt] = mb.autotune(b, cnt, args.precision)[0]
    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    agg = {"gemm_flops": 0.0, "inv_flops": 0.0, "gemm_device_seconds": 0.0, "inv_device_seconds": 0.0,
           "launches": 0, "gemm_launches": 0, "inversions": 0, "peak_device_bytes": 0,
           "pack_device_seconds": 0.0, "inv_panel_device_seconds": 0.0, "inv_panel_flops": 0.0,
           "inv_update_flops": 0.0, "inv_panel_launches": 0, "pack_bytes": 0.0, "frames": 0, "request_frames": 0}
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s & 0xFF)  # L2 flush, outside the timed interval
        ev[s][0].record(stream)
        reps = step(args.warmup + s)
        ev[s][1].record(stream)
        for r in reps:
            for key in agg:
                agg[key] = max(agg[key], r[key]) if key == "peak_device_bytes" else agg[key] + r[key]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    secs = sum(a.elapsed_time(z) for a, z in ev) / 1e3
    if dist:
        t = torch.tensor([secs], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    total_blocks = bps * args.steps * world
    value = total_blocks / secs

    # accuracy of the last step's blocks against a dense LAPACK inverse on the host
    inv_ref = np.linalg.inv(m_host)
    errs = []
    for q, (i, j) in enumerate(rank_blocks(k, rank, world, args.warmup + args.steps - 1, bps)):
        r = inv_ref[i * b:(i + 1) * b, j * b:(j + 1) * b]
        errs.append(float(np.linalg.norm(outs[q].double().cpu().numpy() - r) / np.linalg.norm(r)))
    del inv_ref
    # the plain FP64 CUDA-core path on the same step (same blocks, same
    # refinement, same runs merged): the "mixed vs FP64" half of the metric
    fp64_arm = None
    if args.precision == "fp64_tc" and not args.no_fp64_check:
        fp64_arm = fp64_path_arm(args, M, k, b, bps, rank, world, outs[0], m_host)
    roofline = roofline_of(args, agg, secs)

    line = {"metric": METRIC, "value": value, "unit": "blocks/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(args), "data": "synthetic",
            "config": {"workload": f"n={n} k={k} b={b} {matrix_name(args)}, "
                                   + (f"{args.together} runs merged" if args.together
                                      else "blocks one at a time") + f" ({args.precision}"
                                   + (", principal-Schur variant" if args.variant == "principal" else "") + ")",
                       "blocks_per_step": bps, "precision": args.precision, "slices": args.slices,
                       "refine": args.refine,
                       "l2": "M larger than L2 and a 256 MB L2 flush between timed steps",
                       "max_rel_err_vs_dense_inverse": max(errs),
                       "autotuned_cluster_bias": tuned,
                       "frames_evaluated_per_step": agg["frames"] // args.steps,
                       "frames_of_the_runs_alone_per_step": agg["request_frames"] // args.steps},
            "fp64_path": fp64_arm,
            "speedup_vs_fp64_path": (value / fp64_arm["value"]) if fp64_arm else None,
            "roofline": roofline, "gpu_launches": agg["launches"],
            "peak_device_bytes": agg["peak_device_bytes"], "clocks": clk}
    ctx.close()

    # end to end through the C ABI with host buffers (H2D of M and D2H of the blocks timed)
    if not args.no_e2e and rank == 0:
        mh = torch.tensor(m_host, dtype=dt).pin_memory()
        houts = [torch.empty((b, b), dtype=dt).pin_memory() for _ in range(bps)]
        e2e_steps = max(1, min(args.steps, 3))
        # one context for the stream of matrices (created, planned and warmed
        # up once); every timed step re-reads M from pinned host memory
        # (mbinv_reload: the H2D copy) and returns its blocks to pinned host
        # memory (the D2H copies)
        with mb.Context(mh, k, precision=args.precision, slices=args.slices, refine=args.refine,
                        variant=args.variant) as hc:
            def e2e_step(s):
                hc.reload()
                ij = block_list(k, s * bps, bps)
                if args.together:
                    hc.blocks(ij, outs=houts, width=args.together)
                else:
                    for q, (i, j) in enumerate(ij):
                        hc.block(i, j, out=houts[q])
            e2e_step(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(e2e_steps):
                e2e_step(s)
            torch.cuda.synchronize()
            te = time.perf_counter() - t0
        es = dt.itemsize if hasattr(dt, "itemsize") else (8 if dt == torch.float64 else 4)
        line["e2e"] = {"value": e2e_steps * bps / te, "unit": "blocks/s", "h2d_bytes_per_step": n * n * es,
                       "d2h_bytes_per_step": bps * b * b * es, "steps": e2e_steps,
                       "timing": "host wall clock; one context created and warmed up before the timed steps, "
                                 "each step mbinv_reload (H2D of M) + mbinv_blocks (D2H of the blocks)"}
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        secs_cpu, cores = cpu_oracle_time(m_host, k, block_list(k, 0, args.cpu_sample_blocks), args.cpu_threads)
        line["cpu_baseline"] = {"value": 1.0 / secs_cpu, "unit": "blocks/s", "cores": cores, "kind": "oracle",
                                "sample": f"{args.cpu_sample_blocks} block(s) from (0,0) of the same matrix, "
                                          "memoized recursion, FP64"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
