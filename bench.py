"""Benchmark of the response-density-matrix solve on one or more GB300s.

One step = one full solve (Gershgorin bounds, initial matrices, every TC2 /
first-order iteration with its block-sparse products and truncation, the
polarizability) of the 2,000-atom random-packed cluster (8 orbitals per atom,
N = 16,000, 32 x 32 blocks, truncation 1e-6, H1 for x, y and z).  Inputs are
resident in HBM before the timed region; the working set (X0, X1 for three
directions, ~1 GB in FP64) is far larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode M] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own
copy of the workload (independent problems, weak scaling, no collective on
the data path).  ``--impl reference`` times the CPU oracle (dense FP64 TC2)
on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per P1 solve (block-SpGEMM TFLOP/s alongside), FP64 vs mixed, at |dalpha|/alpha <= 1e-6"
WORKLOAD = "cluster-2000-atoms-N16000-b32-tau1e-6-xyz"
# TC2 iterations of the oracle's stopping rule on this workload, predicted by
# tests/golden/make_golden.py from the spectrum of H0 (oracle only)
ORACLE_ITERS_FILE = os.path.join(ROOT, "tests", "golden", "cfg2_oracle.json")
FP64_PEAK_NOTE = ("GB300 FP64: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz = 1.26 TFLOP/s "
                  "(nominal 1.25 TFLOP/s)")
FP32_PEAK_NOTE = "GB300 FP32: 152 SMs x 128 FMA/clk/SM x 2 flop x 2.07 GHz = 80.5 TFLOP/s"

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged
# over the launches of one solve) of the product kernels on the 2,000-atom
# cluster, from one ncu capture (profiles/); reported only while the code of the
# kernel's source file is unchanged since (SHA-256 of the file with comments and
# whitespace removed, so that a comment edit keeps the figure and a code edit drops it)
PROFILED_TRAFFIC = {
    "tc": {"file": "paper_2009_03551_gb300/csrc/k_tc.cu",
           "sha256": "6a82385f0d0a5f5e14c70eba34567217d1377dd7c2340b3f90a7116d34ac1682",
           "bytes_per_launch": 24744794482, "workload": WORKLOAD},
    "ff": {"file": "paper_2009_03551_gb300/csrc/k_numeric.cu",
           "sha256": "1c9d3e76e36659e5d06b0d237474522761ebecc2732c37eb20f037dc4adcb12e",
           "bytes_per_launch": 10398166912, "workload": WORKLOAD},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default=os.environ.get("RDM_BENCH_MODE", "mixed_fp16"),
                    choices=["fp64", "fp32", "mixed_bf16", "mixed_fp16"])
    ap.add_argument("--atoms", type=int, default=2000, help="atoms of the cluster workload")
    ap.add_argument("--workload", default="cluster",
                    help="cluster (default: the 2,000-atom cluster, or --atoms), batch24 (24 uneven "
                         "chains/clusters, 300-8,000 atoms), slab<N> (30-bohr slab of N atoms)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--tau", type=float, default=1e-6, help="block truncation threshold")
    ap.add_argument("--tau-refine", type=float, default=-1.0,
                    help="threshold of the final (FP64/FP32) tier of the mixed modes (< 0: --tau); the "
                         "FP64 comparison solve runs at this threshold throughout")
    return ap.parse_args()


def profiled_traffic(cls, workload):
    """Bytes per launch of the class's kernel from the committed capture, or None."""
    import hashlib
    rec = PROFILED_TRAFFIC.get(cls)
    if rec is None or rec["workload"] != workload:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), rec["file"])
    try:
        sha = code_sha256(path)
    except OSError:
        return None
    return rec["bytes_per_launch"] if sha == rec["sha256"] else None


def code_sha256(path):
    """SHA-256 of a C/C++/CUDA source file with its comments and all whitespace removed."""
    return code_digest(open(path, encoding="utf-8").read())


def code_digest(src):
    """SHA-256 of C/C++/CUDA source text with its comments and all whitespace removed."""
    import hashlib
    import re
    # string and character literals are kept whole; comments are dropped
    tok = re.compile(r'"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'|//[^\n]*|/\*.*?\*/', re.S)
    code = tok.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", src)
    return hashlib.sha256(re.sub(r"\s+", "", code).encode()).hexdigest()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
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
            parts = [x.strip() for x in ln.split(",")]
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


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def oracle_iterations():
    try:
        with open(ORACLE_ITERS_FILE) as f:
            return int(json.load(f)["tc2_iterations"])
    except Exception:
        return 17


def oracle_sample(sys_, reps: int = 1):
    """Time the oracle's dominant operation on this workload: one dense FP64
    product X0 X0 of the full N x N matrix (numpy / threaded BLAS), then scale
    to one solve = (1 + 2 * n_dirs) products per iteration x iterations."""
    from oracle.tc2 import gershgorin_bounds
    h0 = sys_.h0.to_dense()
    lo, hi = gershgorin_bounds(h0)
    x0 = (hi * np.eye(h0.shape[0]) - h0) / (hi - lo)
    del h0
    times = []
    for _ in range(reps):
        t = time.perf_counter()
        _ = x0 @ x0
        times.append(time.perf_counter() - t)
    iters = oracle_iterations()
    per_product = min(times)
    n_prod = 1 + 2 * len(sys_.h1)
    return per_product, per_product * n_prod * iters, iters, n_prod


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, sys_, rank, wname):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(sys_)
    vals = []
    for _ in range(args.steps):
        per_prod, per_solve, iters, n_prod = oracle_sample(sys_)
        vals.append(per_solve)
    v = float(np.mean(vals))
    sample = (f"one dense FP64 {sys_.n}x{sys_.n} product X0*X0 per step (numpy, threaded BLAS), "
              f"scaled by {n_prod} products/iteration x {iters} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "higher_is_better": False,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "atoms": sys_.n_atoms, "N": sys_.n, "b": sys_.b, "tau": args.tau,
                       "directions": len(sys_.h1)},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def to_device(sys_, torch, dev):
    class M:
        pass

    def conv(m):
        o = M()
        o.nb, o.b, o.n = m.nb, m.b, m.n
        o.row_ptr = torch.from_numpy(m.row_ptr).to(dev)
        o.col_idx = torch.from_numpy(m.col_idx).to(dev)
        o.vals = torch.from_numpy(m.vals).to(dev)
        return o

    class S:
        pass

    s = S()
    s.h0 = conv(sys_.h0)
    s.h1 = [conv(m) for m in sys_.h1]
    s.dirs = sys_.dirs
    s.n_electrons = sys_.n_electrons
    return s


def pinned_system(sys_, torch):
    """The system with its matrices copied into pinned host memory (numpy
    views of pinned torch tensors)."""
    class M:
        pass

    def conv(m):
        o = M()
        o.nb, o.b, o.n = m.nb, m.b, m.n
        o.row_ptr = torch.from_numpy(np.ascontiguousarray(m.row_ptr)).pin_memory().numpy()
        o.col_idx = torch.from_numpy(np.ascontiguousarray(m.col_idx)).pin_memory().numpy()
        o.vals = torch.from_numpy(np.ascontiguousarray(m.vals)).pin_memory().numpy()
        return o

    class S:
        pass

    s = S()
    s.h0 = conv(sys_.h0)
    s.h1 = [conv(m) for m in sys_.h1]
    s.dirs = sys_.dirs
    s.n_electrons = sys_.n_electrons
    return s


def job_seconds_per_solve(t_local, steps, world, dist, torch, device):
    """Whole-job time per solve: the slowest rank's timed region (every rank
    solves its own replica of the workload, `steps` times) divided by the
    solves all ranks completed."""
    t = t_local
    if dist is not None:
        x = torch.tensor([t_local], device=device, dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t / (steps * world)


def alphas(sol, nsys):
    return np.stack([sol.alpha(k) for k in range(nsys)])


def run_ours(args, systems, wname, rank, world, torch, dist):
    from paper_2009_03551_gb300 import rdm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    nsys = len(systems)
    sys_ = systems[0]
    dsys = [to_device(s, torch, dev) for s in systems]
    torch.cuda.synchronize()

    sol = rdm.Solver(dev.index, stream.cuda_stream)
    params = dict(tau=args.tau, tau_refine=args.tau_refine, tol=1e-9, mode=args.mode, max_iter=100)
    tau64 = args.tau_refine if args.tau_refine > 0 else args.tau
    sol.set_params(**params)
    sol.load(dsys)
    for _ in range(args.warmup):
        sol.solve()

    def barrier():
        if dist is not None:
            dist.barrier()

    clk = ClockSampler(dev.index)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = []
    for _ in range(args.steps):
        code, info = sol.solve()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    s_per_solve = job_seconds_per_solve(ms / 1e3, args.steps, world, dist, torch, dev)
    alpha_m = alphas(sol, nsys)
    last = infos[-1]
    useful = float(np.mean([i.useful_flops for i in infos]))
    kms = [float(np.mean([i.kernel_ms[k] for i in infos])) for k in range(7)]
    kfl = [float(np.mean([i.kernel_flops[k] for i in infos])) for k in range(4)]
    launches = int(sum(i.kernel_launches for i in infos))
    sinfo = [sol.info(k) for k in range(nsys)]
    sol.close()   # frees the device buffers before the comparison solves

    # FP64 comparison solve (context for the metric's "FP64 vs mixed")
    fp64 = None
    if not args.no_fp64 and args.mode != "fp64":
        s64 = rdm.Solver(dev.index, stream.cuda_stream)
        s64.set_params(tau=tau64, tol=1e-9, mode="fp64", max_iter=100)
        s64.load(dsys)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        _, i64 = s64.solve()
        a1.record(stream)
        torch.cuda.synchronize()
        t64 = a0.elapsed_time(a1) / 1e3
        alpha64 = alphas(s64, nsys)
        # largest relative alpha error over the systems (each normalised by its own max |alpha|)
        rel = float(max(np.max(np.abs(alpha_m[k] - alpha64[k])) / np.max(np.abs(alpha64[k]))
                        for k in range(nsys)))
        fp64 = {"s_per_solve": t64, "steps": 1, "warmup": 0, "iterations": i64.iterations,
                "tflops": i64.useful_flops / t64 / 1e12, "alpha_rel_diff_mixed_vs_fp64": rel,
                "speedup_mixed_vs_fp64": t64 / s_per_solve}
        s64.close()

    # end to end through the public API with host buffers: the inputs and the
    # P1 outputs live in pinned host memory, allocated once before the timed
    # region (as an application that solves repeatedly would keep them)
    e2e = None
    if args.e2e_steps > 0:
        h2d = sum(m.row_ptr.nbytes + m.col_idx.nbytes + m.vals.nbytes for s in systems for m in [s.h0, *s.h1])
        hsys = [pinned_system(s, torch) for s in systems]
        se = rdm.Solver(dev.index, stream.cuda_stream)
        se.set_params(**params)
        se.load(hsys)
        se.solve()   # warm-up of the host path
        torch.cuda.synchronize()
        outs = {}
        for k in range(nsys):
            for d in range(len(systems[k].h1)):
                cap = rdm.rdm_get_p1_nnzb(se.h, k, d) * 11 // 10 + 16
                nb, b = systems[k].h0.nb, systems[k].h0.b
                outs[k, d] = (torch.empty(nb + 1, dtype=torch.int32, pin_memory=True).numpy(),
                              torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy(),
                              torch.empty(cap * b * b, dtype=torch.float64, pin_memory=True).numpy())
        d2h = 0
        t = time.perf_counter()
        for _ in range(args.e2e_steps):
            se.load(hsys)
            se.solve()
            d2h = 0
            for k in range(nsys):
                d2h += 72
                for d in range(len(systems[k].h1)):
                    p = se.p1(k, d, out=outs[k, d])
                    d2h += p.row_ptr.nbytes + p.col_idx.nbytes + p.vals.nbytes
                _ = se.alpha(k)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t) / args.e2e_steps
        e2e = {"value": te, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        se.close()

    peaks, peak_kind = load_peaks()
    mode = args.mode
    # dominant kernel of the solve (by device time) among the product kernels:
    # tensor-core split products, FP64, FP32 and double-FP32 CUDA-core products
    tc_ms, f64_ms, f32_ms, ff_ms = kms[1], kms[2], kms[3], kms[6]
    classes = {
        "tc": ("k_tc_bf16x3 (tcgen05 split-precision block SpGEMM + fused truncation)", tc_ms, kfl[0],
               peaks["bf16_tflops"] * 1e12 / 3.0, "tensor",
               f"measured bf16 dense burst / 3 (a split product issues 3 MMAs per useful product; {peak_kind}, "
               "MEASURED_PEAKS.json bf16_tflops; fp16 has the same nominal rate)"),
        "fp64": ("k_numeric_simt<32,double> (FP64 block SpGEMM + fused truncation)", f64_ms, kfl[1], 1.26e12,
                 "alu", FP64_PEAK_NOTE + " (derived from unit counts and clock)"),
        "fp32": ("k_numeric_f32_b32 (FP32 block SpGEMM + fused truncation)", f32_ms, kfl[2], 80.5e12, "alu",
                 FP32_PEAK_NOTE + " (derived from unit counts and clock)"),
        "ff": ("k_numeric_f32_b32<double-FP32> (error-free FP32 block SpGEMM + fused truncation)", ff_ms, kfl[3],
               80.5e12 / 12.0, "alu", FP32_PEAK_NOTE + "; 12 FP32-pipe operations per multiply-add "
               "(2 useful flops) -> 6.7 TFLOP/s (derived from unit counts and clock)"),
    }
    dom = max(classes, key=lambda k: classes[k][1])
    kname, k_ms, k_fl, peak, bound, peak_note = classes[dom]
    achieved = k_fl / (k_ms / 1e3) if k_ms > 0 else 0.0
    roofline = {"kernel": kname, "bound": bound, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                "traffic": profiled_traffic(dom, wname),
                "ms_per_solve": k_ms, "peak_source": peak_note, "share_of_solve": k_ms / (s_per_solve * 1e3),
                "per_class": {k: {"ms": v[1], "tflops": (v[2] / (v[1] / 1e3) / 1e12) if v[1] > 0 else None,
                                  "frac": ((v[2] / (v[1] / 1e3)) / v[3]) if v[1] > 0 else None}
                              for k, v in classes.items() if v[2] > 0}}
    num_ms = tc_ms + f64_ms + f32_ms + ff_ms
    achieved_all = useful / (num_ms / 1e3) if num_ms > 0 else 0.0

    line = {"metric": METRIC, "value": s_per_solve, "unit": "s", "higher_is_better": False,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_per_solve * 1e3,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "mixed_bf16": "bf16x3+f64",
                                                                "mixed_fp16": "fp16x3+f64"}[mode],
            "data": "synthetic",
            "config": {"workload": wname, "mode": mode, "systems": nsys,
                       "atoms": int(sum(s.n_atoms for s in systems)), "N": int(sum(s.n for s in systems)),
                       "b": sys_.b, "tau": args.tau, "tau_refine": tau64, "tol": 1e-9, "directions": 3,
                       "iterations": int(max(i.iterations for i in sinfo)),
                       "nnzb_p0": int(sum(i.nnzb_p0 for i in sinfo)),
                       "nnzb_p1": [int(sum(i.nnzb_p1[d] for i in sinfo)) for d in range(3)],
                       "nnzb_per_block_row_p0": float(sum(i.nnzb_p0 for i in sinfo) /
                                                      sum(s.h0.nb for s in systems)),
                       "l2": "working set >> L2 (no flush needed)", "parallelism": f"replicas{world}"},
            "tflops": useful / s_per_solve / 1e12 * 1.0 if world == 1 else None,
            "block_spgemm_tflops": achieved_all / 1e12,
            "alpha_diag": [float(alpha_m[0][k, k]) for k in range(3)],
            "roofline": roofline, "fp64": fp64, "e2e": e2e, "gpu_launches": launches,
            "kernel_ms_per_solve": {"symbolic_pairs_tiles": kms[0], "tensor_core_products": kms[1],
                                    "fp64_products": kms[2], "fp32_products": kms[3], "compaction": kms[4],
                                    "reductions_setup_host": kms[5], "double_fp32_products": kms[6]},
            "tier_iterations": list(last.tier_iters)[:3],
            "device_gb_peak": last.device_bytes_peak / 1e9, "product_groups": int(last.product_groups),
            "clocks": clocks}
    return line


def make_workload(args):
    """(name, list of systems) of the requested workload."""
    from synth import make_batch_config, make_config
    w = args.workload
    def e(x):
        m, ex = f"{x:.0e}".split("e")
        return f"{m}e{int(ex)}"
    ts = f"tau{e(args.tau)}" + (f"-refine{e(args.tau_refine)}" if args.tau_refine > 0 else "")
    if w == "cluster":
        cfg = 2 if args.atoms <= 2000 else 3
        s = make_config(cfg, n_atoms=args.atoms)
        name = f"cluster-{args.atoms}-atoms-N{s.n}-b32-{ts}-xyz"
        return name, [s]
    if w == "batch24":
        return f"batch-24-systems-300-8000-atoms-b32-{ts}-xyz", make_batch_config(24, b=32)
    if w.startswith("slab"):
        n = int(w[4:])
        return f"slab-{n}-atoms-30bohr-b32-{ts}-xyz", [make_config(5, n_atoms=n)]
    raise SystemExit(f"unknown workload {w}")


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    wname, systems = make_workload(args)
    sys_ = systems[0]

    if args.impl == "reference":
        run_reference(args, sys_, rank, wname)
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    from paper_2009_03551_gb300 import build as b
    if rank == 0 or world == 1:
        b.build()
    if dist is not None:
        dist.barrier()
    line = run_ours(args, systems, wname, rank, world, torch, dist)
    if rank == 0 and world == 1 and not args.no_cpu and len(systems) == 1 and sys_.n <= 16000:
        per_prod, per_solve, iters, n_prod = oracle_sample(sys_)
        line["cpu_baseline"] = {"value": per_solve, "unit": "s", "cores": cores(), "kind": "oracle",
                                "sample": f"one dense FP64 {sys_.n}x{sys_.n} product of the oracle's TC2 "
                                          f"({per_prod:.2f} s), scaled by {n_prod} products x {iters} iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
