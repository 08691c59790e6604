"""Benchmark of the response-density-matrix solve on one or more GB300s.

One step = one full solve (Gershgorin bounds, initial matrices, every TC2 /
first-order iteration with its block-sparse products and truncation, the
polarizability) of the default workload: a batch of 24 independent systems of
uneven size (300-8,000 atoms each, 84,131 atoms in all, 8 orbitals per atom,
chains and random-packed clusters, 32 x 32 blocks, truncation 1e-6, H1 for x,
y and z), solved together as one block-diagonal problem in the mixed
fp16 / FP64 ladder.  Inputs are resident in HBM before the timed region; the
working set (hundreds of GB) is far larger than L2, so no flush is needed.
The plain FP64 GPU solve of the same workload runs once beside it, and
|dalpha|/alpha is measured between the two.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode M] [--workload W] [--impl ours|reference]

Prints ONE JSON line (rank 0).  Under torchrun a batch is partitioned: every
rank solves the systems that a greedy work estimate assigns to it (no
collective on the data path; the polarizabilities are gathered afterwards),
so the job's total work is fixed (strong scaling); a single-system workload
runs one replica per rank (weak scaling).  ``--impl reference`` times the CPU
oracle (dense FP64 TC2, oracle B) end to end on a bounded sample of the
workload: a carve-out of one of its clusters.
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
FP64_PEAK_NOTE = ("GB300 FP64: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz = 1.26 TFLOP/s "
                  "(nominal 1.25 TFLOP/s)")
FP32_PEAK_NOTE = "GB300 FP32: 152 SMs x 128 FMA/clk/SM x 2 flop x 2.07 GHz = 80.5 TFLOP/s"
DENSE_MAX_N = 16000       # largest system the dense CPU oracle may be given (N x N FP64: 2 GB)
SAMPLE_ATOMS = 250        # atoms of the carve-out the CPU oracle solves (N = 2,000)
SLICE_PAIRS = 28          # bf16 slice pairs one FP64-class slice product issues per useful product
# MMA work of one K-step of the tensor-core kernel at block size b: 3 products of 128 x 256 x b
def tc_flops_per_kstep(b):
    return 3 * 2 * 128 * 256 * b


# DRAM traffic of the product kernels, from one ncu capture each (profiles/):
# dram__bytes_read.sum + dram__bytes_write.sum per launch, divided by the work
# units of that launch (K-steps for the tensor-core kernel, block triples for
# the CUDA-core kernels), so that a capture on a small case scales to the
# launches of the bench workload by the units they process.  A figure is
# reported only while the code of the kernel's source file is unchanged since
# the capture (SHA-256 of the file with comments and whitespace removed).
PROFILED_TRAFFIC = {
    "tc": {"file": ["paper_2009_03551_gb300/csrc/k_tc.cu", "paper_2009_03551_gb300/csrc/tc_ptx.cuh",
                    "paper_2009_03551_gb300/csrc/tc_plan.cuh"],
           "sha256": "db478c16abca005fcca1f40d0b5bf63327422468ad2a3836d58b99a077079b46",
           "bytes_per_unit": 15071.0, "unit": "K-step", "b": 32,
           "capture": "profiles/k_tc_bf16x3_dram_cluster1000.md"},
    "ff": {"file": "paper_2009_03551_gb300/csrc/k_numeric.cu",
           "sha256": "1c9d3e76e36659e5d06b0d237474522761ebecc2732c37eb20f037dc4adcb12e",
           "bytes_per_unit": None, "unit": "block triple"},
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
    ap.add_argument("--workload", default="batch24",
                    help="batch24 (default: 24 uneven chains/clusters, 300-8,000 atoms, 84,131 in all), "
                         "cluster (the 2,000-atom cluster, or --atoms), slab<N> (30-bohr slab of N atoms)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--tau", type=float, default=1e-6, help="block truncation threshold")
    ap.add_argument("--tau-refine", type=float, default=-1.0,
                    help="threshold of the final (FP64/FP32) tier of the mixed modes (< 0: --tau); the "
                         "FP64 comparison solve runs at this threshold throughout")
    ap.add_argument("--split-directions", type=int, default=0,
                    help="1: solve the field directions one after another (about half the device memory)")
    ap.add_argument("--correct", type=int, default=0,
                    help="1: correct P0 and P1 for the residuals of their defining conditions after the solve "
                         "(two more solves of the same mode)")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1 (default): the library picks the block size of the products in {16, 32, 64} by timed "
                         "probe solves during the warm-up; 0: the uploaded 32 x 32 blocks")
    ap.add_argument("--block-size", type=int, default=0, help="block size of the products (0: uploaded; "
                                                                "ignored with --autotune 1)")
    ap.add_argument("--refine-x0", type=int, default=0,
                    help="final-tier arithmetic of X0^2 (rdm.h RDM_REFINE_*: 0 default, 1 FP64, 3 FP32, "
                         "4 double-FP32, 5 tensor-core slice products)")
    ap.add_argument("--sweep", default="",
                    help="tau or tol: instead of the timed solve, sweep the truncation threshold (or the "
                         "band-energy tolerance) on --workload and print one JSON line per point")
    return ap.parse_args()


def profiled_traffic(cls, units_per_launch, b=32):
    """DRAM bytes per launch of the class's kernel, scaled from the committed
    capture by the units the launch processes; None if there is no capture of
    the current code at this block size."""
    rec = PROFILED_TRAFFIC.get(cls)
    if rec is None or rec["bytes_per_unit"] is None or not units_per_launch or rec.get("b", 32) != b:
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    files = rec["file"] if isinstance(rec["file"], list) else [rec["file"]]
    try:
        sha = code_digest("".join(open(os.path.join(root, f), encoding="utf-8").read() for f in files))
    except OSError:
        return None
    return rec["bytes_per_unit"] * units_per_launch if sha == rec["sha256"] else None


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

def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def dense(m):
    """Dense copy of a BSR matrix for the CPU oracle; refuses systems whose
    dense form would not fit comfortably in host memory."""
    if m.n > DENSE_MAX_N:
        raise ValueError(f"dense oracle refused: N = {m.n} > {DENSE_MAX_N}")
    return m.to_dense()


def oracle_sample_system(systems):
    """The bounded sample the CPU oracle solves: the SAMPLE_ATOMS atoms nearest
    the centre of the smallest cluster of the workload (of its first system if
    it has no cluster), with the same matrix elements (synth.carve_sphere)."""
    from synth import carve_sphere
    clusters = [k for k, s in enumerate(systems) if s.kind != "chain"] or [0]
    k = min(clusters, key=lambda i: systems[i].n_atoms)
    parent = systems[k]
    n_keep = min(SAMPLE_ATOMS, parent.n_atoms)
    s = carve_sphere(parent, n_keep) if n_keep < parent.n_atoms else parent
    desc = (f"oracle B (dense FP64 TC2 with the first-order recursion for x, y, z, block truncation, band-energy "
            f"stop) solved end to end on the {n_keep} atoms nearest the centre of system {k} of the workload "
            f"({parent.kind}, {parent.n_atoms} atoms): N = {s.n}, b = {s.b}")
    return s, k, desc


def timed_oracle_solve(sample, tau, tol=1e-9):
    """Wall time of one full oracle-B solve of the sample (dense FP64, numpy
    with the host's threaded BLAS), and its iteration count."""
    from oracle import tc2_response
    h0 = dense(sample.h0)
    h1s = [dense(m) for m in sample.h1]
    t = time.perf_counter()
    r = tc2_response(h0, h1s, sample.n_occ, sample.b, tau=tau, tol=tol, max_iter=100)
    return time.perf_counter() - t, r.iterations


def dense_cost_model(t_sample, sample, systems):
    """Context only: the sample's time scaled to the whole workload by the
    dense oracle's N^3 cost (iteration counts assumed equal)."""
    return t_sample * sum((s.n / sample.n) ** 3 for s in systems)


def run_reference(args, systems, rank, wname):
    if rank != 0:
        return
    sample, k, desc = oracle_sample_system(systems)
    for _ in range(args.warmup):
        timed_oracle_solve(sample, args.tau)
    vals, iters = [], 0
    for _ in range(args.steps):
        t, iters = timed_oracle_solve(sample, args.tau)
        vals.append(t)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "higher_is_better": False,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "systems": len(systems),
                       "atoms": int(sum(s.n_atoms for s in systems)), "b": systems[0].b, "tau": args.tau,
                       "directions": len(systems[0].h1),
                       "sample": {"system": k, "atoms": sample.n_atoms, "N": sample.n, "iterations": iters}},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores(), "kind": "oracle",
                             "sample": desc + f"; one such solve per step ({iters} iterations)"},
            "scaled_to_workload": {"kind": "model", "value": dense_cost_model(v, sample, systems), "unit": "s",
                                   "basis": "the timed sample scaled by the dense N^3 cost to every system of "
                                            "the workload (not measured)"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# partition of a batch over ranks
# ---------------------------------------------------------------------------

def work_estimate(s):
    """Cost proxy of one system's solve: the block triples of H0 H0
    (sum over block rows of the squared blocks per row)."""
    rp = np.asarray(s.h0.row_ptr, dtype=np.int64)
    k = np.diff(rp)
    return float(np.sum(k * k))


def partition(works, world):
    """Greedy longest-processing-time partition: systems in decreasing order
    of work, each to the rank with the least work so far (ties: lowest rank).
    Returns, per rank, the sorted indices of its systems."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(works)), key=lambda i: (-works[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += works[i]
    return [sorted(x) for x in out]


def gather_results(local, world, dist):
    """{system index: result} of every rank, merged (all ranks get the merge)."""
    if dist is None or world == 1:
        return dict(local)
    parts = [None] * world
    dist.all_gather_object(parts, dict(local))
    merged = {}
    for p in parts:
        merged.update(p)
    return merged


def job_seconds_per_solve(t_local, steps, world, dist, torch, device, replicas=True):
    """Whole-job time per solve: the slowest rank's timed region divided by
    the solves of the whole workload that all ranks completed (with replicas
    every rank completes `steps` solves; with a partition the ranks together
    complete `steps` solves of the one workload)."""
    t = t_local
    if dist is not None:
        x = torch.tensor([t_local], device=device, dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return t / (steps * (world if replicas else 1))


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _copy_system(sys_, conv):
    class S:
        pass

    s = S()
    s.h0 = conv(sys_.h0)
    s.h1 = [conv(m) for m in sys_.h1]
    s.dirs = sys_.dirs
    s.n_electrons = sys_.n_electrons
    return s


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

    return _copy_system(sys_, conv)


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

    return _copy_system(sys_, conv)


def alphas(sol, nsys):
    return np.stack([sol.alpha(k) for k in range(nsys)])


def rel_alpha_diff(a, b):
    """Largest |a - b| over the 3 x 3 tensor, relative to max |b|, worst over systems."""
    return float(max(np.max(np.abs(a[k] - b[k])) / np.max(np.abs(b[k])) for k in range(len(b))))


def run_ours(args, systems, wname, rank, world, torch, dist):
    from paper_2009_03551_gb300 import rdm

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    # a batch is partitioned over the ranks; a single system is replicated
    replicas = len(systems) == 1 or world == 1
    if replicas:
        mine = list(range(len(systems)))
    else:
        mine = partition([work_estimate(s) for s in systems], world)[rank]
    local = [systems[k] for k in mine]
    nsys = len(local)
    sys_ = systems[0]
    dsys = [to_device(s, torch, dev) for s in local]
    torch.cuda.synchronize()

    sol = rdm.Solver(dev.index, stream.cuda_stream)
    params = dict(tau=args.tau, tau_refine=args.tau_refine, tol=1e-9, mode=args.mode, max_iter=100,
                  autotune=args.autotune, block_size=args.block_size, refine_x0=args.refine_x0,
                  split_directions=args.split_directions, correct=args.correct)
    tau64 = args.tau_refine if args.tau_refine > 0 else args.tau
    sol.set_params(**params)
    if nsys:
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
    for _ in range(args.steps if nsys else 0):
        code, info = sol.solve()
        infos.append(info)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    s_per_solve = job_seconds_per_solve(ms / 1e3, args.steps, world, dist, torch, dev, replicas)
    alpha_m = alphas(sol, nsys) if nsys else np.zeros((0, 3, 3))
    infos = infos or [rdm.rdm_info()]
    last = infos[-1]
    useful = float(np.mean([i.useful_flops for i in infos]))
    issued = float(np.mean([i.issued_flops for i in infos]))
    kms = [float(np.mean([i.kernel_ms[k] for i in infos])) for k in range(8)]
    kfl = [float(np.mean([i.kernel_flops[k] for i in infos])) for k in range(5)]
    tc_launches = float(np.mean([i.tc_launches for i in infos]))
    launches = int(sum(i.kernel_launches for i in infos))
    sinfo = [sol.info(k) for k in range(nsys)]
    sol.close()   # frees the device buffers before the comparison solves

    # FP64 comparison solve (context for the metric's "FP64 vs mixed")
    fp64 = None
    if not args.no_fp64 and args.mode != "fp64":
        t64, it64, fl64 = 0.0, 0, 0.0
        alpha64 = np.zeros((0, 3, 3))
        if nsys:
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
            it64, fl64 = i64.iterations, i64.useful_flops
            alpha64 = alphas(s64, nsys)
            s64.close()
        t64 = job_seconds_per_solve(t64, 1, world, dist, torch, dev, replicas=False)
        a_m = gather_results({k: alpha_m[q] for q, k in enumerate(mine)}, world, dist)
        a_64 = gather_results({k: alpha64[q] for q, k in enumerate(mine)}, world, dist)
        ks = sorted(a_64)
        fp64 = {"s_per_solve": t64, "steps": 1, "warmup": 0, "iterations": it64,
                "tflops": fl64 / t64 / 1e12 if t64 > 0 and world == 1 else None,
                "alpha_rel_diff_mixed_vs_fp64": rel_alpha_diff([a_m[k] for k in ks], [a_64[k] for k in ks]),
                "speedup_mixed_vs_fp64": t64 / s_per_solve}

    # end to end through the public API with host buffers: the inputs and the
    # P1 outputs live in pinned host memory, allocated once before the timed
    # region (as an application that solves repeatedly would keep them)
    e2e = None
    if args.e2e_steps > 0:
        h2d = sum(m.row_ptr.nbytes + m.col_idx.nbytes + m.vals.nbytes for s in local for m in [s.h0, *s.h1])
        hsys = [pinned_system(s, torch) for s in local]
        se = rdm.Solver(dev.index, stream.cuda_stream)
        se.set_params(**params)
        outs = {}
        if nsys:
            se.load(hsys)
            se.solve()   # warm-up of the host path
            torch.cuda.synchronize()
            for k in range(nsys):
                for d in range(len(local[k].h1)):
                    cap = rdm.rdm_get_p1_nnzb(se.h, k, d) * 11 // 10 + 16
                    nb, b = local[k].h0.nb, local[k].h0.b
                    outs[k, d] = (torch.empty(nb + 1, dtype=torch.int32, pin_memory=True).numpy(),
                                  torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy(),
                                  torch.empty(cap * b * b, dtype=torch.float64, pin_memory=True).numpy())
        barrier()
        d2h = 0
        t = time.perf_counter()
        for _ in range(args.e2e_steps if nsys else 0):
            se.load(hsys)
            se.solve()
            d2h = 0
            for k in range(nsys):
                d2h += 72
                for d in range(len(local[k].h1)):
                    p = se.p1(k, d, out=outs[k, d])
                    d2h += p.row_ptr.nbytes + p.col_idx.nbytes + p.vals.nbytes
                _ = se.alpha(k)
        torch.cuda.synchronize()
        te = job_seconds_per_solve((time.perf_counter() - t), args.e2e_steps, world, dist, torch, dev, replicas)
        if dist is not None:
            x = torch.tensor([float(h2d), float(d2h)], device=dev, dtype=torch.float64)
            dist.all_reduce(x)
            h2d, d2h = x.tolist()
            if replicas:
                h2d, d2h = h2d / world, d2h / world
        e2e = {"value": te, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        se.close()

    peaks, peak_kind = load_peaks()
    mode = args.mode
    # dominant kernel of the solve (by device time) among the product kernels:
    # tensor-core split products, FP64, FP32 and double-FP32 CUDA-core products
    tc_ms, f64_ms, f32_ms, ff_ms, oz_ms = kms[1], kms[2], kms[3], kms[6], kms[7]
    issued_tc = max(0.0, issued - (kfl[1] + kfl[2] + kfl[3]) - kfl[4] * SLICE_PAIRS)
    bsz = int(last.block_size) or sys_.b
    ksteps_per_launch = issued_tc / tc_flops_per_kstep(bsz) / tc_launches if tc_launches else 0.0
    classes = {
        "tc": ("k_tc_bf16x3 (tcgen05 split-precision block SpGEMM + fused truncation)", tc_ms, kfl[0],
               peaks["bf16_tflops"] * 1e12 / 3.0, "tensor",
               f"measured bf16 dense burst / 3 (a split product issues 3 MMAs per useful product; {peak_kind}, "
               "MEASURED_PEAKS.json bf16_tflops; fp16 has the same nominal rate)"),
        "fp64": ("k_numeric_simt<32,double> (FP64 block SpGEMM + fused truncation)", f64_ms, kfl[1], 1.26e12,
                 "alu", FP64_PEAK_NOTE + " (derived from unit counts and clock)"),
        "fp32": ("k_numeric_f32_t84 (FP32 block SpGEMM + fused truncation)", f32_ms, kfl[2], 80.5e12, "alu",
                 FP32_PEAK_NOTE + " (derived from unit counts and clock)"),
        "ff": ("k_numeric_ff_b32 (double-FP32 block SpGEMM, error-free transformations, + fused truncation)", ff_ms, kfl[3],
               80.5e12 / 12.0, "alu", FP32_PEAK_NOTE + "; 12 FP32-pipe operations per multiply-add "
               "(2 useful flops) -> 6.7 TFLOP/s (derived from unit counts and clock)"),
        "oz": ("k_tc_oz (tcgen05 exact bf16 slice products, FP64-class, + fused truncation)", oz_ms, kfl[4],
               peaks["bf16_tflops"] * 1e12 / SLICE_PAIRS, "tensor",
               f"measured bf16 dense burst / {SLICE_PAIRS} (28 slice-pair MMAs per useful product; {peak_kind}, "
               "MEASURED_PEAKS.json bf16_tflops)"),
    }
    dom = max(classes, key=lambda k: classes[k][1])
    kname, k_ms, k_fl, peak, bound, peak_note = classes[dom]
    achieved = k_fl / (k_ms / 1e3) if k_ms > 0 else 0.0
    traffic = profiled_traffic("tc", ksteps_per_launch, bsz) if dom == "tc" else None
    roofline = {"kernel": kname, "bound": bound, "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak if peak else None, "traffic": traffic,
                "ms_per_solve": k_ms, "peak_source": peak_note, "share_of_solve": k_ms / (s_per_solve * 1e3),
                "launches_per_solve": tc_launches if dom == "tc" else None,
                "ksteps_per_launch": ksteps_per_launch if dom == "tc" else None,
                "per_class": {k: {"ms": v[1], "tflops": (v[2] / (v[1] / 1e3) / 1e12) if v[1] > 0 else None,
                                  "frac": ((v[2] / (v[1] / 1e3)) / v[3]) if v[1] > 0 else None}
                              for k, v in classes.items() if v[2] > 0}}
    num_ms = tc_ms + f64_ms + f32_ms + ff_ms + oz_ms
    achieved_all = useful / (num_ms / 1e3) if num_ms > 0 else 0.0

    line = {"metric": METRIC, "value": s_per_solve, "unit": "s", "higher_is_better": False,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_per_solve * 1e3,
            "scaling": "weak" if replicas else "strong", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "mixed_bf16": "bf16x3+f64", "mixed_fp16": "fp16x3+f64"}[mode],
            "data": "synthetic",
            "config": {"workload": wname, "mode": mode, "systems": len(systems),
                       "atoms": int(sum(s.n_atoms for s in systems)), "N": int(sum(s.n for s in systems)),
                       "b": sys_.b, "tau": args.tau, "tau_refine": tau64, "tol": 1e-9, "directions": 3,
                       "split_directions": int(args.split_directions), "correct": int(args.correct),
                       "iterations": int(max([i.iterations for i in sinfo], default=0)),
                       "nnzb_p0": int(sum(i.nnzb_p0 for i in sinfo)),
                       "nnzb_p1": [int(sum(i.nnzb_p1[d] for i in sinfo)) for d in range(3)],
                       "nnzb_per_block_row_p0": float(sum(i.nnzb_p0 for i in sinfo) /
                                                      max(1, sum(s.h0.nb for s in local))),
                       "l2": "working set >> L2 (no flush needed)",
                       "parallelism": f"replicas{world}" if replicas else f"partition{world}",
                       "systems_on_rank0": mine if rank == 0 else None},
            "tflops": useful / s_per_solve / 1e12 if world == 1 else None,
            "block_spgemm_tflops": achieved_all / 1e12,
            "alpha_diag": [float(alpha_m[0][k, k]) for k in range(3)] if nsys else None,
            "roofline": roofline, "fp64": fp64, "e2e": e2e, "gpu_launches": launches,
            "kernel_ms_per_solve": {"symbolic_pairs_tiles": kms[0], "tensor_core_products": kms[1],
                                    "fp64_products": kms[2], "fp32_products": kms[3], "compaction": kms[4],
                                    "reductions_setup_host": kms[5], "double_fp32_products": kms[6],
                                    "slice_products": kms[7]},
            "block_size": {"products": int(last.block_size), "uploaded": sys_.b,
                           "autotune": {"on": bool(args.autotune), "probe_ms_b16_b32_b64": list(last.probe_ms),
                                        "probe_total_ms": last.autotune_ms} if args.autotune else None},
            "tier_iterations": list(last.tier_iters)[:3],
            "device_gb_peak": last.device_bytes_peak / 1e9, "product_groups": int(last.product_groups),
            "clocks": clocks}
    return line


def gpu_sample_seconds(args, sample, torch, reps=3):
    """Device time of one solve of the oracle's sample alone, in the bench's
    mode (the like-for-like partner of cpu_baseline)."""
    from paper_2009_03551_gb300 import rdm
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.current_stream(dev)
    sol = rdm.Solver(dev.index, stream.cuda_stream)
    sol.set_params(tau=args.tau, tau_refine=args.tau_refine, tol=1e-9, mode=args.mode, max_iter=100)
    sol.load([to_device(sample, torch, dev)])
    sol.solve()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sol.solve()
    e1.record(stream)
    torch.cuda.synchronize()
    sol.close()
    return e0.elapsed_time(e1) / 1e3 / reps


def sweep(args, systems, wname, torch):
    """Threshold (or tolerance) study on one GPU: for every point, the mixed
    and the FP64 solve of the workload, their times and |dalpha|/alpha against
    the exact sum-over-states alpha when the workload is small enough for the
    dense oracle (else against the FP64 solve at the smallest threshold)."""
    from paper_2009_03551_gb300 import rdm
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    dsys = [to_device(s, torch, dev) for s in systems]
    exact = None
    if all(s.n <= 8000 for s in systems):
        from oracle import exact_response, polarizability
        exact = []
        for s in systems:
            h0 = dense(s.h0)
            h1s = [dense(m) for m in s.h1]
            _, p1s, _, _ = exact_response(h0, h1s, s.n_occ)
            exact.append(polarizability(p1s, h1s))
    pts = [1e-4, 1e-5, 1e-6, 1e-7, 1e-8] if args.sweep == "tau" else [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-9]
    rows = []
    for x in pts:
        for mode in (args.mode, "fp64"):
            tau, tol = (x, 1e-9) if args.sweep == "tau" else (args.tau, x)
            sol = rdm.Solver(dev.index, stream.cuda_stream)
            sol.set_params(tau=tau, tol=tol, mode=mode, max_iter=100)
            sol.load(dsys)
            sol.solve()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            code, info = sol.solve()
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            a = alphas(sol, len(systems))
            infos = [sol.info(k) for k in range(len(systems))]
            sol.close()
            rows.append({"sweep": args.sweep, "value": x, "mode": mode, "tau": tau, "tol": tol, "s_per_solve": t,
                         "iterations": int(max(i.iterations for i in infos)),
                         "nnzb_per_block_row_p0": float(sum(i.nnzb_p0 for i in infos) /
                                                        sum(s.h0.nb for s in systems)),
                         "tflops": info.useful_flops / t / 1e12, "alpha": a})
    # without the exact alpha: the FP64 solve at the last (tightest) point
    ref = exact if exact is not None else [r for r in rows if r["mode"] == "fp64"][-1]["alpha"]
    for r in rows:
        r["alpha_rel_err"] = rel_alpha_diff(r.pop("alpha"), ref)
        r["alpha_ref"] = "exact (sum over states, oracle A)" if exact is not None else "FP64 GPU solve"
        r["workload"] = wname
        print(json.dumps(r), flush=True)


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
    if args.impl == "reference" and rank != 0:
        return    # the CPU oracle runs on rank 0 alone
    wname, systems = make_workload(args)

    if args.impl == "reference":
        run_reference(args, systems, rank, wname)
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
    if args.sweep:
        if rank == 0:
            sweep(args, systems, wname, torch)
        if dist is not None:
            dist.destroy_process_group()
        return
    line = run_ours(args, systems, wname, rank, world, torch, dist)
    if rank == 0 and world == 1 and not args.no_cpu:
        sample, k, desc = oracle_sample_system(systems)
        t_cpu, iters = timed_oracle_solve(sample, args.tau)
        line["cpu_baseline"] = {"value": t_cpu, "unit": "s", "cores": cores(), "kind": "oracle",
                                "sample": desc + f" ({iters} iterations), timed once",
                                "gpu_same_sample_s": gpu_sample_seconds(args, sample, torch),
                                "scaled_to_workload": {"kind": "model",
                                                       "value": dense_cost_model(t_cpu, sample, systems),
                                                       "basis": "the timed sample scaled by the dense N^3 cost "
                                                                "to every system of the workload (not measured)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
