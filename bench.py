"""Benchmark: gate-pass HBM GB/s vs peak, and emulate-vs-simulate speedups.

Workload (one step; n = 30 qubits, complex128 = 16 GiB, larger than L2):
  |0...0>  ->  depth-20 random circuit (600 Haar U(2) + 300 CNOT), fused into
  blocks of up to max_k qubits  ->  emulated QFT on all 30 qubits (FFT)  ->
  emulated addition of a random constant to the register [0, 16)  ->
  transverse-field Ising energy and the marginal of qubits (0, 1, 2).
The headline runs in the FP64 mode (53-bit arithmetic; dense blocks as exact
products of 56-bit splittings on the tensor cores); the same step in the fast
double-float mode is reported beside it.
value = algorithmic bytes of a step / step time (GB/s).  The algorithmic
bytes count the passes the method needs, whatever the implementation does:
each fused gate block moves 2 * 2^n * 16 bytes (Sec. III-B's byte count), the
QFT ceil(n/11) such passes (radix-2^11 tiles, the bit reversal folded), the
addition one, the Ising energy ceil(n/11) reads of the state (every X_i
needs qubit i inside a tile once) and the marginal one read.  The
emulate-vs-simulate comparison of the configuration (30-qubit QFT on a random
normalised state: one FFT vs 30 H + 435 CR gates; the addition: one
permutation vs a ripple of multi-controlled NOTs) is measured once after the
timed steps and reported with its accuracy.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-pass HBM GB/s vs peak; emulate-vs-simulate speedup at stated fidelity"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--depth", type=int, default=20)
    ap.add_argument("--max-k", type=int, default=0, help="fusion width (0: planner default)")
    ap.add_argument("--arith", default="fp64", choices=["fp64", "df64"],
                    help="complex128 arithmetic of the headline (fp64: 53-bit mode; df64: fast mode)")
    ap.add_argument("--fusion-comparison", action="store_true",
                    help="also time the step with fusion up to 2 qubits")
    ap.add_argument("--quick", action="store_true", help="skip e2e, CPU baseline and the comparison")
    ap.add_argument("--only", default="", choices=["", "batch", "tensor_cores", "config4", "qft", "qpe"],
                    help="run one secondary configuration alone (sizes from --n) and print its JSON")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"], help="state type for --only qft")
    ap.add_argument("--kernel-case", default="", choices=["", *KERNEL_CASES],
                    help="run a few launches of one hot kernel on a small state (the ncu capture cases)")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the nvidia-smi clock samples of the timed region in this file")
    return ap.parse_args()


# small single-kernel workloads for ncu captures: (dtype, n, what)
KERNEL_CASES = {
    "tc128": "complex128 5-qubit block on qubits (3,7,11,15,19) of a 24-qubit state, FP64 mode (7 digits), 3 passes",
    "tc128df": "complex128 5-qubit block on qubits (3,7,11,15,19) of a 24-qubit state, double-float mode (6 digits), "
               "3 passes",
    "tc64": "complex64 5-qubit block on qubits (3,7,11,15,19) of a 26-qubit state, 3 passes",
    "direct2": "complex128 2-qubit block on qubits (5,17) of a 26-qubit state (fusion width 2), 3 passes",
    "expect": "TFIM energy of a 26-qubit complex128 state (fixed-point register rounds), 2 evaluations",
    "fft": "emulated 25-qubit QFT of a complex128 state, FP64 mode (5-qubit digit passes), 2 transforms",
    "fftdf": "emulated 26-qubit QFT of a complex128 state, double-float mode (radix-2 shared-memory passes), "
             "2 transforms",
    "qpegemm": "one squaring of a 2^10 x 2^10 complex128 matrix on the tensor cores (digit splitting + product), "
               "2 products",
    "addc": "emulated add-constant on qubits [0,16) of a 26-qubit complex128 state (1 MiB slices, eight CTAs "
            "each, bulk copies), 2 additions",
    "mul": "emulated multiplication c += a b of 8-qubit registers (index = a b c) of a 26-qubit complex128 "
           "state (planes in shared memory), 2 multiplications",
    "batch": "512 ansatz circuits, n ~ U{10..20}, 8 layers, TFIM energy each, complex128 double-float, "
             "default plan, 2 runs",
}


def run_kernel_case(qe, I, which):
    """A few launches of one hot kernel on a small state (a few hundred MB)."""
    import torch
    rng = np.random.default_rng(0)

    def unitary(d):
        z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        q, r = np.linalg.qr(z)
        return q * (np.diag(r) / abs(np.diag(r)))[None, :]

    df = which.endswith("df")
    if which in ("tc128", "tc128df", "tc64"):
        with qe.State(26 if which == "tc64" else 24, "c64" if which == "tc64" else "c128") as st:
            if df:
                st.set_arith(qe.ARITH_DF64)
            st.set_policy(qe.POLICY_AUTO, 5)
            st.init_random(3)
            U = unitary(32)
            for _ in range(3):
                st.apply_gate([3, 7, 11, 15, 19], U)
                st.flush()
    elif which == "direct2":
        with qe.State(26, "c128") as st:
            st.set_policy(qe.POLICY_AUTO, 2)
            st.init_random(3)
            U = unitary(4)
            for _ in range(3):
                st.apply_gate([5, 17], U)
                st.flush()
    elif which == "addc":
        with qe.State(26, "c128") as st:
            st.set_policy(qe.POLICY_EMULATE, 1)
            st.init_random(2)
            for _ in range(2):
                st.add_const(list(range(16)), 40503)
            st.flush()
    elif which == "mul":
        with qe.State(26, "c128") as st:
            st.set_policy(qe.POLICY_EMULATE, 1)
            st.init_random(2)
            for _ in range(2):
                st.mul(list(range(16, 24)), list(range(8, 16)), list(range(8)))
            st.flush()
    elif which == "batch":
        ns = I.batch_sizes(512, 10, 20, 3)
        angles = [I.ansatz_angles(int(nq), 8, 300000 + i) for i, nq in enumerate(ns)]
        with qe.Batch(ns, angles, 0.7, "c128") as b:
            for _ in range(2):
                b.run()
    elif which == "qpegemm":
        D = 1 << 10
        z = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
        with qe.State(20, "c128") as a, qe.State(20, "c128") as c:
            a.set(np.ascontiguousarray(z).reshape(-1))
            for _ in range(2):
                c.matmul(a, a)
    elif which == "expect":
        with qe.State(26, "c128") as st:
            if df:
                st.set_arith(qe.ARITH_DF64)
            st.init_random(2)
            xm, zm, cf = I.tfim_terms(26)
            for _ in range(2):
                st.expectation(xm, zm, cf)
    else:
        n = 26 if df else 25
        with qe.State(n, "c128") as st:
            if df:
                st.set_arith(qe.ARITH_DF64)
            st.set_policy(qe.POLICY_EMULATE, 1)
            st.init_random(2)
            for _ in range(2):
                st.apply_qft(0, n)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": which, "workload": KERNEL_CASES[which]}), flush=True)


def workload_desc(n, depth, max_k):
    return (f"n={n} complex128 state ({16 << n >> 30} GiB): |0..0> -> depth-{depth} random circuit "
            f"({depth * n} Haar U(2) + {depth * (n // 2)} CNOT) fused to k<={max_k} -> emulated "
            f"{n}-qubit QFT -> add-constant on qubits [0,16) -> TFIM energy + 3-qubit marginal")


# ------------------------------------------------------------------ oracle
def host_cpu():
    """(model name, logical CPU count) of the host cores."""
    model = "unknown"
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


class OracleSample:
    """The oracle gate by gate on the config-1 workload itself: the first
    gates of the depth-20 random circuit on the n-qubit complex128 state
    (bounded samples of the step's gate passes).  GB/s counts 2 * 2^n * 16
    bytes per gate, as the GPU line counts a gate pass."""

    def __init__(self, n, depth, seed=0):
        import oracle
        from paper_1604_06460_gb300 import inputs as I
        self.oracle = oracle
        self.n = n
        self.gates = I.random_circuit(n, depth, seed)
        self.psi = oracle.zero_state(n)
        self.pos = 0

    def run(self, count, threads):
        o = self.oracle
        o.set_threads(threads)
        used = o.max_threads()
        t0 = time.perf_counter()
        for _ in range(count):
            g = self.gates[self.pos % len(self.gates)]
            self.pos += 1
            o.apply_gate(self.psi, g.qubits, g.matrix, inplace=True)
        dt = time.perf_counter() - t0
        return count * 2.0 * (16 << self.n) / dt / 1e9, dt, used

    def close(self):
        self.psi = None


def cpu_baseline(n=30, depth=20, gates_1=2, gates_all=16):
    """Single-thread and all-core oracle runs on bounded samples of the
    config-1 circuit at its full size (about 10-20 s of CPU work each)."""
    model, ncpu = host_cpu()
    smp = OracleSample(n, depth)
    v1, t1, _ = smp.run(gates_1, 1)
    va, ta, used = smp.run(gates_all, ncpu)
    smp.close()
    desc = (f"oracle (plain C, FP64) applying gates of the config-1 random circuit gate by gate to the "
            f"{n}-qubit complex128 state ({16 << n >> 30} GiB): {gates_all} gates on {used} threads "
            f"(OpenMP over amplitude groups) and {gates_1} on one thread; GB/s = gates x 2 x 2^{n} x 16 B "
            f"/ wall time")
    return {"value": va, "unit": "GB/s", "cores": used, "kind": "oracle", "sample": desc, "seconds": ta,
            "cpu_model": model, "nproc": ncpu,
            "single_thread": {"value": v1, "unit": "GB/s", "cores": 1, "gates": gates_1, "seconds": t1},
            "all_cores": {"value": va, "unit": "GB/s", "cores": used, "gates": gates_all, "seconds": ta}}


def run_reference(args):
    """The oracle as it stands on all host cores, each step a bounded sample
    (two gates of the config-1 circuit on the full 30-qubit state)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    model, ncpu = host_cpu()
    smp = OracleSample(args.n, args.depth)
    for _ in range(args.warmup):
        smp.run(1, ncpu)
    vals, secs, used = [], 0.0, 1
    for _ in range(args.steps):
        v, dt, used = smp.run(2, ncpu)
        vals.append(v)
        secs += dt
    smp.close()
    value = float(np.mean(vals))
    desc = (f"oracle (plain C, FP64, {used} OpenMP threads on {model}) applying two gates of the config-1 "
            f"random circuit per step to the {args.n}-qubit complex128 state; GB/s = 2 x 2 x 2^{args.n} x 16 B "
            f"per step / wall time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.n, args.depth, 1) + " (oracle: bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": used, "kind": "oracle", "sample": desc,
                         "cpu_model": model, "nproc": ncpu},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- helpers
class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs, written to
    `path` (a temporary file, removed after summary(), when `path` is None)."""

    def __init__(self, index, path=None):
        self.index = index
        self.proc = None
        self.keep = path is not None
        if path is None:
            fd, path = tempfile.mkstemp(prefix="clocks_bench_", suffix=".csv")
            os.close(fd)
        self.path = path

    def __enter__(self):
        try:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
        if getattr(self, "f", None):
            self.f.close()

    def summary(self):
        try:
            lines = open(self.path).read().splitlines() if self.proc else []
        finally:
            if not self.keep and os.path.exists(self.path):
                os.remove(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Source files each profiled kernel is built from (its summary's hash covers
# only these, so an edit elsewhere keeps the counters valid).
KERNEL_SOURCES = {
    "gate_tc_k5_c128": ["tc_c128.cu", "qe_oz.cuh", "qe_tc.cuh", "qe_arith.cuh"],
    "oz_zgemm": ["oz_gemm.cu", "qe_oz.cuh", "qe_tc.cuh"],
    "add": ["perm.cu", "qe_arith.cuh"],
    "arith": ["arith.cu", "qe_arith.cuh"],
    "batch": ["batch.cu", "qe_batch.h", "qe_arith.cuh"],
    "fft_twiddle": ["fft.cu", "qe_arith.cuh"],
    "digitrev": ["fft.cu", "qe_arith.cuh"],
    "gate_tc_k5": ["tcgen05.cu", "qe_tc.cuh", "qe_arith.cuh"],
    "gate_direct": ["gates.cu", "qe_arith.cuh"],
    "expect_fx": ["reduce.cu", "qe_oz.cuh", "qe_tc.cuh", "qe_arith.cuh"],
    "fft": ["fft.cu", "qe_arith.cuh"],
}


def kernel_traffic(name, bytes_per_launch_now):
    """DRAM traffic per launch for kernel `name` from the committed ncu
    summary profiles/<name>_n*.md, if it was taken on the kernel's current
    source."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{name}_n*.md"))):
        text = open(path).read()
        m = re.search(r"traffic_bytes_per_launch_full:\s*([0-9.eE+]+)", text)
        h = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
        if m and h and h.group(1) == source_hash(name):
            return float(m.group(1))
    return None


def source_hash(kernel=None):
    """sha256 (16 hex digits) of the kernel's source files (all of csrc/ when
    the kernel is not listed)."""
    d = os.path.join(ROOT, "paper_1604_06460_gb300", "csrc")
    files = sorted(os.listdir(d))
    for prefix in sorted(KERNEL_SOURCES, key=len, reverse=True):
        if kernel and kernel.startswith(prefix):
            files = KERNEL_SOURCES[prefix]
            break
    hs = hashlib.sha256()
    for f in files:
        hs.update(open(os.path.join(d, f), "rb").read())
    return hs.hexdigest()[:16]


def aggregate_over_ranks(ms, nbytes, world):
    """Replicas: the slowest rank's time and the bytes of all ranks (the
    only collective is this bookkeeping, none on the data path)."""
    if world <= 1:
        return ms, nbytes
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([nbytes], dtype=torch.float64, device=dev)
    dist.all_reduce(b)
    return float(t.item()), float(b.item())


# ------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    if args.kernel_case:
        torch.cuda.set_device(0)
        from paper_1604_06460_gb300 import build as B
        from paper_1604_06460_gb300 import inputs as I
        from paper_1604_06460_gb300 import qe
        B.build()
        qe.load()
        run_kernel_case(qe, I, args.kernel_case)
        return 0
    if args.only:
        torch.cuda.set_device(0)
        from paper_1604_06460_gb300 import build as B
        from paper_1604_06460_gb300 import inputs as I
        from paper_1604_06460_gb300 import qe
        B.build()
        qe.load()
        if args.only == "batch":
            res = bench_batch(qe, I)
        elif args.only == "qft":
            res = bench_qft(qe, args.n, args.dtype)
        elif args.only == "qpe":
            res = bench_qpe(qe, I)
        elif args.only == "tensor_cores":
            res = bench_tensor_cores(qe, I, n=args.n, n_err=min(args.n, 24))
        else:
            res = bench_config4(qe, I, n=args.n)
        print(json.dumps({"only": args.only, "n": args.n, **res}), flush=True)
        return 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1604_06460_gb300 import build as B
    from paper_1604_06460_gb300 import inputs as I
    from paper_1604_06460_gb300 import qe

    B.build()
    qe.load()
    n, depth = args.n, args.depth
    st = qe.State(n, "c128")
    arith = qe.ARITH_FP64 if args.arith == "fp64" else qe.ARITH_DF64
    st.set_arith(arith)
    max_k = args.max_k or 5
    st.set_policy(qe.POLICY_AUTO, max_k)
    gates = I.random_circuit(n, depth, seed=0)
    reg = list(range(min(16, n)))
    cconst = I.random_constant(len(reg), seed=1)
    xm, zm, cf = I.tfim_terms(n)
    stream = st.stream

    def step(from_host=None):
        if from_host is None:
            st.init_basis(0)
        else:
            st.set(from_host)
        for g in gates:
            st.apply(g)
        st.apply_qft(0, n)
        st.add_const(reg, cconst)
        e = st.expectation(xm, zm, cf)
        p = st.probs([0, 1, 2])
        return e, p

    pinned = e2e_input(st, n) if rank == 0 and not args.quick else None
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    st.reset_stats()
    st.profile(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device(), args.clocks_csv) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            energy, probs = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    stats = st.stats()
    prof = st.profile_read()
    st.profile(False)
    blocks_per_step = stats["fused_blocks"] / args.steps
    step_bytes = algorithmic_step_bytes(n, blocks_per_step)
    ms, total_bytes = aggregate_over_ranks(ms, step_bytes * args.steps, world)
    value = total_bytes / (ms * 1e-3) / 1e9
    roofline = roofline_of(prof, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.arith == "fp64" else "df64",
        "arith": ARITH_DESC[args.arith],
        "data": "synthetic",
        "config": {"workload": workload_desc(n, depth, max_k), "n": n, "depth": depth, "max_k": max_k,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (state 16 GiB vs 129 MB L2)"},
        "gpu_launches": int(stats["launches"]),
        "gates_per_s": len(gates) * args.steps / (ms * 1e-3),
        "passes_per_step": stats["passes"] / args.steps,
        "algorithmic_bytes_per_step": step_bytes,
        "implementation": {"bytes_per_step": stats["algorithmic_bytes"] / args.steps,
                           "GB_per_s": stats["algorithmic_bytes"] / (ms * 1e-3) / 1e9 * world,
                           "note": "bytes of the passes the library ran (extra FFT, bit-reversal and "
                                   "expectation passes included)"},
        "energy": energy,
        "roofline": roofline,
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.quick:
        line["e2e"] = e2e(st, step, n, step_bytes, pinned)
        pinned = None
        line["fast_mode_df64"] = other_mode(st, qe, step, n, max_k, qe.ARITH_DF64 if arith == qe.ARITH_FP64
                                            else qe.ARITH_FP64, ms / args.steps)
        line["emulation"] = compare(st, qe, n, reg, cconst)
        if args.fusion_comparison:
            line["fusion_width_comparison"] = fusion_comparison(st, step, max_k)
    st.close()
    if rank == 0 and not args.quick:
        torch.cuda.empty_cache()
        line["accuracy_vs_oracle"] = step_accuracy(qe, I, max_k=max_k)
        line["cpu_baseline"] = cpu_baseline(n, depth)
        # the config-2 oracle reference (minutes of host work) runs on the
        # host cores while the GPU runs the other configurations
        from concurrent.futures import ThreadPoolExecutor
        pool = ThreadPoolExecutor(max_workers=1)
        ref28 = pool.submit(_config2_oracle, 28, 30, max(1, (os.cpu_count() or 2) - 1))
        for key, fn in (("config0_gate_by_gate", bench_config0), ("batch_config3", bench_batch),
                        ("config4_and_cost_model", bench_config4), ("phase_estimation", bench_qpe),
                        ("tensor_core_config2", lambda q, i: bench_tensor_cores(q, i, oracle_reference=ref28))):
            try:
                line[key] = fn(qe, I)
            except Exception as exc:   # report, keep the headline line
                line[key] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
        pool.shutdown()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


ARITH_DESC = {
    "fp64": ("complex128 in the FP64 mode: 3-5-qubit blocks as exact fp16-digit products of 56-bit "
             "splittings on the tensor cores (each input rounded to 2^-56 of its 32-amplitude group's "
             "scale, one rounding per output), everything else (FFT, reductions, smaller gates) in native "
             "FP64"),
    "df64": ("complex128 in the fast mode: 3-5-qubit blocks as exact fp16-digit products of 48-bit "
             "splittings on the tensor cores, smaller blocks, the FFT and the reductions in double-float "
             "(f32 pair, 47-bit) arithmetic"),
}


def algorithmic_step_bytes(n, blocks_per_step):
    """Bytes the method must move in one step (see the module docstring)."""
    amp = 16 << n
    passes = -(-n // 11)
    return (2 * blocks_per_step + 2 * passes + 2 + passes + 1) * amp


def roofline_of(prof, ms):
    """Roofline of the kernel with the largest share of the event time among
    full-state passes: its algorithmic bytes per launch over its average
    CUDA-event duration, against the measured copy bandwidth."""
    full = {k: v for k, v in prof.items() if v[2] > 0}
    dom = max(full, key=lambda k: full[k][1])
    launches, tot_ms, dbytes = full[dom]
    achieved = (dbytes / launches) / (tot_ms / launches * 1e-3) / 1e9
    peak, peak_src = peak_hbm()
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": kernel_traffic(dom, dbytes / launches),
            "algorithmic_bytes_per_launch": dbytes / launches,
            "share_of_step_time": tot_ms / ms,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3), "GB/s": round(v[2] / max(v[1], 1e-9) / 1e6, 1)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}


def other_mode(st, qe, step, n, max_k, arith, ms_headline, steps=3):
    """The same step in the other complex128 arithmetic mode (the fast
    double-float mode beside the FP64 headline), with its own roofline."""
    import torch
    st.set_arith(arith)
    st.set_policy(qe.POLICY_AUTO, max_k)
    step()
    torch.cuda.synchronize()
    st.reset_stats()
    st.profile(True)
    e0, e1 = _events()
    e0.record(st.stream)
    for _ in range(steps):
        step()
    e1.record(st.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    stats = st.stats()
    prof = st.profile_read()
    st.profile(False)
    step_bytes = algorithmic_step_bytes(n, stats["fused_blocks"] / steps)
    rf = roofline_of(prof, ms)
    rf.pop("kernels", None)
    out = {"arith": ARITH_DESC["df64" if arith == qe.ARITH_DF64 else "fp64"],
           "dtype": "df64" if arith == qe.ARITH_DF64 else "f64",
           "ms_per_step": ms / steps, "value": step_bytes * steps / (ms * 1e-3) / 1e9, "unit": "GB/s",
           "speedup_vs_headline": ms_headline / (ms / steps), "roofline": rf,
           "kernels_ms_per_step": {k: round(v[1] / steps, 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}}
    st.set_arith(qe.ARITH_FP64 if arith == qe.ARITH_DF64 else qe.ARITH_DF64)
    st.set_policy(qe.POLICY_AUTO, max_k)
    return out


def step_accuracy(qe, I, n=24, depth=20, max_k=5):
    """The bench step at n = 24 (same generators and seeds) on the GPU in
    both arithmetic modes against the oracle run gate by gate on the host
    cores: final state (max-abs, fidelity), Ising energy and marginal."""
    import oracle
    gates = I.random_circuit(n, depth, seed=0)
    reg = list(range(min(16, n)))
    cconst = I.random_constant(len(reg), seed=1)
    xm, zm, cf = I.tfim_terms(n)
    t0 = time.perf_counter()
    oracle.set_threads(os.cpu_count() or 1)
    ref = oracle.zero_state(n)
    for g in gates:
        oracle.apply_gate(ref, g.qubits, g.matrix, inplace=True)
    ref = oracle.qft_circuit(ref, 0, n)
    ref = oracle.add_const(ref, reg, cconst)
    e_ref = oracle.expectation(ref, xm, zm, cf)
    p_ref = oracle.probs(ref, [0, 1, 2])
    out = {"n": n, "depth": depth, "oracle_s": time.perf_counter() - t0,
           "oracle": "gate by gate, QFT as its H/CR/swap circuit, addition as the index map"}
    for label, arith in (("fp64", qe.ARITH_FP64), ("df64", qe.ARITH_DF64)):
        with qe.State(n, "c128") as st:
            st.set_arith(arith)
            st.set_policy(qe.POLICY_AUTO, max_k)
            for g in gates:
                st.apply(g)
            st.apply_qft(0, n)
            st.add_const(reg, cconst)
            e = st.expectation(xm, zm, cf)
            p = st.probs([0, 1, 2])
            got = st.get()
        out[label] = {"max_abs": float(np.max(np.abs(got - ref))), "fidelity": oracle.fidelity(ref, got),
                      "one_minus_fidelity": 1.0 - oracle.fidelity(ref, got),
                      "abs_dE": abs(e - e_ref), "max_abs_dprob": float(np.max(np.abs(p - p_ref)))}
    return out


def fusion_comparison(st, step, max_k):
    """The same step with fusion up to 2 qubits (elementwise blocks only):
    more passes, longer time to solution."""
    import torch
    from paper_1604_06460_gb300 import qe as Q
    out = {}
    for k in (2, max_k):
        st.set_policy(Q.POLICY_AUTO, k)
        step()
        torch.cuda.synchronize()
        st.reset_stats()
        e0, e1 = _events()
        e0.record(st.stream)
        step()
        e1.record(st.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        s = st.stats()
        out[f"k<={k}"] = {"ms_per_step": ms, "passes": s["passes"],
                          "GB_per_s": s["algorithmic_bytes"] / ms / 1e6}
    st.set_policy(Q.POLICY_AUTO, max_k)
    return out


def e2e_input(st, n):
    """The pinned host copy of an input state for e2e(), made before the
    timed work so that the host's memory management has settled when e2e()
    runs (pinning 16 GiB just before it measured steps ~50 % slower)."""
    import torch
    host = torch.empty(2 << n, dtype=torch.float64, pin_memory=True)
    view = host.numpy().view(np.complex128)
    st.init_random(11)
    st.get(out=view)
    return host, view


def e2e(st, step, n, bytes_per_step, pinned, steps=5):
    """The same step through the public API with the input state in pinned
    host memory (`pinned` from e2e_input): host->device copy of the state and
    device->host read of the energy and marginals inside the timed region;
    the median of `steps` steps, and the host->device rate of the same copies
    timed alone."""
    import torch
    host, view = pinned
    ts, h2d, cpu = [], [], []
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(steps):
            t0, c0 = time.perf_counter(), time.process_time()
            step(from_host=view)
            ts.append(time.perf_counter() - t0)
            cpu.append(time.process_time() - c0)
    for _ in range(3):
        t0 = time.perf_counter()
        st.set(view)
        h2d.append(time.perf_counter() - t0)
    dt = float(np.median(ts))
    return {"value": bytes_per_step / dt / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 16 << n,
            "d2h_bytes_per_step": 8 + 8 * 8, "ms_per_step": dt * 1e3, "steps": steps,
            "ms_per_step_all": [round(t * 1e3, 1) for t in ts],
            "host_cpu_ms_per_step": [round(t * 1e3, 1) for t in cpu],
            "h2d_GB_per_s": (16 << n) / float(np.median(h2d)) / 1e9, "clocks": clk.summary()}


def compare(st, qe, n, reg, cconst):
    """Emulated vs simulated subroutines on the same GPU and input."""
    import torch
    out = {}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record(st.stream)
        fn()
        st.flush()
        ev1.record(st.stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    # QFT on all n qubits of a random normalised state
    st.set_policy(qe.POLICY_EMULATE, 1)
    st.init_random(5)
    t_emu = timed(lambda: st.apply_qft(0, n))
    emu = st.tensor.clone()
    st.set_policy(qe.POLICY_SIMULATE, 1)
    st.init_random(5)
    t_sim = timed(lambda: st.apply_qft(0, n))
    a = torch.view_as_complex(emu.view(-1, 2))
    b = torch.view_as_complex(st.tensor.view(-1, 2))
    max_abs = float((a - b).abs().max().item())
    ov = torch.vdot(a, b)
    fid = float((ov.abs() ** 2 / (torch.vdot(a, a).real * torch.vdot(b, b).real)).item())
    out["qft"] = {"emulated_ms": t_emu, "simulated_ms": t_sim, "speedup": t_sim / t_emu,
                  "simulated_gates": n + n * (n - 1) // 2, "max_abs_diff": max_abs, "fidelity": fid,
                  "analytic_speedup_hint": None}
    del emu
    # addition of a constant: one permutation vs the multi-controlled-NOT ripple
    st.set_policy(qe.POLICY_EMULATE, 1)
    st.init_random(6)
    t_emu = timed(lambda: st.add_const(reg, cconst))
    emu = st.tensor.clone()
    st.set_policy(qe.POLICY_SIMULATE, 1)
    st.init_random(6)
    t_sim = timed(lambda: st.add_const(reg, cconst))
    out["add_const"] = {"emulated_ms": t_emu, "simulated_ms": t_sim, "speedup": t_sim / t_emu,
                        "register": [reg[0], reg[-1] + 1], "c": cconst,
                        "bit_exact": bool(torch.equal(emu, st.tensor))}
    del emu
    # multiplication and division of N = n/3-qubit registers in the paper's
    # layout (index = a b c, c in the low qubits; Sec. III-A, Sec. IV-B)
    N = n // 3
    qc, qb, qa = list(range(N)), list(range(N, 2 * N)), list(range(2 * N, 3 * N))
    st.set_policy(qe.POLICY_EMULATE, 1)
    st.init_random(7)
    t_emu = timed(lambda: st.mul(qa, qb, qc))
    emu = st.tensor.clone()
    st.set_policy(qe.POLICY_SIMULATE, 1)
    st.init_random(7)
    st.reset_stats()
    t_sim = timed(lambda: st.mul(qa, qb, qc))
    gates = st.stats()["gates_applied"]
    out["mul"] = {"N": N, "emulated_ms": t_emu, "simulated_ms": t_sim, "speedup": t_sim / t_emu,
                  "simulated_gates": gates, "emulated_GB_per_s": 2 * (16 << n) / t_emu / 1e6,
                  "bit_exact": bool(torch.equal(emu, st.tensor))}
    del emu
    st.set_policy(qe.POLICY_EMULATE, 1)
    st.init_random(8)
    t_div = timed(lambda: st.div(qa, qb, qc))
    out["div"] = {"N": N, "emulated_ms": t_div, "emulated_GB_per_s": 4 * (16 << n) / t_div / 1e6,
                  "note": "planes of 2^(2N) amplitudes through the scratch buffer (gather + copy back: "
                          "4 x state bytes); no simulated division (its circuit needs work qubits)"}
    st.set_policy(qe.POLICY_AUTO, 2)
    return out


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def bench_qft(qe, n, dtype, reps=3):
    """Emulated QFT on all n qubits of a random normalised state."""
    with qe.State(n, dtype) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.init_random(5)
        st.apply_qft(0, n)
        ts = []
        for _ in range(reps):
            e0, e1 = _events()
            e0.record(st.stream)
            st.apply_qft(0, n)
            e1.record(st.stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        st.reset_stats()
        st.apply_qft(0, n)
        stats = st.stats()
    ms = float(np.median(ts))
    return {"dtype": dtype, "emulated_ms": ms, "passes": stats["passes"],
            "GB_per_s": stats["algorithmic_bytes"] / ms / 1e6}


def bench_config0(qe, I, n=20, layers=10, seed=0):
    """n=20 complex128 from |0..0>, 10 layers of (20 Haar U(2) + 10 CNOT),
    gate by gate without fusion (L2-resident: launch-bound, not HBM-bound);
    gates/s, time to solution and the error against the oracle."""
    import torch
    import oracle
    gates = I.random_circuit(n, layers, seed)
    with qe.State(n, "c128") as st:
        st.set_policy(qe.POLICY_AUTO, 1)
        for g in gates:
            st.apply(g)
        st.flush()
        ts = []
        for _ in range(5):
            st.init_basis(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for g in gates:
                st.apply(g)
            st.sync()
            ts.append(time.perf_counter() - t0)
        got = st.get()
        # the same run once more with per-launch device timing: the kernels'
        # own time, apart from the host's enqueue and launch overhead
        st.init_basis(0)
        st.sync()
        st.profile(True)
        for g in gates:
            st.apply(g)
        prof = st.profile_read()
        st.profile(False)
    ref = oracle.zero_state(n)
    for g in gates:
        ref = oracle.apply_gate(ref, g.qubits, g.matrix)
    dt = float(np.median(ts))
    launches = sum(v[0] for v in prof.values())
    dev_ms = sum(v[1] for v in prof.values())
    return {"n": n, "gates": len(gates), "time_to_solution_ms": dt * 1e3, "gates_per_s": len(gates) / dt,
            "device_ms": dev_ms, "launches": launches, "device_us_per_launch": dev_ms * 1e3 / max(launches, 1),
            "host_overhead_us_per_gate": (dt * 1e3 - dev_ms) * 1e3 / len(gates),
            "max_abs_vs_oracle": float(np.max(np.abs(got - ref))),
            "fidelity_vs_oracle": float(abs(np.vdot(ref, got)) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real)),
            "note": "host-timed through the public API (enqueue + kernels + sync); 32 MB state is L2-resident; "
                    "device_ms: the kernels' own time (CUDA events per launch, one run)"}


def bench_batch(qe, I, count=4096, layers=8, seed=3):
    """4096 ansatz circuits, n ~ U{10..22}, 8 layers, TFIM energy each; one
    persistent launch replayed as a CUDA graph; c128 and c64."""
    import oracle
    ns = I.batch_sizes(count, 10, 22, seed)
    angles = [I.ansatz_angles(int(nq), layers, seed * 100000 + i) for i, nq in enumerate(ns)]
    out = {"circuits": count, "layers": layers, "n_range": [10, 22],
           "sum_amplitudes": float(sum(2.0 ** int(v) for v in ns))}
    for dtype in ("c128", "c64"):
        with qe.Batch(ns, angles, 0.7, dtype) as b:
            t0 = time.perf_counter()
            plan = b.tune(reps=1)
            tune_s = time.perf_counter() - t0
            b.run()
            reps = 3
            t0 = time.perf_counter()
            for _ in range(reps):
                e = b.run()
            dt = (time.perf_counter() - t0) / reps
            info = b.info()
            e64 = None
            if dtype == "c128":
                # the same batch in native FP64 (gates and energy sums), on the
                # plan tuned for double-float
                b.set_arith(qe.ARITH_FP64)
                b.run()
                t0 = time.perf_counter()
                e64 = b.run()
                dt64 = time.perf_counter() - t0
        # oracle energies on sampled circuits of the batch: four that run in
        # shared memory (n <= 12) and two HBM-resident ones (n = 20, 22)
        idx = [i for i in range(count) if ns[i] <= 12][:4]
        idx += [next(i for i in range(count) if ns[i] == v) for v in (20, 22) if v in set(int(x) for x in ns)]
        err = err64 = 0.0
        oracle.set_threads(os.cpu_count() or 1)
        for i in idx:
            psi = oracle.zero_state(int(ns[i]))
            for g in I.ansatz_circuit(int(ns[i]), layers, seed * 100000 + i):
                psi = oracle.apply_gate(psi, g.qubits, g.matrix, inplace=True)
            xm, zm, cf = I.tfim_terms(int(ns[i]), 0.7)
            ref = oracle.expectation(psi, xm, zm, cf)
            err = max(err, abs(e[i] - ref))
            if e64 is not None:
                err64 = max(err64, abs(e64[i] - ref))
        out[dtype] = {"arith": ("double-float (47-bit significands) gates and float-pair energy sums"
                                if dtype == "c128" else "FP32 gates, float-pair energy sums"),
                      "time_to_solution_ms": dt * 1e3, "circuits_per_s": count / dt,
                      "pass_bytes_GB_per_s": info["hbm_bytes"] / dt / 1e9, "items": info["items"],
                      "pass_bytes_note": "state bytes the passes of the large circuits read and write; waves of "
                                         "<= 64 MiB keep them largely in L2, so DRAM moves less",
                      "plan": plan, "tune_s": tune_s, "max_abs_dE_vs_oracle_sampled": err,
                      **({"fp64_mode": {"arith": "native FP64 gates and FP64 energy sums (same plan)",
                                        "time_to_solution_ms": dt64 * 1e3, "circuits_per_s": count / dt64,
                                        "max_abs_dE_vs_oracle_sampled": err64}} if e64 is not None else {}),
                      "sampled_circuits": len(idx), "sampled_n": [int(ns[i]) for i in idx]}
    return out


def _config2_oracle(n_err, depth, threads=None):
    """The FP64 oracle's state of the config-2 circuit at n_err qubits, gate
    by gate on the host cores; returns (state, seconds)."""
    import oracle
    from paper_1604_06460_gb300 import inputs as I
    t0 = time.perf_counter()
    oracle.set_threads(threads or os.cpu_count() or 1)
    ref = oracle.zero_state(n_err)
    for g in I.random_circuit(n_err, depth, seed=5):
        oracle.apply_gate(ref, g.qubits, g.matrix, inplace=True)
    return ref, time.perf_counter() - t0


def bench_tensor_cores(qe, I, n=32, depth=30, n_err=28, oracle_reference=None):
    """complex64 state, depth-30 random circuit fused into 5-qubit blocks on
    the tcgen05 tensor cores (3xTF32, FP32 accumulation); the error at n_err
    on the same seed against the FP64 oracle, run gate by gate on the host
    cores (oracle_reference: a future of that run started earlier, so that it
    overlaps the GPU work of other configurations)."""
    import torch
    import oracle
    gates = I.random_circuit(n, depth, seed=5)
    out = {"n": n, "depth": depth, "gates": len(gates)}
    with qe.State(n, "c64") as st:
        st.set_policy(qe.POLICY_AUTO, 5)
        st.init_basis(0)
        for g in gates:
            st.apply(g)
        st.flush()
        st.reset_stats()
        st.profile(True)
        e0, e1 = _events()
        st.init_basis(0)
        torch.cuda.synchronize()
        e0.record(st.stream)
        for g in gates:
            st.apply(g)
        st.flush()
        e1.record(st.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        prof = st.profile_read()
        stats = st.stats()
    tc = prof.get("gate_tc_k5", (0, 0.0, 0.0))
    peak, _ = peak_hbm()
    out.update({"ms": ms, "passes": stats["passes"], "GB_per_s": stats["algorithmic_bytes"] / ms / 1e6,
                "tc_launches": tc[0], "tc_GB_per_s": tc[2] / max(tc[1], 1e-9) / 1e6,
                "tc_frac_of_copy": tc[2] / max(tc[1], 1e-9) / 1e6 / peak,
                "tc_share": tc[1] / ms})
    gates = I.random_circuit(n_err, depth, seed=5)
    with qe.State(n_err, "c64") as st:
        st.set_policy(qe.POLICY_AUTO, 5)
        for g in gates:
            st.apply(g)
        got = st.get()
    ref, t_or = oracle_reference.result() if oracle_reference is not None else _config2_oracle(n_err, depth)
    max_abs, ov, nr, ng = 0.0, 0j, 0.0, 0.0
    chunk = 1 << 22
    for i0 in range(0, ref.size, chunk):
        r = ref[i0:i0 + chunk]
        g = got[i0:i0 + chunk].astype(np.complex128)
        max_abs = max(max_abs, float(np.max(np.abs(g - r))))
        ov += np.vdot(r, g)
        nr += np.vdot(r, r).real
        ng += np.vdot(g, g).real
    fid = float(abs(ov) ** 2 / (nr * ng))
    out["error_at_n%d" % n_err] = {"max_abs": max_abs, "fidelity": fid, "one_minus_fidelity": 1.0 - fid,
                                   "reference": "oracle (FP64, gate by gate on the host cores)",
                                   "oracle_s": t_or, "oracle_threads": oracle.max_threads()}
    del ref, got
    return out


def bench_qpe(qe, I, ns=(8, 9, 10, 11, 12)):
    """Phase estimation, simulated vs emulated (Sec. III-C; Table II's
    quantities on one GPU): U is one Trotter step of the 1-D transverse-field
    Ising evolution (G = 4n - 3 gates).  T_apply: the circuit applied once,
    gate by gate, to an (n+1)-qubit state (the one-ancilla simulation needs
    2^b - 1 of them); T_build: the dense 2^n x 2^n matrix of U (identity state
    plus the gates); T_gemm: one squaring, on the tensor cores (exact digit
    products, 128-bit sums) and with the FP64 kernel (QE_GEMM_F64=1).  The
    cross-over is the smallest b with (2^b - 1) T_apply >= T_build + (b - 1)
    T_gemm."""
    import torch
    out = {}
    for n in ns:
        gates = I.tfim_trotter_step(n)
        with qe.State(n + 1, "c128") as st:
            st.set_policy(qe.POLICY_AUTO, 1)
            st.init_random(1)
            for g in gates:
                st.apply(g)
            st.flush()
            reps = 20
            e0, e1 = _events()
            e0.record(st.stream)
            for _ in range(reps):
                for g in gates:
                    st.apply(g)
                st.flush()
            e1.record(st.stream)
            e1.synchronize()
            t_apply = e0.elapsed_time(e1) / reps
        with qe.State(2 * n, "c128") as u, qe.State(2 * n, "c128") as u2:
            u.set_policy(qe.POLICY_AUTO, 0)
            torch.cuda.synchronize()
            e0, e1 = _events()
            e0.record(u.stream)
            u.init_identity(n)
            for g in gates:
                u.apply(g)
            u.flush()
            e1.record(u.stream)
            e1.synchronize()
            t_build = e0.elapsed_time(e1)
            gemm = {}
            for label in ("tensor_cores", "fp64"):
                if label == "fp64":
                    os.environ["QE_GEMM_F64"] = "1"
                try:
                    u2.matmul(u, u)
                    torch.cuda.synchronize()
                    e0, e1 = _events()
                    e0.record(u2.stream)
                    u2.matmul(u, u)
                    e1.record(u2.stream)
                    e1.synchronize()
                    gemm[label] = (e0.elapsed_time(e1), u2.get())
                finally:
                    os.environ.pop("QE_GEMM_F64", None)
        t_gemm, t_f64 = gemm["tensor_cores"][0], gemm["fp64"][0]
        diff = float(np.max(np.abs(gemm["tensor_cores"][1] - gemm["fp64"][1])))

        def crossover(tg):
            b = 1
            while (2 ** b - 1) * t_apply < t_build + (b - 1) * tg and b < 64:
                b += 1
            return b
        out[f"n{n}"] = {"G": len(gates), "apply_U_ms": t_apply, "build_dense_U_ms": t_build,
                        "zgemm_ms": t_gemm, "zgemm_TFLOPs": 8.0 * 8 ** n / (t_gemm * 1e-3) / 1e12,
                        "zgemm_fp64_ms": t_f64, "zgemm_fp64_TFLOPs": 8.0 * 8 ** n / (t_f64 * 1e-3) / 1e12,
                        "tensor_core_vs_fp64_max_abs": diff,
                        "crossover_bits": crossover(t_gemm), "crossover_bits_fp64_gemm": crossover(t_f64)}
        torch.cuda.empty_cache()
    out["note"] = ("Table II of the paper (Xeon, MKL zgemm) gives cross-overs 6, 9, 12, 15, 18 bits for "
                   "n = 8..12 (context only)")
    return out


def bench_config4(qe, I, n=33):
    """n=33 complex128 (128 GiB) random state: add-constant on a 16-qubit
    register (emulated permutation vs multi-controlled-NOT ripple) and the QFT
    on it (digit passes vs 136 gates).  The learned cost model is trained on
    timing sweeps at the sizes of configurations 1-3 (gate passes of the
    30-qubit complex128 and 32-qubit complex64 states, subroutines on 24-, 26-
    and 28-qubit states) and scored, with the analytic rule, on held-out
    emulate-or-simulate decisions at n = 30 and on this configuration's two
    subroutines: regret = time of the chosen paths / time of the best - 1."""
    import torch
    from paper_1604_06460_gb300 import costmodel
    t0 = time.perf_counter()
    Xg, yg = costmodel.sweep_gate_passes([30], dtypes=("c128",), seed=0)
    Xc, yc = costmodel.sweep_gate_passes([32], dtypes=("c64",), seed=0)
    Xs, ys = costmodel.sweep_subroutines([24, 26, 28], dtypes=("c128",), seed=0)
    X = np.concatenate([Xg, Xc, Xs])
    y = np.concatenate([yg, yc, ys])
    model, loss = costmodel.train(X, y, epochs=4000, lr=3e-3, seed=0)
    out = {"cost_model": {"samples": int(len(y)), "train_loss": loss, "sweep_and_train_s": time.perf_counter() - t0,
                          "sweeps": "gate passes k=1..5 at n=30 (c128) and n=32 (c64); QFTs and additions at "
                                    "n=24, 26, 28 (c128)"}}
    t0 = time.perf_counter()
    res, regret = costmodel.evaluate_decisions(30, costmodel.decision_cases(30), model)
    out["decisions_n30"] = {"cases": len(res), "regret": regret,
                            "learned_differs_from_analytic": sum(r["learned"] != r["analytic"] for r in res),
                            "analytic_wrong": sum(r["analytic"] != r["best"] for r in res),
                            "learned_wrong": sum(r["learned"] != r["best"] for r in res),
                            "seconds": time.perf_counter() - t0}
    torch.cuda.empty_cache()
    c = I.random_constant(16, 7)
    results = {}
    with qe.State(n, "c128") as st:
        for reg_lo in (0, 17):
            reg = list(range(reg_lo, reg_lo + 16))
            for label, pol in (("emulated", qe.POLICY_EMULATE), ("simulated", qe.POLICY_SIMULATE)):
                st.init_random(9)
                st.set_policy(pol, 1)
                e0, e1 = _events()
                e0.record(st.stream)
                st.add_const(reg, c)
                e1.record(st.stream)
                e1.synchronize()
                results[f"add_{reg_lo}_{label}"] = e0.elapsed_time(e1)
                # bit-exact check on a slice: both paths from the same input
                results[f"add_{reg_lo}_{label}_sample"] = st.get(min(12345 << 17, (1 << n) - 1024), 1024).copy()
        for label, pol in (("emulated", qe.POLICY_EMULATE), ("simulated", qe.POLICY_SIMULATE)):
            st.init_random(9)
            st.set_policy(pol, 1)
            e0, e1 = _events()
            e0.record(st.stream)
            st.apply_qft(0, 16)
            e1.record(st.stream)
            e1.synchronize()
            results[f"qft_{label}"] = e0.elapsed_time(e1)
            results[f"qft_{label}_sample"] = st.get(777 << 16, 4096).copy()
        # which path each policy takes for this configuration's subroutines
        chosen = {}
        for pname, pol, mdl in (("analytic", qe.POLICY_ANALYTIC, None), ("learned", qe.POLICY_AUTO, model)):
            st.set_cost_model(mdl)
            st.set_policy(pol, 2)
            st.init_random(9)
            st.profile(True)
            st.apply_qft(0, 16)
            q = costmodel._path(st.profile_read())
            st.profile(False)
            st.profile(True)
            st.add_const(list(range(16)), c)
            a = costmodel._path(st.profile_read())
            st.profile(False)
            chosen[pname] = (q, a)
        st.set_cost_model(None)
    for r in (0, 17):
        out[f"add_const_reg_{r}_{r + 16}"] = {
            "emulated_ms": results[f"add_{r}_emulated"], "simulated_ms": results[f"add_{r}_simulated"],
            "speedup": results[f"add_{r}_simulated"] / results[f"add_{r}_emulated"],
            "bit_exact_sample": bool(np.array_equal(results[f"add_{r}_emulated_sample"],
                                                    results[f"add_{r}_simulated_sample"])),
            "emulated_GB_per_s": 2 * (16 << n) / results[f"add_{r}_emulated"] / 1e6}
    a, b = results["qft_emulated_sample"], results["qft_simulated_sample"]
    out["qft_reg_0_16"] = {"emulated_ms": results["qft_emulated"], "simulated_ms": results["qft_simulated"],
                           "speedup": results["qft_simulated"] / results["qft_emulated"],
                           "simulated_gates": 16 + 120, "max_abs_sample": float(np.max(np.abs(a - b)))}
    best_qft = "emulated" if results["qft_emulated"] <= results["qft_simulated"] else "simulated"
    best_add = "emulated" if results["add_0_emulated"] <= results["add_0_simulated"] else "simulated"
    for pname in ("analytic", "learned"):
        q, a_ = chosen[pname]
        out[f"{pname}_choice_n33"] = {"qft": q, "add_const": a_,
                                      "qft_regret": results[f"qft_{q}"] / results[f"qft_{best_qft}"] - 1,
                                      "add_regret": results[f"add_0_{a_}"] / results[f"add_0_{best_add}"] - 1}
    model.close()
    return out


if __name__ == "__main__":
    sys.exit(main())
