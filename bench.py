#!/usr/bin/env python
"""Benchmark of the statevector hot path: a 30-qubit complex128 statevector
(16 GiB, random normalised Gaussian amplitudes) through a seeded 500-operation
circuit (one-qubit Haar unitaries; Haar unitaries on 2-5 targets with 0-5
controls; 1-3-qubit diagonal phase gates; Pauli gadgets of weight 1-30).

One step = the whole 500-operation circuit applied in place on the resident
state.  Prints ONE JSON line on rank 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/qsim_oracle.py) as it stands, on
a bounded sample of the same workload, on the host cores.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gates/s & HBM GB/s on 30q FP64 SV; fused-TC speedup at 1e-6 infidelity"
UNIT = "gates/s"
NUM_OPS = 500
CIRCUIT_TAG = "sv30-circuit"
STATE_SEED = 2311015121
CPU_SAMPLE_QUBITS = 20
ARITH_CODE = {"fx": 2, "df": 0, "f64": 1}     # qs_arith
DTYPE = {
    "fx": ("c128 storage; arithmetic at least FP64: one- and two-target gates, diagonals and gadgets in 60-bit "
           "block fixed point with exact integer products and one rounding per output (error <= 2^-53 |y| + "
           "2^-55 max|x| max|m|, 2^-54 for the two-target gates' eight terms), 3-5-target gates as eight exact "
           "7-bit slices (56-bit operands) on the bf16 tensor cores"),
    "df": "c128 storage, double-float (2xf32, 47-bit) arithmetic",
    "f64": "c128 storage, native f64 arithmetic",
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--qubits", type=int, default=30, help="statevector size (the workload is 30)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--arith", choices=["fx", "df", "f64"], default="fx",
                    help="complex128 arithmetic: block fixed point with exact integer products and one "
                         "rounding, at least the 53 bits of FP64 (default); double-float on the FP32 pipes "
                         "(47-bit); or native FP64")
    ap.add_argument("--f64-share", type=int, default=0,
                    help="sixteenths of one-target-gate work done in native FP64 beside double-float")
    ap.add_argument("--no-fused", action="store_true", help="skip the fused tensor-core comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (15- and 6-qubit density matrices, the 4096-state batch, "
                         "the 31-qubit complex128 fused case)")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end leg (at most --steps)")
    ap.add_argument("--relabel-ab", action="store_true",
                    help="also time the fused form with forced lazy relabelling (one run per setting)")
    ap.add_argument("--fused-qubits", type=int, default=32,
                    help="qubits of the fused comparison (32: the complex64 fused workload's size)")
    ap.add_argument("--fused-max-block", type=int, default=6,
                    help="widest fused block the cost-model planner may form (6 on complex64; complex128 stops at 5)")
    ap.add_argument("--fused-prec", choices=("c64", "c128"), default="c64",
                    help="precision of the fused form: complex64 (3xTF32 blocks) or complex128 (bf16 integer slices)")
    ap.add_argument("--detail", default="", help="write per-kernel-family statistics to this JSON file")
    ap.add_argument("--cpu-sample", type=int, default=0, help=argparse.SUPPRESS)
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# Workload description shared by both arms
# ---------------------------------------------------------------------------

def make_ops(nq):
    from paper_2311_01512_gb300 import workloads as wl
    return wl.statevector_circuit(nq, NUM_OPS, wl.rng_for(CIRCUIT_TAG))


def op_family(op):
    """Kernel family the CUDA path launches for one operation record."""
    kind = op["op"]
    if kind == "unitary":
        return "k_gate1" if len(op["targs"]) == 1 else "k_dense<%d>" % len(op["targs"])
    if kind == "diagonal":
        return "k_diag"
    if kind == "gadget":
        return "k_gadget" if any(p in (1, 2) for p in op["paulis"]) else "k_phase"
    raise ValueError(kind)


def op_bytes(op, nq, amp_bytes):
    """Algorithmic HBM bytes of one operation: every amplitude it updates is
    read once and written once, 2 * sizeof(amp) * (amplitudes touched).
    A gate with s controls touches 2^(N - s) amplitudes."""
    if op["op"] == "unitary":
        return 2 * amp_bytes * (1 << (nq - len(op["ctrls"])))
    return 2 * amp_bytes * (1 << nq)


def op_h2d_bytes(op):
    """Host-to-device bytes the C ABI moves for one operation (the staged
    matrix of a dense gate; small parameters travel in the launch)."""
    if op["op"] == "unitary" and len(op["targs"]) > 1:
        return 16 * (1 << (2 * len(op["targs"])))
    return 0


def config_dict(nq, args):
    return {"workload": "%d-qubit complex128 statevector, seeded %d-op circuit "
                        "(1q Haar; 2-5 target Haar with 0-5 controls; 1-3q diagonal phases; "
                        "Pauli gadgets of weight 1-%d)" % (nq, NUM_OPS, nq),
            "qubits": nq, "ops_per_step": NUM_OPS, "amp": "complex128",
            "state_bytes": 16 * (1 << nq),
            "l2": "inputs larger than L2 (state 16 GiB vs 129 MB L2); no flush",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# CPU oracle sample (runs in a fresh process; never imports torch or CUDA)
# ---------------------------------------------------------------------------

def host_cpu_info():
    """nproc and the CPU model of this host (from /proc/cpuinfo or lscpu)."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.startswith("Model name:"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "model": model or platform.machine(), "arch": platform.machine()}


def cpu_sample_main(num_ops):
    """The oracle on the first num_ops operations of the circuit recipe (all
    500: the whole circuit) at CPU_SAMPLE_QUBITS, one thread."""
    import numpy as np
    from oracle import qsim_oracle as orc
    from paper_2311_01512_gb300 import workloads as wl
    nq = CPU_SAMPLE_QUBITS
    ops = make_ops(nq)[:num_ops]
    psi = wl.random_statevector(nq, wl.rng_for("cpu-sample"))
    t0 = time.perf_counter()
    psi = orc.run_ops(psi, ops, is_density=False)
    dt = time.perf_counter() - t0
    scale = 2.0 ** (nq - 30)
    print(json.dumps({"ops": len(ops), "seconds": dt, "qubits": nq,
                      "value_30q_equiv": len(ops) / dt * scale,
                      "norm": float(np.sum(np.abs(psi) ** 2))}))


def one_thread_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def run_cpu_sample(num_ops):
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample", str(num_ops)],
                         capture_output=True, text=True, env=one_thread_env(), cwd=ROOT, timeout=900)
    if out.returncode != 0:
        raise RuntimeError("cpu sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline_dict(res, sample):
    info = host_cpu_info()
    return {"value": res["value_30q_equiv"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_nproc": info["nproc"], "host_cpu": info["model"], "host_arch": info["arch"],
            "sample": sample}


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Distributed helpers (replicas: each rank runs the whole workload)
# ---------------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def device_random_state(nq, device):
    """Seeded complex Gaussian amplitudes, normalised (input generation)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(STATE_SEED)
    psi = torch.randn(1 << nq, dtype=torch.complex128, device=device, generator=g)
    psi /= torch.linalg.vector_norm(psi)
    return psi


def fill_random_state(dst, nq, device, seed=STATE_SEED + 7):
    """Seeded complex Gaussian amplitudes written into dst (complex64 or
    complex128) in chunks of 2^26, then normalised: no state-sized temporary
    (input generation)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    step = 1 << min(26, nq)
    ss = 0.0
    for i in range(0, 1 << nq, step):
        c = torch.randn(step, dtype=torch.complex128, device=device, generator=g)
        ss += float(torch.vdot(c, c).real.item())
        dst[i:i + step].copy_(c)
        del c
    scale = 1.0 / ss ** 0.5
    for i in range(0, 1 << nq, step):
        dst[i:i + step] *= scale


def load_traffic(family):
    """DRAM bytes per launch measured by ncu for a kernel family, if the record
    matches the current kernel sources (profiles/dram_traffic.json)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
        from paper_2311_01512_gb300 import build as b
        if rec.get("sources_sha256") != b.sources_digest():
            return None
        return rec.get("families", {}).get(family)
    except Exception:
        return None


def main_ours(args):
    world, rank, local = dist_setup(args)
    cpu_res = None
    sections = {}
    t_sec = time.perf_counter()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_res = run_cpu_sample(NUM_OPS)   # before the first GPU call; a separate process
    sections["cpu_baseline"] = time.perf_counter() - t_sec
    t_sec = time.perf_counter()
    import torch
    from paper_2311_01512_gb300 import qs
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    nq = args.qubits
    ops = make_ops(nq)
    stream = torch.cuda.Stream(device=device)
    with torch.cuda.stream(stream):
        psi = device_random_state(nq, device)
    stream.synchronize()
    st = qs.State(nq, density=False, prec=qs.QS_C128, stream=stream, storage=psi)
    h = st.handle
    qs.qs_set_arithmetic(h, ARITH_CODE[args.arith], args.f64_share)
    fams = [op_family(op) for op in ops]
    nbytes = [op_bytes(op, nq, 16) for op in ops]

    for _ in range(args.warmup):
        for op in ops:
            qs.apply_op(h, op)
    stream.synchronize()

    # timed region: K steps, events around every operation on the launching stream
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(NUM_OPS + 1)] for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        for i, op in enumerate(ops):
            evs[k][i].record(stream)
            qs.apply_op(h, op)
        evs[k][NUM_OPS].record(stream)
    t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(total_ms, world, device)
    ms_per_step = total_ms / args.steps

    # per-family statistics from the per-operation events
    fam_time, fam_bytes, fam_count = {}, {}, {}
    for k in range(args.steps):
        for i in range(NUM_OPS):
            dt = evs[k][i].elapsed_time(evs[k][i + 1])
            f = fams[i]
            fam_time[f] = fam_time.get(f, 0.0) + dt
            fam_bytes[f] = fam_bytes.get(f, 0) + nbytes[i]
            fam_count[f] = fam_count.get(f, 0) + 1
    dom = max(fam_time, key=fam_time.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    achieved = fam_bytes[dom] / (fam_time[dom] * 1e-3) / 1e9
    traffic = load_traffic(dom)
    step_bytes = sum(nbytes)
    value = world * NUM_OPS * args.steps / (total_ms * 1e-3)

    norm = qs.qs_calc_norm_or_trace(h).real

    e2e = None
    if not args.no_e2e:
        # Each step uploads its whole input from pinned host memory through
        # qs_set_amps, runs the circuit and reads the norm back, one after the
        # other.  (Overlapping the next upload with the circuit on a second
        # state was slower on GB300: measured with a 16 GiB upload, the copy
        # engine gets under 20 GB/s while the streaming kernels saturate HBM,
        # and beside the whole circuit the upload took 674 ms and lengthened
        # the circuit by 601 ms, against 81 ms for the upload alone.)
        pinned = torch.empty(1 << nq, dtype=torch.complex128, pin_memory=True)
        with torch.cuda.stream(stream):
            fresh = device_random_state(nq, device)
        stream.synchronize()
        pinned.copy_(fresh)
        del fresh
        h2d = 16 * (1 << nq) + sum(op_h2d_bytes(op) for op in ops)
        qs.qs_set_amps_ptr(h, pinned.data_ptr(), 0, 1 << nq)      # untimed warm-up step
        for op in ops:
            qs.apply_op(h, op)
        qs.qs_calc_norm_or_trace(h)
        K = max(1, min(args.steps, args.e2e_steps))
        ev_u0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ev_u1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        e_clocks = ClockSampler(local)
        e_clocks.start()
        barrier(world)
        torch.cuda.synchronize()
        e_start.record(stream)
        for k in range(K):
            ev_u0[k].record(stream)
            qs.qs_set_amps_ptr(h, pinned.data_ptr(), 0, 1 << nq)
            ev_u1[k].record(stream)
            for op in ops:
                qs.apply_op(h, op)
            out_norm = qs.qs_calc_norm_or_trace(h)     # device -> host read of the step's result
        e_end.record(stream)
        e_end.synchronize()
        barrier(world)
        e_clk = e_clocks.stop()
        e_total = max_over_ranks(e_start.elapsed_time(e_end), world, device)
        up_ms = [ev_u0[k].elapsed_time(ev_u1[k]) for k in range(K)]
        e2e = {"value": world * NUM_OPS * K / (e_total * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16,
               "upload_ms_per_step": sum(up_ms) / len(up_ms), "ms_per_step": e_total / K, "steps": K,
               "clocks": e_clk,
               "note": ("pinned host state uploaded through qs_set_amps every step (read by the library's copy "
                        "kernel from page-locked memory), %d ops, norm read back, in sequence on one device state"
                        % NUM_OPS),
               "final_norm": out_norm.real}

    fused = None
    extra = None
    sections["main_and_e2e"] = time.perf_counter() - t_sec
    single = rank == 0 and world == 1          # the comparisons run on one GPU only
    if (not args.no_fused or not args.no_extra) and single:
        st.close()
        del psi
        torch.cuda.empty_cache()
    if not args.no_fused and single:
        t_sec = time.perf_counter()
        fused = fused_comparison(args, device)
        sections["fused_c64_32q"] = time.perf_counter() - t_sec
    if not args.no_extra and single:
        extra = other_workloads(args, device, sections)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.arith],
            "data": "synthetic", "config": config_dict(nq, args),
            "hbm_gbs": step_bytes / (ms_per_step * 1e-3) / 1e9,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "time_share": fam_time[dom] / sum(fam_time.values())},
            "gpu_launches": NUM_OPS * args.steps,
            "clocks": clk,
            "final_norm": norm,
        }
        if e2e is not None:
            line["e2e"] = e2e
        if fused is not None:
            line["fused_tc"] = fused
        if extra is not None:
            line["other_workloads"] = extra
        line["bench_sections_s"] = sections
        if cpu_res is not None:
            line["cpu_baseline"] = cpu_baseline_dict(
                cpu_res, "the whole %d-op circuit of the same recipe on a %d-qubit complex128 state "
                         "(oracle/qsim_oracle.py, numpy, one thread; %.1f s); gates/s scaled to 30 qubits "
                         "by 2^(%d-30), the ratio of the bytes each operation streams"
                % (cpu_res["ops"], cpu_res["qubits"], cpu_res["seconds"], cpu_res["qubits"]))
        print(json.dumps(line), flush=True)
        detail = {f: {"launches": fam_count[f], "ms_total": fam_time[f],
                      "share": fam_time[f] / sum(fam_time.values()),
                      "gbs": fam_bytes[f] / (fam_time[f] * 1e-3) / 1e9} for f in fam_time}
        print("per-family: " + json.dumps(detail), file=sys.stderr)
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump({"line": line, "families": detail,
                           "per_op_ms": [[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(NUM_OPS)]
                                         for k in range(args.steps)],
                           "ops": [{"op": op["op"], "targs": op["targs"], "ctrls": op.get("ctrls", []),
                                    "family": fams[i]} for i, op in enumerate(ops)]}, f)
    if not ((not args.no_fused or not args.no_extra) and single):
        st.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Fused tensor-core form vs the plain per-gate FP64 form (same GPU)
# ---------------------------------------------------------------------------

FUSED_OPS = 1000


def fused_comparison(args, device, nq=None, prec=None, max_block=None):
    """The 1000-gate unitary circuit of the fused workload (1q Haar; 1-2-target
    Haar with 0-3 controls; gadgets of weight 1-6) on one random state: the
    plain per-gate form in complex128 (native FP64, and block fixed point,
    which is at least FP64-accurate) against cost-model-planned fused blocks
    on the tensor cores (complex64 with 3xTF32 blocks, or complex128 with
    eight-slice integer blocks).  Every timed run starts from the seeded
    initial state; times are medians of three runs after a warm-up on the
    first 20 gates, except native FP64 (one warmed run: about a minute at 32
    qubits).  The plan (cost-model DP and FP64 block composition) is timed
    apart from the fused runs.  1 - fidelity and max |delta amp| of the fused
    result are taken against both complex128 per-gate results."""
    import torch
    from paper_2311_01512_gb300 import costmodel, qs
    from paper_2311_01512_gb300 import workloads as wl
    nq = nq or args.fused_qubits
    c64 = (prec or args.fused_prec) == "c64"
    ops = wl.unitary_circuit(nq, FUSED_OPS, wl.rng_for("fused-tc-circuit"))
    stream = torch.cuda.Stream(device=device)

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def reset(dst):
        # the seeded initial state, written on the circuit's stream
        with torch.cuda.stream(stream):
            fill_random_state(dst, nq, device)
        stream.synchronize()

    def runs(dst, fn, n):
        out = []
        for _ in range(n):
            reset(dst)
            out.append(timed(fn))
        return out

    def per_gate(handle, tensor, arith, n):
        qs.qs_set_arithmetic(handle, arith)
        warm = qs.Circuit(nq, ops[:20])
        warm.plan(qs.QS_PLAN_NONE, 1)
        warm.apply(handle)
        warm.close()
        circ = qs.Circuit(nq, ops)
        circ.plan(qs.QS_PLAN_NONE, 1)
        t = runs(tensor, lambda: circ.apply(handle), n)
        circ.close()
        return t

    out = {"qubits": nq, "ops": FUSED_OPS, "fused_amp": "complex64" if c64 else "complex128"}
    with torch.cuda.stream(stream):
        r64 = torch.empty(1 << nq, dtype=torch.complex128, device=device)
        rfx = torch.empty_like(r64)
    stream.synchronize()
    s64 = qs.State(nq, prec=qs.QS_C128, stream=stream, storage=r64)
    sfx = qs.State(nq, prec=qs.QS_C128, stream=stream, storage=rfx)
    out["per_gate_f64_ms_runs"] = per_gate(s64.handle, r64, qs.QS_ARITH_F64, 1)
    out["per_gate_f64_ms"] = out["per_gate_f64_ms_runs"][0]
    out["per_gate_fx_ms_runs"] = per_gate(sfx.handle, rfx, qs.QS_ARITH_FX, 3)
    out["per_gate_fx_ms"] = statistics.median(out["per_gate_fx_ms_runs"])
    # fused form, planned by the learned cost model
    with torch.cuda.stream(stream):
        tf = torch.empty(1 << nq, dtype=torch.complex64 if c64 else torch.complex128, device=device)
    sf = qs.State(nq, prec=qs.QS_C64 if c64 else qs.QS_C128, stream=stream, storage=tf)
    model, meta = costmodel.load()
    circf = qs.Circuit(nq, ops)
    width = min(max_block or args.fused_max_block, 6 if c64 else 5)
    t0 = time.perf_counter()
    plan = circf.plan_cost(model, sf.handle, max_block_qubits=width, window=24)
    out["plan_ms"] = (time.perf_counter() - t0) * 1e3
    plan["max_block_qubits"] = width
    reset(tf)
    circf.apply(sf.handle)                                  # warm-up
    out["fused_ms_runs"] = runs(tf, lambda: circf.apply(sf.handle), 3)
    out["fused_ms"] = statistics.median(out["fused_ms_runs"])
    # lazy relabelling: SWAPs that move tensor-core blocks' qubits off the 5
    # lowest positions where the cost model predicts a saving above a SWAP
    # pass (1.2 one-target passes); kept as the fused form only if faster.
    # --relabel-ab also times forced relabelling (any predicted saving; every
    # low qubit), one warmed run each.
    if c64:
        if getattr(args, "relabel_ab", False):
            ab = {}
            for name, price in (("any_predicted_saving", 0.0), ("every_low_qubit", -1e30)):
                nsw = circf.plan_relabel(model, sf.handle, low_qubits=5, swap_passes=price)
                reset(tf)
                circf.apply(sf.handle)
                ab[name] = {"swaps": nsw, "ms": runs(tf, lambda: circf.apply(sf.handle), 1)[0]}
            out["relabel_ab"] = ab
        nsw = circf.plan_relabel(model, sf.handle, low_qubits=5, swap_passes=1.2)
        out["relabel_swaps"] = nsw
        if nsw:
            reset(tf)
            circf.apply(sf.handle)
            out["fused_relabel_ms_runs"] = runs(tf, lambda: circf.apply(sf.handle), 3)
            out["fused_relabel_ms"] = statistics.median(out["fused_relabel_ms_runs"])
            if out["fused_relabel_ms"] >= out["fused_ms"]:
                circf.plan_relabel(model, sf.handle, low_qubits=0)
                reset(tf)
                circf.apply(sf.handle)          # the result below: the faster form
            else:
                out["fused_ms_without_relabel"] = out["fused_ms"]
                out["fused_ms"] = out["fused_relabel_ms"]
    out["plan"] = plan
    out["plan_note"] = ("plan_ms: cost-model DP over the circuit and FP64 composition of the fused blocks on "
                        "the device, done once per circuit, outside fused_ms")
    out["costmodel_holdout_median_time_error"] = meta.get("holdout_median_abs_rel_time_error")
    out["costmodel_test_median_time_error"] = meta.get("test_median_abs_rel_time_error")
    # max |delta amp| and fidelity of the fused result (tf, one application
    # from the initial state) against both per-gate complex128 results, in
    # slices of 2^26 amplitudes
    for name, ref in (("f64", r64), ("fx", rfx)):
        dmax, ov, na, nb = 0.0, 0.0 + 0.0j, 0.0, 0.0
        step = 1 << min(26, nq)
        with torch.cuda.stream(stream):
            for i in range(0, 1 << nq, step):
                a = ref[i:i + step]
                b = tf[i:i + step].to(torch.complex128)
                dmax = max(dmax, float((a - b).abs().max().item()))
                ov += complex(torch.vdot(a, b).item())
                na += float(torch.vdot(a, a).real.item())
                nb += float(torch.vdot(b, b).real.item())
        stream.synchronize()
        out["max_abs_delta_amp_vs_" + name] = dmax
        out["one_minus_fidelity_vs_" + name] = 1.0 - abs(ov) ** 2 / (na * nb)
    out["one_minus_fidelity"] = out["one_minus_fidelity_vs_f64"]
    out["max_abs_delta_amp"] = out["max_abs_delta_amp_vs_f64"]
    out["reference"] = ("per-gate complex128 results from the same initial state: native FP64 (f64) and block "
                        "fixed point (fx, at least FP64; both oracle-checked at small sizes)")
    # unfused, same precision as the fused form (complex128: that is fx)
    if c64:
        circn = qs.Circuit(nq, ops)
        circn.plan(qs.QS_PLAN_NONE, 1)
        out["per_gate_same_prec_ms_runs"] = runs(tf, lambda: circn.apply(sf.handle), 3)
        out["per_gate_same_prec_ms"] = statistics.median(out["per_gate_same_prec_ms_runs"])
        circn.close()
    else:
        out["per_gate_same_prec_ms"] = out["per_gate_fx_ms"]
    out["speedup_vs_per_gate_f64"] = out["per_gate_f64_ms"] / out["fused_ms"]
    out["speedup_vs_per_gate_fx"] = out["per_gate_fx_ms"] / out["fused_ms"]
    for h in (s64, sfx, sf):
        h.close()
    circf.close()
    model.close()
    del r64, rfx, tf
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# The other workloads, each on its own (after the main state is freed)
# ---------------------------------------------------------------------------

def other_workloads(args, device, sections):
    """The density-matrix workloads (15 qubits: 400 operations, GB/s by kind;
    6 qubits: microseconds per operation, per call, recorded and batched),
    the 4096-state batch in complex64 and complex128 (gates/s, speedup over
    launching each circuit separately, 1 - fidelity of 8 sampled states), and
    the 31-qubit complex128 fused case.  A workload that fails is reported
    with its error instead of stopping the run."""
    import traceback
    import torch
    from paper_2311_01512_gb300 import batch_bench, dm_bench, qs
    from paper_2311_01512_gb300 import workloads as wl
    peak = None
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except Exception:
        pass
    jobs = [
        ("densmatr_15q_400ops", lambda: dm_bench.large(qs, wl, torch, peak, reps=3)),
        ("densmatr_6q_300ops", lambda: dm_bench.small(qs, wl, torch, 20)),
        ("batch_4096_c64", lambda: batch_bench.run(0, 4096, 3, True, 8)),
        ("batch_4096_c128", lambda: batch_bench.run(1, 4096, 3, True, 8)),
        ("fused_c128_31q", lambda: fused_comparison(args, device, nq=31, prec="c128", max_block=5)),
    ]
    out = {}
    for name, fn in jobs:
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:          # reported, not hidden: the error text goes into the line
            out[name] = {"error": "%s: %s" % (type(e).__name__, e), "trace": traceback.format_exc()[-1500:]}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        sections[name] = time.perf_counter() - t0
    return out


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle on a bounded sample, on the host cores
# ---------------------------------------------------------------------------

REF_OPS_PER_STEP = 100


def main_reference(args):
    """The CPU oracle as it stands on the host cores, one thread: the same
    500-op circuit recipe at CPU_SAMPLE_QUBITS, REF_OPS_PER_STEP successive
    operations per step (step k applies operations k*100 .. k*100+99 of the
    circuit, cycling through it), on one evolving state."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for k, v in one_thread_env().items():
        os.environ[k] = v
    from oracle import qsim_oracle as orc
    from paper_2311_01512_gb300 import workloads as wl
    nq = CPU_SAMPLE_QUBITS
    ops = make_ops(nq)
    psi = wl.random_statevector(nq, wl.rng_for("cpu-sample"))
    m = REF_OPS_PER_STEP

    def step(k):
        first = (k * m) % NUM_OPS
        return orc.run_ops(psi, ops[first:first + m], is_density=False)

    for k in range(args.warmup):
        psi = step(k)
    secs = 0.0
    for k in range(args.warmup, args.warmup + args.steps):
        t0 = time.perf_counter()
        psi = step(k)
        secs += time.perf_counter() - t0
    value = m * args.steps / secs * 2.0 ** (nq - 30)
    first_op = (args.warmup * m) % NUM_OPS
    sample = ("%d timed steps of %d successive operations each (operations %d onward of the %d-op circuit, "
              "cycling) on a %d-qubit complex128 state after %d warm-up steps; oracle/qsim_oracle.py, numpy, "
              "one thread, %.1f s; gates/s scaled to 30 qubits by 2^(%d-30)"
              % (args.steps, m, first_op, NUM_OPS, nq, args.warmup, secs, nq))
    cb = cpu_baseline_dict({"value_30q_equiv": value}, sample)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (numpy f64)",
            "data": "synthetic", "config": config_dict(30, args), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_sample:
        cpu_sample_main(args.cpu_sample)
        return
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
