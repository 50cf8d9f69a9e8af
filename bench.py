"""Throughput benchmark: MPS simulation of a parameterised ansatz plus its
Pauli-sum energy, at chi=128 on 40 qubits.

One step = the whole hot path for one batch of parameter vectors:
reset to |0...0>, apply the 10-layer Ry/Rz + CNOT-ladder ansatz (390
two-qubit gates per state, the middle bonds saturate at chi=128 after 7
layers), then evaluate E(theta) = sum_k c_k <P_k> over the 157-term
Heisenberg chain for every state.

Prints ONE JSON line. ``value`` = Pauli-term expectations per second
(whole job: states x terms / step time, the state simulation included);
``gates_per_s`` = two-qubit gate applications per second; the dominant
kernel's roofline (the one-sided Jacobi SVD) is measured live with CUDA
events on the library's stream, against the FP32 (or FP64) FMA rate measured
in the same run by the library's peak kernel (``alu_peaks``).
``random_terms`` reports the metric's second term set (2000 random strings of
weight <= 4) as one expectation pass over the final states, with the
tensor-core sweep kernel's roofline. ``accuracy`` compares the line's energy
of theta row 0 with the FP64 oracle on the same row (target |dE| <= 1e-6
sum|c_k|). ``fp64_form`` times one step of the plain FP64 form (complex128
everywhere) on the same workload, with its own roofline and accuracy.

  python bench.py [--gpus N --steps K --warmup W] [--dtype c64_bf16split|c64|c128] [--batch B]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)
Under torchrun each rank simulates its own batch (replicas; weak scaling).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1807_07914_gb300 import inputs  # noqa: E402

METRIC = "Pauli-term expectations/sec and gates/sec at chi=128, 40 qubits; % roofline"
UNIT = "expectations/s"

def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def profiled_traffic(name, key="traffic_bytes"):
    """DRAM bytes (read + write) of a kernel from its committed ncu summary in
    profiles/: the figures of its machine-readable lines, kept only while the
    sha256 of the kernel's sources equals the one recorded with the capture
    (a changed kernel has no traffic figure until it is captured again)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ":" in ln and ln.split(":", 1)[0].strip() in (
                key, "traffic_unit", "sources", "sources_sha256"):
            k, v = ln.split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if not {key, "sources", "sources_sha256"} <= kv.keys():
        return None
    h = hashlib.sha256()
    for src in kv["sources"].split():
        try:
            h.update(open(os.path.join(ROOT, src), "rb").read())
        except OSError:
            return None
    if h.hexdigest() != kv["sources_sha256"]:
        return None
    return {"bytes": float(kv[key]), "unit": kv.get("traffic_unit", "per launch"),
            "source": "profiles/" + name}


def workload_cfg(args):
    wl = inputs.workload("chi128", rep=args.rank_seed)
    n, chi, eps = wl["n"], wl["chi_max"], wl["eps"]
    return wl, n, chi, eps


def config_dict(args, n, chi, B, P, T, state_bytes):
    return {
        "workload": f"hea40_chi128: n={n}, 10 layers (Ry,Rz on every qubit; CNOT ladder), "
                    f"chi_max={chi}, cutoff 1e-10, {B} theta/GPU, Heisenberg chain {T} terms",
        "n_qubits": n, "chi_max": chi, "layers": 10, "params": P, "batch_per_gpu": B,
        "terms": T, "gates2q_per_state": 390,
        "l2": f"inputs larger than L2 (state arena {state_bytes / 2**30:.2f} GiB per GPU)",
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ distributed
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x, ws, device=None):
    """Max of a float over ranks (timing only; not on the data path)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, ws, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(wl, n_theta=1, n_terms=None, energies=None):
    """Time the FP64 oracle (as it stands) on a bounded sample of the same
    workload: the full circuit for n_theta parameter rows and the per-term
    energy sweeps. Returns (seconds, states, terms_per_state, gates); the
    energies of the rows are appended to ``energies`` when given."""
    from oracle import mps as OM
    terms = wl["terms"] if n_terms is None else wl["terms"][:n_terms]
    t0 = time.perf_counter()
    gates = 0
    for b in range(n_theta):
        m = OM.MPS(wl["n"], wl["chi_max"], wl["eps"]).run(wl["circuit"], wl["thetas"][b])
        gates += len(m.step_weights)
        e = 0.0
        for c, s, p in terms:
            e += c * m.expect_pauli(s, p).real
        if energies is not None:
            energies.append(e)
    return time.perf_counter() - t0, n_theta, len(terms), gates


def blas_threads():
    for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            return int(os.environ[k])
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return int(max(i.get("num_threads", 1) for i in info))
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(wl, energies=None):
    dt, states, T, gates = oracle_sample(wl, 1, energies=energies)
    out = {"value": states * T / dt, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "gates_per_s": gates / dt,
           "sample": f"FP64 oracle (numpy/LAPACK) on 1 of the theta rows: full 390-gate "
                     f"circuit + {T} per-term sweeps, {dt:.1f} s"}
    one = cpu_baseline_one_thread()
    if one is not None:
        out["one_thread"] = one
    return out


def cpu_baseline_one_thread():
    """The same oracle sample with one BLAS thread: the reference arm run in a
    child process whose thread pools are limited by the environment."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference",
                            "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                           text=True, timeout=600)
        line = json.loads(r.stdout.strip().splitlines()[-1])
        return {"value": line["value"], "unit": line["unit"], "cores": 1,
                "ms_per_sample": line["ms_per_step"]}
    except (OSError, ValueError, IndexError, KeyError, subprocess.SubprocessError):
        return None


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    wl, n, chi, eps = workload_cfg(args)
    for _ in range(args.warmup):
        oracle_sample(wl, 1)
    times = []
    tot_terms = 0
    for _ in range(args.steps):
        dt, states, T, gates = oracle_sample(wl, 1)
        times.append(dt)
        tot_terms += states * T
    tot = sum(times)
    v = tot_terms / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(config_dict(args, n, chi, args.batch, wl["n_params"], len(wl["terms"]), 0),
                       l2="host oracle: the FP64 MPS of one state at a time in host memory"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                         "sample": f"per step: 1 of the {args.batch} theta rows of the workload, "
                                   "full circuit + all terms"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def random_terms_pass(args, m, wl, energy, stream, ws, device, chunk):
    """One timed expectation pass of the 2000 random strings over the batch's
    final states; the environment updates' algorithmic flops come from the
    library's counters and the sweep GEMMs are event-timed on its stream."""
    import torch
    from paper_1807_07914_gb300 import tnmps
    ps = tnmps.PauliSum(wl["n"], wl["terms_random"])
    T = len(wl["terms_random"])
    m.expect_dev(ps, energy, chunk=chunk)       # warm-up: workspace, plan upload
    torch.cuda.synchronize(device)
    s0 = m.stats()
    m.profile(("env", "env_tc"))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.expect_dev(ps, energy, chunk=chunk)
    e1.record(stream)
    torch.cuda.synchronize(device)
    prof = m.profile_read()
    m.profile(None)
    s1 = m.stats()
    m.check()
    t = reduce_max(e0.elapsed_time(e1) / 1000.0, ws, device)
    flops = s1["env_flops"] - s0["env_flops"]
    out = {"terms": T, "weight_max": 4, "chunk": chunk,
           "value": reduce_sum(m.batch, ws, device) * T / t, "unit": UNIT, "ms_per_pass": 1000 * t,
           "env_updates": s1["env_updates"] - s0["env_updates"],
           "env_alg_tflops": flops / t / 1e12}
    peaks = load_peaks()
    if args.dtype == "c64_bf16split":
        tc_ms = prof["env_tc"][0]
        alg = flops / (tc_ms / 1000.0) / 1e12
        peak = float(peaks.get("bf16_tflops", 1933.1))
        out["roofline"] = {
            "kernel": "k_swtc (transfer-sweep GEMM steps on tcgen05, BF16 split)",
            "bound": "tensor", "achieved": alg, "peak": peak, "unit": "TFLOP/s",
            "frac": alg / peak, "traffic": None, "gemm_ms": tc_ms,
            "executed_tflops": 3 * alg, "executed_frac": 3 * alg / peak,
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)",
            "note": "achieved = algorithmic complex-GEMM flops (4 real MACs per complex MAC); "
                    "executed = 3 x (hi*hi + hi*lo + lo*hi), padding to 32-wide tiles not counted"}
        fused = m.get_tuning()["sweep_fused"] == 1
        tr = profiled_traffic("k_swtc_bf16split_chi128_8states.md",
                              "traffic_bytes_fused" if fused else "traffic_bytes")
        out["sweep_form"] = "fused (k_sweep_fused)" if fused else "two launches per level"
        if tr is not None:
            upd = out["env_updates"]
            out["roofline"]["traffic"] = tr["bytes"] * upd
            out["roofline"]["traffic_source"] = (
                tr["source"] + f": {tr['bytes'] / 1e3:.0f} KB of DRAM {tr['unit']} (ncu, one "
                "trie level of 8 states) x the node-state updates of this pass")
            # algorithmic: the parent environment read and the new one written (BF16 hi/lo
            # row-K form, 128 KB each at chi = 128) per update
            out["roofline"]["alg_bytes"] = 2 * 131072 * upd
            out["roofline"]["traffic_over_alg_bytes"] = tr["bytes"] / (2 * 131072)
    return out


def measure_alu_peaks(device):
    """FMA throughput of the CUDA cores in FP32 and FP64 (the ceilings of the
    Jacobi SVD), from the library's peak kernel: full occupancy (8 CTAs of
    256 threads per SM), best of 5 event-timed launches after 2 warm-ups."""
    import torch
    from paper_1807_07914_gb300 import tnmps
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = 8 * sms
    out = {}
    for bits, iters, dt in ((32, 40000, torch.float32), (64, 600, torch.float64)):
        sink = torch.empty(blocks * 256, dtype=dt, device=device)
        stream = torch.cuda.current_stream(device)
        for _ in range(2):
            flops = tnmps.alu_peak_dev(bits, blocks, iters, sink)
        best = None
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tnmps.alu_peak_dev(bits, blocks, iters, sink)
            e1.record(stream)
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out[f"fp{bits}_tflops"] = flops / (best / 1000.0) / 1e12
        out[f"fp{bits}_ms"] = best
    out["how"] = (f"tnmps_alu_peak_dev: {blocks} CTAs x 256 threads, 8 independent FMA chains "
                  "per thread, 2 flop per FMA, best of 5 event-timed launches")
    return out


def jacobi_roofline(st, prof_jac, steps, t_local, peak, peak_src, prof_lq=None):
    """The Jacobi SVD's roofline object: algorithmic flops per launch (device
    counters) over its average event-timed launch duration; with prof_lq, the
    event-timed share of the LQ factorisation that precedes each Jacobi."""
    jac_ms, jac_n = prof_jac
    alg_flops = 8 * st["jacobi_pair_rows"] + 18 * st["jacobi_rot_rows"]
    exe_flops = 16 * st["jacobi_pair_rows"] + 18 * st["jacobi_rot_rows"]
    launches_per_step = jac_n / steps
    avg_launch_s = jac_ms / 1000.0 / max(jac_n, 1)
    per_launch_alg = alg_flops / max(launches_per_step, 1)
    achieved = per_launch_alg / avg_launch_s / 1e12
    alg_bytes = st["jacobi_alg_bytes"] / max(launches_per_step, 1)
    return {"kernel": "k_jacobi (one-sided Jacobi SVD, K3)", "bound": "alu",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "alg_bytes_per_launch": alg_bytes, "peak_source": peak_src,
            "executed_tflops": exe_flops / max(launches_per_step, 1) / avg_launch_s / 1e12,
            "alg_flops_per_launch": per_launch_alg, "avg_launch_ms": 1000 * avg_launch_s,
            "share_of_step": jac_ms / steps / (1000 * t_local / steps),
            "sweeps_per_svd": st["jacobi_sweeps"] / max(st["svds"], 1),
            "preconditioner": None if not prof_lq or not prof_lq[1] else {
                "kernel": "k_lq_theta (Theta = L Q^H, Householder QR of Theta^H; the Jacobi "
                          "runs on L)",
                "ms_per_step": prof_lq[0] / steps, "launches_per_step": prof_lq[1] / steps,
                "share_of_step": prof_lq[0] / steps / (1000 * t_local / steps)}}


def accuracy(e_gpu, e_oracle, terms):
    if e_oracle is None:
        return None
    scale = sum(abs(t[0]) for t in terms)
    d = abs(float(e_gpu) - float(e_oracle))
    return {"theta_row": 0, "energy": float(e_gpu), "energy_oracle": float(e_oracle),
            "abs_dE": d, "rel_to_sum_abs_c": d / scale, "target_rel": 1e-6,
            "oracle": "FP64 oracle MPS (LAPACK SVD, rule R, per-term full sweeps) on the same row"}


def fp64_form(args, wl, th_row0, e_oracle, alu, device):
    """The plain FP64 form (complex128 state, FP64 Jacobi, sweeps and split)
    on the same workload: one timed step of 152 states (one SVD per SM), the
    kernels loaded first by a one-layer warm-up circuit."""
    import torch
    from paper_1807_07914_gb300 import tnmps
    n, chi, P, T = wl["n"], wl["chi_max"], wl["n_params"], len(wl["terms"])
    B = args.fp64_batch
    th = inputs.thetas(B, P, inputs.rng_for(5, 200))
    th[0] = th_row0
    m = tnmps.MPSBatch(n, chi, B, dtype="c128", max_params=P, eps=wl["eps"], device=device)
    ps = tnmps.PauliSum(n, wl["terms"])
    th_dev = torch.tensor(th, dtype=torch.float64, device=device)
    energy = torch.empty(B, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    warm, _ = inputs.hea_circuit(n, 1, ("RY", "RZ"))
    m.apply_circuit_dev(tnmps.gate_array(warm), th_dev)
    m.expect_dev(ps, energy)
    torch.cuda.synchronize(device)
    gates_c = tnmps.gate_array(wl["circuit"])
    m.reset()
    m.profile(("jacobi", "svd_lq"))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    m.apply_circuit_dev(gates_c, th_dev)
    m.expect_dev(ps, energy)
    e1.record(stream)
    torch.cuda.synchronize(device)
    prof = m.profile_read()
    m.profile(None)
    m.check()
    st = m.stats()
    t = e0.elapsed_time(e1) / 1000.0
    roof = jacobi_roofline(st, prof["jacobi"], 1, t, alu["fp64_tflops"],
                           "measured FP64 FMA rate (tnmps_alu_peak_dev, this run)",
                           prof["svd_lq"])
    return {"dtype": "c128", "batch": B, "steps": 1, "ms_per_step": 1000 * t,
            "value": B * T / t, "unit": UNIT, "gates_per_s": B * 390 / t,
            "gates_chi128_per_s": st["gates2q_full"] / t, "roofline": roof,
            "accuracy": accuracy(energy[0].item(), e_oracle, wl["terms"])}


def run_gpu(args):
    import torch
    ws, rank, local = dist_setup()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    from paper_1807_07914_gb300 import tnmps

    args.rank_seed = rank
    wl, n, chi, eps = workload_cfg(args)
    B = args.batch
    P = wl["n_params"]
    th = inputs.thetas(B, P, inputs.rng_for(5, 100 + rank))
    if rank == 0:
        th[0] = wl["thetas"][0]        # the row the CPU baseline and the accuracy check sample
    terms = wl["terms"]
    T = len(terms)
    alu = measure_alu_peaks(device)
    m = tnmps.MPSBatch(n, chi, B, dtype=args.dtype, max_params=P, eps=eps, device=device)
    if args.dtype != "c128":
        m.set_svd_tolerance(args.svd_tolerance)
    m.set_svd_precondition(args.svd_precondition)
    ps = tnmps.PauliSum(n, terms)
    gates_c = tnmps.gate_array(wl["circuit"])
    th_dev = torch.tensor(th, dtype=torch.float64, device=device)
    energy = torch.empty(B, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    # ---- launch shapes picked by the autotuner on this workload (untimed)
    heis_chunk, rand_chunk, tune = 0, args.random_chunk, None
    if not args.no_tune:
        from paper_1807_07914_gb300 import autotune
        sets = {"heisenberg": ps}
        if not args.no_random_terms:
            sets["random"] = tnmps.PauliSum(n, wl["terms_random"])
        rep = autotune.tune_context(m, gates_c, th_dev, sets)
        heis_chunk = rep["chunk"]["heisenberg"]
        rand_chunk = rep["chunk"].get("random", args.random_chunk)
        ex = rep["expect_s"]["heisenberg"]["candidates_s"]
        d_key = "0" if "0" in ex else max(ex, key=int)   # the whole batch when it fits
        default_s = rep["circuit_s"]["default"] + ex[d_key]
        tuned_s = rep["circuit_s"]["tuned"] + ex[str(heis_chunk)]
        tune = {"tuning": rep["tuning"], "chunk": rep["chunk"], "cached": rep["cached"],
                "default_step_s": default_s, "tuned_step_s": tuned_s,
                "gain": default_s / tuned_s, "trials": rep["trials"],
                "expect_candidates_s": {k: v["candidates_s"] for k, v in rep["expect_s"].items()},
                "how": rep["how"] + "; default = all shapes 0, Heisenberg chunk = whole batch, "
                                    f"random-string chunk = {args.random_chunk}"}
        if "random" in rep["expect_s"]:
            rc = rep["expect_s"]["random"]["candidates_s"]
            if str(args.random_chunk) in rc:
                tune["random_pass_gain"] = rc[str(args.random_chunk)] / rc[str(rand_chunk)]
        del sets

    def step(ev=None):
        if ev is not None:  # timed steps sit in an NVTX range (launch lists filter on it)
            torch.cuda.nvtx.range_push("bench_step")
        m.reset()
        if ev is not None:
            ev[0].record(stream)
        m.apply_circuit_dev(gates_c, th_dev)
        if ev is not None:
            ev[1].record(stream)
        m.expect_dev(ps, energy, chunk=heis_chunk)
        if ev is not None:
            ev[2].record(stream)
            torch.cuda.nvtx.range_pop()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)
    m.check()
    # ---- timed region (device time, inputs resident in HBM)
    st0 = m.stats()
    clocks = ClockSampler(local)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(device)
    clocks.start()
    time.sleep(0.3)
    m.profile(tnmps.PROF_CLASSES if args.profile_all else ("jacobi", "svd_lq"))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize(device)
    prof = m.profile_read()
    m.profile(None)
    clk = clocks.stop()
    if ws > 1:
        dist.barrier()
    st1 = m.stats()
    m.check()
    e_row0 = energy[0].item()
    t_local = start.elapsed_time(end) / 1000.0
    circ_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    exp_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    t = reduce_max(t_local, ws, device)
    launches_step = (st1["launches"] - st0["launches"]) / args.steps
    total_states = reduce_sum(B, ws, device) * args.steps
    value = total_states * T / t
    gates_per_s = total_states * 390 / t
    full_per_step = st1["gates2q_full"]
    # ---- dominant kernel: one-sided Jacobi (counters of the last step)
    if args.dtype != "c128":
        peak, peak_src = alu["fp32_tflops"], "measured FP32 FMA rate (tnmps_alu_peak_dev, this run)"
    else:
        peak, peak_src = alu["fp64_tflops"], "measured FP64 FMA rate (tnmps_alu_peak_dev, this run)"
    roof = jacobi_roofline(st1, prof["jacobi"], args.steps, t_local, peak, peak_src,
                           prof["svd_lq"])
    tr = profiled_traffic("k_jacobi_bench_step_304states_dram.md")
    if (tr is not None and args.dtype == "c64_bf16split" and B == 304
            and args.svd_precondition == 1):
        roof["traffic"] = tr["bytes"]
        roof["traffic_over_alg_bytes"] = tr["bytes"] / roof["alg_bytes_per_launch"]
        roof["traffic_source"] = (tr["source"] + ": ncu dram__bytes_read.sum + "
                                  "dram__bytes_write.sum, every Jacobi launch of one timed step, "
                                  "averaged per launch")
    # ---- end to end through the public host API (pinned host buffers)
    th_pin = torch.tensor(th, dtype=torch.float64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m.reset()
        m.apply_circuit(wl["circuit"], th_pin.numpy())
        e_host = m.expect(ps, chunk=heis_chunk)
    t_e2e = reduce_max(time.perf_counter() - t0, ws, device)
    e2e = {"value": reduce_sum(B, ws, device) * e2e_steps * T / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": int(B * P * 8), "d2h_bytes_per_step": int(B * 8),
           "steps": e2e_steps}
    assert np.all(np.isfinite(e_host))
    # ---- the second term set of the metric: 2000 random strings of weight <= 4
    # on the final states (expectation phase alone, states resident)
    rand = None if args.no_random_terms else random_terms_pass(args, m, wl, energy, stream, ws,
                                                                device, rand_chunk)
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.dtype, "data": "synthetic",
            "config": dict(config_dict(args, n, chi, B, P, T, m.arena.numel()),
                           svd_tolerance_factor=args.svd_tolerance if args.dtype != "c128"
                           else 1.0, svd_precondition=args.svd_precondition),
            "gates_per_s": gates_per_s,
            "gates_chi128_per_s": reduce_sum(full_per_step, ws, device) * args.steps / t,
            "phases_ms": {"circuit": circ_ms, "expect": exp_ms},
            "expectations_per_s_sweep_phase": B * T / (exp_ms / 1000.0),
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches_step * args.steps),
            "clocks": clk, "alu_peaks": alu,
        }
        if tune is not None:
            line["autotune"] = tune
        if rand is not None:
            line["random_terms"] = rand
        if args.profile_all:
            line["class_ms_per_step"] = {k: v[0] / args.steps for k, v in prof.items()}
    del m
    # ---- accuracy of this line against the FP64 oracle on theta row 0, the
    # oracle timed on the host cores, and the plain FP64 form
    e_oracle = None
    if rank == 0:
        energies = []
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, energies)
        elif not args.no_accuracy:
            oracle_sample(wl, 1, energies=energies)
        e_oracle = energies[0] if energies else None
        line["accuracy"] = accuracy(e_row0, e_oracle, terms)
    if not args.no_fp64_form and rank == 0:
        line["fp64_form"] = fp64_form(args, wl, wl["thetas"][0], e_oracle, alu, device)
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--dtype", choices=("c64_bf16split", "c64", "c128"), default="c64_bf16split",
                    help="c64_bf16split: complex64 state, FP32 Jacobi with FP64 Gram, sweeps on "
                         "the tensor cores (BF16 split); c64: FP32 CUDA-core sweeps; c128: FP64")
    ap.add_argument("--no-random-terms", action="store_true",
                    help="skip the pass over the 2000 random strings")
    ap.add_argument("--random-chunk", type=int, default=32,
                    help="states per expectation chunk of the random-string pass (untuned default)")
    ap.add_argument("--svd-precondition", type=int, default=1, choices=(0, 1),
                    help="1: the Jacobi SVD runs on L of Theta = L Q^H (default); 0: on Theta")
    ap.add_argument("--svd-tolerance", type=float, default=64.0,
                    help="factor on the Jacobi orthogonality tolerance of the complex64 forms "
                         "(1 = rounding level; 64 keeps the energies at the same accuracy "
                         "against the FP64 oracle with 5 %% fewer sweeps)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch shapes (skip the autotuner)")
    ap.add_argument("--batch", type=int, default=304,
                    help="theta rows per GPU (default 2 x 152 SMs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the FP64 oracle energy of theta row 0 (with --no-cpu-baseline)")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="skip the one-step measurement of the plain FP64 (complex128) form")
    ap.add_argument("--fp64-batch", type=int, default=152,
                    help="states of the FP64-form step (default one per SM)")
    ap.add_argument("--profile-all", action="store_true",
                    help="time every kernel class with events (diagnostic; adds overhead)")
    args = ap.parse_args()
    args.rank_seed = 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
