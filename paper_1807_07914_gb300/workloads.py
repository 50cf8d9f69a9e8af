"""Measurements of the other workload shapes on one GPU, one JSON line each.

  python -m paper_1807_07914_gb300.workloads large100 [--dtype c64_bf16split] [--oracle]
  python -m paper_1807_07914_gb300.workloads rounds [--circuits 10] [--eps 1e-4] [--chi 64]
  python -m paper_1807_07914_gb300.workloads sample [--shots 1024] [--batch 304]
  python -m paper_1807_07914_gb300.workloads supergate [--batch 304] [--sweeps 3] [--oracle]

``large100``: the 100-qubit single state (6 Ry/Rz + CNOT-ladder layers, 1200
parameters, chi_max 256, cutoff 1e-8) and its 5000 random strings of weight
<= 4: circuit time, expectation pass time, bond dimensions; with ``--oracle``
the FP64 oracle is timed on the 20-term subset and its energy compared.

``rounds``: the random-circuit workload of Sec. V.A (round 1 starts with H on
every qubit; each round is a layer of random single-qubit gates followed by
nearest-neighbour CNOTs), for 5..85 qubits in steps of 5 and 2..10 rounds in
steps of 2, ``--circuits`` circuits each, at the paper's default cutoff 1e-4
and a bond cap of ``--chi``: the largest bond dimension, the MPS storage in
bytes (the paper's memory metric) and two-qubit gates per second (one circuit
per launch sequence, so small registers are launch-latency bound).

``sample``: measurement shots of all 40 qubits from the chi=128 benchmark
states (10 ansatz layers), ``--shots`` per state: shots per second.

``supergate``: a six-qubit super-gate (distant CNOT/CZ, a SWAP, rotations)
applied by overlap maximisation (Sec. II general gate action) to the chi=128
benchmark states at chi_max 128 with a fixed number of sweeps: fits per
second, the fidelity of the first iterate (gates one by one with truncation)
and after the sweeps, per-class time shares and the FP32 rate of the fit
GEMMs; with ``--oracle`` the FP64 oracle fits state 0 (time and fidelities).
"""
import argparse
import json
import time

import numpy as np
import torch

from . import inputs, tnmps

ESIZE = {"c128": 16, "c64": 8, "c64_bf16split": 8}


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def large100(a):
    wl = inputs.workload("large100")
    th = torch.tensor(wl["thetas"][:1], dtype=torch.float64, device="cuda")
    m = tnmps.MPSBatch(wl["n"], wl["chi_max"], 1, dtype=a.dtype, max_params=wl["n_params"],
                       eps=wl["eps"])
    gates = tnmps.gate_array(wl["circuit"])
    ps = tnmps.PauliSum(wl["n"], wl["terms"])
    energy = torch.empty(1, dtype=torch.float64, device="cuda")
    for _ in range(2):  # warm-up
        m.reset()
        m.apply_circuit_dev(gates, th)
        m.expect_dev(ps, energy)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e2, e3 = _events()
    m.reset()
    s0 = m.stats()
    e0.record()
    m.apply_circuit_dev(gates, th)
    e1.record()
    e2.record()
    m.expect_dev(ps, energy)
    e3.record()
    torch.cuda.synchronize()
    m.check()
    s1 = m.stats()
    t_circ, t_exp = e0.elapsed_time(e1) / 1e3, e2.elapsed_time(e3) / 1e3
    dims = m.bond_dims()[0]
    out = {"workload": "large100: n=100, 6 layers Ry/Rz + CNOT ladder, chi_max 256, cutoff 1e-8, "
                       "5000 strings of weight <= 4, 1 state",
           "dtype": a.dtype, "circuit_s": t_circ, "expect_s": t_exp,
           "expectations_per_s": len(wl["terms"]) / t_exp,
           "env_alg_tflops": (s1["env_flops"] - s0["env_flops"]) / t_exp / 1e12,
           "max_bond": int(dims.max()), "energy": float(energy[0])}
    if a.oracle:
        from oracle import energy as OE
        sub = wl["terms"][:20]
        t0 = time.perf_counter()
        vals, _ = OE.term_values_mps(wl["n"], wl["circuit"], wl["thetas"][0], sub,
                                     wl["chi_max"], wl["eps"])
        t_or = time.perf_counter() - t0
        e20, pt = m.expect(tnmps.PauliSum(wl["n"], sub), per_term=True)
        out["oracle_20_terms_s"] = t_or
        out["oracle_20_expectations_per_s"] = 20 / t_or
        out["max_abs_dterm_20"] = float(np.max(np.abs(pt[0] - vals)))
        out["dE_20_rel_sum_abs_c"] = float(abs(e20[0] - OE.energy_from_values(sub, vals)) /
                                           sum(abs(t[0]) for t in sub))
    print(json.dumps(out))


def rounds(a):
    res = []
    for n in range(5, 90, 5):
        for r in range(2, 12, 2):
            maxb, bytes_, t, g2 = 0, [], 0.0, 0
            for k in range(a.circuits):
                rng = np.random.default_rng(10000 * n + 100 * r + k)
                circ = inputs.rounds_circuit(n, r, rng)
                m = tnmps.MPSBatch(n, a.chi, 1, dtype=a.dtype, max_params=0, eps=a.eps)
                e0, e1 = _events()
                e0.record()
                m.apply_circuit(circ, None)
                e1.record()
                torch.cuda.synchronize()
                m.check()
                t += e0.elapsed_time(e1) / 1e3
                g2 += sum(1 for gt in circ if gt[0] == "CNOT")
                d = np.concatenate([[1], m.bond_dims()[0], [1]])
                maxb = max(maxb, int(d.max()))
                bytes_.append(int(np.sum(d[:-1] * 2 * d[1:])) * ESIZE[a.dtype])
            res.append({"n": n, "rounds": r, "max_bond": maxb, "mps_bytes_mean": float(np.mean(bytes_)),
                        "mps_bytes_max": int(np.max(bytes_)), "gates2q_per_s": g2 / t})
    print(json.dumps({"workload": f"Sec. V.A rounds circuits, {a.circuits} per (n, rounds), "
                                  f"cutoff {a.eps}, chi cap {a.chi}, {a.dtype}", "rows": res}))


def sample(a):
    wl = inputs.workload("chi128")
    B, T = a.batch, a.shots
    th = torch.tensor(inputs.thetas(B, wl["n_params"], inputs.rng_for(5, 7)), dtype=torch.float64,
                      device="cuda")
    m = tnmps.MPSBatch(40, 128, B, dtype=a.dtype, max_params=wl["n_params"], eps=wl["eps"])
    m.apply_circuit_dev(tnmps.gate_array(wl["circuit"]), th)
    u = torch.rand((B, T, 40), dtype=torch.float64, device="cuda",
                   generator=torch.Generator(device="cuda").manual_seed(1))
    bits = torch.empty((B, T, 40), dtype=torch.uint8, device="cuda")
    m.sample_dev(u, bits)  # warm-up (also moves the centre to the last site)
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    m.sample_dev(u, bits)
    e1.record()
    torch.cuda.synchronize()
    m.check()
    t = e0.elapsed_time(e1) / 1e3
    print(json.dumps({"workload": f"{B} chi=128 states (40 qubits, 10 layers), {T} shots each, "
                                  "all 40 qubits measured", "dtype": a.dtype, "seconds": t,
                      "shots_per_s": B * T / t, "max_bond": int(m.bond_dims().max()),
                      "mean_ones": float(bits.float().mean())}))


def _fit_flops(F, P, w, p, q):
    """Real flops of the fit GEMMs of one state: one overlap pass and one sweep
    (8 flops per complex MAC). F, P: bond dimensions of phi and psi indexed by
    bond + 1 (bond -1 .. n-1); phi's are those after the fit (a sweep after the
    first sees them)."""
    def wb(bond):
        return int(w[bond + 1 - p])

    f = lambda bond: int(F[bond + 1])
    d = lambda bond: int(P[bond + 1])

    def left(i):  # T1, T2, EnvL at site i
        fa = f(i - 1)
        return 8 * (fa * wb(i - 1) * 2 * d(i) * d(i - 1) + 2 * wb(i) * fa * d(i) * 2 * wb(i - 1) +
                    f(i) * wb(i) * d(i) * 2 * fa)

    def right(i):  # V1, V2, EnvR at site i
        return 8 * (2 * d(i - 1) * f(i) * wb(i) * d(i) + 2 * wb(i - 1) * d(i - 1) * f(i) * 2 * wb(i) +
                    f(i - 1) * wb(i - 1) * d(i - 1) * 2 * f(i))

    def grad(i):  # T1..T4 and Theta at the pair (i, i+1)
        fa = f(i - 1)
        return 8 * (fa * wb(i - 1) * 2 * d(i) * d(i - 1) + 2 * wb(i) * fa * d(i) * 2 * wb(i - 1) +
                    fa * 2 * wb(i) * 2 * d(i + 1) * d(i) +
                    2 * wb(i + 1) * 2 * fa * d(i + 1) * 2 * wb(i) +
                    4 * fa * f(i + 1) * wb(i + 1) * d(i + 1))

    env_l = lambda i: 8 * f(i) * wb(i) * d(i) * 2 * f(i - 1)
    overlap = sum(left(i) for i in range(p, q + 1))
    sweep = (sum(right(i) for i in range(q, p + 1, -1)) +
             sum(grad(i) + env_l(i) for i in range(p, q)) + left(q))
    return overlap, sweep


def supergate(a):
    wl = inputs.workload("chi128")
    B, P = a.batch, wl["n_params"]
    th = inputs.thetas(B, P, inputs.rng_for(5, 12))
    th[0] = wl["thetas"][0]  # the row the oracle fits
    th = torch.tensor(th, dtype=torch.float64, device="cuda")
    m = tnmps.MPSBatch(40, 128, B, dtype=a.dtype, max_params=P, eps=wl["eps"])
    gates = tnmps.gate_array(wl["circuit"])
    block, bth = inputs.supergate_block(a.first, inputs.rng_for(5, 11))
    sg = tnmps.Supergate(40, block, bth)
    kw = dict(chi_max=128, target=1e-10, tol=-1.0, max_sweeps=a.sweeps)

    def fresh():
        m.reset()
        m.apply_circuit_dev(gates, th)
        torch.cuda.synchronize()

    def fit():  # the fit alone sits in an NVTX range (launch lists filter on it)
        torch.cuda.nvtx.range_push("supergate_fit")
        r = m.apply_supergate(sg, **kw)
        torch.cuda.nvtx.range_pop()
        return r

    fresh()
    psi_dims = np.concatenate([np.ones((B, 1), np.int64), m.bond_dims(), np.ones((B, 1), np.int64)], 1)
    fit()  # warm-up
    t_tot, F, F0 = 0.0, [], []
    for _ in range(a.reps):
        fresh()
        t0 = time.perf_counter()
        f, f0, info = fit()
        t_tot += time.perf_counter() - t0
        F.append(f)
        F0.append(f0)
    phi_dims = np.concatenate([np.ones((B, 1), np.int64), m.bond_dims(), np.ones((B, 1), np.int64)], 1)
    win = phi_dims[:, sg.first:sg.last + 2]  # bonds first-1 .. last
    fresh()  # one more run with per-class event timing
    m.profile(tnmps.PROF_CLASSES)
    t0 = time.perf_counter()
    fit()
    t_prof = time.perf_counter() - t0
    prof = m.profile_read()
    m.profile(None)
    fit_flops = 0
    for z in range(B):
        ov, sw = _fit_flops(phi_dims[z], psi_dims[z], sg.bonds, sg.first, sg.last)
        fit_flops += ov + a.sweeps * sw
    fit_s = prof["fit"][0] / 1e3
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    F, F0 = np.concatenate(F), np.concatenate(F0)
    out = {"workload": f"super-gate on qubits {sg.first}..{sg.last} (distant CNOT/CZ, SWAP, "
                       f"rotations) of {B} chi=128 states (40 qubits, 10 layers), chi_max 128, "
                       f"{a.sweeps} sweeps", "dtype": a.dtype, "batch": B, "reps": a.reps,
           "mpo_bonds": [int(x) for x in sg.bonds],
           "fits_per_s": B * a.reps / t_tot, "s_per_batch": t_tot / a.reps,
           "fidelity_first_iterate_mean": float(F0.mean()), "fidelity_mean": float(F.mean()),
           "window_bond_min_mean": [int(win.min()), float(win.mean())],
           "class_share": {k: v[0] / 1e3 / t_prof for k, v in prof.items() if v[1]},
           "fit_gemm": {"kernel": "k_gemm fit problems (FP32 CUDA-core tile GEMM)",
                        "bound": "alu", "alg_flops": fit_flops, "seconds": fit_s,
                        "achieved": fit_flops / fit_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                        "frac": fit_flops / fit_s / 1e12 / peak,
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}}
    if a.oracle:
        import copy

        from oracle import mps as OM
        from oracle import supergate as OSG
        om = OM.MPS(40, 128, wl["eps"]).run(wl["circuit"], wl["thetas"][0])
        t0 = time.perf_counter()
        _, f_or, _, _, f0_or = OSG.apply_supergate(copy.deepcopy(om), block, bth, **kw)
        out["oracle_s_per_fit"] = time.perf_counter() - t0
        out["oracle_fits_per_s"] = 1.0 / out["oracle_s_per_fit"]
        out["state0_fidelity_gpu_vs_oracle"] = [float(F[0]), float(f_or)]
        out["state0_first_iterate_gpu_vs_oracle"] = [float(F0[0]), float(f0_or)]
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=("large100", "rounds", "sample", "supergate"))
    ap.add_argument("--shots", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=304)
    ap.add_argument("--dtype", default="c64_bf16split", choices=tuple(ESIZE))
    ap.add_argument("--oracle", action="store_true")
    ap.add_argument("--circuits", type=int, default=10)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--first", type=int, default=17, help="supergate: first qubit of the block")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=3)
    a = ap.parse_args()
    {"large100": large100, "rounds": rounds, "sample": sample, "supergate": supergate}[a.case](a)


if __name__ == "__main__":
    main()
