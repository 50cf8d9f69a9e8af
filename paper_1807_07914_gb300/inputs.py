"""Seeded synthetic inputs shared by the tests, the oracle checks and the bench.

This module holds no simulation arithmetic: it only builds gate lists, Pauli
sums and parameter vectors. Both the CUDA library and the CPU oracle consume
what it returns, and neither imports the other.

A gate record is ``(name, q0, q1, param, angle, scale)``; the effective angle
of a rotation is ``angle + scale * theta[param]`` when ``param >= 0``, else
``angle``. Two-qubit gates use ``q0`` as the first operand (the control of a
CNOT). A Pauli sum is a list of ``(coeff, sites, paulis)`` with codes
1=X, 2=Y, 3=Z; an empty term is the identity.

Workload shapes follow the paper's two demonstrations (Sec. V.A random
"rounds" circuits, Sec. V.B parameterised VQE ansatz with a Pauli-sum
Hamiltonian) at the sizes of the benchmark configurations.
"""
import numpy as np

ROT = ("RX", "RY", "RZ")


def rng_for(config_idx, rep=0):
    return np.random.default_rng(1000 * int(config_idx) + int(rep))


# ---------------------------------------------------------------- circuits
def hea_circuit(n, layers, rotations=("RY",)):
    """Hardware-efficient ansatz: per layer, the listed rotations on every
    qubit (each with its own parameter), then CNOT(i, i+1) for i = 0..n-2.
    Returns (gates, n_params)."""
    gates = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            for r in rotations:
                gates.append((r, q, -1, p, 0.0, 1.0))
                p += 1
        for q in range(n - 1):
            gates.append(("CNOT", q, q + 1, -1, 0.0, 1.0))
    return gates, p


def h2_ansatz():
    """Two-qubit, one-parameter ansatz of the paper's VQE demonstration
    (Sec. V.B listing), with the printed literal angles; parameter 0 is t0.
    "CNOT 1 0" is read as control 1, target 0."""
    gates = [
        ("RX", 0, -1, -1, 3.1415926, 1.0),
        ("RY", 1, -1, -1, 1.57079, 1.0),
        ("RX", 0, -1, -1, 7.85397, 1.0),
        ("CNOT", 1, 0, -1, 0.0, 1.0),
        ("RZ", 0, -1, 0, 0.0, 1.0),
        ("CNOT", 1, 0, -1, 0.0, 1.0),
        ("RY", 1, -1, -1, 7.8539752, 1.0),
        ("RX", 0, -1, -1, 1.57079, 1.0),
    ]
    return gates, 1


def rounds_circuit(n, rounds, rng):
    """Random "rounds" circuit of Sec. V.A: round 1 starts with H on every
    qubit; every round has a layer of random single-qubit gates (Paulis or
    rotations with angle ~ U(-pi, pi)) and then nearest-neighbour CNOTs.
    The paper does not give the single-qubit distribution; here it is uniform
    over {X, Y, Z, RX, RY, RZ}."""
    gates = []
    for r in range(rounds):
        if r == 0:
            gates += [("H", q, -1, -1, 0.0, 1.0) for q in range(n)]
        for q in range(n):
            k = int(rng.integers(6))
            name = ("X", "Y", "Z", "RX", "RY", "RZ")[k]
            ang = float(rng.uniform(-np.pi, np.pi)) if k >= 3 else 0.0
            gates.append((name, q, -1, -1, ang, 1.0))
        for q in range(n - 1):
            gates.append(("CNOT", q, q + 1, -1, 0.0, 1.0))
    return gates


def thetas(batch, n_params, rng):
    return rng.uniform(-np.pi, np.pi, size=(batch, n_params))


# ---------------------------------------------------------------- Pauli sums
def heisenberg_terms(n, rng, pbc=False):
    """H = sum_i (X_i X_{i+1} + Y_i Y_{i+1} + Z_i Z_{i+1}) + sum_i h_i Z_i with
    h_i ~ U(-1, 1); open chain: 3(n-1) + n terms."""
    terms = []
    bonds = n if pbc else n - 1
    for i in range(bonds):
        j = (i + 1) % n
        for p in (1, 2, 3):
            terms.append((1.0, (i, j), (p, p)))
    h = rng.uniform(-1.0, 1.0, size=n)
    for i in range(n):
        terms.append((float(h[i]), (i,), (3,)))
    return terms


def random_pauli_terms(n, count, w_max, rng, scale_by_weight=False):
    """``count`` distinct Pauli strings (at most as many as exist); weight
    w ~ U{1..min(w_max, n)}, sites uniform
    without replacement, Paulis uniform over {X, Y, Z}, coefficients
    ~ N(0, 1) (divided by w when ``scale_by_weight``)."""
    from math import comb
    w_top = min(w_max, n)
    count = min(count, sum(comb(n, w) * 3 ** w for w in range(1, w_top + 1)))
    seen = set()
    terms = []
    while len(terms) < count:
        w = int(rng.integers(1, w_top + 1))
        sites = tuple(sorted(int(s) for s in rng.choice(n, size=w, replace=False)))
        paulis = tuple(int(p) for p in rng.integers(1, 4, size=w))
        key = (sites, paulis)
        if key in seen:
            continue
        seen.add(key)
        c = float(rng.normal())
        if scale_by_weight:
            c /= w
        terms.append((c, sites, paulis))
    return terms


def all_two_qubit_terms(rng):
    """Random real coefficients on all 16 two-qubit Pauli strings (the
    identity included as the empty term)."""
    terms = [(float(rng.normal()), (), ())]
    for p0 in range(4):
        for p1 in range(4):
            if p0 == 0 and p1 == 0:
                continue
            sites, paulis = [], []
            if p0:
                sites.append(0)
                paulis.append(p0)
            if p1:
                sites.append(1)
                paulis.append(p1)
            terms.append((float(rng.normal()), tuple(sites), tuple(paulis)))
    return terms


def terms_to_csr(terms):
    """(term_off[int32, T+1], sites[int32], paulis[uint8], coeffs[float64])."""
    off = [0]
    sites, paulis, coeffs = [], [], []
    for c, s, p in terms:
        sites += list(s)
        paulis += list(p)
        off.append(len(sites))
        coeffs.append(float(c))
    return (np.asarray(off, dtype=np.int32), np.asarray(sites, dtype=np.int32),
            np.asarray(paulis, dtype=np.uint8), np.asarray(coeffs, dtype=np.float64))


def batch_jobs(count, rng, n_range=(16, 64), depth_range=(2, 8), chi_range=(32, 128),
               terms_range=(50, 2000), w_max=4):
    """Heterogeneous job list: per job n ~ U{n_range}, ansatz depth ~ U{depth},
    chi_max ~ U{chi_range}, Pauli sums of ~U{terms_range} strings of weight
    <= w_max with coefficients ~ N(0, 1) / weight, theta ~ U(-pi, pi)."""
    jobs = []
    for _ in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        chi = int(rng.integers(chi_range[0], chi_range[1] + 1))
        T = int(rng.integers(terms_range[0], terms_range[1] + 1))
        circ, P = hea_circuit(n, depth, ("RY", "RZ"))
        jobs.append(dict(n=n, chi=chi, depth=depth, circuit=circ, n_params=P,
                         theta=thetas(1, P, rng)[0],
                         terms=random_pauli_terms(n, T, w_max, rng, scale_by_weight=True)))
    return jobs


# ---------------------------------------------------------------- workloads
def supergate_block(first, rng):
    """A super-gate on the six qubits first..first+5: distant and reversed
    two-qubit gates, a SWAP and two parameterised rotations (angles drawn from
    rng). Returns (gates, theta)."""
    f = int(first)
    gates = [("CNOT", f, f + 4, -1, 0.0, 1.0), ("RY", f + 2, -1, 0, 0.0, 1.0),
             ("CZ", f + 5, f + 1, -1, 0.0, 1.0), ("H", f + 3, -1, -1, 0.0, 1.0),
             ("CNOT", f + 1, f + 2, -1, 0.0, 1.0), ("SWAP", f + 3, f, -1, 0.0, 1.0),
             ("RX", f + 4, -1, 1, 0.0, 1.0), ("CNOT", f + 5, f + 3, -1, 0.0, 1.0)]
    return gates, rng.uniform(-np.pi, np.pi, 2)


def workload(name, rep=0):
    """Named synthetic workloads. Returns a dict with n, chi_max, eps,
    circuit, n_params, thetas, terms (and extra term sets for the bench)."""
    if name == "hea8":            # plain method, small, dense-checkable
        rng = rng_for(0, rep)
        circ, P = hea_circuit(8, 2, ("RY",))
        th = thetas(16, P, rng)
        terms = random_pauli_terms(8, 32, 3, rng)
        # "no truncation": the paper's default cutoff 1e-4 would drop real Schmidt
        # values (~7e-5 occur), so the cutoff only removes rounding noise here.
        return dict(name=name, n=8, chi_max=16, eps=1e-12, circuit=circ, n_params=P,
                    thetas=th, terms=terms)
    if name == "heis40":          # precision configuration
        rng = rng_for(1, rep)
        circ, P = hea_circuit(40, 4, ("RY", "RZ"))
        th = thetas(256, P, rng)
        terms = heisenberg_terms(40, rng)
        return dict(name=name, n=40, chi_max=64, eps=1e-10, circuit=circ, n_params=P,
                    thetas=th, terms=terms)
    if name == "large100":        # large single state
        rng = rng_for(3, rep)
        circ, P = hea_circuit(100, 6, ("RY", "RZ"))
        th = thetas(1, P, rng)
        terms = random_pauli_terms(100, 5000, 4, rng)
        return dict(name=name, n=100, chi_max=256, eps=1e-8, circuit=circ, n_params=P,
                    thetas=th, terms=terms)
    if name == "chi128":          # the chi=128, 40-qubit throughput workload
        rng = rng_for(5, rep)
        circ, P = hea_circuit(40, 10, ("RY", "RZ"))
        th = thetas(256, P, rng)
        heis = heisenberg_terms(40, rng)
        rand = random_pauli_terms(40, 2000, 4, rng, scale_by_weight=True)
        return dict(name=name, n=40, chi_max=128, eps=1e-10, circuit=circ, n_params=P,
                    thetas=th, terms=heis, terms_random=rand)
    raise KeyError(name)
