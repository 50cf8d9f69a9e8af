"""Shot sampling of a computational-basis measurement of every qubit (oracle
side; test infrastructure only).

Paper passage (arXiv:1807.07914, Sec. V.B): the kernels of the VQE example
end in MEASURE instructions on the measured qubits. Here the measurement of
all n qubits is sampled exactly ("perfect sampling"): qubits n-1, n-2, ..., 0
in turn, each drawn from its probability conditioned on the outcomes already
drawn. The random numbers are inputs: u[k][q] in [0, 1) decides qubit q of
shot k, outcome 0 if u < P(q = 0 | outcomes of the qubits above q), else 1,
so a sampler is a deterministic function of its uniforms (the contract the
GPU sampler follows too).

Two forms that share nothing but that rule:

* ``sample_dense``: from the state vector, conditional probabilities by
  summing |psi|^2 over the basis states consistent with the outcomes drawn;
* ``sample_mps``: from the FP64 MPS with its orthogonality centre on site
  n-1 (sites 0..n-2 left isometries), where P(s | outcomes above q) is
  ||X_q[:, s, :] v||^2 for the normalised conditional vector v.

Both return (bits [shots][n] uint8, margin [shots]) with margin the smallest
|u - P(0 | ...)| over the qubits of the shot: comparisons skip shots that
rounding could have decided differently.

Pins: ``tests/test_oracle_sampling.py`` -- the two forms agree bit for bit,
the Born rule on histograms, GHZ (all equal, decided by the first draw) and
the product-state closed form (qubit q is 1 iff u >= cos^2(theta_q / 2)).
"""
import copy

import numpy as np


def _decide(u, p0, p1):
    tot = p0 + p1
    pz = p0 / tot if tot > 0 else 1.0
    return (0 if u < pz else 1), abs(u - pz)


def sample_dense(psi, n, uniforms):
    psi = np.asarray(psi, dtype=np.complex128)
    prob = np.abs(psi) ** 2
    uniforms = np.asarray(uniforms, dtype=np.float64)
    shots = uniforms.shape[0]
    idx = np.arange(1 << n)
    bits = np.zeros((shots, n), np.uint8)
    margin = np.full(shots, np.inf)
    for k in range(shots):
        consistent = np.ones(1 << n, dtype=bool)
        for q in range(n - 1, -1, -1):
            b = (idx >> q) & 1
            p0 = prob[consistent & (b == 0)].sum()
            p1 = prob[consistent & (b == 1)].sum()
            s, m = _decide(uniforms[k, q], p0, p1)
            bits[k, q] = s
            margin[k] = min(margin[k], m)
            consistent &= b == s
    return bits, margin


def sample_mps(mps, uniforms):
    m = copy.deepcopy(mps)  # the caller's gauge stays as it was
    m.move_centre(m.n - 1)
    uniforms = np.asarray(uniforms, dtype=np.float64)
    shots, n = uniforms.shape[0], m.n
    bits = np.zeros((shots, n), np.uint8)
    margin = np.full(shots, np.inf)
    for k in range(shots):
        v = np.ones(1, dtype=np.complex128)  # right boundary, D_{n-1} = 1
        for q in range(n - 1, -1, -1):
            A = m.tensors[q]
            w = [A[:, s, :] @ v for s in (0, 1)]
            p = [float(np.vdot(x, x).real) for x in w]
            s, mg = _decide(uniforms[k, q], p[0], p[1])
            bits[k, q] = s
            margin[k] = min(margin[k], mg)
            v = w[s] / np.sqrt(p[s])
    return bits, margin
