"""What the trained surrogate gains: surrogate-proposed Adam steps, each
verified by the GPU MPS, reach the energy of plain parameter-shift Adam with
fewer MPS evaluations (8 qubits, 48 parameters, 32 random Pauli strings)."""
import numpy as np
import pytest

from paper_1807_07914_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1807_07914_gb300 import vqe  # noqa: E402


def test_param_shift_gradient_against_oracle():
    from oracle import energy as OE
    n = 6
    circ, P = inputs.hea_circuit(n, 2, ("RY", "RZ"))
    rng = np.random.default_rng(2)
    terms = inputs.random_pauli_terms(n, 12, 3, rng)
    th = rng.uniform(-np.pi, np.pi, P)
    en = vqe.MPSEnergy(n, 8, 1e-12, circ, P, terms, "c128", 2 * P + 1)
    e0, g, _, _ = vqe.param_shift(en, th)
    assert en.evals == 2 * P + 1
    assert abs(e0 - OE.energy(n, circ, th, terms, "dense")) < 1e-10
    assert np.allclose(g, OE.parameter_shift_gradient(n, circ, th, terms, "dense"), atol=1e-10)


def test_surrogate_reaches_plain_best_with_fewer_evaluations():
    n = 8
    circ, P = inputs.hea_circuit(n, 3, ("RY", "RZ"))
    rng = np.random.default_rng(11)
    terms = inputs.random_pauli_terms(n, 32, 3, rng)
    gen = vqe.MPSEnergy(n, 16, 1e-12, circ, P, terms, "c64", 2048)
    X = rng.uniform(-np.pi, np.pi, (20000, P))
    sur = vqe.Surrogate(P)
    sur.add(X, gen(X))
    sur.fit(30, 1e-3, restandardise=True)
    theta0 = np.random.default_rng(5).uniform(-np.pi, np.pi, P)
    budget = 20000
    plain = vqe.MPSEnergy(n, 16, 1e-12, circ, P, terms, "c128", 2 * P + 1)
    hp, bp = vqe.plain_adam(plain, theta0, 0.05, budget)
    verifier = vqe.MPSEnergy(n, 16, 1e-12, circ, P, terms, "c128", 2 * P + 1)
    hs, bs, st = vqe.surrogate_adam(verifier, sur, theta0, 0.05, budget)
    # every reported energy is an MPS energy; the surrogate run is monotone
    assert all(b[1] <= a[1] for a, b in zip(hs, hs[1:]))
    assert st["accepted"] > 0
    ev = vqe.evals_to(hs, bp[0])
    assert ev is not None and ev < vqe.evals_to(hp, bp[0])
