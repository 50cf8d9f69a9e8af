"""Small, self-contained launches of single kernels for profiler captures.

  python -m paper_1807_07914_gb300.prof_case jacobi --dtype c64 --batch 304 --m 256 --n 256
  python -m paper_1807_07914_gb300.prof_case circuit --dtype c64 --batch 152 --layers 9
  python -m paper_1807_07914_gb300.prof_case sweep --dtype c64_bf16split --batch 8 --terms 2000

``jacobi`` runs the standalone batched SVD on random complex matrices (the
shape of a saturated chi=128 two-site block) ``--reps`` times; ``circuit``
runs the chi=128 ansatz on a reduced batch and then the Heisenberg energy;
``sweep`` builds the chi=128 states (7 layers saturate the middle bonds) and
then evaluates the first ``--terms`` of the 2000 random strings ``--reps``
times (one state chunk; ``--sweep-fused 1`` runs both steps of a trie level in
one launch). All exit non-zero on any library error.
"""
import argparse
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1807_07914_gb300 import inputs, tnmps  # noqa: E402


def jacobi(a):
    rng = np.random.default_rng(7)
    tdt = torch.complex64 if a.dtype == "c64" else torch.complex128
    host = rng.normal(size=(a.batch, a.n, a.m)) + 1j * rng.normal(size=(a.batch, a.n, a.m))
    src = torch.tensor(host, dtype=tdt, device="cuda")
    buf = torch.empty_like(src)
    sig = torch.zeros((a.batch, a.n), dtype=torch.float64, device="cuda")
    sw = torch.zeros(a.batch, dtype=torch.int32, device="cuda")
    for _ in range(a.reps):
        buf.copy_(src)
        tnmps.jacobi_svd_dev(buf, a.m, a.n, sig, sw)
    torch.cuda.synchronize()
    print("sweeps", sw.float().mean().item())


def circuit(a):
    wl = inputs.workload("chi128")
    circ, P = inputs.hea_circuit(40, a.layers, ("RY", "RZ"))
    m = tnmps.MPSBatch(40, 128, a.batch, dtype=a.dtype, max_params=P, eps=wl["eps"])
    th = inputs.thetas(a.batch, P, inputs.rng_for(5, 7))
    m.apply_circuit(circ, th)
    e = m.expect(tnmps.PauliSum(40, wl["terms"]))
    assert np.all(np.isfinite(e))
    print("energy[0]", e[0])


def sweep(a):
    wl = inputs.workload("chi128")
    circ, P = inputs.hea_circuit(40, a.layers, ("RY", "RZ"))
    m = tnmps.MPSBatch(40, 128, a.batch, dtype=a.dtype, max_params=P, eps=wl["eps"])
    th = inputs.thetas(a.batch, P, inputs.rng_for(5, 7))
    m.apply_circuit(circ, th)
    m.set_tuning(sweep_fused=a.sweep_fused)
    ps = tnmps.PauliSum(40, wl["terms_random"][:a.terms])
    energy = torch.empty(a.batch, dtype=torch.float64, device="cuda")
    for _ in range(a.reps):
        m.expect_dev(ps, energy, chunk=a.batch)
    torch.cuda.synchronize()
    m.check()
    assert bool(torch.all(torch.isfinite(energy)))
    print("energy[0]", float(energy[0]), "bonds", int(m.bond_dims().max()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=("jacobi", "circuit", "sweep"))
    ap.add_argument("--dtype", default="c64", choices=("c64", "c128", "c64_bf16split"))
    ap.add_argument("--terms", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=152)
    ap.add_argument("--m", type=int, default=256)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--layers", type=int, default=9)
    ap.add_argument("--sweep-fused", type=int, default=0,
                    help="sweep: both steps of a trie level in one launch (tnmps_tuning)")
    a = ap.parse_args()
    {"jacobi": jacobi, "circuit": circuit, "sweep": sweep}[a.case](a)


if __name__ == "__main__":
    main()
