"""FP64 matrix-product state, step by step as the paper describes it
(oracle side; test infrastructure only).

Paper passages followed (arXiv:1807.07914):

* Sec. IV (ITensor MPS implementation): n rank-3 tensors, O(n chi^2)
  numbers; the register starts as a product state; single-qubit gates are
  contracted into the site tensor; a two-qubit gate on adjacent qubits
  contracts the two rank-3 tensors and the gate into a rank-4 tensor, which
  an SVD splits back into two rank-3 tensors and a diagonal matrix, with
  singular values below a cutoff epsilon truncated (default 1e-4).
* Sec. II, Fig. "mpssvd": accelerated update of adjacent qubit pairs.

Readings where the paper is silent:

* Cutoff rule R: with sigma sorted descending and sigma_norm = sqrt(sum
  sigma^2), keep sigma_i >= eps * sigma_norm, then cap at chi_max keeping
  the largest, keep at least one; the discarded weight of the step is
  w = sum_{i>=k} sigma_i^2 / sigma_norm^2 and the kept sigma are rescaled so
  the state has unit norm.
* Gauge: mixed canonical form with an orthogonality centre; before a
  two-qubit gate on (l, l+1) the centre is moved to l by QR (rightward) or
  LQ (leftward) steps; after the gate it sits on l+1.
* Non-adjacent two-qubit gates are brought together with SWAP chains and the
  SWAPs undone afterwards (Sec. IV).
* Expectation values: one full left-to-right transfer sweep over all n sites
  per term, starting from the 1x1 identity -- the slow form with no prefix
  sharing and no use of the canonical gauge.

Pins: ``tests/test_oracle_mps.py`` -- agreement with the dense brute force
when nothing is truncated, norm 1 after every gate, the truncation error of
one step equal to its discarded weight, GHZ and product-state closed forms at
n=40, bond-dimension bounds, and the cutoff semantics; ``cut_margin`` against
closed forms (a two-value Schmidt spectrum at the cutoff, a planted gap at the
cap, the exact tie of a Bell pair cut to one value).
"""
import numpy as np

from . import gates as g


def truncation_rank(sigma, chi_max, eps):
    """Rule R (see module docstring). ``sigma`` sorted descending.
    Returns (k, discarded_weight, kept_norm)."""
    s2 = sigma.astype(np.float64) ** 2
    total = float(np.sum(s2))
    norm = np.sqrt(total)
    keep = int(np.count_nonzero(sigma >= eps * norm))
    k = max(1, min(int(chi_max), keep))
    w = float(np.sum(s2[k:])) / total if total > 0 else 0.0
    return k, w, float(np.sqrt(np.sum(s2[:k])))


def cut_margin(sigma, chi_max, eps):
    """How far one step's truncation decision is from changing, relative to
    sigma_0. Returns (d_cut, d_cap): d_cut is the smallest distance of any
    sigma_i from the cutoff eps * sigma_norm (a perturbation of the sigma
    below it keeps the same count above the cutoff); d_cap, when the chi_max
    cap binds, is the gap sigma_{k-1} - sigma_k between the last kept and the
    first dropped value (below it the kept subspace is not unique: a tie at
    the cut), else inf. Diagnostic only: no part of the simulation uses it.
    ``sigma`` sorted descending."""
    s = np.asarray(sigma, dtype=np.float64)
    if s.size == 0 or not s[0] > 0:
        return float("inf"), float("inf")
    norm = np.sqrt(float(np.sum(s ** 2)))
    d_cut = float(np.min(np.abs(s - eps * norm))) / s[0]
    keep = int(np.count_nonzero(s >= eps * norm))
    d_cap = float(s[chi_max - 1] - s[chi_max]) / s[0] if keep > chi_max else float("inf")
    return d_cut, d_cap


class MPS:
    """MPS of n qubits; ``tensors[i]`` has shape (D_{i-1}, 2, D_i)."""

    def __init__(self, n, chi_max=1 << 30, eps=1e-4):
        self.n = int(n)
        self.chi_max = int(chi_max)
        self.eps = float(eps)
        self.tensors = []
        for _ in range(self.n):
            t = np.zeros((1, 2, 1), dtype=np.complex128)
            t[0, 0, 0] = 1.0          # |0> on every site (Sec. IV)
            self.tensors.append(t)
        self.centre = 0
        self.discarded = 0.0          # sum of per-step discarded weights
        self.step_weights = []
        self.cut_margins = []         # per two-qubit step: (d_cut, d_cap), see cut_margin

    # ---- gauge moves -------------------------------------------------
    def _move_right(self):
        c = self.centre
        A = self.tensors[c]
        Dl, _, Dr = A.shape
        Q, R = np.linalg.qr(A.reshape(Dl * 2, Dr))
        r = Q.shape[1]
        self.tensors[c] = Q.reshape(Dl, 2, r)
        self.tensors[c + 1] = np.einsum("rm,msb->rsb", R, self.tensors[c + 1])
        self.centre = c + 1

    def _move_left(self):
        c = self.centre
        A = self.tensors[c]
        Dl, _, Dr = A.shape
        # LQ of A as Dl x (2 Dr) == conjugate transpose of QR of its adjoint.
        Q, R = np.linalg.qr(A.reshape(Dl, 2 * Dr).conj().T)
        r = Q.shape[1]
        self.tensors[c] = Q.conj().T.reshape(r, 2, Dr)
        self.tensors[c - 1] = np.einsum("asm,mr->asr", self.tensors[c - 1], R.conj().T)
        self.centre = c - 1

    def move_centre(self, target):
        while self.centre < target:
            self._move_right()
        while self.centre > target:
            self._move_left()

    # ---- gates -------------------------------------------------------
    def apply_1q(self, U, q):
        self.tensors[q] = np.einsum("ts,asb->atb", U, self.tensors[q])

    def apply_2q_adjacent(self, G, l):
        """G (4x4, basis 2*s_l + s_{l+1}) on sites (l, l+1)."""
        self.move_centre(l)
        A, B = self.tensors[l], self.tensors[l + 1]
        Dl, Dr = A.shape[0], B.shape[2]
        theta = np.einsum("asm,mtb->astb", A, B)
        theta = np.einsum("stuv,auvb->astb", G.reshape(2, 2, 2, 2), theta)
        U, S, Vh = np.linalg.svd(theta.reshape(Dl * 2, 2 * Dr), full_matrices=False)
        k, w, kept = truncation_rank(S, self.chi_max, self.eps)
        self.tensors[l] = U[:, :k].reshape(Dl, 2, k)
        self.tensors[l + 1] = ((S[:k, None] / kept) * Vh[:k]).reshape(k, 2, Dr)
        self.centre = l + 1
        self.discarded += w
        self.step_weights.append(w)
        self.cut_margins.append(cut_margin(S, self.chi_max, self.eps))

    def apply_2q(self, G, qa, qb):
        """G (basis 2*s_qa + s_qb) on qubits (qa, qb), any distance."""
        if abs(qa - qb) == 1:
            if qa < qb:
                self.apply_2q_adjacent(G, qa)
            else:
                # reorder the basis to (s_qb, s_qa) for the site pair (qb, qa)
                P = g.two_qubit("SWAP")
                self.apply_2q_adjacent(P @ G @ P, qb)
            return
        # SWAP chain: bring qb next to qa, apply, then undo (Sec. IV).
        sw = g.two_qubit("SWAP")
        step = 1 if qb > qa else -1
        pos = qb
        while abs(pos - qa) > 1:
            lo = min(pos, pos - step)
            self.apply_2q_adjacent(sw, lo)
            pos -= step
        self.apply_2q(G, qa, pos)
        while pos != qb:
            lo = min(pos, pos + step)
            self.apply_2q_adjacent(sw, lo)
            pos += step

    def run(self, circuit, theta):
        for gate in circuit:
            if g.is_two_qubit(gate):
                self.apply_2q(g.two_qubit(gate[0]), gate[1], gate[2])
            else:
                self.apply_1q(g.one_qubit_matrix(gate, theta), gate[1])
        return self

    # ---- observables -------------------------------------------------
    def bond_dims(self):
        return [t.shape[2] for t in self.tensors[:-1]]

    def expect_pauli(self, sites, paulis):
        """<psi|P|psi> by a full left-to-right transfer sweep from the 1x1
        identity over all n sites (no prefix sharing, no gauge shortcut)."""
        ops = {int(q): int(p) for q, p in zip(sites, paulis)}
        L = np.ones((1, 1), dtype=np.complex128)
        for i, A in enumerate(self.tensors):
            P = g.PAULI[ops.get(i, 0)]
            # L'[c,d] = sum_{a,b,s,t} L[a,b] conj(A[a,s,c]) P[s,t] A[b,t,d]
            L = np.einsum("ab,asc,st,btd->cd", L, A.conj(), P, A, optimize=True)
        return complex(L[0, 0])

    def norm2(self):
        return self.expect_pauli([], []).real

    def to_dense(self):
        """State vector in the qubit-q = bit-q convention (small n only)."""
        v = self.tensors[0].reshape(2, -1)
        for A in self.tensors[1:]:
            v = np.einsum("xm,msb->xsb", v, A).reshape(-1, A.shape[2])
        v = v.reshape((2,) * self.n)
        # axis i of v is site i; numpy C order makes axis 0 the MSB, so
        # reverse the axes to put qubit 0 on the least significant bit.
        return np.transpose(v, tuple(range(self.n - 1, -1, -1))).reshape(-1)
