"""Super-gate application by overlap maximisation (oracle side; test
infrastructure only).

Paper passage (arXiv:1807.07914, Sec. II, the general algorithm for the action
of a super-gate on a tensor-network wave-function, and Sec. IV, the ExaTENSOR
MPS visitor that implements it): an aggregate of gates on any qubits acts on
the input network TN_inp by
  (1) attaching the gates to TN_inp, which gives TN_mid;
  (3) instantiating the output network TN_out as a copy of TN_inp;
  (4) joining TN_mid with the conjugate of TN_out into the closed, scalar
      network TN_opt = <TN_out|TN_mid>;
  (5) optimising the tensors of TN_out to maximise TN_opt, using the gradient
      of TN_opt with respect to the output tensors;
  (6) while the value reached is not acceptable, enlarging the auxiliary
      (bond) dimensions of TN_out and repeating (5).

Readings where the paper is silent:

* TN_mid's gates form a matrix-product operator W over the window [p, q] of
  qubits the super-gate touches (the identity elsewhere). W[i] has shape
  (w_{i-1}, 2, 2, w_i), index order [left bond, output, input, right bond].
  A two-qubit gate enters through its operator-Schmidt decomposition
  sum_k A_k (x) B_k (an SVD of the gate regrouped as (out_a in_a) x
  (out_b in_b)); the Schmidt index k runs along the bonds between its two
  qubits, and the sites in between carry the identity. A one-qubit gate
  multiplies its site's output leg. Gates act in list order.
* TN_out stays an MPS in mixed-canonical gauge. Its tensors outside the window
  are those of TN_inp: the super-gate is the identity there, and with TN_inp's
  orthogonality centre moved into the window the environments of the window
  boundaries are identity matrices.
* First iterate of (5). Started from the plain copy of (3), two-site updates
  cannot build entanglement between distant qubits: every update sees TN_mid
  projected onto the fixed remainder of TN_out, so a bond-1 copy stays stuck
  at a local optimum (F = 1/2 for a distant CNOT on |+>|0...0>, whatever the
  bond cap). The optimisation therefore starts from the copy with the gates
  applied one by one by the accelerated route (adjacent pairs, SWAP chains,
  SVD truncation at the stage's bond cap), which is itself a valid TN_out of
  those dimensions; the sweeps only raise its overlap with TN_mid.
* (5): with every other tensor of TN_out isometric around a two-site block,
  the gradient of <TN_out|TN_mid> with respect to the conjugated block is the
  open network Theta_grad (left environment, the two MPO tensors, the two
  TN_inp tensors, right environment). On the unit sphere the maximiser of the
  overlap over that block is Theta_grad / ||Theta_grad||, which each update
  takes; it is split by SVD with the cutoff rule R of ``mps.truncation_rank``
  and the stage's bond cap (two sites, so that bonds can grow). One sweep
  updates the pairs (p, p+1), ..., (q-1, q) left to right; before each sweep
  the centre goes back to site p by LQ steps.
* The value of TN_opt after a sweep is O = <TN_out|TN_mid> and the fidelity
  F = |O|^2 (TN_out and TN_mid have unit norm: the gates are unitary). A stage
  of (5) ends when a sweep raises F by less than ``tol``, or after
  ``max_sweeps`` sweeps. (6) calls F acceptable when 1 - F <= ``target``;
  otherwise the bond cap (initially the largest bond of TN_inp inside the
  window: the dimensions of the copy) doubles, up to ``chi_max``, and the
  stage repeats from (3) with the larger cap.
* The discarded weight of the result is that of TN_inp plus 1 - F.

Pins (``tests/test_oracle_supergate.py``): the MPO contracted densely equals
the product of the gate matrices applied by the state-vector module; without
truncation the result is the exact state G|psi> of the state-vector module;
the closed form F = 1/2 of a distant CNOT on |+>|0...0> at bond cap 1; a
single adjacent gate reproduces the SVD-truncated gate application of
``mps`` (Eckart-Young) with F = 1 - its discarded weight; the sweeps never
lower the fidelity of their first iterate; and an independent dense-vector
formulation of the same alternating updates gives the same fidelities.
"""
import copy

import numpy as np

from . import gates as g
from .mps import truncation_rank


def window(circuit):
    """First and last qubit the gate list touches."""
    qs = []
    for gate in circuit:
        qs.append(int(gate[1]))
        if g.is_two_qubit(gate):
            qs.append(int(gate[2]))
    if not qs:
        raise ValueError("empty super-gate")
    return min(qs), max(qs)


def mpo_from_gates(circuit, theta):
    """(p, q, W): the super-gate as an MPO over sites p..q, W[i - p] of shape
    (w_left, 2, 2, w_right) = [bond, out, in, bond]."""
    p, q = window(circuit)
    W = [np.eye(2, dtype=np.complex128).reshape(1, 2, 2, 1) for _ in range(q - p + 1)]
    swap = g.two_qubit("SWAP")
    for gate in circuit:
        if not g.is_two_qubit(gate):
            U = g.one_qubit_matrix(gate, theta)
            i = int(gate[1]) - p
            W[i] = np.einsum("ot,atsb->aosb", U, W[i])
            continue
        G = g.two_qubit(gate[0])
        qa, qb = int(gate[1]), int(gate[2])
        if qa > qb:  # reorder the basis to (s_left, s_right)
            G = swap @ G @ swap
            qa, qb = qb, qa
        # G[(oa ob), (ia ib)] regrouped as M[(oa ia), (ob ib)] = sum_k A_k B_k
        M = G.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
        U, S, Vh = np.linalg.svd(M)
        r = int(np.count_nonzero(S > 1e-14 * S[0]))
        A = (U[:, :r] * S[:r]).T.reshape(r, 2, 2)  # A[k, out, in] on qa
        B = Vh[:r].reshape(r, 2, 2)                # B[k, out, in] on qb
        i, j = qa - p, qb - p
        # left end: the Schmidt index joins the right bond
        t = np.einsum("kot,atsb->aosbk", A, W[i])
        a, _, _, b, _ = t.shape
        W[i] = t.reshape(a, 2, 2, b * r)
        # bridge: identity on the Schmidt index
        for m in range(i + 1, j):
            a, _, _, b = W[m].shape
            t = np.einsum("aosb,kl->akosbl", W[m], np.eye(r))
            W[m] = t.reshape(a * r, 2, 2, b * r)
        # right end: the Schmidt index joins the left bond
        t = np.einsum("kot,atsb->akosb", B, W[j])
        a, _, _, _, b = t.shape
        W[j] = t.reshape(a * r, 2, 2, b)
    return p, q, W


def mpo_dense(W):
    """The window operator as a dense matrix in the qubit-q = bit-q order of
    the window (bit 0 = site p)."""
    T = W[0][0]  # (2, 2, w)
    m = 1
    for Wi in W[1:]:
        # T[(o..), (i..), b] x Wi[b, o, s, c]
        T = np.einsum("xyb,bosc->xoysc", T, Wi)
        m += 1
        T = T.reshape(2 ** m, 2 ** m, -1)
    # site order p..q is C-order (site p most significant): reverse the bits
    T = T[:, :, 0].reshape((2,) * (2 * m))
    perm = tuple(range(m - 1, -1, -1)) + tuple(range(2 * m - 1, m - 1, -1))
    return T.transpose(perm).reshape(2 ** m, 2 ** m)


def _env_left(L, phi, W, psi):
    # L'[b', beta, b] = sum L[a', alpha, a] conj(phi[a', o, b']) W[alpha, o, s, beta] psi[a, s, b],
    # summed one operand at a time (psi, then W, then phi)
    t = np.einsum("xya,asc->xysc", L, psi, optimize=True)
    t = np.einsum("xysc,yosz->xozc", t, W, optimize=True)
    return np.einsum("xozc,xob->bzc", t, phi.conj(), optimize=True)


def _env_right(R, phi, W, psi):
    # R'[c', gamma, c] = sum conj(phi[c', o, d']) W[gamma, o, s, delta] psi[c, s, d] R[d', delta, d],
    # summed one operand at a time (R, then W, then phi)
    t = np.einsum("csy,dhy->csdh", psi, R, optimize=True)
    t = np.einsum("csdh,gosh->cdgo", t, W, optimize=True)
    return np.einsum("cdgo,xod->xgc", t, phi.conj(), optimize=True)


def _theta_grad(L, W1, W2, psi1, psi2, R):
    # Theta[a', o1, o2, c'] = sum L[a', al, a] W1[al, o1, s1, be] W2[be, o2, s2, ga]
    #                             psi1[a, s1, m] psi2[m, s2, c] R[c', ga, c],
    # summed one operand at a time (psi1, W1, psi2, W2, R)
    t = np.einsum("xya,asm->xysm", L, psi1, optimize=True)
    t = np.einsum("xysm,yosb->xobm", t, W1, optimize=True)
    t = np.einsum("xobm,mtc->xobtc", t, psi2, optimize=True)
    t = np.einsum("xobtc,bptg->xopgc", t, W2, optimize=True)
    return np.einsum("xopgc,zgc->xopz", t, R, optimize=True)


def apply_supergate(mps, circuit, theta, chi_max, target=1e-10, tol=1e-12, max_sweeps=8):
    """Apply the gate list ``circuit`` to ``mps`` by overlap maximisation.

    Returns (phi, F, history, chi, F_start): the output MPS (centre on the
    last site of the window), the final fidelity |<phi|G psi>|^2, the fidelity
    after every sweep, the final bond cap and the fidelity of the last
    stage's first iterate."""
    p, q, W = mpo_from_gates(circuit, theta)
    psi = copy.deepcopy(mps)
    psi.move_centre(p)
    if p == q:                                             # no bond to fit
        phi = copy.deepcopy(psi)
        phi.tensors[p] = np.einsum("osb,asc->aoc", W[0][0], psi.tensors[p])
        return phi, 1.0, [1.0], 0, 1.0
    chi = max(psi.tensors[i].shape[2] for i in range(p, q))
    chi = max(1, min(int(chi_max), chi))
    history = []
    while True:
        phi = copy.deepcopy(psi)                           # step (3)
        phi.chi_max = chi
        phi.run(circuit, theta)                            # first iterate
        F_start = overlap_fidelity(phi, psi, p, q, W)
        F, F_prev = F_start, None
        for _ in range(max_sweeps):                        # step (5)
            F = sweep(phi, psi, p, q, W, chi)
            history.append(F)
            if F_prev is not None and F - F_prev < tol:
                break
            F_prev = F
        if 1.0 - F <= target or chi >= chi_max:
            break
        chi = min(int(chi_max), 2 * chi)                    # step (6)
    phi.discarded = mps.discarded + max(0.0, 1.0 - F)
    return phi, F, history, chi, F_start


def overlap_fidelity(phi, psi, p, q, W):
    """|<phi|G psi>|^2 over the window (phi and psi equal and isometric
    outside it), by left environments from the identity at bond p-1."""
    Dp = phi.tensors[p].shape[0]
    L = np.eye(Dp, dtype=np.complex128).reshape(Dp, 1, Dp)
    for i in range(p, q + 1):
        L = _env_left(L, phi.tensors[i], W[i - p], psi.tensors[i])
    return abs(complex(np.trace(L[:, 0, :]))) ** 2


def sweep(phi, psi, p, q, W, chi):
    """One left-to-right sweep of two-site updates over the window; returns
    the fidelity after it."""
    phi.move_centre(p)
    Dq = phi.tensors[q].shape[2]
    R = {q + 1: np.eye(Dq, dtype=np.complex128).reshape(Dq, 1, Dq)}
    for i in range(q, p + 1, -1):
        R[i] = _env_right(R[i + 1], phi.tensors[i], W[i - p], psi.tensors[i])
    Dp = phi.tensors[p].shape[0]
    L = np.eye(Dp, dtype=np.complex128).reshape(Dp, 1, Dp)
    for i in range(p, q):
        grad = _theta_grad(L, W[i - p], W[i + 1 - p], psi.tensors[i], psi.tensors[i + 1],
                           R[i + 2])
        Fa, Fc = grad.shape[0], grad.shape[3]
        U, S, Vh = np.linalg.svd(grad.reshape(2 * Fa, 2 * Fc), full_matrices=False)
        k, _, kept = truncation_rank(S, chi, phi.eps)
        phi.tensors[i] = U[:, :k].reshape(Fa, 2, k)
        phi.tensors[i + 1] = ((S[:k, None] / kept) * Vh[:k]).reshape(k, 2, Fc)
        phi.centre = i + 1
        L = _env_left(L, phi.tensors[i], W[i - p], psi.tensors[i])
    L = _env_left(L, phi.tensors[q], W[q - p], psi.tensors[q])
    return abs(complex(np.trace(L[:, 0, :]))) ** 2
