"""Plain, slow FP64 CPU oracle for MPS circuit simulation and Pauli-sum energies.

TEST INFRASTRUCTURE ONLY. Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may use it. It shares no code, table or helper with the
CUDA library in ``paper_1807_07914_gb300``; both sides only consume the plain
input descriptions (gate lists, Pauli terms, parameter vectors) produced by
``paper_1807_07914_gb300.inputs``.

What the oracle computes, and the paper passage each part follows
(McCaskey et al., "Validating Quantum-Classical Programming Models with Tensor
Network Simulations", arXiv:1807.07914):

* ``gates``       -- textbook one- and two-qubit gate matrices (the gate set of
                     the VQE listing in Sec. V.B and of the random rounds
                     circuits in Sec. V.A).
* ``statevector`` -- dense 2^n brute-force simulation (the exact method that
                     Sec. I contrasts with tensor networks), n <= 12 here.
* ``mps``         -- FP64 matrix-product state: product-state initialisation
                     (Sec. IV, ITensor MPS implementation), single-qubit gates
                     contracted into the site tensor, adjacent two-qubit gates
                     by contraction to a rank-4 tensor followed by SVD with a
                     singular-value cutoff (Sec. II, Fig. "mpssvd"; Sec. IV),
                     and expectation values of Pauli strings by a full
                     left-to-right transfer-matrix sweep per term.
* ``energy``      -- E(theta) = sum_k c_k <psi(theta)|P_k|psi(theta)>, the
                     quantity the VQE loop of Sec. V.B evaluates per parameter
                     value, plus the parameter-shift gradient.
* ``mlp``         -- FP64 reference of the small MLP surrogate (forward,
                     backward, Adam) that checks the GPU training kernels.
* ``sampling``    -- exact shot sampling of a measurement of every qubit (the
                     MEASURE instructions of the Sec. V.B kernels), from the
                     state vector and from the MPS, driven by input uniforms.
* ``supergate``   -- application of an aggregate of gates on any qubits by
                     maximising the overlap of an output MPS with the input
                     network plus the gates (Sec. II, general gate action;
                     Sec. IV, ExaTENSOR MPS visitor): the gates as an MPO,
                     left/right environments and two-site updates.

Parity status of each function is stated in its docstring; every function
here is pinned by a ``-m "not gpu"`` test against a closed form, a textbook
identity, a library routine or brute force, except where a docstring says
"parity unpinned".
"""
