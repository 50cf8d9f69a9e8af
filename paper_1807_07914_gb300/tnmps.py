"""Thin ctypes binding of ``libtnmps.so`` (the C ABI in ``include/tnmps.h``).

Argument marshalling only: every step of circuit application and energy
evaluation runs in the library's CUDA kernels. PyTorch provides device
memory (the context arena and expectation workspaces are uint8 CUDA tensors)
and the current CUDA stream. There is no CPU fallback: importing this module
without the built library, or using it without a CUDA device, raises.
"""
import ctypes as C
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libtnmps.so")

OPS = {"I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "RX": 8, "RY": 9,
       "RZ": 10, "CNOT": 16, "CZ": 17, "SWAP": 18}
DTYPES = {"c128": 0, "c64": 1, "c64_bf16split": 2}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_NOMEM", 3: "ERR_UNSUPPORTED", 4: "ERR_NOT_CONVERGED",
          5: "ERR_NUMERIC", 6: "ERR_CUDA", 7: "ERR_INJECTED", 8: "ERR_TIMEOUT"}


class TnmpsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Gate(C.Structure):
    _fields_ = [("op", C.c_int32), ("q0", C.c_int32), ("q1", C.c_int32), ("param", C.c_int32),
                ("angle", C.c_double), ("scale", C.c_double)]


class Job(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("chi_max", C.c_int32), ("gates", C.c_void_p),
                ("n_gates", C.c_int32), ("theta", C.c_void_p), ("n_params", C.c_int32),
                ("term_off", C.c_void_p), ("sites", C.c_void_p), ("paulis", C.c_void_p),
                ("coeffs", C.c_void_p), ("n_terms", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("jacobi_shape", C.c_int32 * 3), ("gemm_stages", C.c_int32),
                ("sweep_fused", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(k, C.c_uint64) for k in ("gates2q", "gates2q_full", "jacobi_pair_rows",
                                          "jacobi_rotations", "jacobi_sweeps", "svds",
                                          "env_updates", "env_flops", "jacobi_rot_rows",
                                          "launches", "jacobi_alg_bytes")]


PROF_CLASSES = ("theta", "jacobi", "split", "move", "gate1", "env", "term", "env_tc", "fit",
                "svd_lq")


_lib = None


def lib():
    """Load the library once; raise if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libtnmps.so not built ({_LIB_PATH}); run "
                           "`python -m paper_1807_07914_gb300.build`")
    L = C.CDLL(_LIB_PATH)
    P, I, S, D = C.c_void_p, C.c_int, C.c_size_t, C.c_double
    sig = {
        "tnmps_status_string": (C.c_char_p, [I]),
        "tnmps_version": (C.c_char_p, []),
        "tnmps_state_bytes": (S, [I, I, I, I, I]),
        "tnmps_init": (I, [C.POINTER(P), I, I, I, I, I, P, S]),
        "tnmps_free": (None, [P]),
        "tnmps_set_cutoff": (I, [P, D]),
        "tnmps_set_stream": (I, [P, P]),
        "tnmps_reset": (I, [P]),
        "tnmps_apply_circuit": (I, [P, P, S, P, S]),
        "tnmps_apply_circuit_batched": (I, [P, P, S, P, S]),
        "tnmps_apply_circuit_batched_dev": (I, [P, P, S, P, S]),
        "tnmps_terms_create": (I, [C.POINTER(P), I, P, P, P, P, S]),
        "tnmps_terms_free": (None, [P]),
        "tnmps_terms_info": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_int64)]),
        "tnmps_expect_workspace_bytes": (S, [P, P, I]),
        "tnmps_expect_pauli_sum": (I, [P, P, P, S, P, P]),
        "tnmps_expect_pauli_sum_dev": (I, [P, P, P, S, P, P]),
        "tnmps_check": (I, [P]),
        "tnmps_get_bond_dims": (I, [P, P]),
        "tnmps_get_discarded_weight": (I, [P, P]),
        "tnmps_get_site": (I, [P, I, I, P, S, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "tnmps_get_centre": (I, [P]),
        "tnmps_get_stats": (I, [P, C.POINTER(Stats)]),
        "tnmps_last_error": (C.c_char_p, [P]),
        "tnmps_jacobi_svd_dev": (I, [I, I, I, I, P, I, P, P, I, P]),
        "tnmps_debug_inject": (I, [P, I, I]),
        "tnmps_expect_pauli_sum_noalloc": (I, [P, P, P, P]),
        "tnmps_sample_dev": (I, [P, P, I, P]),
        "tnmps_supergate_create": (I, [C.POINTER(P), I, P, S, P, S]),
        "tnmps_supergate_free": (None, [P]),
        "tnmps_supergate_info": (I, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), P]),
        "tnmps_supergate_mpo": (I, [P, P, S]),
        "tnmps_supergate_workspace_bytes": (S, [P, P]),
        "tnmps_apply_supergate": (I, [P, P, I, D, D, I, P, S, P, P, P]),
        "tnmps_gemm_bf16_dev": (I, [I, I, I, P, I, P, I, P, I, P]),
        "tnmps_mlp_bytes": (S, [I, I, I]),
        "tnmps_mlp_num_params": (C.c_int64, [I, I]),
        "tnmps_mlp_init": (I, [C.POINTER(P), I, I, I, P, S]),
        "tnmps_mlp_free": (None, [P]),
        "tnmps_mlp_set_stream": (I, [P, P]),
        "tnmps_mlp_last_error": (C.c_char_p, [P]),
        "tnmps_mlp_set_params": (I, [P, P]),
        "tnmps_mlp_get_params": (I, [P, P]),
        "tnmps_mlp_forward": (I, [P, P, I, P]),
        "tnmps_mlp_backward": (I, [P, P, P, I, P, P, P, P]),
        "tnmps_mlp_train_step": (I, [P, P, P, I, C.c_float, I, P]),
        "tnmps_batch_create": (I, [C.POINTER(P), P, I, D]),
        "tnmps_batch_bytes": (S, [P, I]),
        "tnmps_batch_bind": (I, [P, P, S, I, I, P]),
        "tnmps_batch_capture_graph": (I, [P]),
        "tnmps_batch_launch": (I, [P]),
        "tnmps_batch_results": (I, [P, P, P]),
        "tnmps_batch_info": (I, [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_double)]),
        "tnmps_batch_last_error": (C.c_char_p, [P]),
        "tnmps_batch_free": (None, [P]),
        "tnmps_profile": (I, [P, C.c_uint32]),
        "tnmps_profile_read": (I, [P, P, P]),
        "tnmps_alu_peak_dev": (I, [I, I, I, P, C.POINTER(C.c_double), P]),
        "tnmps_set_tuning": (I, [P, C.POINTER(Tuning)]),
        "tnmps_debug_wait_timeout": (I, [P, C.c_int64]),
        "tnmps_set_svd_tolerance": (I, [P, D]),
        "tnmps_set_svd_precondition": (I, [P, I]),
        "tnmps_mlp_check": (I, [P]),
        "tnmps_get_tuning": (I, [P, C.POINTER(Tuning)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def gate_array(circuit):
    """Gate records (name, q0, q1, param, angle, scale) -> ctypes array."""
    arr = (Gate * max(len(circuit), 1))()
    for i, (name, q0, q1, param, angle, scale) in enumerate(circuit):
        arr[i] = Gate(OPS[name], int(q0), int(q1 if q1 is not None else -1),
                      int(param if param is not None else -1), float(angle), float(scale))
    return arr


def _stream_handle(device):
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class PauliSum:
    """A term set in the library's trie form (host side)."""

    def __init__(self, n_qubits, terms):
        off, sites, paulis, coeffs = _csr(terms)
        self.n = int(n_qubits)
        self.n_terms = len(terms)
        h = C.c_void_p()
        st = lib().tnmps_terms_create(C.byref(h), self.n, _ptr(off), _ptr(sites), _ptr(paulis),
                                      _ptr(coeffs), self.n_terms)
        if st != 0:
            raise TnmpsError(st, "invalid Pauli terms")
        self._h = h
        self._keep = (off, sites, paulis, coeffs)

    def info(self):
        nn, dep, ml = C.c_int64(), C.c_int32(), C.c_int64()
        lib().tnmps_terms_info(self._h, C.byref(nn), C.byref(dep), C.byref(ml))
        return {"nodes": nn.value, "depth": dep.value, "max_level_nodes": ml.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().tnmps_terms_free(self._h)
            self._h = None

    __del__ = close


class Supergate:
    """An ordered aggregate of gates on any qubits, bound to parameter values,
    held by the library as a matrix-product operator over the qubits it
    touches (host side; no device work)."""

    def __init__(self, n_qubits, circuit, theta=None):
        self.n = int(n_qubits)
        th = np.ascontiguousarray(theta if theta is not None else [0.0], dtype=np.float64)
        arr = gate_array(circuit)
        h = C.c_void_p()
        st = lib().tnmps_supergate_create(C.byref(h), self.n, arr, len(circuit), _ptr(th),
                                          0 if theta is None else th.size)
        if st != 0:
            raise TnmpsError(st, "invalid super-gate")
        self._h = h
        first, last = C.c_int32(), C.c_int32()
        lib().tnmps_supergate_info(h, C.byref(first), C.byref(last), None)
        self.first, self.last = first.value, last.value
        bonds = np.zeros(self.last - self.first + 2, np.int32)
        lib().tnmps_supergate_info(h, None, None, _ptr(bonds))
        self.bonds = bonds

    def mpo(self):
        """The MPO site tensors [w_left, 2 out, 2 in, w_right], complex128."""
        w = self.bonds
        sizes = [int(w[i]) * 4 * int(w[i + 1]) for i in range(len(w) - 1)]
        buf = np.zeros(2 * sum(sizes), np.float64)
        st = lib().tnmps_supergate_mpo(self._h, _ptr(buf), buf.size)
        if st != 0:
            raise TnmpsError(st, "MPO read failed")
        z = buf.view(np.complex128)
        out, o = [], 0
        for i, n in enumerate(sizes):
            out.append(z[o:o + n].reshape(int(w[i]), 2, 2, int(w[i + 1])).copy())
            o += n
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().tnmps_supergate_free(self._h)
            self._h = None

    __del__ = close


def _csr(terms):
    off = [0]
    s, p, c = [], [], []
    for coeff, sites, paulis in terms:
        s += [int(x) for x in sites]
        p += [int(x) for x in paulis]
        off.append(len(s))
        c.append(float(coeff))
    return (np.asarray(off, np.int32), np.asarray(s if s else [0], np.int32),
            np.asarray(p if p else [0], np.uint8), np.asarray(c if c else [0.0], np.float64))


class MPSBatch:
    """``batch`` MPS states of ``n`` qubits on one CUDA device."""

    def __init__(self, n, chi_max, batch=1, dtype="c128", max_params=0, eps=1e-4,
                 device="cuda:0"):
        if not torch.cuda.is_available():
            raise RuntimeError("tnmps needs a CUDA device; there is no CPU fallback")
        L = lib()
        self.device = torch.device(device)
        self.n, self.chi, self.batch, self.dtype = int(n), int(chi_max), int(batch), dtype
        self.max_params = int(max_params)
        nbytes = L.tnmps_state_bytes(self.n, self.chi, DTYPES[dtype], self.batch, self.max_params)
        if nbytes == 0:
            raise TnmpsError(1, "invalid sizes")
        with torch.cuda.device(self.device):
            self.arena = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            h = C.c_void_p()
            st = L.tnmps_init(C.byref(h), self.n, self.chi, DTYPES[dtype], self.batch,
                              self.max_params, _ptr(self.arena), nbytes)
        if st != 0:
            raise TnmpsError(st, "init failed")
        self._h = h
        self._ws = {}
        self._sg_ws = None
        self.set_stream()
        self.set_cutoff(eps)

    # -------------------------------------------------------------- helpers
    def _check(self, st):
        if st != 0:
            raise TnmpsError(st, lib().tnmps_last_error(self._h).decode())

    def set_stream(self, stream=None):
        s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(
            self.device).cuda_stream
        self._check(lib().tnmps_set_stream(self._h, C.c_void_p(s)))

    def set_cutoff(self, eps):
        self._check(lib().tnmps_set_cutoff(self._h, float(eps)))

    def set_svd_tolerance(self, factor):
        """Factor on the Jacobi SVD's orthogonality tolerance (1 = rounding level)."""
        self._check(lib().tnmps_set_svd_tolerance(self._h, float(factor)))

    def set_svd_precondition(self, mode):
        """1 (default): the Jacobi SVD runs on L of Theta = L Q^H (same singular
        values and left vectors, fewer sweeps); 0: on Theta itself."""
        self._check(lib().tnmps_set_svd_precondition(self._h, int(mode)))

    def reset(self):
        self._check(lib().tnmps_reset(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().tnmps_free(self._h)
            self._h = None

    __del__ = close

    # -------------------------------------------------------------- circuits
    def apply_circuit(self, circuit, thetas=None):
        """thetas: None, [n_params] (shared) or [batch, n_params] (host)."""
        g = gate_array(circuit)
        if thetas is None:
            self._check(lib().tnmps_apply_circuit(self._h, g, len(circuit), None, 0))
            return
        th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64))
        if th.ndim == 1:
            self._check(lib().tnmps_apply_circuit(self._h, g, len(circuit), _ptr(th), th.size))
        else:
            assert th.shape[0] == self.batch
            self._check(lib().tnmps_apply_circuit_batched(self._h, g, len(circuit), _ptr(th),
                                                          th.shape[1]))

    def apply_circuit_dev(self, gates_c, thetas_dev, n_gates=None):
        """Asynchronous: gates_c from gate_array(), thetas_dev a float64 CUDA
        tensor [batch, n_params]."""
        assert thetas_dev.is_cuda and thetas_dev.dtype == torch.float64
        assert thetas_dev.dim() == 2 and thetas_dev.shape[0] == self.batch, \
            "thetas_dev must hold one row per state"
        assert thetas_dev.is_contiguous()
        ng = len(gates_c) if n_gates is None else n_gates
        self._check(lib().tnmps_apply_circuit_batched_dev(self._h, gates_c, ng, _ptr(thetas_dev),
                                                          thetas_dev.shape[-1]))

    # -------------------------------------------------------------- energies
    def workspace(self, terms, chunk=0):
        key = (id(terms), chunk)
        ws = self._ws.get(key)
        if ws is None:
            nb = lib().tnmps_expect_workspace_bytes(self._h, terms._h, int(chunk))
            if nb == 0:
                raise TnmpsError(1, "workspace size query failed")
            ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self._ws = {key: ws}
        return ws

    def device_name(self):
        return torch.cuda.get_device_name(self.device)

    def workspace_bytes(self, terms, chunk=0):
        """Device bytes of an expectation workspace for ``chunk`` states at a
        time (0: the whole batch); 0 on a mismatch."""
        return int(lib().tnmps_expect_workspace_bytes(self._h, terms._h, int(chunk)))

    def drop_workspaces(self):
        """Release the cached expectation workspace (PyTorch memory)."""
        self._ws = {}

    def expect(self, terms, per_term=False, chunk=0):
        """Energies [batch] (and Re<P_k> [batch, T]) as numpy, synchronous."""
        ws = self.workspace(terms, chunk)
        e = np.zeros(self.batch, np.float64)
        pt = np.zeros((self.batch, terms.n_terms), np.float64) if per_term else None
        self._check(lib().tnmps_expect_pauli_sum(self._h, terms._h, _ptr(ws), ws.numel(),
                                                 _ptr(e), _ptr(pt)))
        return (e, pt) if per_term else e

    def expect_dev(self, terms, energy, per_term=None, chunk=0):
        """Asynchronous: energy (and per_term) float64 CUDA tensors."""
        ws = self.workspace(terms, chunk)
        self._check(lib().tnmps_expect_pauli_sum_dev(self._h, terms._h, _ptr(ws), ws.numel(),
                                                     _ptr(energy), _ptr(per_term)))

    def expect_noalloc(self, terms, energy, per_term=None):
        """Like expect_dev, for callers that cannot allocate device memory:
        the library's own static scratch replaces the workspace. Asynchronous
        when the scratch already holds this context's plan for these terms;
        otherwise the plan upload synchronises the stream first."""
        self._check(lib().tnmps_expect_pauli_sum_noalloc(self._h, terms._h, _ptr(energy),
                                                         _ptr(per_term)))

    # -------------------------------------------------------------- measurement
    def sample_dev(self, uniforms_dev, bits_dev):
        """Asynchronous: uniforms_dev float64 CUDA tensor [batch, shots, n] in
        [0, 1); bits_dev uint8 CUDA tensor of the same shape receives the
        outcomes (qubit q of shot k is 0 iff u[b, k, q] < P(0 | qubits above))."""
        assert uniforms_dev.is_cuda and uniforms_dev.dtype == torch.float64
        assert bits_dev.is_cuda and bits_dev.dtype == torch.uint8
        assert uniforms_dev.shape == (self.batch, uniforms_dev.shape[1], self.n)
        assert bits_dev.shape == uniforms_dev.shape
        self._check(lib().tnmps_sample_dev(self._h, _ptr(uniforms_dev), uniforms_dev.shape[1],
                                           _ptr(bits_dev)))

    def sample(self, uniforms):
        """Measurement shots as a uint8 numpy array [batch, shots, n] for
        host uniforms [batch, shots, n] (synchronous)."""
        u = torch.as_tensor(np.ascontiguousarray(uniforms, dtype=np.float64)).to(self.device)
        bits = torch.empty(u.shape, dtype=torch.uint8, device=self.device)
        self.sample_dev(u, bits)
        self.check()
        return bits.cpu().numpy()

    # -------------------------------------------------------------- super-gates
    def apply_supergate(self, sg, chi_max=None, target=1e-10, tol=1e-12, max_sweeps=8):
        """Apply a Supergate by overlap maximisation (synchronous). Returns
        (fidelity [batch], fidelity of the first iterate [batch],
        {"sweeps", "stages", "chi"})."""
        nb = lib().tnmps_supergate_workspace_bytes(self._h, sg._h)
        if nb == 0:
            raise TnmpsError(1, "super-gate workspace query failed")
        if self._sg_ws is None or self._sg_ws.numel() < nb:
            self._sg_ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
        f = np.zeros(self.batch, np.float64)
        f0 = np.zeros(self.batch, np.float64)
        info = np.zeros(3, np.int32)
        self._check(lib().tnmps_apply_supergate(
            self._h, sg._h, int(chi_max if chi_max is not None else self.chi), float(target),
            float(tol), int(max_sweeps), _ptr(self._sg_ws), self._sg_ws.numel(), _ptr(f),
            _ptr(f0), _ptr(info)))
        return f, f0, {"sweeps": int(info[0]), "stages": int(info[1]), "chi": int(info[2])}

    # -------------------------------------------------------------- inspection
    def check(self):
        self._check(lib().tnmps_check(self._h))

    def bond_dims(self):
        d = np.zeros((self.batch, max(self.n - 1, 1)), np.int32)
        self._check(lib().tnmps_get_bond_dims(self._h, _ptr(d)))
        return d[:, : self.n - 1]

    def discarded(self):
        w = np.zeros(self.batch, np.float64)
        self._check(lib().tnmps_get_discarded_weight(self._h, _ptr(w)))
        return w

    def site(self, b, i):
        cap = self.chi * 2 * self.chi
        buf = np.zeros(2 * cap, np.float64)
        dl, dr = C.c_int32(), C.c_int32()
        self._check(lib().tnmps_get_site(self._h, b, i, _ptr(buf), cap, C.byref(dl), C.byref(dr)))
        z = buf[: 2 * dl.value * 2 * dr.value].view(np.complex128)
        return z.reshape(dl.value, 2, dr.value)

    def centre(self):
        return lib().tnmps_get_centre(self._h)

    def stats(self):
        s = Stats()
        self._check(lib().tnmps_get_stats(self._h, C.byref(s)))
        return {k: int(getattr(s, k)) for k, _ in Stats._fields_}

    def profile(self, classes=PROF_CLASSES):
        """Start CUDA-event timing of the named kernel classes (None = stop)."""
        mask = 0
        for k in classes or ():
            mask |= 1 << PROF_CLASSES.index(k)
        self._check(lib().tnmps_profile(self._h, mask))

    def profile_read(self):
        ms = np.zeros(len(PROF_CLASSES), np.float64)
        cnt = np.zeros(len(PROF_CLASSES), np.uint64)
        self._check(lib().tnmps_profile_read(self._h, _ptr(ms), _ptr(cnt)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_CLASSES)}

    def set_tuning(self, jacobi_shape=(0, 0, 0), gemm_stages=0, sweep_fused=0):
        """Launch shapes of the context's kernels (see tnmps_tuning in
        include/tnmps.h); the results do not depend on them."""
        t = Tuning()
        for i, v in enumerate(jacobi_shape):
            t.jacobi_shape[i] = int(v)
        t.gemm_stages = int(gemm_stages)
        t.sweep_fused = int(sweep_fused)
        self._check(lib().tnmps_set_tuning(self._h, C.byref(t)))

    def get_tuning(self):
        t = Tuning()
        self._check(lib().tnmps_get_tuning(self._h, C.byref(t)))
        return {"jacobi_shape": [int(v) for v in t.jacobi_shape], "gemm_stages": int(t.gemm_stages),
                "sweep_fused": int(t.sweep_fused)}

    def debug_wait_timeout(self, max_cycles=2000000):
        """Enqueue a device wait that runs out after max_cycles SM clocks and
        raises the timeout flag (failure-detection tests)."""
        self._check(lib().tnmps_debug_wait_timeout(self._h, int(max_cycles)))

    def inject(self, nth, status):
        self._check(lib().tnmps_debug_inject(self._h, int(nth), int(status)))


class Surrogate:
    """The MLP surrogate d_in -> width -> width -> 1 (SiLU) on one GPU."""

    def __init__(self, d_in, width=256, max_batch=4096, device="cuda:0"):
        L = lib()
        self.device = torch.device(device)
        self.d, self.w, self.max_batch = int(d_in), int(width), int(max_batch)
        nb = L.tnmps_mlp_bytes(self.d, self.w, self.max_batch)
        if nb == 0:
            raise TnmpsError(1, "invalid surrogate sizes")
        self.n_params = int(L.tnmps_mlp_num_params(self.d, self.w))
        self.arena = torch.empty(nb, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        st = L.tnmps_mlp_init(C.byref(h), self.d, self.w, self.max_batch, _ptr(self.arena), nb)
        if st != 0:
            raise TnmpsError(st, "surrogate init failed")
        self._h = h
        self._check(L.tnmps_mlp_set_stream(h, C.c_void_p(
            torch.cuda.current_stream(self.device).cuda_stream)))
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step = 0

    def _check(self, st):
        if st != 0:
            raise TnmpsError(st, lib().tnmps_mlp_last_error(self._h).decode())

    def check(self):
        """Synchronise; raise if a tensor-core GEMM wait ran out since the last check."""
        self._check(lib().tnmps_mlp_check(self._h))

    def set_params(self, p):
        p = torch.as_tensor(p, dtype=torch.float32, device=self.device).contiguous()
        assert p.numel() == self.n_params
        self._check(lib().tnmps_mlp_set_params(self._h, _ptr(p)))
        torch.cuda.current_stream(self.device).synchronize()
        self.step = 0

    def get_params(self):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        self._check(lib().tnmps_mlp_get_params(self._h, _ptr(p)))
        return p

    def forward(self, x):
        x = x.contiguous()
        y = torch.empty(x.shape[0], dtype=torch.float32, device=self.device)
        self._check(lib().tnmps_mlp_forward(self._h, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def backward(self, x, target=None, want_params=True, want_x=True):
        x = x.contiguous()
        B = x.shape[0]
        y = torch.empty(B, dtype=torch.float32, device=self.device)
        gp = torch.empty(self.n_params, dtype=torch.float32, device=self.device) if want_params else None
        gx = torch.empty_like(x) if want_x else None
        self._check(lib().tnmps_mlp_backward(self._h, _ptr(x), _ptr(target), B, _ptr(y),
                                             _ptr(self.loss), _ptr(gp), _ptr(gx)))
        return y, gp, gx

    def train_step(self, x, target, lr):
        self.step += 1
        self._check(lib().tnmps_mlp_train_step(self._h, _ptr(x.contiguous()),
                                               _ptr(target.contiguous()), x.shape[0],
                                               float(lr), self.step, _ptr(self.loss)))
        return self.loss

    def close(self):
        if getattr(self, "_h", None):
            lib().tnmps_mlp_free(self._h)
            self._h = None

    __del__ = close


class Batch:
    """Many independent circuits (each: n, chi_max, gate list, theta, Pauli
    sum) evaluated in one persistent launch (complex64 state, FP64 energies)."""

    def __init__(self, jobs, cutoff=1e-10, ctas=None, block_cols=32, device="cuda:0"):
        L = lib()
        self.device = torch.device(device)
        self._keep = []
        arr = (Job * len(jobs))()
        for i, jb in enumerate(jobs):
            g = gate_array(jb["circuit"])
            th = np.ascontiguousarray(np.asarray(jb["theta"], dtype=np.float64))
            off, sites, paulis, coeffs = _csr(jb["terms"])
            self._keep += [g, th, off, sites, paulis, coeffs]
            arr[i] = Job(jb["n"], jb["chi"], C.cast(g, C.c_void_p), len(jb["circuit"]),
                         th.ctypes.data, th.size, off.ctypes.data, sites.ctypes.data,
                         paulis.ctypes.data, coeffs.ctypes.data, len(jb["terms"]))
        h = C.c_void_p()
        st = L.tnmps_batch_create(C.byref(h), arr, len(jobs), float(cutoff))
        if st != 0:
            raise TnmpsError(st, "batch planning failed")
        self._h = h
        self.n_jobs = len(jobs)
        props = torch.cuda.get_device_properties(self.device)
        self.ctas = ctas or props.multi_processor_count
        nb = L.tnmps_batch_bytes(h, self.ctas)
        self.arena = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self._check(L.tnmps_batch_bind(h, _ptr(self.arena), nb, self.ctas, block_cols,
                                       C.c_void_p(self.stream.cuda_stream)))

    def _check(self, st):
        if st != 0:
            raise TnmpsError(st, lib().tnmps_batch_last_error(self._h).decode())

    def capture_graph(self):
        self._check(lib().tnmps_batch_capture_graph(self._h))

    def launch(self):
        self._check(lib().tnmps_batch_launch(self._h))

    def results(self):
        e = np.zeros(self.n_jobs)
        w = np.zeros(self.n_jobs)
        self._check(lib().tnmps_batch_results(self._h, _ptr(e), _ptr(w)))
        return e, w

    def run(self):
        self.launch()
        return self.results()[0]

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_double()
        lib().tnmps_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c))
        return {"ops": a.value, "trie_nodes": b.value, "est_cost": c.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().tnmps_batch_free(self._h)
            self._h = None

    __del__ = close


def gemm_bf16(a, b, out=None, stream=None):
    """C = A B^T on the tensor cores: a [M, K] and b [N, K] bfloat16 CUDA
    tensors (K-major), result float32 [M, N]."""
    assert a.dtype == torch.bfloat16 and b.dtype == torch.bfloat16 and a.is_cuda and b.is_cuda
    M, K = a.shape
    N = b.shape[0]
    out = torch.empty((M, N), dtype=torch.float32, device=a.device) if out is None else out
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(a.device).cuda_stream
    st = lib().tnmps_gemm_bf16_dev(M, N, K, _ptr(a), a.stride(0), _ptr(b), b.stride(0), _ptr(out),
                                   out.stride(0), C.c_void_p(s))
    if st != 0:
        raise TnmpsError(st, "gemm_bf16 failed")
    return out


def alu_peak_dev(bits, blocks, iters, sink, stream=None):
    """Enqueue the FMA-throughput kernel (FP32 for bits = 32, FP64 for 64)
    into ``sink`` (a float32 / float64 CUDA tensor of blocks * 256 values);
    returns the launch's floating-point operation count."""
    assert sink.is_cuda and sink.numel() >= blocks * 256
    assert sink.dtype == {32: torch.float32, 64: torch.float64}[bits]
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(sink.device).cuda_stream
    fl = C.c_double()
    st = lib().tnmps_alu_peak_dev(int(bits), int(blocks), int(iters), _ptr(sink), C.byref(fl),
                                  C.c_void_p(s))
    if st != 0:
        raise TnmpsError(st, "alu_peak_dev failed")
    return fl.value


def jacobi_svd_dev(a, m, n, sigma, sweeps, max_sweeps=0, stream=None):
    """One-sided Jacobi on a [batch, n, lda] complex CUDA tensor (column j of
    matrix b is a[b, j, :m]); in place. sigma float64 [batch, n], sweeps int32
    [batch]."""
    dt = {torch.complex128: 0, torch.complex64: 1}[a.dtype]
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(a.device).cuda_stream
    st = lib().tnmps_jacobi_svd_dev(dt, a.shape[0], int(m), int(n), _ptr(a), a.shape[2],
                                    _ptr(sigma), _ptr(sweeps), int(max_sweeps), C.c_void_p(s))
    if st != 0:
        raise TnmpsError(st, "jacobi_svd_dev failed")
