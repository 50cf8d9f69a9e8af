"""Launch-shape autotuner of a context's hot kernels, run on the caller's own
workload.

Knobs (``tnmps_tuning`` in include/tnmps.h, plus the expectation chunk):

* ``jacobi_shape[c]`` -- CTA shape of the complex64 Jacobi SVD for blocks of up
  to 64, 128 and 256 rows (two CTAs of 256 threads per SM with 16-column
  blocks, or one CTA of 512 threads per SM with 32-column blocks);
* ``gemm_stages`` -- shared-memory ring depth (2 or 3) of the tensor-core
  GEMMs of the BF16-split form (two-site block, split, transfer sweeps);
* ``sweep_fused`` -- the transfer sweeps of the BF16-split form as two
  launches per trie level or as one launch running both steps per CTA;
* ``chunk`` -- states per expectation chunk of each term set (the workspace
  size: a wider chunk fills more SMs per trie level, a narrower one keeps the
  environments in L2).

Every choice computes the same results (up to FP32 summation order); only the
time differs. The tuner starts from the defaults and goes through the knobs
one at a time (coordinate descent), timing each candidate on the caller's
circuit or term set with CUDA events on the context's stream and keeping the
fastest. The result is cached in a JSON table (``$TNMPS_AUTOTUNE_CACHE``,
default ``~/.cache/tnmps/autotune.json``) keyed by the device, the register
size, bond cap, arithmetic form, batch and the term sets' sizes.
"""
import hashlib
import json
import os

import torch

DEFAULT = {"jacobi_shape": [0, 0, 0], "gemm_stages": 0, "sweep_fused": 0}


def cache_path():
    return os.environ.get("TNMPS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tnmps",
                                       "autotune.json"))


def _key(m, term_sets):
    h = hashlib.sha1()
    h.update(str(m.device_name()).encode())
    h.update(repr((m.n, m.chi, m.dtype, m.batch)).encode())
    for name, ps in term_sets.items():
        h.update(repr((name, ps.n_terms, ps.info()["max_level_nodes"])).encode())
    return h.hexdigest()[:16]


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    try:
        os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
        with open(cache_path(), "w") as f:
            json.dump(table, f, indent=1)
    except OSError:
        pass


class CudaTimer:
    """Seconds of ``fn`` by CUDA events on the context's current stream."""

    def __init__(self, device):
        self.device = device
        self.stream = torch.cuda.current_stream(device)

    def sync(self):
        torch.cuda.synchronize(self.device)

    def __call__(self, fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        fn()
        e1.record(self.stream)
        torch.cuda.synchronize(self.device)
        return e0.elapsed_time(e1) / 1000.0


def tune_context(m, gates_c, thetas_dev, term_sets, chunk_candidates=(8, 16, 32, 64),
                 max_workspace_bytes=40 << 30, use_cache=True, timer=None, energy=None,
                 margin=0.01):
    """Tune the context ``m`` for the circuit (``gates_c`` from gate_array,
    ``thetas_dev`` [batch, n_params] on the device) and the named term sets
    (``{name: PauliSum}``). Leaves the best launch shapes set on ``m``.

    ``timer`` (default: CUDA events on the context's stream) times a callable
    and ``timer.sync()`` waits for the device; ``energy`` is the device output
    buffer of the trial passes (default: a new one). A candidate replaces the
    current choice only when it is faster by more than ``margin`` (relative),
    so that timing noise does not move a knob away from its default.

    Returns a report: the chosen ``tuning`` and ``chunk`` per term set, the
    seconds of the circuit and of each term set's pass with the defaults and
    with the chosen configuration, every candidate's time, and whether it came
    from the cache."""
    key = _key(m, term_sets)
    table = _load() if use_cache else {}
    if key in table:
        rep = dict(table[key])
        m.set_tuning(**rep["tuning"])
        rep["cached"] = True
        return rep
    timer = timer or CudaTimer(m.device)
    if energy is None:
        energy = torch.empty(m.batch, dtype=torch.float64, device=m.device)

    def circuit():
        m.reset()
        m.apply_circuit_dev(gates_c, thetas_dev)

    def circuit_time(cfg):
        m.set_tuning(**cfg)
        circuit()                    # first pass loads the kernels of this shape
        timer.sync()
        return min(timer(circuit), timer(circuit))

    cfg = json.loads(json.dumps(DEFAULT))
    trials = []
    best_t = circuit_time(cfg)
    default_circuit = best_t
    trials.append({"tuning": json.loads(json.dumps(cfg)), "circuit_s": best_t})
    alternatives = [("jacobi_shape", 2, 1), ("jacobi_shape", 1, 1), ("jacobi_shape", 0, 1)]
    if m.dtype == "c64_bf16split":
        alternatives.append(("gemm_stages", None, 2))
    if m.dtype == "c128":
        alternatives = []            # complex128 has a single shape
    for name, idx, val in alternatives:
        cand = json.loads(json.dumps(cfg))
        if idx is None:
            cand[name] = val
        else:
            cand[name][idx] = val
        t = circuit_time(cand)
        trials.append({"tuning": cand, "circuit_s": t})
        if t < (1 - margin) * best_t:
            best_t, cfg = t, cand
    m.set_tuning(**cfg)
    circuit()
    timer.sync()
    # states per expectation chunk, per term set (on the circuit's final states)
    chunks, passes = {}, {}
    for name, ps in term_sets.items():
        res = {}
        for ch in (0,) + tuple(c for c in chunk_candidates if c < m.batch):
            nb = m.workspace_bytes(ps, ch)
            if nb == 0 or nb > max_workspace_bytes:
                continue
            m.expect_dev(ps, energy, chunk=ch)       # workspace, plan upload
            timer.sync()
            res[ch] = min(timer(lambda: m.expect_dev(ps, energy, chunk=ch)) for _ in range(2))
        m.drop_workspaces()
        best = min(res, key=res.get)
        first = 0 if 0 in res else min(res)           # the whole batch when it fits
        if not res[best] < (1 - margin) * res[first]:
            best = first
        chunks[name] = int(best)
        passes[name] = {"candidates_s": {str(k): v for k, v in res.items()},
                        "default_chunk": 0 if 0 in res else int(min(res)),
                        "best_s": res[best]}
    # the sweep form, on the sum of the term sets' passes at their chunks
    if m.dtype == "c64_bf16split" and passes:
        def passes_time():
            tot = 0.0
            for name, ps in term_sets.items():
                m.expect_dev(ps, energy, chunk=chunks[name])
                timer.sync()
                tot += min(timer(lambda: m.expect_dev(ps, energy, chunk=chunks[name]))
                           for _ in range(2))
            m.drop_workspaces()
            return tot
        base = passes_time()
        alt = json.loads(json.dumps(cfg))
        alt["sweep_fused"] = 1
        m.set_tuning(**alt)
        t_alt = passes_time()
        trials.append({"tuning": alt, "expect_passes_s": t_alt, "versus": base})
        if t_alt < (1 - margin) * base:
            cfg = alt
        m.set_tuning(**cfg)
    rep = {"tuning": cfg, "chunk": chunks, "circuit_s": {"default": default_circuit,
                                                          "tuned": best_t},
           "expect_s": passes, "trials": trials, "cached": False,
           "how": "coordinate descent from the defaults; each candidate timed with CUDA events "
                  "on the caller's workload (best of two circuit passes, one expectation pass)"}
    table[key] = {k: v for k, v in rep.items() if k != "cached"}
    if use_cache:
        _store(table)
    return rep
