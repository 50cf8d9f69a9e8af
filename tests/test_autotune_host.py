"""The autotuner's search on a fake context with a known cost model (no GPU):
coordinate descent over the launch shapes from the defaults, the chunk of
each term set, the sweep form on the sum of the passes, workspace limits and
the cache round trip."""
import json

import pytest

from paper_1807_07914_gb300 import autotune


class FakeTerms:
    def __init__(self, n_terms, width):
        self.n_terms, self.width = n_terms, width

    def info(self):
        return {"max_level_nodes": self.width}


class FakeCtx:
    """Costs: the circuit depends on the Jacobi shapes and the ring depth, a
    pass on the chunk and on the sweep form; the clock advances by them."""

    def __init__(self, circuit_cost, pass_cost, dtype="c64_bf16split", batch=304):
        self.n, self.chi, self.dtype, self.batch = 40, 128, dtype, batch
        self.device = None
        self.circuit_cost, self.pass_cost = circuit_cost, pass_cost
        self.cfg = dict(autotune.DEFAULT)
        self.clock = 0.0
        self.dropped = 0

    def device_name(self):
        return "fake-gpu"

    def set_tuning(self, jacobi_shape=(0, 0, 0), gemm_stages=0, sweep_fused=0):
        self.cfg = {"jacobi_shape": list(jacobi_shape), "gemm_stages": gemm_stages,
                    "sweep_fused": sweep_fused}

    def get_tuning(self):
        return json.loads(json.dumps(self.cfg))

    def reset(self):
        pass

    def apply_circuit_dev(self, gates, th):
        self.clock += self.circuit_cost(self.cfg)

    def expect_dev(self, ps, energy, chunk=0):
        self.clock += self.pass_cost(ps, chunk, self.cfg)

    def workspace_bytes(self, ps, chunk):
        return (chunk or self.batch) * ps.width * 1000

    def drop_workspaces(self):
        self.dropped += 1


class FakeTimer:
    def __init__(self, m):
        self.m = m

    def sync(self):
        pass

    def __call__(self, fn):
        t0 = self.m.clock
        fn()
        return self.m.clock - t0


def circuit_cost(cfg):
    js = cfg["jacobi_shape"]
    # class 1 and 0 prefer the alternative, class 2 the default, stages 2 is worse
    return (3.0 - 0.06 * js[1] - 0.04 * js[0] + 0.2 * js[2] + 0.05 * (cfg["gemm_stages"] == 2)
            - 0.01 * cfg["sweep_fused"])


def pass_cost(ps, chunk, cfg):
    base = {0: 1.0, 8: 1.3, 16: 1.2, 32: 1.05, 64: 0.98}[chunk] * ps.n_terms / 1000
    if not cfg["sweep_fused"]:
        return base
    return base * (0.9 if ps.n_terms < 500 else 1.05)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    monkeypatch.setenv("TNMPS_AUTOTUNE_CACHE", str(tmp_path / "t.json"))
    return tmp_path / "t.json"


def test_coordinate_descent_chunks_and_sweep_form(cache):
    m = FakeCtx(circuit_cost, pass_cost)
    sets = {"heis": FakeTerms(157, 118), "rand": FakeTerms(2000, 808)}
    rep = autotune.tune_context(m, None, None, sets, max_workspace_bytes=304 * 500 * 1000,
                                timer=FakeTimer(m), energy=object())
    assert rep["tuning"]["jacobi_shape"] == [1, 1, 0] and rep["tuning"]["gemm_stages"] == 0
    assert m.get_tuning() == rep["tuning"]
    assert rep["circuit_s"]["default"] == pytest.approx(3.0)
    assert rep["circuit_s"]["tuned"] == pytest.approx(2.90)
    # the whole batch fits for the chain (118 x 304 kB) but not for the random set
    assert rep["chunk"] == {"heis": 64, "rand": 64}
    assert "0" in rep["expect_s"]["heis"]["candidates_s"]
    assert "0" not in rep["expect_s"]["rand"]["candidates_s"]
    # fused: 10 % faster on the chain only, slower in sum -> two launches kept
    assert rep["tuning"]["sweep_fused"] == 0 and m.dropped >= 2
    again = autotune.tune_context(FakeCtx(circuit_cost, pass_cost), None, None, sets,
                                  timer=FakeTimer(m), energy=object())
    assert again["cached"] and again["tuning"] == rep["tuning"]
    assert json.loads(cache.read_text())


def test_sweep_form_taken_when_the_sum_drops(cache):
    m = FakeCtx(circuit_cost, pass_cost)
    sets = {"heis": FakeTerms(157, 118)}
    rep = autotune.tune_context(m, None, None, sets, use_cache=False, timer=FakeTimer(m),
                                energy=object())
    assert rep["tuning"]["sweep_fused"] == 1 and not cache.exists()


def test_gains_below_the_margin_keep_the_default(cache):
    m = FakeCtx(lambda cfg: 3.0 - 0.02 * cfg["jacobi_shape"][1], pass_cost)
    rep = autotune.tune_context(m, None, None, {"heis": FakeTerms(157, 118)}, use_cache=False,
                                timer=FakeTimer(m), energy=object(), margin=0.01)
    assert rep["tuning"]["jacobi_shape"] == [0, 0, 0]          # 0.7 % is noise-level
    rep = autotune.tune_context(m, None, None, {"heis": FakeTerms(157, 118)}, use_cache=False,
                                timer=FakeTimer(m), energy=object(), margin=0.001)
    assert rep["tuning"]["jacobi_shape"] == [0, 1, 0]


def test_complex128_has_one_shape(cache):
    m = FakeCtx(circuit_cost, pass_cost, dtype="c128")
    rep = autotune.tune_context(m, None, None, {"heis": FakeTerms(157, 118)}, use_cache=False,
                                timer=FakeTimer(m), energy=object())
    assert rep["tuning"] == autotune.DEFAULT and len(rep["trials"]) == 1
