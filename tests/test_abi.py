"""The C-ABI library builds, loads without a GPU and exports every function
that include/tnmps.h declares; host-only entry points behave."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libt():
    from paper_1807_07914_gb300 import build, tnmps
    build.build()
    return tnmps


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(tnmps_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("tnmps_init", "tnmps_apply_circuit", "tnmps_apply_circuit_batched",
                 "tnmps_expect_pauli_sum", "tnmps_expect_pauli_sum_dev", "tnmps_free"):
        assert must in names


def test_library_exports_every_declared_symbol(libt):
    L = C.CDLL(libt._LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_host_only_entry_points(libt):
    L = libt.lib()
    assert L.tnmps_version().decode().startswith("tnmps")
    assert L.tnmps_status_string(4).decode() == "SVD did not converge"
    assert L.tnmps_status_string(8).decode() == "device wait timed out"
    # arena size: grows with batch, rejects bad sizes
    a = L.tnmps_state_bytes(40, 128, 0, 1, 800)
    b = L.tnmps_state_bytes(40, 128, 0, 2, 800)
    assert 0 < a < b
    assert L.tnmps_state_bytes(0, 16, 0, 1, 0) == 0
    assert L.tnmps_state_bytes(8, 1000, 0, 1, 0) == 0
    assert L.tnmps_state_bytes(8, 16, 5, 1, 0) == 0
    # complex64 arena is smaller than complex128
    assert L.tnmps_state_bytes(40, 128, 1, 4, 0) < L.tnmps_state_bytes(40, 128, 0, 4, 0)


def test_term_trie_on_host(libt):
    """The prefix trie shares left-environment prefixes: Heisenberg-type
    terms XX, YY, ZZ, Z starting at a site need 6 nodes per start site."""
    n = 6
    terms = []
    for i in range(n - 1):
        for p in (1, 2, 3):
            terms.append((1.0, (i, i + 1), (p, p)))
    for i in range(n):
        terms.append((0.5, (i,), (3,)))
    ps = libt.PauliSum(n, terms)
    info = ps.info()
    assert info["depth"] == 2
    # start sites 0..4: X, Y, Z at level 1 and XX, YY, ZZ at level 2; site 5: Z only
    assert info["nodes"] == 6 * (n - 1) + 1
    # identical prefixes are shared: ZZ..., ZX... share the Z node
    ps2 = libt.PauliSum(4, [(1.0, (0, 1), (3, 3)), (1.0, (0, 1), (3, 1)), (1.0, (0,), (3,))])
    assert ps2.info()["nodes"] == 3
    # invalid terms are rejected on the host
    with pytest.raises(libt.TnmpsError):
        libt.PauliSum(4, [(1.0, (0, 0), (1, 1))])
    with pytest.raises(libt.TnmpsError):
        libt.PauliSum(4, [(1.0, (7,), (1,))])
    with pytest.raises(libt.TnmpsError):
        libt.PauliSum(4, [(1.0, (1,), (4,))])
