"""C ABI checks that need no GPU: every declared symbol is exported, argument
validation, and the host-side code construction (GF(2) elimination, positions,
parity map) against the oracle, bit for bit."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import ldpc_synth as S
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2201_04265_gb300 import build_lib
    build_lib.build()
    import paper_2201_04265_gb300 as L
    return L


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ldpc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    from paper_2201_04265_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared_functions()
    assert "ldpc_decode" in names and "ldpc_encode" in names and "ldpc_code_create" in names
    for name in names:
        assert hasattr(lib, name), name
    # and the binding knows every one of them
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def _a_from_oracle(sysm):
    kw = (sysm.k + 31) // 32
    return S.pack_bits(sysm.A) if sysm.rank else np.zeros((0, kw), np.uint32)


@pytest.mark.parametrize("maker", [
    lambda: S.fig1_code(),
    lambda: S.fig2_code(),
    lambda: S.gallager_regular(504, 3, 6, seed=1),
    lambda: S.random_regular(1008, 3, 9, seed=41),
    lambda: S.table1_code(0.25, seed=6),
    lambda: S.dense_to_code(np.random.default_rng(5).integers(0, 2, (37, 70), dtype=np.uint8)),
])
def test_host_code_matches_oracle(L, maker):
    code = maker()
    c = L.Code.from_csr_code(code, host_only=True)
    sysm = oracle.systematic(code)
    assert (c.n, c.m, c.k, c.rank, c.nnz) == (code.n, code.m, sysm.k, sysm.rank, code.nnz)
    info, par = c.positions()
    np.testing.assert_array_equal(info, sysm.info_pos)
    np.testing.assert_array_equal(par, sysm.parity_pos)
    np.testing.assert_array_equal(c.parity_map(), _a_from_oracle(sysm))
    c.close()


def test_qc_description_equals_expanded_csr(L):
    base = S.qc_base_matrix(6, 10, 30, 3, 8, 16, seed=3)
    code = S.qc_expand(base, 16)
    a = L.Code.from_qc(base, 16, host_only=True)
    b = L.Code.from_csr_code(code, host_only=True)
    assert (a.n, a.m, a.k, a.rank, a.nnz) == (b.n, b.m, b.k, b.rank, b.nnz)
    np.testing.assert_array_equal(a.parity_map(), b.parity_map())
    np.testing.assert_array_equal(a.positions()[0], b.positions()[0])


@pytest.mark.parametrize("bad", [
    dict(n=4, m=1, rp=[0, 2], ci=[1, 1]),          # repeated column
    dict(n=4, m=1, rp=[0, 2], ci=[2, 1]),          # unsorted row
    dict(n=4, m=1, rp=[0, 2], ci=[1, 4]),          # column out of range
    dict(n=4, m=2, rp=[0, 2, 1], ci=[0, 1]),       # row_ptr not monotone
    dict(n=0, m=1, rp=[0, 0], ci=[]),              # no bits
    dict(n=2, m=2, rp=[0, 1, 2], ci=[0, 1]),       # rank(H) = n, no information bits
])
def test_malformed_h_is_rejected(L, bad):
    with pytest.raises(L.LdpcError) as ei:
        L.Code(bad["n"], bad["m"], np.array(bad["rp"]), np.array(bad["ci"] or [0]), host_only=True)
    assert ei.value.status == -1


def test_bad_qc_shift_rejected(L):
    with pytest.raises(L.LdpcError):
        L.Code.from_qc(np.array([[0, 5]]), 4, host_only=True)


def test_host_only_code_cannot_decode(L):
    import torch
    code = S.fig1_code()
    c = L.Code.from_csr_code(code, host_only=True)
    # the check happens before any device access
    st = c._lib.ldpc_encode(c.handle, None, None, 1, None)
    assert st == -1
    assert b"host-only" in c._lib.ldpc_last_error()
    # so do the encoder-table calls (no device memory is touched)
    with pytest.raises(L.LdpcError, match="host-only"):
        c.build_encode_tables()
    with pytest.raises(L.LdpcError, match="host-only"):
        c.free_encode_tables()
    del torch


@pytest.mark.parametrize("maker,conflict_free", [  # regular codes: nearly conflict-free
    (lambda: S.random_regular(8064, 3, 6, seed=2), True),
    (lambda: S.gallager_regular(504, 3, 6, seed=1), True),
    (lambda: S.random_regular(2016, 3, 12, seed=47), True),
    (lambda: S.dense_to_code(np.random.default_rng(5).integers(0, 2, (37, 70), dtype=np.uint8)), False),
])
def test_check_schedule_is_a_row_permutation(L, maker, conflict_free):
    code = maker()
    c = L.Code.from_csr_code(code, host_only=True)
    order, unplaced = c.schedule()
    for r in range(code.m):
        lo, hi = code.row_ptr[r], code.row_ptr[r + 1]
        assert sorted(order[lo:hi].tolist()) == list(range(lo, hi))
    if conflict_free:   # at most 1 % of edges outside a conflict-free step
        assert unplaced <= 0.01 * code.nnz, unplaced
