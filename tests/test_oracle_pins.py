"""Pins the FP64 oracle to what the paper and the mathematics fix (no GPU).

Every expected value here comes from the paper's printed examples (golden
files), closed forms derived from parity probabilities, brute-force
enumeration, or invariants -- never from the oracle itself.
"""

from fractions import Fraction
import math

import numpy as np
import pytest

import ldpc_synth as S
import oracle
from oracle import brute
from conftest import read_golden


def _fig1():
    g = read_golden("fig1_tanner.txt")
    h = np.array([[int(x) for x in row] for row in g["H"]], dtype=np.uint8)
    return h, g["edge"]


# ----------------------------------------------------------- paper examples


def test_fig1_matrix_and_graph_agree():
    h, edges = _fig1()
    from_edges = np.zeros_like(h)
    for v, c in edges:
        from_edges[int(c[1:]) - 1, int(v[1:]) - 1] = 1
    np.testing.assert_array_equal(h, from_edges)
    assert np.all(h.sum(0) == 2) and np.all(h.sum(1) == 4)  # (2,4)-regular


def test_fig1_rank_and_codewords():
    h, _ = _fig1()
    code = S.dense_to_code(h)
    sysm = oracle.systematic(code)
    # rows 1+3 and 2+4 both equal e7+e8, so one row is dependent
    assert brute.rank_gf2(h) == 3
    assert sysm.rank == 3 and sysm.k == 5
    cws = brute.codewords(h)
    assert len(cws) == 32
    # the oracle's encoder spans exactly the code
    msgs = brute.all_words(5)
    enc = oracle.encode(sysm, msgs)
    assert len({tuple(r) for r in enc}) == 32
    assert {tuple(r) for r in enc} == {tuple(r) for r in cws}


def test_fig2_worked_encoding():
    g = read_golden("fig2_encoding.txt")
    p_cols = [[int(x) for x in c] for c in g["P_col"]]
    m = np.array([[int(x) for x in g["m"][0]]], dtype=np.uint8)
    p = np.array([int(x) for x in g["p"][0]], dtype=np.uint8)
    # H = [P^T | I_4] is the parity-check matrix of G = [I_4 | P]
    h = np.zeros((4, 8), dtype=np.uint8)
    for j, col in enumerate(p_cols):
        h[j, :4] = col
        h[j, 4 + j] = 1
    code = S.dense_to_code(h)
    sysm = oracle.systematic(code)
    np.testing.assert_array_equal(sysm.info_pos, [0, 1, 2, 3])
    np.testing.assert_array_equal(sysm.parity_pos, [4, 5, 6, 7])
    np.testing.assert_array_equal(oracle.encode(sysm, m)[0], p)
    # the figure's G is not Fig. 1's code: its row-1 check fails on p
    h1, _ = _fig1()
    assert (h1[0].astype(int) @ p.astype(int)) % 2 == 1


# ------------------------------------------------------------- GF(2) / Eq. 1


@pytest.mark.parametrize("maker", [
    lambda: S.gallager_regular(504, 3, 6, seed=1),
    lambda: S.random_regular(240, 3, 9, seed=7),
    lambda: S.qc_expand(S.qc_base_matrix(6, 10, 30, 3, 8, 8, seed=3), 8),
    lambda: S.dense_to_code(np.random.default_rng(5).integers(0, 2, (13, 29), dtype=np.uint8)),
])
def test_encoded_codewords_satisfy_parity(maker):
    code = maker()
    sysm = oracle.systematic(code)
    h = code.dense()
    assert sysm.rank == brute.rank_gf2(h)
    msgs = S.info_bits(64, sysm.k, seed=3)
    cw = oracle.encode(sysm, msgs)
    assert not ((cw.astype(np.int64) @ h.T.astype(np.int64)) % 2).any()      # H c^T = 0
    np.testing.assert_array_equal(cw[:, sysm.info_pos], msgs)               # systematic
    # G H^T = 0: every row of G (encoding of a unit vector) is a codeword
    eye = np.eye(sysm.k, dtype=np.uint8)
    g_rows = oracle.encode(sysm, eye)
    assert not ((g_rows.astype(np.int64) @ h.T.astype(np.int64)) % 2).any()
    # rank(G) = k: the info columns of G are the identity
    np.testing.assert_array_equal(g_rows[:, sysm.info_pos], eye)


def test_gallager_rank_deficiency():
    code = S.gallager_regular(504, 3, 6, seed=1)
    sysm = oracle.systematic(code)
    assert code.m == 252 and sysm.rank <= 252 - 2 and sysm.k >= 254


def test_syndrome_matches_dense_product():
    code = S.random_regular(96, 3, 6, seed=2)
    bits = np.random.default_rng(0).integers(0, 2, (20, code.n), dtype=np.uint8)
    want = (bits.astype(np.int64) @ code.dense().T.astype(np.int64)) % 2
    np.testing.assert_array_equal(oracle.syndrome(code, bits), want)


# --------------------------------------------------- check/variable updates


def _p_odd(ps):
    """P(an odd number of independent bits are 1), by direct recursion."""
    odd = Fraction(0)
    for p in ps:
        odd = odd * (1 - p) + (1 - odd) * p
    return odd


def _extrinsic_llr(ratios):
    """Exact check message for a parity check whose other inputs have
    likelihood ratios p1/p0 = ratios: our bit equals the XOR of the others."""
    ps = [Fraction(a) / (1 + Fraction(a)) for a in ratios]
    po = _p_odd(ps)
    return math.log(po / (1 - po))


def test_fig1_single_iteration_closed_form():
    h, _ = _fig1()
    code = S.dense_to_code(h)
    R = np.full((1, 8), math.log(3.0))
    res = oracle.decode(code, R, iters=1)
    e = _extrinsic_llr([3, 3, 3])            # = ln(9/7)
    assert abs(e - math.log(9 / 7)) < 1e-15
    np.testing.assert_allclose(res.post[0], math.log(3) + 2 * e, rtol=0, atol=1e-13)


def test_odd_degree_sign():
    # a degree-3 check with inputs ln 3: the message is ln(3/5) < 0, which
    # fixes the (-1)^{d_c} factor of the sign-corrected Eq. 5
    code = S.dense_to_code([[1, 1, 1]])
    res = oracle.decode(code, np.full((1, 3), math.log(3.0)), iters=1)
    assert abs(_extrinsic_llr([3, 3]) - math.log(3 / 5)) < 1e-15
    np.testing.assert_allclose(res.post[0], math.log(3) + math.log(3 / 5), atol=1e-13)


def test_mixed_rational_inputs():
    code = S.dense_to_code([[1, 1, 1, 1]])
    ratios = [3, 9, 2, 5]
    R = np.log(np.array([ratios], dtype=np.float64))
    res = oracle.decode(code, R, iters=1)
    for v in range(4):
        others = ratios[:v] + ratios[v + 1:]
        np.testing.assert_allclose(res.post[0, v], math.log(ratios[v]) + _extrinsic_llr(others),
                                   atol=1e-13)


def test_degree_two_check_is_repetition():
    code = S.dense_to_code([[1, 1]])
    R = np.array([[0.7, -2.5]])
    res = oracle.decode(code, R, iters=1)
    np.testing.assert_allclose(res.post[0], [0.7 - 2.5, -2.5 + 0.7], atol=1e-15)


def test_single_parity_check_is_map():
    code = S.dense_to_code([[1, 1, 1, 1, 1]])
    R = np.random.default_rng(1).normal(0, 2, (8, 5))
    res = oracle.decode(code, R, iters=1)
    np.testing.assert_allclose(res.post, brute.bitwise_map_llr(code.dense(), R), atol=1e-12)


def _random_tree_code(nv_target, seed):
    """A cycle-free Tanner graph: checks attach to one existing bit plus new bits."""
    rng = np.random.default_rng(seed)
    rows = []
    nv = 1
    while nv < nv_target:
        d = int(rng.integers(2, 5))
        old = int(rng.integers(nv))
        new = list(range(nv, nv + d - 1))
        rows.append([old] + new)
        nv += d - 1
    h = np.zeros((len(rows), nv), dtype=np.uint8)
    for c, r in enumerate(rows):
        h[c, r] = 1
    return S.dense_to_code(h)


@pytest.mark.parametrize("which", ["two_checks", "random_tree"])
def test_tree_code_bp_equals_map(which):
    if which == "two_checks":
        code = S.dense_to_code([[1, 1, 1, 0, 0], [0, 0, 1, 1, 1]])
        T = 3
    else:
        code = _random_tree_code(15, seed=4)
        T = 2 * code.m + 2
    R = np.random.default_rng(2).normal(0.5, 2.0, (16, code.n))
    res = oracle.decode(code, R, iters=T)
    np.testing.assert_allclose(res.post, brute.bitwise_map_llr(code.dense(), R), atol=1e-12)


# ------------------------------------------------------------- invariants


def _c1_frames(F=8, seed=11, ebn0=2.0):
    code = S.gallager_regular(504, 3, 6, seed=1)
    sysm = oracle.systematic(code)
    msgs = S.info_bits(F, sysm.k, seed)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, ebn0, sysm.k / code.n, S.frame_noise(F, code.n, seed + 1))
    return code, sysm, cw, llr


def test_sign_flip_symmetry():
    code, sysm, cw, llr = _c1_frames(F=4)
    R = llr.astype(np.float64)
    base = oracle.decode(code, R, iters=7)
    c = cw[1].astype(bool)                      # support of a codeword
    flipped = R.copy()
    flipped[:, c] = -flipped[:, c]
    res = oracle.decode(code, flipped, iters=7)
    want = base.post.copy()
    want[:, c] = -want[:, c]
    np.testing.assert_allclose(res.post, want, rtol=1e-14, atol=0)


def test_noiseless_input_decodes_in_one_iteration():
    code, sysm, cw, _ = _c1_frames(F=3)
    R = 20.0 * (2.0 * cw - 1.0)
    res = oracle.decode(code, R, iters=50, early_stop=True)
    assert np.all(res.iters == 1) and np.all(res.ok == 1)
    np.testing.assert_array_equal(res.hard, cw)


def test_unit_weights_equal_plain_bp():
    code, _, _, llr = _c1_frames(F=3)
    plain = oracle.decode(code, llr, iters=5)
    wbp = oracle.decode(code, llr, iters=5, weights=np.ones((5, code.nnz)))
    np.testing.assert_array_equal(plain.post, wbp.post)


def test_zero_iterations_return_channel_llrs():
    code, _, _, llr = _c1_frames(F=2)
    res = oracle.decode(code, llr, iters=0, early_stop=True)
    np.testing.assert_array_equal(res.post, llr.astype(np.float64))
    assert np.all(res.iters == 0)
    np.testing.assert_array_equal(res.hard, (llr >= 0).astype(np.uint8))


def test_early_stop_matches_fixed_iterations_prefix():
    code, _, cw, llr = _c1_frames(F=16, ebn0=2.5)
    es = oracle.decode(code, llr, iters=30, early_stop=True)
    for f in range(16):
        fixed = oracle.decode(code, llr[f:f + 1], iters=int(es.iters[f]))
        np.testing.assert_array_equal(fixed.post[0], es.post[f])
        if es.ok[f]:
            # the stopped word satisfies every check (Eq. 1)
            assert not oracle.syndrome(code, es.hard[f:f + 1]).any()


def test_clipping_bounds_messages():
    # with a single degree-2 check the message is the other input, clipped
    code = S.dense_to_code([[1, 1]])
    res = oracle.decode(code, np.array([[50.0, 1.0]]), iters=1, clip=20.0)
    np.testing.assert_allclose(res.post[0], [50.0 + 1.0, 1.0 + 20.0])


def test_bp_agrees_with_ml_at_high_snr():
    h, _ = _fig1()
    code = S.dense_to_code(h)
    sysm = oracle.systematic(code)
    msgs = S.info_bits(400, sysm.k, seed=8)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, 6.0, sysm.k / code.n, S.frame_noise(400, code.n, 9))
    res = oracle.decode(code, llr, iters=10)
    ml = brute.block_ml(h, llr)
    agree = np.mean(np.all(res.hard == ml, axis=1))
    assert agree > 0.95, agree


# ------------------------------------------------------------ gradient


def _bce_loss_np(L, bits):
    # mean of softplus(L) - c L, the BCE of sigmoid(L) against c
    return float(np.mean(np.logaddexp(0.0, L) - bits * L))


def test_wbp_reference_gradient_against_finite_differences():
    from oracle import wbp_ref
    code = S.random_regular(96, 3, 6, seed=5)
    sysm = oracle.systematic(code)
    F, T = 4, 4
    msgs = S.info_bits(F, sysm.k, seed=51)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, 1.0, sysm.k / code.n, S.frame_noise(F, code.n, 52)).astype(np.float64)
    w = 1.0 + 0.2 * np.random.default_rng(53).standard_normal((T, code.nnz))
    loss, gw, gR, Lv = wbp_ref.loss_and_grads(code, llr, w, cw)
    # two independent forward implementations agree (C oracle vs torch restatement)
    fwd = oracle.decode(code, llr, iters=T, weights=w)
    np.testing.assert_allclose(Lv, fwd.post, rtol=1e-11, atol=1e-11)
    assert abs(loss - _bce_loss_np(fwd.post, cw)) < 1e-12
    # central differences of the C oracle's loss, h = 1e-3
    h = 1e-3
    rng = np.random.default_rng(54)
    coords = [(int(rng.integers(T)), int(rng.integers(code.nnz))) for _ in range(64)]
    fd = []
    for (t, e) in coords:
        wp = w.copy(); wp[t, e] += h
        wm = w.copy(); wm[t, e] -= h
        lp = _bce_loss_np(oracle.decode(code, llr, iters=T, weights=wp).post, cw)
        lm = _bce_loss_np(oracle.decode(code, llr, iters=T, weights=wm).post, cw)
        fd.append((lp - lm) / (2 * h))
    ref = np.array([gw[t, e] for (t, e) in coords])
    scale = np.max(np.abs(gw))
    np.testing.assert_allclose(ref, fd, rtol=1e-4, atol=1e-6 * scale)
    # and along R
    rcoords = [(int(rng.integers(F)), int(rng.integers(code.n))) for _ in range(16)]
    for (f, v) in rcoords:
        Rp = llr.copy(); Rp[f, v] += h
        Rm = llr.copy(); Rm[f, v] -= h
        d = (_bce_loss_np(oracle.decode(code, Rp, iters=T, weights=w).post, cw)
             - _bce_loss_np(oracle.decode(code, Rm, iters=T, weights=w).post, cw)) / (2 * h)
        assert abs(d - gR[f, v]) <= 1e-4 * abs(d) + 1e-6 * np.max(np.abs(gR))
