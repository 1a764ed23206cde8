"""Cluster-resident decoder (quasi-cyclic codes created from their base matrix).

It shares the check arithmetic and the evaluation and summation orders with
the plain decoder, so the two must agree bit for bit: posteriors, hard
decisions, iteration counts and flags, with and without early stop, in FP32
and binary16 message storage, on clusters of 2, 4 and 8 CTAs and on ragged
batches.  Against the FP64 oracle it meets the FP32 parity gate.
"""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle
from parity_util import assert_fp32_parity

pytestmark = pytest.mark.gpu

# (mb, nb, nonzeros, row weight min, max, z, seed): clusters of 2 CTAs
# (z = 64), 4 (the 46 x 68, z = 384 workload code) and, with binary16
# messages, 8 (a 24 x 48 base lifted by 768)
QC = {
    "z64": (8, 16, 40, 3, 8, 64, 2),
    "c3_z384": (46, 68, 316, 3, 19, 384, 3),
    "z768": (24, 48, 200, 3, 14, 768, 4),
}
CTAS = {("z64", True): 2, ("z64", False): 2, ("c3_z384", True): 4, ("c3_z384", False): 4,
        ("z768", True): 8, ("z768", False): 4}


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


_made = {}


def qc_code(L, name):
    if name not in _made:
        mb, nb, nnz, lo, hi, z, seed = QC[name]
        base = S.qc_base_matrix(mb, nb, nnz, lo, hi, z, seed=seed)
        _made[name] = (S.qc_expand(base, z), L.Code.from_qc(base, z))
    return _made[name]


def zero_word_llr(n, rate, F, ebn0, seed):
    """The all-zero codeword (valid for every linear code) through BPSK/AWGN."""
    return S.bpsk_awgn_llr(np.zeros((F, n), dtype=np.uint8), ebn0, rate, S.frame_noise(F, n, seed))


def _run(L, code, llr, **kw):
    r = L.decode(code, llr, **kw)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in (r.post, r.hard, r.iters, r.ok)]


@pytest.mark.parametrize("name", list(QC))
@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("early_stop", [False, True])
def test_cluster_matches_plain_bit_for_bit(L, name, fp16, early_stop):
    h, code = qc_code(L, name)
    ctas, group, local = code.cluster_layout(fp16)
    assert (ctas, group) == (CTAS[name, fp16], 2 if fp16 else 1)
    assert 0.4 < local <= 1.0   # share of base entries whose row and column share a CTA
    F = 9 if name == "z768" else 37   # odd: the last binary16 group holds one frame
    llr = torch.from_numpy(zero_word_llr(code.n, code.k / code.n, F, 2.0, seed=810)).cuda()
    kw = dict(max_iters=25, early_stop=early_stop, msg_fp16=fp16)
    a = _run(L, code, llr, schedule="plain", **kw)
    b = _run(L, code, llr, schedule="cluster", **kw)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    if early_stop:
        assert len(np.unique(a[2])) > 1   # frames stopped at different iterations


@pytest.mark.parametrize("early_stop", [False, True])
def test_cluster_against_oracle(L, early_stop):
    """Random codewords of the z = 64 code encoded by the oracle, FP32
    messages, 20 iterations: the FP32 parity gate."""
    h, code = qc_code(L, "z64")
    sysm = oracle.systematic(h)
    F = 64
    msgs = S.info_bits(F, sysm.k, 820)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, 2.5, sysm.k / h.n, S.frame_noise(F, h.n, 821))
    post, hard, iters, ok = _run(L, code, torch.from_numpy(llr).cuda(), max_iters=20,
                                 early_stop=early_stop, schedule="cluster")
    assert_fp32_parity(h, llr, 20, post, S.unpack_bits(hard.view(np.uint32), h.n), iters, ok,
                       early_stop=early_stop, max_excluded=0.05)


def test_cluster_is_the_default_for_the_large_qc_code(L):
    """The n = 26112 code does not fit one SM, so the default schedule takes
    the cluster decoder (its workspace is the 256-byte work counter)."""
    _, code = qc_code(L, "c3_z384")
    for fp16 in (False, True):
        assert L.decode_workspace_size(code, 4096, msg_fp16=fp16) == 256
        assert L.decode_workspace_size(code, 4096, msg_fp16=fp16, schedule="plain") > 256


@pytest.mark.parametrize("fp16", [False, True])
def test_cluster_zero_iterations_single_frame_and_empty(L, fp16):
    h, code = qc_code(L, "c3_z384")
    llr = torch.from_numpy(zero_word_llr(code.n, code.k / code.n, 3, 1.5, seed=830)).cuda()
    post, hard, iters, ok = _run(L, code, llr, max_iters=0, schedule="cluster", msg_fp16=fp16)
    np.testing.assert_array_equal(post, llr.cpu().numpy())
    np.testing.assert_array_equal(S.unpack_bits(hard.view(np.uint32), code.n),
                                  (llr.cpu().numpy() >= 0).astype(np.uint8))
    assert (iters == 0).all()
    np.testing.assert_array_equal(
        ok, (~oracle.syndrome(h, S.unpack_bits(hard.view(np.uint32), code.n)).any(axis=1)).astype(np.uint8))
    one = _run(L, code, llr[1:2].contiguous(), max_iters=12, schedule="cluster", msg_fp16=fp16)
    ref = _run(L, code, llr[1:2].contiguous(), max_iters=12, schedule="plain", msg_fp16=fp16)
    for x, y in zip(one, ref):
        np.testing.assert_array_equal(x, y)
    empty = L.decode(code, llr[:0], max_iters=5, schedule="cluster", msg_fp16=fp16)
    assert empty.hard.shape == (0, code.NW)


def test_cluster_rejects_codes_without_a_cluster_layout(L):
    h = S.random_regular(1008, 3, 6, seed=5)          # not created from a base matrix
    code = L.Code.from_csr_code(h)
    assert code.cluster_shape(True) == (0, 0)
    with pytest.raises(L.LdpcError) as ei:
        L.decode(code, torch.zeros((2, code.n), device="cuda"), schedule="cluster")
    assert ei.value.status == -5
