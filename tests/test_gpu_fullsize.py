"""Parity at the benchmark sizes, on sampled frames the oracle recomputes one by one.

n = 8064 random (3,6) code, 65536 frames, 50 fixed iterations (the benchmark
batch): the GPU encodes every frame and decodes the whole batch in the
benchmark's configuration (resident decoder, binary16 and FP32 messages).
For a sample of frames the oracle regenerates the information bits and the
noise from their per-frame seeds, encodes them itself (the GPU codeword must
match bit for bit) and decodes them.  Quasi-cyclic n = 26112 code, 4096 frames,
25 iterations: encoding is checked by properties that hold at any size, and
decoding on the all-zero codeword (valid for every linear code), so no oracle
input depends on the CUDA path.
"""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle
from parity_util import CLIP, assert_fp32_parity

pytestmark = pytest.mark.gpu

F2, T2, EBN0_2, SEED2 = 65536, 50, 2.0, 7100
CH = 4096   # frames per host-side chunk, to bound host memory


def _pack(bits):
    return np.concatenate([S.pack_bits(bits[i:i + CH]) for i in range(0, bits.shape[0], CH)])


def _unpack(words, n):
    return np.concatenate([S.unpack_bits(words[i:i + CH], n) for i in range(0, words.shape[0], CH)])


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.fixture(scope="module")
def c2(L):
    h = S.random_regular(8064, 3, 6, seed=2)
    sysm = oracle.systematic(h)
    code = L.Code.from_csr_code(h)
    rate = sysm.k / h.n
    # all frames: info bits and noise from per-frame seeds, GPU encoding
    info = S.info_bits(F2, sysm.k, SEED2)
    cw_words = L.encode(code, torch.from_numpy(_pack(info).view(np.int32)).cuda())
    cw = _unpack(cw_words.cpu().numpy().view(np.uint32), h.n)
    llr = np.empty((F2, h.n), dtype=np.float32)
    for f0 in range(0, F2, 8192):
        fr = np.arange(f0, f0 + 8192)
        llr[f0:f0 + 8192] = S.bpsk_awgn_llr(cw[fr], EBN0_2, rate, S.frame_noise(F2, h.n, SEED2 + 1, frames=fr))
    sample = np.random.default_rng(5).choice(F2, 40, replace=False)
    return h, sysm, code, cw, torch.from_numpy(llr).cuda(), sample, rate


def _oracle_frames(h, sysm, rate, frames):
    msgs = S.info_bits(F2, sysm.k, SEED2, frames=frames)
    cw = oracle.encode(sysm, msgs)
    llr = S.bpsk_awgn_llr(cw, EBN0_2, rate, S.frame_noise(F2, h.n, SEED2 + 1, frames=frames))
    return cw, llr


def test_c2_encode_full_batch(L, c2):
    h, sysm, code, cw, _, sample, rate = c2
    want, _ = _oracle_frames(h, sysm, rate, sample)
    np.testing.assert_array_equal(cw[sample], want)
    # every codeword of the batch satisfies H c^T = 0 (Eq. 1)
    _, ok = L.syndrome(code, torch.from_numpy(_pack(cw).view(np.int32)).cuda(), want_syn=False)
    assert bool(ok.all())


def test_c2_encode_full_batch_tables(L, c2):
    """The whole 65536-frame batch through the Four-Russians tables: the same
    codewords as the AND/XOR form, and the oracle's on the sampled frames."""
    h, sysm, code, cw, _, sample, rate = c2
    info = torch.from_numpy(_pack(S.info_bits(F2, sysm.k, SEED2)).view(np.int32)).cuda()
    code.build_encode_tables()
    try:
        words = L.encode(code, info)
    finally:
        code.free_encode_tables()
    got = _unpack(words.cpu().numpy().view(np.uint32), h.n)
    np.testing.assert_array_equal(got, cw)
    want, _ = _oracle_frames(h, sysm, rate, sample)
    np.testing.assert_array_equal(got[sample], want)


@pytest.mark.parametrize("fp16", [False, True])
def test_c2_decode_full_batch_sampled_frames(L, c2, fp16):
    """The whole 65536-frame batch on the resident decoder in the benchmark's
    configuration; 40 sampled frames against the FP64 oracle.  FP32 messages:
    the FP32 parity gate.  Binary16 messages (parity unpinned at 1e-3 by
    design): hard decisions of every frame the oracle decodes agree, and the
    clipped LLR error against FP64 is bounded by what binary16 rounding of
    messages of up to 20 can add over 50 iterations."""
    h, sysm, code, cw, llr, sample, rate = c2
    res = L.decode(code, llr, max_iters=T2, schedule="resident", msg_fp16=fp16)
    torch.cuda.synchronize()
    post = res.post.cpu().numpy()[sample]
    hard = S.unpack_bits(res.hard.cpu().numpy()[sample].view(np.uint32), h.n)
    ok = res.ok.cpu().numpy()[sample]
    iters = res.iters.cpu().numpy()[sample]
    _, ollr = _oracle_frames(h, sysm, rate, sample)
    np.testing.assert_array_equal(ollr, llr.cpu().numpy()[sample])   # identical inputs
    if not fp16:
        assert_fp32_parity(h, ollr, T2, post, hard, iters, ok, max_excluded=0.05)
    else:
        ref = oracle.decode(h, ollr, iters=T2, nthreads=16)
        good = ref.ok.astype(bool)
        np.testing.assert_array_equal(hard[good], ref.hard[good])
        err = np.abs(np.clip(post, -CLIP, CLIP) - np.clip(ref.post, -CLIP, CLIP))
        print(f"binary16 messages, C2 at {EBN0_2} dB: max |dL| {err.max():.4g}, mean {err.mean():.4g}")
        assert err.mean() < 0.05 and err.max() <= 2 * CLIP
    assert (res.iters.cpu().numpy() == T2).all()


def test_c2_fp16_resident_and_fp32_plain_equal_frame_errors(L, c2):
    """The headline comparison's gate on the full batch: the binary16 resident
    decoder and the plain FP32 decoder fail on the same number of frames to
    within 0.1 % of the batch, and disagree in their hard decisions on at most
    0.1 % of the frames."""
    h, sysm, code, cw, llr, sample, rate = c2
    a = L.decode(code, llr, max_iters=T2, schedule="resident", msg_fp16=True, want_post=False)
    b = L.decode(code, llr, max_iters=T2, schedule="plain", msg_fp16=False, want_post=False)
    torch.cuda.synchronize()
    fail16 = int((a.ok == 0).sum())
    fail32 = int((b.ok == 0).sum())
    differ = int((a.hard != b.hard).any(dim=1).sum())
    assert abs(fail16 - fail32) <= 0.001 * F2, (fail16, fail32)
    assert differ <= 0.001 * F2, differ


@pytest.fixture(scope="module")
def qc(L):
    base = S.qc_base_matrix(46, 68, 316, 3, 19, 384, seed=3)
    return S.qc_expand(base, 384), L.Code.from_qc(base, 384)


def test_qc_encode_full_batch_properties(L, qc):
    h, code = qc
    F = 4096
    info = S.info_bits(F, code.k, 7300)
    words = L.encode(code, torch.from_numpy(S.pack_bits(info).view(np.int32)).cuda())
    _, ok = L.syndrome(code, words, want_syn=False)
    assert bool(ok.all())                                   # H c^T = 0 for all 4096
    bits = S.unpack_bits(words.cpu().numpy()[:64].view(np.uint32), code.n)
    info_pos, _ = code.positions()
    np.testing.assert_array_equal(bits[:, info_pos], info[:64])   # systematic
    assert not oracle.syndrome(h, bits).any()               # checked by the oracle too


def test_qc_encode_full_batch_tables(L, qc):
    """4096 frames of the n = 26112 code through the Four-Russians tables
    (about 600 MB): same codewords as the AND/XOR form, all satisfy H c^T = 0,
    and the oracle's syndrome agrees on a sample."""
    h, code = qc
    F = 4096
    info_bits = S.info_bits(F, code.k, 7301)
    info = torch.from_numpy(S.pack_bits(info_bits).view(np.int32)).cuda()
    ref = L.encode(code, info)
    code.build_encode_tables()
    try:
        words = L.encode(code, info)
    finally:
        code.free_encode_tables()
    assert torch.equal(words, ref)
    _, ok = L.syndrome(code, words, want_syn=False)
    assert bool(ok.all())
    bits = S.unpack_bits(words.cpu().numpy()[:32].view(np.uint32), code.n)
    info_pos, _ = code.positions()
    np.testing.assert_array_equal(bits[:, info_pos], info_bits[:32])
    assert not oracle.syndrome(h, bits).any()


@pytest.fixture(scope="module")
def qc_sys(qc):
    h, _ = qc
    return oracle.systematic(h)   # about a minute: GF(2) elimination of the 17664 x 26112 H


@pytest.mark.parametrize("ebn0", [1.0, 2.0])
def test_qc_decode_random_codewords_against_oracle(L, qc, qc_sys, ebn0):
    """32 random codewords of the n = 26112 quasi-cyclic code, encoded by the
    oracle, 25 iterations with FP32 messages through the schedule this code
    takes by default, against the FP64 oracle (FP32 parity gate).  At 1.0 dB
    no frame decodes; at 2.0 dB all do."""
    h, code = qc
    F, T = 32, 25
    msgs = S.info_bits(F, qc_sys.k, 9000)
    cw = oracle.encode(qc_sys, msgs)
    llr = S.bpsk_awgn_llr(cw, ebn0, qc_sys.k / h.n, S.frame_noise(F, h.n, 9001))
    res = L.decode(code, torch.from_numpy(llr).cuda(), max_iters=T, msg_fp16=False)
    torch.cuda.synchronize()
    hard = S.unpack_bits(res.hard.cpu().numpy().view(np.uint32), h.n)
    assert_fp32_parity(h, llr, T, res.post.cpu().numpy(), hard, res.iters.cpu().numpy(),
                       res.ok.cpu().numpy(), max_excluded=0.05)


@pytest.mark.parametrize("ebn0", [1.85, 2.0])
def test_qc_decode_full_batch_fp16_frame_errors(L, qc, ebn0):
    """The full 4096-frame, 25-iteration batch on the all-zero codeword (valid
    for every linear code, so no input depends on the CUDA path): binary16
    message storage fails on the same number of frames as FP32 messages, to
    within 0.1 % of the batch."""
    h, code = qc
    F, T = 4096, 25
    rate = code.k / code.n
    zero = np.zeros((1, code.n), dtype=np.uint8)
    llr = np.empty((F, code.n), dtype=np.float32)
    for f0 in range(0, F, 1024):
        fr = np.arange(f0, f0 + 1024)
        llr[f0:f0 + 1024] = S.bpsk_awgn_llr(np.broadcast_to(zero, (1024, code.n)), ebn0, rate,
                                            S.frame_noise(F, code.n, 7400, frames=fr))
    d_llr = torch.from_numpy(llr).cuda()
    r32 = L.decode(code, d_llr, max_iters=T, msg_fp16=False, want_post=False)
    r16 = L.decode(code, d_llr, max_iters=T, msg_fp16=True, want_post=False)
    torch.cuda.synchronize()
    fe32 = int((r32.hard != 0).any(dim=1).sum())
    fe16 = int((r16.hard != 0).any(dim=1).sum())
    assert 0 < fe32 < F or ebn0 == 2.0
    assert abs(fe32 - fe16) <= 0.001 * F, (fe32, fe16)
