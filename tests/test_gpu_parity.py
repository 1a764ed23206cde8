"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Encoding and syndromes must match bit for bit.  FP32 decoding must keep total
LLRs within 1e-4 relative or 1e-3 absolute (both clipped to |L| <= 20) with
identical hard decisions except where the oracle's |L| < 1e-3.
"""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle
from conftest import read_golden
from parity_util import (CODES, assert_fp32_parity, code_and_sys, hard_close, llr_close,
                         workload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


_codes = {}


def dev_code(L, name):
    if name not in _codes:
        code, _ = code_and_sys(name)
        _codes[name] = L.Code.from_csr_code(code)
    return _codes[name]


def to_dev_words(bits):
    return torch.from_numpy(S.pack_bits(bits).view(np.int32)).cuda()


def from_dev_words(t, L_bits):
    return S.unpack_bits(t.cpu().numpy().view(np.uint32), L_bits)


# ------------------------------------------------------------------ encode


@pytest.mark.parametrize("name", [n for n in CODES if n != "c2_random_8064"])
@pytest.mark.parametrize("F", [1, 33, 200])
def test_encode_bit_exact(L, name, F):
    code, sysm = code_and_sys(name)
    c = dev_code(L, name)
    msgs = S.info_bits(F, sysm.k, seed=100 + F)
    want = oracle.encode(sysm, msgs)
    got = from_dev_words(L.encode(c, to_dev_words(msgs)), code.n)
    np.testing.assert_array_equal(got, want)
    # pad bits of the last word stay zero
    raw = L.encode(c, to_dev_words(msgs)).cpu().numpy().view(np.uint32)
    if code.n % 32:
        assert not (raw[:, -1] >> np.uint32(code.n % 32)).any()


@pytest.mark.parametrize("name", ["c1_gallager_504", "qc_small", "qc_irregular_512", "table1_r025",
                                  "table1_r075", "reg312_2016"])
@pytest.mark.parametrize("F", [1, 33, 300])
def test_encode_tables_bit_exact(L, name, F):
    """Four-Russians tables: the oracle's codewords, whatever the bits beyond k
    in the last information word; freeing the tables returns to the AND/XOR
    form with the same result."""
    code, sysm = code_and_sys(name)
    c = L.Code.from_csr_code(code)   # its own object: the tables change its encode path
    msgs = S.info_bits(F, sysm.k, seed=400 + F)
    want = oracle.encode(sysm, msgs)
    info = to_dev_words(msgs)
    if sysm.k % 32:   # garbage in the pad bits of the last word
        junk = np.random.default_rng(F).integers(0, 2 ** 31, F).astype(np.int32) << (sysm.k % 32)
        info[:, -1] |= torch.from_numpy(junk).cuda()
    nbytes = c.build_encode_tables()
    assert nbytes == 4096 * (-(-(-(-c.rank // 32)) // 4)) * (-(-c.k // 8))
    got = from_dev_words(L.encode(c, info), code.n)
    np.testing.assert_array_equal(got, want)
    c.free_encode_tables()
    np.testing.assert_array_equal(from_dev_words(L.encode(c, info), code.n), want)
    c.close()


def test_encode_tables_rejected_when_scratch_does_not_fit(L):
    """A 70-bit code has 3 words per codeword, fewer than the 4 scratch words
    of one parity slice: no tables, and encoding keeps the AND/XOR form."""
    code, sysm = code_and_sys("irregular_37x70")
    c = L.Code.from_csr_code(code)
    with pytest.raises(L.LdpcError):
        c.build_encode_tables()
    msgs = S.info_bits(9, sysm.k, seed=5)
    np.testing.assert_array_equal(from_dev_words(L.encode(c, to_dev_words(msgs)), code.n),
                                  oracle.encode(sysm, msgs))
    c.close()


def test_encode_fig2_worked_example(L):
    g = read_golden("fig2_encoding.txt")
    c = L.Code.from_csr_code(S.fig2_code())
    m = np.array([[int(x) for x in g["m"][0]]], dtype=np.uint8)
    p = np.array([int(x) for x in g["p"][0]], dtype=np.uint8)
    np.testing.assert_array_equal(from_dev_words(L.encode(c, to_dev_words(m)), 8)[0], p)


def test_encode_empty_batch(L):
    c = dev_code(L, "c1_gallager_504")
    out = L.encode(c, torch.zeros((0, c.KW), dtype=torch.int32, device="cuda"))
    assert out.shape == (0, c.NW)


# ---------------------------------------------------------------- syndrome


@pytest.mark.parametrize("name", ["c1_gallager_504", "irregular_37x70", "qc_small", "reg39_1008"])
def test_syndrome_bit_exact(L, name):
    code, sysm = code_and_sys(name)
    c = dev_code(L, name)
    rng = np.random.default_rng(7)
    words = rng.integers(0, 2, (77, code.n), dtype=np.uint8)
    words[:10] = oracle.encode(sysm, S.info_bits(10, sysm.k, seed=8))  # some codewords
    syn, ok = L.syndrome(c, to_dev_words(words))
    want = oracle.syndrome(code, words)
    np.testing.assert_array_equal(from_dev_words(syn, code.m), want)
    np.testing.assert_array_equal(ok.cpu().numpy(), (~want.any(axis=1)).astype(np.uint8))
    assert ok.cpu().numpy()[:10].all()


# ------------------------------------------------------------------ decode


def _gpu_decode(L, c, llr, **kw):
    res = L.decode(c, torch.from_numpy(np.ascontiguousarray(llr)).cuda(), **kw)
    torch.cuda.synchronize()
    return (res.post.cpu().numpy(), from_dev_words(res.hard, c.n), res.iters.cpu().numpy(),
            res.ok.cpu().numpy())


@pytest.mark.parametrize("T", [0, 1, 2, 5])
@pytest.mark.parametrize("name", ["c1_gallager_504", "reg39_1008", "irregular_37x70", "qc_small"])
def test_decode_fp32_few_iterations_all_frames(L, name, T):
    """Before rounding has room to grow, every frame meets the tolerance."""
    w = workload(name, 96, 2.0, seed=21)
    c = dev_code(L, name)
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=T, schedule="plain")
    ref = oracle.decode(w.code, w.llr, iters=T)
    assert llr_close(post, ref.post).all(), np.abs(post - ref.post).max()
    assert hard_close(hard, ref.hard, ref.post).all()
    np.testing.assert_array_equal(iters, ref.iters)
    np.testing.assert_array_equal(ok, ref.ok)
    if T == 0:
        np.testing.assert_array_equal(post, w.llr)


@pytest.mark.parametrize("name", ["table1_r025", "table1_r050", "table1_r075"])
def test_decode_table1_paper_setting(L, name):
    """The paper's Table I workload (n = 1032, 12 ones per row, 9/6/3 per
    column, 10 fixed iterations) through the default schedule, which decodes
    all three codes on chip (nine message planes for column weights 9 and 6)."""
    w = workload(name, 200, 3.0, seed=31)
    c = dev_code(L, name)
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=10)
    assert_fp32_parity(w.code, w.llr, 10, post, hard, iters, ok, max_excluded=0.05)
    assert (iters == 10).all()


@pytest.mark.parametrize("name,ebn0", [("c1_gallager_504", 2.0), ("reg312_2016", 3.5),
                                       ("table1_r050", 2.5)])
def test_decode_fp32_fixed_20_iterations(L, name, ebn0):
    """Config-1 style run (20 fixed iterations): every frame whose FP64 decode
    is stable under FP32-sized input rounding must meet the tolerance."""
    w = workload(name, 400, ebn0, seed=11)
    c = dev_code(L, name)
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=20, schedule="plain")
    assert_fp32_parity(w.code, w.llr, 20, post, hard, iters, ok, max_excluded=0.05)
    assert (iters == 20).all()


def test_decode_early_stop(L):
    w = workload("c1_gallager_504", 300, 2.5, seed=31)
    c = dev_code(L, "c1_gallager_504")
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=50, early_stop=True,
                                        schedule="plain")
    assert_fp32_parity(w.code, w.llr, 50, post, hard, iters, ok, early_stop=True, max_excluded=0.05)
    # a stopped frame's hard decisions satisfy every check
    done = ok.astype(bool) & (iters < 50)
    assert not oracle.syndrome(w.code, hard[done]).any()
    assert (iters >= 1).all()


def test_decode_noiseless_one_iteration(L):
    w = workload("reg39_1008", 8, 2.0, seed=3)
    c = dev_code(L, "reg39_1008")
    llr = (20.0 * (2.0 * w.cw - 1.0)).astype(np.float32)
    post, hard, iters, ok = _gpu_decode(L, c, llr, max_iters=50, early_stop=True)
    assert (iters == 1).all() and ok.all()
    np.testing.assert_array_equal(hard, w.cw)


def test_decode_sign_flip_symmetry_bit_exact(L):
    w = workload("c1_gallager_504", 32, 2.0, seed=41)
    c = dev_code(L, "c1_gallager_504")
    base = _gpu_decode(L, c, w.llr, max_iters=12, schedule="plain")[0]
    s = w.cw[3].astype(bool)
    flipped = w.llr.copy()
    flipped[:, s] = -flipped[:, s]
    got = _gpu_decode(L, c, flipped, max_iters=12, schedule="plain")[0]
    want = base.copy()
    want[:, s] = -want[:, s]
    np.testing.assert_array_equal(got, want)


def test_decode_deterministic(L):
    w = workload("reg36_1008", 64, 1.5, seed=5)
    c = dev_code(L, "reg36_1008")
    a = _gpu_decode(L, c, w.llr, max_iters=30, schedule="plain")
    b = _gpu_decode(L, c, w.llr, max_iters=30, schedule="plain")
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_decode_fp16_storage_frame_errors(L):
    """FP16 message storage: LLR parity is not pinned at 1e-3 (binary16's ulp at
    16 is 1/64); the gate is equal frame-error counts within 0.1% of frames."""
    w = workload("reg36_1008", 2000, 2.0, seed=61)
    c = dev_code(L, "reg36_1008")
    p32, h32, _, _ = _gpu_decode(L, c, w.llr, max_iters=30, schedule="plain")
    p16, h16, _, _ = _gpu_decode(L, c, w.llr, max_iters=30, schedule="plain", msg_fp16=True)
    fe32 = np.any(h32 != w.cw, axis=1).sum()
    fe16 = np.any(h16 != w.cw, axis=1).sum()
    assert abs(int(fe32) - int(fe16)) <= max(1, int(0.001 * len(w.cw))), (fe32, fe16)


def test_decode_fp16_storage_llr_error_at_1_5db(L):
    """Binary16 message storage against the FP64 oracle where frames fail
    (1.5 dB on the n = 1008 (3,6) code, 50 iterations): parity at 1e-3 is not
    pinned by design, so this states the error and gates it on what binary16
    rounding allows -- the mean clipped |dL| stays below 1e-2 and the hard
    decisions of every frame the oracle decodes agree.  Measured on GB300 for
    the n = 8064 code at the same point: max 0.13, mean 4e-4; for this code max 9.1
    (a frame that does not converge), mean 7e-3."""
    w = workload("reg36_1008", 400, 1.5, seed=62)
    c = dev_code(L, "reg36_1008")
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=50, schedule="resident", msg_fp16=True)
    ref = oracle.decode(w.code, w.llr, iters=50, nthreads=16)
    err = np.abs(np.clip(post.astype(np.float64), -20, 20) - np.clip(ref.post, -20, 20))
    print(f"binary16 messages, n=1008 at 1.5 dB: max |dL| {err.max():.4g}, mean {err.mean():.4g}, "
          f"oracle FER {(ref.hard != w.cw).any(axis=1).mean():.3f}")
    assert 0 < ref.ok.mean() < 1          # an informative point: some frames fail
    assert err.mean() < 1e-2
    good = ref.ok.astype(bool)            # frames near the threshold may flip under binary16 rounding
    assert (hard[good] == ref.hard[good]).all(axis=1).mean() >= 0.99


def test_decode_empty_and_single_frame(L):
    c = dev_code(L, "c1_gallager_504")
    res = L.decode(c, torch.zeros((0, c.n), device="cuda"), max_iters=5)
    assert res.hard.shape == (0, c.NW)
    w = workload("c1_gallager_504", 1, 2.0, seed=2)
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=5, schedule="plain")
    ref = oracle.decode(w.code, w.llr, iters=5)
    assert llr_close(post, ref.post).all()


def test_decode_rejects_bad_arguments(L):
    c = dev_code(L, "c1_gallager_504")
    x = torch.zeros((4, c.n), device="cuda")
    with pytest.raises(L.LdpcError):
        L.decode(c, x, max_iters=-1)
    with pytest.raises(L.LdpcError):
        L.decode(c, x, clip=0.0)
    with pytest.raises(ValueError):
        L.decode(c, x[:, :10].contiguous())


# ------------------------------------------------- resident (on-chip) decoder


@pytest.mark.parametrize("name", ["c1_gallager_504", "reg39_1008", "reg312_2016", "reg36_1008"])
@pytest.mark.parametrize("fp16", [False, True])
@pytest.mark.parametrize("early_stop", [False, True])
def test_resident_matches_plain_bit_for_bit(L, name, fp16, early_stop):
    """Both schedules share the check arithmetic and the summation order, so
    they must agree exactly, in FP32 and in FP16 storage alike."""
    w = workload(name, 203, 2.0, seed=71)   # odd F: the last frame group is ragged
    c = dev_code(L, name)
    kw = dict(max_iters=25, early_stop=early_stop, msg_fp16=fp16)
    a = _gpu_decode(L, c, w.llr, schedule="plain", **kw)
    b = _gpu_decode(L, c, w.llr, schedule="resident", **kw)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("dc,npad_log", [(6, 12), (9, 12), (9, 13), (12, 12), (12, 13)])
@pytest.mark.parametrize("early_stop", [False, True])
def test_resident_fixed_plane_instances_bit_for_bit(L, dc, npad_log, early_stop):
    """Regular codes with binary16 messages and planes of 2^12 or 2^13 words
    take the resident instances with the plane size fixed at compile time
    (rows of 6, 9 and 12); they give the plain decoder's bits.  All-zero
    codewords at Eb/N0 from 1 to 4 dB over the frames, so that with early
    stop some frames stop at different iterations and some run them all."""
    n = {12: 4032, 13: 8064}[npad_log] // dc * dc
    h = S.random_regular(n, 3, dc, seed=60 + dc)
    c = L.Code.from_csr_code(h)
    F = 13
    llr = S.bpsk_awgn_llr(np.zeros((F, n), dtype=np.uint8), np.linspace(1.0, 4.0, F), 1 - 3 / dc,
                          S.frame_noise(F, n, 72))
    kw = dict(max_iters=30, early_stop=early_stop, msg_fp16=True)
    a = _gpu_decode(L, c, llr, schedule="plain", **kw)
    b = _gpu_decode(L, c, llr, schedule="resident", **kw)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    if early_stop:
        assert len(np.unique(a[2])) > 1
    c.close()


@pytest.mark.parametrize("name", ["c1_gallager_504", "reg312_2016", "qc_irregular_512",
                                  "table1_r025", "table1_r050", "table1_r075"])
@pytest.mark.parametrize("F", [1, 37])
@pytest.mark.parametrize("early_stop", [False, True])
def test_resident_small_batch_plan_bit_for_bit(L, name, F, early_stop):
    """With FP32 messages and no more frames than SMs the resident decoder
    spreads each frame's checks over more threads (the small-batch plan).
    Check and bit arithmetic keep their order, so it must agree exactly with
    the plain decoder, and each frame's result must not depend on the batch it
    came in (a batch larger than the SM count takes the throughput plan)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = workload(name, F, 2.0, seed=83)
    c = dev_code(L, name)
    kw = dict(max_iters=15, early_stop=early_stop)
    try:
        b = _gpu_decode(L, c, w.llr, schedule="resident", **kw)
    except L.LdpcError:
        pytest.skip("code has no resident layout")
    a = _gpu_decode(L, c, w.llr, schedule="plain", **kw)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    big = np.concatenate([w.llr] * (sms // F + 1))[: sms + 5]
    d = _gpu_decode(L, c, big, schedule="resident", **kw)
    for x, y in zip(b, d):
        np.testing.assert_array_equal(x, y[:F])


def test_resident_against_oracle(L):
    w = workload("c1_gallager_504", 1000, 2.0, seed=11)
    c = dev_code(L, "c1_gallager_504")
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=20, schedule="resident")
    assert_fp32_parity(w.code, w.llr, 20, post, hard, iters, ok, max_excluded=0.05)


def test_resident_zero_iterations_and_auto_schedule(L):
    w = workload("reg36_1008", 9, 2.0, seed=72)
    c = dev_code(L, "reg36_1008")
    post, hard, iters, ok = _gpu_decode(L, c, w.llr, max_iters=0, schedule="resident")
    np.testing.assert_array_equal(post, w.llr)
    np.testing.assert_array_equal(hard, (w.llr >= 0).astype(np.uint8))
    assert (iters == 0).all()
    np.testing.assert_array_equal(ok, (~oracle.syndrome(w.code, hard).any(axis=1)).astype(np.uint8))
    # a code that fits on chip decodes resident under "auto"
    assert L.decode_workspace_size(c, 9, schedule="auto") == L.decode_workspace_size(
        c, 9, schedule="resident")


def test_resident_rejects_code_that_does_not_fit(L):
    c = dev_code(L, "irregular_37x70")   # column degree > 3
    with pytest.raises(L.LdpcError) as ei:
        L.decode(c, torch.zeros((2, c.n), device="cuda"), schedule="resident")
    assert ei.value.status == -5


# ------------------------------------------------------ decode from host memory


@pytest.mark.parametrize("pinned", [True, False])
def test_decode_from_host_memory_equals_device_decode(L, pinned):
    """ldpc_decode_host: chunked, copy-overlapped decoding from host memory gives
    the same bits as ldpc_decode on the device (ragged last chunk included)."""
    w = workload("reg36_1008", 1000, 2.0, seed=91)
    c = dev_code(L, "reg36_1008")
    host = torch.from_numpy(w.llr)
    if pinned:
        host = host.pin_memory()
    dec = L.HostDecoder(c, chunk=384, max_iters=20, early_stop=True, msg_fp16=True)
    out = dec.outputs(1000, want_post=True)
    dec.decode(host, out=out)
    torch.cuda.synchronize()
    ref = L.decode(c, host.cuda(), max_iters=20, early_stop=True, msg_fp16=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.post.numpy(), ref.post.cpu().numpy())
    np.testing.assert_array_equal(out.hard.numpy(), ref.hard.cpu().numpy())
    np.testing.assert_array_equal(out.iters.numpy(), ref.iters.cpu().numpy())
    np.testing.assert_array_equal(out.ok.numpy(), ref.ok.cpu().numpy())


def test_probe_xu_rates(L):
    """The roofline's measured per-op rates (results per SM per clock) lie in a
    sane range: at least a few, at most one warp's worth per scheduler."""
    ex2, rcp, lg2 = L.probe_xu_rates()
    for r in (ex2, rcp, lg2):
        assert 4.0 <= r <= 128.0, (ex2, rcp, lg2)
