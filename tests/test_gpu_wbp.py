"""Weighted belief propagation on the GPU: forward against the oracle, and the
hand-written adjoint against the FP64 autograd reference and finite
differences."""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle
from oracle import wbp_ref
from parity_util import code_and_sys, fp32_conditioned_frames, llr_close, workload

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
        _codes[name] = L.Code.from_csr_code(code_and_sys(name)[0])
    return _codes[name]


def _weights(T, E, seed, spread=0.2):
    return (1.0 + spread * np.random.default_rng(seed).standard_normal((T, E))).astype(np.float32)


def test_unit_weights_equal_plain_decoder_bit_for_bit(L):
    w = workload("reg36_1008", 130, 2.0, seed=81)
    c = dev_code(L, "reg36_1008")
    llr = torch.from_numpy(w.llr).cuda()
    ones = torch.ones((10, c.nnz), dtype=torch.float32, device="cuda")
    post = L.weighted_bp(c, llr, ones)
    ref = L.decode(c, llr, max_iters=10, schedule="plain")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(post.cpu().numpy(), ref.post.cpu().numpy())


@pytest.mark.parametrize("T", [1, 3, 10])
def test_forward_matches_oracle_with_random_weights(L, T):
    wl = workload("reg36_1008", 64, 2.0, seed=82)
    c = dev_code(L, "reg36_1008")
    wts = _weights(T, c.nnz, seed=83)
    post = L.weighted_bp(c, torch.from_numpy(wl.llr).cuda(), torch.from_numpy(wts).cuda())
    ref = oracle.decode(wl.code, wl.llr, iters=T, weights=wts.astype(np.float64))
    assert llr_close(post.cpu().numpy(), ref.post).all()


def _gpu_loss_grads(L, c, llr, wts, bits):
    llr_t = torch.from_numpy(llr).cuda().requires_grad_(True)
    w_t = torch.from_numpy(wts).cuda().requires_grad_(True)
    post = L.weighted_bp(c, llr_t, w_t)
    loss = torch.nn.functional.binary_cross_entropy_with_logits(
        post, torch.from_numpy(bits.astype(np.float32)).cuda(), reduction="mean")
    loss.backward()
    return float(loss.detach()), w_t.grad.cpu().numpy().astype(np.float64), llr_t.grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("T,ebn0", [(3, 2.0), (10, 2.0)])
def test_backward_matches_fp64_reference_gradient(L, T, ebn0):
    """Config-5 shape: (3,6) code n = 1008, T unrolled iterations, BCE loss."""
    wl = workload("reg36_1008", 16, ebn0, seed=84)
    c = dev_code(L, "reg36_1008")
    wts = _weights(T, c.nnz, seed=85)
    loss, gw, gR = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    rloss, rgw, rgR, _ = wbp_ref.loss_and_grads(wl.code, wl.llr.astype(np.float64), wts.astype(np.float64), wl.cw)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss) + 1e-7
    # Tolerance (reading of the gradient bar for FP32): the FP64 reference itself
    # moves by up to ~5e-3 relative on coordinates below 1e-4 of the largest when
    # its inputs are rounded to FP32, so the relative bound applies from 1e-3 of
    # the largest coordinate up, and an absolute bound of 1e-5 of it everywhere.
    for got, ref in ((gw, rgw), (gR, rgR)):
        cos = float(np.dot(got.ravel(), ref.ravel()) / (np.linalg.norm(got) * np.linalg.norm(ref)))
        assert cos >= 0.9999, cos
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
        mx = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-5 * mx
        big = np.abs(ref) >= 1e-3 * mx
        rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
        assert rel.max() <= 1e-3, rel.max()


def test_backward_against_finite_differences_of_gpu_forward(L):
    wl = workload("reg36_1008", 32, 2.0, seed=86)
    c = dev_code(L, "reg36_1008")
    T = 4
    wts = _weights(T, c.nnz, seed=87)
    _, gw, _ = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    bits = torch.from_numpy(wl.cw.astype(np.float32)).cuda()
    llr_t = torch.from_numpy(wl.llr).cuda()

    def loss_of(wv):
        post = L.weighted_bp(c, llr_t, torch.from_numpy(wv).cuda())
        # float64 reduction of the FP32 posteriors
        return float(torch.nn.functional.binary_cross_entropy_with_logits(
            post.double(), bits.double(), reduction="mean"))

    h = 1e-3
    idx = np.argsort(-np.abs(gw).ravel())[:24]   # coordinates with a clear signal
    for flat in idx:
        t, e = divmod(int(flat), c.nnz)
        wp = wts.copy(); wp[t, e] += h
        wm = wts.copy(); wm[t, e] -= h
        fd = (loss_of(wp) - loss_of(wm)) / (2 * h)
        assert abs(fd - gw[t, e]) <= 2e-2 * abs(gw[t, e]) + 1e-7, (t, e, fd, gw[t, e])


def test_backward_deterministic_and_zero_iterations(L):
    wl = workload("c1_gallager_504", 200, 2.0, seed=88)
    c = dev_code(L, "c1_gallager_504")
    wts = _weights(5, c.nnz, seed=89)
    a = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    b = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    # T = 0: the posterior is the input and its gradient passes through
    llr_t = torch.from_numpy(wl.llr).cuda().requires_grad_(True)
    post = L.weighted_bp(c, llr_t, torch.zeros((0, c.nnz), device="cuda"))
    np.testing.assert_array_equal(post.detach().cpu().numpy(), wl.llr)
    post.sum().backward()
    assert torch.all(llr_t.grad == 1)


def _check_grads(got_ref_pairs):
    for got, ref in got_ref_pairs:
        cos = float(np.dot(got.ravel(), ref.ravel()) / (np.linalg.norm(got) * np.linalg.norm(ref)))
        assert cos >= 0.9999, cos
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)
        mx = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-5 * mx
        big = np.abs(ref) >= 1e-3 * mx
        rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
        assert rel.max() <= 1e-3, rel.max()


def test_backward_at_256_frames_against_fp64_reference_and_finite_differences(L):
    """The gradient bar at 256 frames of the configuration-5 code (n = 1008,
    T = 10, 2 dB): against the FP64 autograd reference, and central finite
    differences (h = 1e-3) of the GPU forward on the 24 largest coordinates."""
    wl = workload("reg36_1008", 256, 2.0, seed=90)
    c = dev_code(L, "reg36_1008")
    T = 10
    wts = _weights(T, c.nnz, seed=91)
    loss, gw, gR = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    rloss, rgw, rgR, _ = wbp_ref.loss_and_grads(wl.code, wl.llr.astype(np.float64), wts.astype(np.float64), wl.cw)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss) + 1e-7
    _check_grads(((gw, rgw), (gR, rgR)))
    bits = torch.from_numpy(wl.cw.astype(np.float32)).cuda()
    llr_t = torch.from_numpy(wl.llr).cuda()

    def loss_of(wv):
        post = L.weighted_bp(c, llr_t, torch.from_numpy(wv).cuda())
        return float(torch.nn.functional.binary_cross_entropy_with_logits(post.double(), bits.double(),
                                                                          reduction="mean"))

    h = 1e-3
    for flat in np.argsort(-np.abs(gw).ravel())[:24]:
        t, e = divmod(int(flat), c.nnz)
        wp = wts.copy(); wp[t, e] += h
        wm = wts.copy(); wm[t, e] -= h
        fd = (loss_of(wp) - loss_of(wm)) / (2 * h)
        assert abs(fd - gw[t, e]) <= 2e-2 * abs(gw[t, e]) + 1e-7, (t, e, fd, gw[t, e])


def test_backward_deterministic_at_4096_frames(L):
    """The configuration-5 batch (4096 frames, T = 10): two backward passes
    give identical weight and input gradients (fixed-order frame reduction)."""
    wl = workload("reg36_1008", 4096, 2.0, seed=92)
    c = dev_code(L, "reg36_1008")
    wts = _weights(10, c.nnz, seed=93)
    a = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    b = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])
    assert np.isfinite(a[1]).all() and np.abs(a[1]).max() > 0


def test_table1_code_rows_of_12(L):
    """The paper's Table I code of rate 1/2 (rows of 12 ones): unit weights give
    the plain decoder's bits, random weights the oracle's forward, and the
    adjoint the FP64 reference gradient."""
    wl = workload("table1_r050", 24, 3.0, seed=94)
    c = dev_code(L, "table1_r050")
    llr = torch.from_numpy(wl.llr).cuda()
    post = L.weighted_bp(c, llr, torch.ones((6, c.nnz), dtype=torch.float32, device="cuda"))
    ref = L.decode(c, llr, max_iters=6, schedule="plain")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(post.cpu().numpy(), ref.post.cpu().numpy())
    T = 3
    wts = _weights(T, c.nnz, seed=95)
    post = L.weighted_bp(c, llr, torch.from_numpy(wts).cuda())
    oref = oracle.decode(wl.code, wl.llr, iters=T, weights=wts.astype(np.float64))
    assert llr_close(post.cpu().numpy(), oref.post).all()
    loss, gw, gR = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    rloss, rgw, rgR, _ = wbp_ref.loss_and_grads(wl.code, wl.llr.astype(np.float64), wts.astype(np.float64), wl.cw)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss) + 1e-7
    _check_grads(((gw, rgw), (gR, rgR)))


@pytest.mark.parametrize("F", [1, 37])
def test_irregular_code_and_ragged_batch(L, F):
    """Rows of 3 to 7 edges and columns of 1 to 4 (a lifted quasi-cyclic code):
    every row is shorter than the kernel's width of 8 and takes the guarded
    path (the regular codes above take the unguarded one), and a batch
    that is not a multiple of the frames a thread takes leaves padding frames
    beside real ones.  Unit weights give the plain decoder's bits, random
    weights the oracle's forward, the adjoint the FP64 reference gradient."""
    wl = workload("qc_irregular_512", F, 2.5, seed=96)
    c = dev_code(L, "qc_irregular_512")
    rows = np.diff(wl.code.row_ptr)
    assert rows.max() < 8 and rows.min() < rows.max()
    llr = torch.from_numpy(wl.llr).cuda()
    post = L.weighted_bp(c, llr, torch.ones((8, c.nnz), dtype=torch.float32, device="cuda"))
    ref = L.decode(c, llr, max_iters=8, schedule="plain")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(post.cpu().numpy(), ref.post.cpu().numpy())
    T = 5
    wts = _weights(T, c.nnz, seed=97)
    post = L.weighted_bp(c, llr, torch.from_numpy(wts).cuda())
    oref = oracle.decode(wl.code, wl.llr, iters=T, weights=wts.astype(np.float64))
    assert llr_close(post.cpu().numpy(), oref.post).all()
    loss, gw, gR = _gpu_loss_grads(L, c, wl.llr, wts, wl.cw)
    rloss, rgw, rgR, _ = wbp_ref.loss_and_grads(wl.code, wl.llr.astype(np.float64), wts.astype(np.float64), wl.cw)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss) + 1e-7
    _check_grads(((gw, rgw), (gR, rgR)))
