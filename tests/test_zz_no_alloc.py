"""ldpc_decode_noalloc: decoding for callers that cannot allocate device memory.

Such callers (a real-time receive thread that must not block in an
allocator, or a framework that owns every device buffer) get their scratch
from the library's one static device array.  This test calls the entry point
through the C ABI twice in a row, on different batches, and checks each
result against ldpc_decode with the plain schedule; the second call must not
see anything left in the shared array by the first.  It also checks that a
batch needing more scratch than the array holds is refused.  The file is
named so that pytest collects it last.
"""

import ctypes

import numpy as np
import pytest
import torch

import ldpc_synth as S
from parity_util import hard_close, llr_close, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


def _abi_noalloc(L, code, llr, T, early_stop, schedule=0):
    from paper_2201_04265_gb300 import _lib
    F = llr.shape[0]
    dev = llr.device
    post = torch.empty((F, code.n), dtype=torch.float32, device=dev)
    hard = torch.empty((F, code.NW), dtype=torch.int32, device=dev)
    iters = torch.empty((F,), dtype=torch.int32, device=dev)
    ok = torch.empty((F,), dtype=torch.uint8, device=dev)
    opts = _lib.DecodeOpts(T, int(early_stop), 0, schedule, 20.0)
    st = code._lib.ldpc_decode_noalloc(code.handle, ctypes.c_void_p(llr.data_ptr()), F, ctypes.byref(opts),
                                       ctypes.c_void_p(post.data_ptr()), ctypes.c_void_p(hard.data_ptr()),
                                       ctypes.c_void_p(iters.data_ptr()), ctypes.c_void_p(ok.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, post, hard, iters, ok


@pytest.mark.parametrize("name", ["c1_gallager_504", "reg39_1008"])
def test_noalloc_matches_decode_on_two_calls_in_a_row(L, name):
    from parity_util import code_and_sys
    h, _ = code_and_sys(name)
    code = L.Code.from_csr_code(h)
    for call, (F, ebn0, T, es) in enumerate([(300, 2.0, 20, False), (171, 2.5, 30, True)]):
        w = workload(name, F, ebn0, seed=500 + call)
        llr = torch.from_numpy(w.llr).cuda()
        st, post, hard, iters, ok = _abi_noalloc(L, code, llr, T, es)
        assert st == 0, code._lib.ldpc_last_error()
        ref = L.decode(code, llr, max_iters=T, early_stop=es, schedule="plain")
        torch.cuda.synchronize()
        p, rp = post.cpu().numpy(), ref.post.cpu().numpy()
        assert llr_close(p, rp).all()
        h_got = S.unpack_bits(hard.cpu().numpy().view(np.uint32), code.n)
        h_ref = S.unpack_bits(ref.hard.cpu().numpy().view(np.uint32), code.n)
        assert hard_close(h_got, h_ref, rp).all()
        np.testing.assert_array_equal(iters.cpu().numpy(), ref.iters.cpu().numpy())
        np.testing.assert_array_equal(ok.cpu().numpy(), ref.ok.cpu().numpy())


def _same_as_plain(L, code, llr, got, T, es, fp16=False):
    post, hard, iters, ok = got
    ref = L.decode(code, llr, max_iters=T, early_stop=es, schedule="plain", msg_fp16=fp16)
    torch.cuda.synchronize()
    p, rp = post.cpu().numpy(), ref.post.cpu().numpy()
    assert llr_close(p, rp).all()
    h_got = S.unpack_bits(hard.cpu().numpy().view(np.uint32), code.n)
    h_ref = S.unpack_bits(ref.hard.cpu().numpy().view(np.uint32), code.n)
    assert hard_close(h_got, h_ref, rp).all()
    np.testing.assert_array_equal(iters.cpu().numpy(), ref.iters.cpu().numpy())
    np.testing.assert_array_equal(ok.cpu().numpy(), ref.ok.cpu().numpy())
    return iters.cpu().numpy()


def test_noalloc_leftover_stop_flags_do_not_carry_over(L):
    """Two early-stop calls of the same size: the first, at high Eb/N0, stops
    most frames after a few iterations and leaves their stop marks and
    unsatisfied-check flags in the shared array; the second, at low Eb/N0,
    must still run every frame until it converges or reaches the cap."""
    from parity_util import code_and_sys
    h, _ = code_and_sys("c1_gallager_504")
    code = L.Code.from_csr_code(h)
    F, T = 256, 40
    its = []
    for call, ebn0 in enumerate((5.0, 1.0)):
        w = workload("c1_gallager_504", F, ebn0, seed=520 + call)
        llr = torch.from_numpy(w.llr).cuda()
        st, *got = _abi_noalloc(L, code, llr, T, True)
        assert st == 0, code._lib.ldpc_last_error()
        its.append(_same_as_plain(L, code, llr, got, T, True))
    assert np.median(its[0]) <= 5 and (its[1] == T).mean() > 0.2, (np.median(its[0]), (its[1] == T).mean())


def test_noalloc_binary16_messages_through_the_binding(L):
    """The binding's decode_noalloc with binary16 messages equals the plain
    schedule's binary16 decode, on two calls in a row."""
    from parity_util import code_and_sys
    h, _ = code_and_sys("reg36_1008")
    code = L.Code.from_csr_code(h)
    for call, (F, T, es) in enumerate([(200, 25, False), (200, 25, True)]):
        w = workload("reg36_1008", F, 2.0, seed=540 + call)
        llr = torch.from_numpy(w.llr).cuda()
        r = L.decode_noalloc(code, llr, max_iters=T, early_stop=es, msg_fp16=True)
        _same_as_plain(L, code, llr, (r.post, r.hard, r.iters, r.ok), T, es, fp16=True)


def test_noalloc_refuses_the_resident_schedule(L):
    from parity_util import code_and_sys
    h, _ = code_and_sys("c1_gallager_504")
    code = L.Code.from_csr_code(h)
    llr = torch.zeros((4, code.n), dtype=torch.float32, device="cuda")
    assert _abi_noalloc(L, code, llr, 5, False, schedule=2)[0] == -1
    assert b"plain schedule" in code._lib.ldpc_last_error()


def test_noalloc_refuses_batches_beyond_the_static_scratch(L):
    from paper_2201_04265_gb300 import _lib
    from parity_util import code_and_sys
    h, _ = code_and_sys("reg36_1008")
    code = L.Code.from_csr_code(h)
    per_frame = L.decode_workspace_size(code, 64, schedule="plain") / 64
    F = int(_lib.NOALLOC_SCRATCH_BYTES / per_frame) + 64
    llr = torch.zeros((F, code.n), dtype=torch.float32, device="cuda")
    st = _abi_noalloc(L, code, llr, 5, False)[0]
    assert st == -1
    assert b"static array" in code._lib.ldpc_last_error()
