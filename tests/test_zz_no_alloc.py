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


def _abi_noalloc(L, code, llr, T, early_stop):
    from paper_2201_04265_gb300 import _lib
    F = llr.shape[0]
    dev = llr.device
    post = torch.empty((F, code.n), dtype=torch.float32, device=dev)
    hard = torch.empty((F, code.NW), dtype=torch.int32, device=dev)
    iters = torch.empty((F,), dtype=torch.int32, device=dev)
    ok = torch.empty((F,), dtype=torch.uint8, device=dev)
    opts = _lib.DecodeOpts(T, int(early_stop), 0, 0, 20.0)
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
