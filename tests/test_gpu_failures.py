"""Error paths made on the host: a device allocation that fails (injected by
the library's test hook, no GPU fault involved) must come back as
LDPC_ENOMEM from every call that allocates, leave nothing allocated behind,
and leave the library usable."""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle

pytestmark = pytest.mark.gpu

ENOMEM = -2


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.fixture()
def hook(L):
    from paper_2201_04265_gb300 import _lib
    lib = _lib.load()
    yield lib.ldpc_test_fail_allocation
    lib.ldpc_test_fail_allocation(-1)


def test_code_creation_fails_cleanly_at_every_allocation(L, hook):
    h = S.random_regular(1008, 3, 6, seed=5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for after in range(40):
        hook(after)
        try:
            c = L.Code.from_csr_code(h)
        except L.LdpcError as e:
            assert e.status == ENOMEM, e
            failures += 1
            continue
        hook(-1)                      # more allocations than this code makes: nothing failed
        c.close()
        break
    assert failures >= 10             # every device table of the code was a failure point
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 8 << 20   # the failed creations freed their tables
    # the library still decodes afterwards
    sysm = oracle.systematic(h)
    cw = oracle.encode(sysm, S.info_bits(4, sysm.k, 7))
    llr = S.bpsk_awgn_llr(cw, 3.0, sysm.k / h.n, S.frame_noise(4, h.n, 8))
    c = L.Code.from_csr_code(h)
    r = L.decode(c, torch.from_numpy(llr).cuda(), max_iters=20)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(S.unpack_bits(r.hard.cpu().numpy().view(np.uint32), h.n),
                                  oracle.decode(h, llr, iters=20).hard)


def test_encode_tables_and_mixed_plan_report_enomem(L, hook):
    h = S.gallager_regular(504, 3, 6, seed=1)
    c = L.Code.from_csr_code(h)
    sysm = oracle.systematic(h)
    msgs = S.info_bits(5, sysm.k, 11)
    info = torch.from_numpy(S.pack_bits(msgs).view(np.int32)).cuda()
    for after in (0, 1):              # the column table, then the tables themselves
        hook(after)
        with pytest.raises(L.LdpcError) as ei:
            c.build_encode_tables()
        assert ei.value.status == ENOMEM
    hook(-1)
    # encoding falls back to the AND/XOR form with the oracle's codewords
    got = S.unpack_bits(L.encode(c, info).cpu().numpy().view(np.uint32), h.n)
    np.testing.assert_array_equal(got, oracle.encode(sysm, msgs))
    codes = [L.Code.from_csr_code(S.random_regular(504, 3, 6, seed=40)),
             L.Code.from_csr_code(S.random_regular(1008, 3, 9, seed=41))]
    for after in (0, 1, 2):           # slot tables of each code, then the descriptors
        hook(after)
        with pytest.raises(L.LdpcError) as ei:
            L.MixedPlan(codes)
        assert ei.value.status == ENOMEM
    hook(-1)
    plan = L.MixedPlan(codes)         # and a plan builds once the device has memory again
    assert plan.config()["groups_per_item"] >= 1
