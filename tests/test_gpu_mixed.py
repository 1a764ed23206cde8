"""Mixed-code batches (one persistent launch over frames of 15 codes): every
frame must decode exactly as the single-code decoder decodes it, under any
launch configuration, eagerly and replayed from a captured CUDA graph."""

import numpy as np
import pytest
import torch

import ldpc_synth as S
import oracle
from parity_util import assert_fp32_parity

pytestmark = pytest.mark.gpu

NS = (504, 1008, 2016, 4032, 8064)
DEGS = ((3, 6), (3, 9), (3, 12))


@pytest.fixture(scope="module")
def L():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2201_04265_gb300 as L
    torch.cuda.set_device(0)
    return L


@pytest.fixture(scope="module")
def mixed(L):
    """The serving mix: n in {504..8064} x degree pairs (3,6), (3,9), (3,12)."""
    hs, syss = [], []
    for i, n in enumerate(NS):
        for j, (dv, dc) in enumerate(DEGS):
            h = S.random_regular(n, dv, dc, seed=40 + 3 * i + j)
            hs.append(h)
            syss.append(oracle.systematic(h))
    codes = [L.Code.from_csr_code(h) for h in hs]
    return hs, syss, codes


def _batch(mixed, F, seed, fc=None):
    hs, syss, _ = mixed
    rng = np.random.default_rng(seed)
    if fc is None:
        fc = rng.integers(0, len(hs), F).astype(np.int32)
    ebn0 = rng.uniform(1.0, 4.0, F)
    llrs = []
    for f in range(F):
        h, sy = hs[fc[f]], syss[fc[f]]
        msg = S.info_bits(1, sy.k, seed, frames=[f])
        cw = oracle.encode(sy, msg)
        llrs.append(S.bpsk_awgn_llr(cw, ebn0[f], sy.k / h.n, S.frame_noise(1, h.n, seed + 1, frames=[f]))[0])
    return fc, llrs


def _single(L, codes, fc, llrs, **kw):
    out = []
    for f in range(len(fc)):
        r = L.decode(codes[fc[f]], torch.from_numpy(llrs[f][None]).cuda(), schedule="resident", **kw)
        out.append((r.post.cpu().numpy()[0], r.hard.cpu().numpy()[0], int(r.iters.item()), int(r.ok.item())))
    return out


def _split(plan, b, res, fc):
    post, hard = res.post.cpu().numpy(), res.hard.cpu().numpy()
    lo, ho = b.llr_off.cpu().numpy(), b.hard_off.cpu().numpy()
    it, ok = res.iters.cpu().numpy(), res.ok.cpu().numpy()
    out = []
    for f in range(len(fc)):
        c = plan.codes[fc[f]]
        out.append((post[lo[f]:lo[f] + c.n], hard[ho[f]:ho[f] + c.NW], int(it[f]), int(ok[f])))
    return out


@pytest.mark.parametrize("fp16", [True, False])
def test_mixed_equals_single_code_decoding(L, mixed, fp16):
    _, _, codes = mixed
    fc, llrs = _batch(mixed, 150, seed=401)
    plan = L.MixedPlan(codes, msg_fp16=fp16)
    b = plan.batch(fc)
    llr = torch.from_numpy(np.concatenate(llrs)).cuda()
    kw = dict(max_iters=50, early_stop=True)
    got = _split(plan, b, plan.decode(b, llr, **kw), fc)
    want = _single(L, codes, fc, llrs, msg_fp16=fp16, **kw)
    for f, (g, w) in enumerate(zip(got, want)):
        np.testing.assert_array_equal(g[0], w[0], err_msg=f"frame {f}")
        np.testing.assert_array_equal(g[1], w[1])
        assert g[2:] == w[2:], (f, g[2:], w[2:])
    # configurations change the schedule, never the bits
    for order, gpi, cps in ((1, 1, 1), (0, 4, 2), (1, 2, 2)):
        plan.set_config(order, gpi, cps)
        again = _split(plan, b, plan.decode(b, llr, **kw), fc)
        for g, a in zip(got, again):
            np.testing.assert_array_equal(g[0], a[0])
            assert g[2:] == a[2:]


def test_mixed_autotune_graph_replay_and_bad_code(L, mixed):
    _, _, codes = mixed
    fc, llrs = _batch(mixed, 120, seed=402)
    fc[7] = 99                     # out of range: left undecoded
    plan = L.MixedPlan(codes)
    b = plan.batch(np.where(fc == 99, 0, fc))
    b.frame_code[7] = 99
    llr = torch.from_numpy(np.concatenate([llrs[f] if fc[f] != 99 else llrs[f][:codes[0].n] * 0
                                           for f in range(len(fc))])).cuda()
    cfg = plan.autotune(b, llr, reps=2)
    assert cfg["order"] in (0, 1) and cfg["groups_per_item"] >= 1
    eager = plan.decode(b, llr)
    assert int(eager.iters[7]) == -1 and int(eager.ok[7]) == 0
    # capture one decode in a CUDA graph and replay it on new inputs
    out = plan.outputs(b)
    ws = plan.workspace(len(fc))
    static_llr = llr.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.decode(b, static_llr, out=out, workspace=ws)   # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.decode(b, static_llr, out=out, workspace=ws)
    # frame 7 (no valid code) leaves its output region unwritten: compare the rest
    keep = np.ones(b.n_llr, dtype=bool)
    o7 = int(b.llr_off[7])
    keep[o7:o7 + codes[0].n] = False
    for scale in (1.0, 1.7):
        static_llr.copy_(llr * scale)
        g.replay()
        ref = plan.decode(b, llr * scale)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.post.cpu().numpy()[keep], ref.post.cpu().numpy()[keep])
        np.testing.assert_array_equal(out.iters.cpu().numpy(), ref.iters.cpu().numpy())


def test_mixed_matches_the_oracle_on_every_code(L, mixed):
    """Every one of the 15 codes of the serving mix, 6 frames each, decoded in
    one mixed launch (FP32 messages, early stop after at most 50 iterations,
    Eb/N0 ~ U[1, 4] dB per frame) against the FP64 oracle: the FP32 parity
    gate per frame, with equal iteration counts on the stable frames."""
    hs, _, codes = mixed
    per = 6
    fc = np.repeat(np.arange(len(hs), dtype=np.int32), per)
    np.random.default_rng(403).shuffle(fc)
    fc, llrs = _batch(mixed, len(fc), seed=403, fc=fc)
    plan = L.MixedPlan(codes, msg_fp16=False)
    b = plan.batch(fc)
    res = plan.decode(b, torch.from_numpy(np.concatenate(llrs)).cuda(), max_iters=50, early_stop=True)
    torch.cuda.synchronize()
    got = _split(plan, b, res, fc)
    excluded = 0
    for c, h in enumerate(hs):
        fr = np.nonzero(fc == c)[0]
        assert fr.size == per
        llr = np.stack([llrs[f] for f in fr])
        post = np.stack([got[f][0] for f in fr])
        hard = S.unpack_bits(np.stack([got[f][1] for f in fr]).view(np.uint32), h.n)
        its = np.array([got[f][2] for f in fr])
        ok = np.array([got[f][3] for f in fr])
        rep = assert_fp32_parity(h, llr, 50, post, hard, its, ok, early_stop=True, max_excluded=None)
        excluded += rep.excluded
    assert excluded <= 0.05 * len(fc), excluded
