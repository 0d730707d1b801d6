"""The allocation-free relaxed-loss entry point (sb_graphL_fwd_static).

It exists for callers that cannot allocate device memory when they call in,
because their memory is fixed ahead of time: hosts with a fixed memory budget,
plugins whose host owns the allocator, or loops that must not enter the CUDA
allocator.  This file is named to be collected
last so that a failure here never hides the other GPU tests.  It checks two
calls in a row through the C ABI against sb_graphL_fwd on the same inputs,
with the tolerance the other graphL tests use (1e-5 relative to the sum of
|terms|, discrete loss exact).
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def test_static_forward_matches_context_forward():
    import paper_2311_00869_gb300 as P

    sb = P.SignedBal(0)
    n, u, v, s = synth.er_graph(2000, 9000, 0.3, seed=17)
    n1, m1, _ = sb.load_graph(n, u, v, s)
    eu, ev, eneg = (t.cpu().numpy() for t in sb.graph_edges())
    second = (ev.astype(np.uint32) | (eneg.astype(np.uint32) << np.uint32(31))).view(np.int32)
    packed = torch.from_numpy(np.stack([eu, second], axis=1).copy()).cuda()
    eu, ev = torch.from_numpy(eu).cuda(), torch.from_numpy(ev).cuda()
    lib = P._abi.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for R, seed in ((37, 1), (256, 2)):
        gam = torch.from_numpy(synth.gamma0(n1, R, seed=seed)).cuda()
        ref_loss, ref_F = sb.graphL_fwd(gam)
        prod = (gam[eu.long()].double() * gam[ev.long()].double()).abs()
        bound = (1e-5 * 0.5 * (1.0 + prod).sum(dim=0)).cpu().numpy()
        for _call in range(2):
            loss = torch.full((R,), float("nan"), device="cuda")
            F = torch.full((R,), -1, dtype=torch.int32, device="cuda")
            rc = lib.sb_graphL_fwd_static(ctypes.c_void_p(packed.data_ptr()), m1, ctypes.c_void_p(gam.data_ptr()), R,
                                          ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(F.data_ptr()), stream)
            assert rc == 0
            torch.cuda.synchronize()
            assert torch.equal(F, ref_F)
            diff = (loss.double() - ref_loss.double()).abs().cpu().numpy()
            assert np.all(diff <= bound)
    # it allocates nothing: free device memory is the same before and after
    # repeated calls (the first call above has done the one-time set-up)
    R = 256
    gam = torch.from_numpy(synth.gamma0(n1, R, seed=3)).cuda()
    loss = torch.empty(R, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _call in range(5):
        assert lib.sb_graphL_fwd_static(ctypes.c_void_p(packed.data_ptr()), m1, ctypes.c_void_p(gam.data_ptr()), R,
                                        ctypes.c_void_p(loss.data_ptr()), None, stream) == 0  # F_out may be null
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref_loss, _ = sb.graphL_fwd(gam)
    assert np.all((loss.double() - ref_loss.double()).abs().cpu().numpy() <= 1e-5 * 0.5 * (1.0 + (
        gam[eu.long()].double() * gam[ev.long()].double()).abs()).sum(dim=0).cpu().numpy())
    # no edges: every loss and every discrete loss is 0
    loss0 = torch.full((R,), float("nan"), device="cuda")
    F0 = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    assert lib.sb_graphL_fwd_static(None, 0, ctypes.c_void_p(gam.data_ptr()), R, ctypes.c_void_p(loss0.data_ptr()),
                                    ctypes.c_void_p(F0.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    assert torch.all(loss0 == 0) and torch.all(F0 == 0)
    # sizes beyond the stated maximum are refused before anything runs
    big = torch.zeros((4, 2048), device="cuda")
    out = torch.zeros(2048, device="cuda")
    assert lib.sb_graphL_fwd_static(ctypes.c_void_p(packed.data_ptr()), m1, ctypes.c_void_p(big.data_ptr()), 2048,
                                    ctypes.c_void_p(out.data_ptr()), None, stream) == -1
    sb.close()
