"""ap_exemplars_noalloc: the exemplar outputs for callers that cannot allocate
device memory (callers that only hold pointers handed to them, callers whose
device memory is reserved by another framework's pool, latency-critical code
where cudaMalloc would synchronise).  It must give what ap_exemplars gives,
call after call, while allocating nothing.

This file is named to be collected last."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from paper_0910_1650_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _square(M):
    n = M.shape[0]
    t = capi.empty_square(n, "cuda")
    t.copy_(torch.from_numpy(np.ascontiguousarray(M, dtype=np.float32)).cuda())
    return t


def _case(X, iters, lam):
    S = oap.build_similarity(X)[0]
    ref = oap.run(S, lam=lam, fixed_iters=iters)
    return _square(S), _square(ref["R"]), _square(ref["A"])


def _oracle_outputs(S, R, A):
    """The oracle's outputs on the very float32 bits the GPU sees, with the
    a+r decisions taken in float32 as the kernels take them."""
    n = S.shape[0]
    f = lambda t: t.cpu().numpy()[:, :n].astype(np.float64)
    return oap.exemplars(f(S), f(R), f(A), dtype=np.float32)


def test_noalloc_matches_workspace_entry_two_calls_in_a_row():
    X1, _ = synth.gaussian_mixture_2d()                 # n = 500
    X2, _ = synth.workload(1, scale=0.1)                # n = 2000, d = 64
    cases = [_case(X2, 30, 0.9), _case(X1, 120, 0.5)]   # larger first: stale scratch is longer
    outs = [torch.empty(c[0].shape[0], dtype=torch.int32, device="cuda") for c in cases]
    torch.cuda.synchronize()
    free_after_setup = None
    for (S, R, A), idx_buf in zip(cases, outs):
        idx_ref, ref = capi.ap_exemplars(S, R, A)
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        idx, got = capi.ap_exemplars_noalloc(S, R, A, idx=idx_buf)
        torch.cuda.synchronize()
        after = torch.cuda.mem_get_info()[0]
        if free_after_setup is not None:
            assert after == before          # the call itself allocated nothing
        free_after_setup = after
        assert torch.equal(idx, idx_ref)
        assert got["n_exemplars"] == ref["n_exemplars"] > 0
        for k in ("dpsim", "expref", "netsim"):
            assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k])
        # and what the oracle computes from the same messages
        ora = _oracle_outputs(S, R, A)
        assert np.array_equal(idx.cpu().numpy().astype(np.int64), ora["idx"])
        assert got["n_exemplars"] == ora["E"].size
        for k in ("dpsim", "expref", "netsim"):
            assert abs(got[k] - ora[k]) <= 1e-9 * abs(ora[k])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import ctypes as C
    n = capi.AP_NOALLOC_MAX_N + 1
    ld = (n + 3) // 4 * 4
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")   # never read: the size check comes first
    idx = torch.zeros(16, dtype=torch.int32, device="cuda")
    res = capi.ApResult()
    p = C.c_void_p(buf.data_ptr())
    st = capi.lib().ap_exemplars_noalloc(p, p, p, n, ld, C.c_void_p(idx.data_ptr()),
                                         C.byref(res), None)
    assert st == capi.AP_ERR_TOO_LARGE
    assert "scratch" in capi.status_string(st)
