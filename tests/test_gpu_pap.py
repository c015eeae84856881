"""Batched AP and partition AP (Algorithm 2) through the C ABI against the
float64 oracle (same float32 S bits on both sides)."""
import numpy as np
import pytest
import torch

from oracle import ap as oap
from oracle import pap as opap
from paper_0910_1650_gb300 import capi, synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


def rel_inf(x, ref):
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-300))


def s32(X):
    return oap.build_similarity(X)[0].astype(np.float32).astype(np.float64)


def pack(mats):
    """1-D float32 arena with each matrix at a 16-byte aligned offset, ld % 32 == 0."""
    offs, lds, at = [], [], 0
    for M in mats:
        n = M.shape[0]
        ld = (n + 31) // 32 * 32
        offs.append(at)
        lds.append(ld)
        at += n * ld
    arena = np.zeros(at, dtype=np.float32)
    for M, o, ld in zip(mats, offs, lds):
        n = M.shape[0]
        arena[o:o + n * ld].reshape(n, ld)[:, :n] = M
    return torch.from_numpy(arena).cuda(), offs, lds


def unpack(arena, offs, ns, lds):
    a = arena.cpu().numpy().astype(np.float64)
    return [a[o:o + n * ld].reshape(n, ld)[:, :n] for o, n, ld in zip(offs, ns, lds)]


def _mixtures():
    out = []
    for j, n in enumerate([37, 120, 500, 256, 1999]):
        X, _ = synth.gaussian_mixture(n, 6, 3 + j, 900 + j, 5.0, 1.0)
        out.append(s32(X))
    return out


def test_batched_fixed_iterations_matches_oracle():
    mats = _mixtures()
    Sa, offs, lds = pack(mats)
    Ra = torch.zeros_like(Sa)
    Aa = torch.zeros_like(Sa)
    ns = [m.shape[0] for m in mats]
    res, dec = capi.ap_iterate_batched(Sa, Ra, Aa, offs, ns, lds, damping=0.9, max_iter=12,
                                       conv_iter=0, decisions=True)
    Rs, As = unpack(Ra, offs, ns, lds), unpack(Aa, offs, ns, lds)
    d = dec.cpu().numpy()
    at = 0
    for S, R, A, r, n in zip(mats, Rs, As, res, ns):
        ref = oap.run(S, lam=0.9, fixed_iters=12)
        assert r["iters"] == 12
        assert rel_inf(R, ref["R"]) <= TOL and rel_inf(A, ref["A"]) <= TOL
        assert np.array_equal(d[at:at + n], oap.decisions(R, A, dtype=np.float32))
        at += n


def test_batched_convergence_each_problem_stops_on_its_own():
    mats = _mixtures()
    Sa, offs, lds = pack(mats)
    Ra = torch.zeros_like(Sa)
    Aa = torch.zeros_like(Sa)
    ns = [m.shape[0] for m in mats]
    res, _ = capi.ap_iterate_batched(Sa, Ra, Aa, offs, ns, lds, damping=0.9, max_iter=1000,
                                     conv_iter=15)
    Rs, As = unpack(Ra, offs, ns, lds), unpack(Aa, offs, ns, lds)
    iters = []
    for S, R, A, r in zip(mats, Rs, As, res):
        ref = oap.run(S, lam=0.9, max_iter=1000, convits=15)
        assert r["converged"] == 1 and ref["converged"]
        assert abs(r["iters"] - ref["iters"]) <= max(5, 0.15 * ref["iters"])
        e_gpu = oap.exemplars(S, R, A, dtype=np.float32)
        e_ref = oap.exemplars(S, ref["R"], ref["A"])
        assert np.array_equal(e_gpu["idx"], e_ref["idx"])
        iters.append(r["iters"])
    assert len(set(iters)) > 1          # the problems really stopped at different times


def _pap_case(n=600):
    X, lab = synth.gaussian_mixture(n, 8, 6, 4242, 5.0, 1.0)
    return s32(X)


@pytest.mark.parametrize("k,part", [(4, None), (3, [0, 150, 420, 600])])
def test_pap_fixed_iterations_matches_oracle(k, part):
    S = _pap_case()
    n = S.shape[0]
    Sd = capi.empty_square(n, "cuda")
    Sd.copy_(torch.from_numpy(S.astype(np.float32)).cuda())
    R, A, idx, res = capi.pap_run(Sd, k, part, damping=0.9, max_iter=15, conv_iter=0)
    offs = part if part is not None else opap.equal_partition(n, k)
    ref = opap.run(S, offs, lam=0.9, fixed_iters=15)
    assert res["k"] == k and res["sub_iters_max"] == 15 and res["final"]["iters"] == 15
    assert rel_inf(R.cpu().numpy().astype(np.float64), ref["final"]["R"]) <= TOL
    assert rel_inf(A.cpu().numpy().astype(np.float64), ref["final"]["A"]) <= TOL


@pytest.mark.parametrize("k,part", [(4, None), (3, [0, 150, 420, 600])])
def test_pap_carry_r_matches_oracle(k, part):
    """The variant that starts Step 4 from the block-diagonal R as well as A'."""
    S = _pap_case()
    n = S.shape[0]
    Sd = capi.empty_square(n, "cuda")
    Sd.copy_(torch.from_numpy(S.astype(np.float32)).cuda())
    R, A, idx, res = capi.pap_run(Sd, k, part, damping=0.9, max_iter=15, conv_iter=0, carry_r=True)
    offs = part if part is not None else opap.equal_partition(n, k)
    ref = opap.run(S, offs, lam=0.9, fixed_iters=15, carry_r=True)
    assert rel_inf(R.cpu().numpy().astype(np.float64), ref["final"]["R"]) <= TOL
    assert rel_inf(A.cpu().numpy().astype(np.float64), ref["final"]["A"]) <= TOL
    # and it differs from the paper's form, which starts Step 4 from R = 0
    R0, _, _, _ = capi.pap_run(Sd, k, part, damping=0.9, max_iter=15, conv_iter=0)
    assert not torch.equal(R0, R)


def test_pap_converged_matches_oracle_and_plain_ap():
    S = _pap_case(1200)
    n = S.shape[0]
    Sd = capi.empty_square(n, "cuda")
    Sd.copy_(torch.from_numpy(S.astype(np.float32)).cuda())
    R, A, idx, res = capi.pap_run(Sd, 4, None, damping=0.9, max_iter=1000, conv_iter=15)
    ref = opap.run(S, opap.equal_partition(n, 4), lam=0.9, max_iter=1000, convits=15)
    e_ref = oap.exemplars(S, ref["final"]["R"], ref["final"]["A"])
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), e_ref["idx"])
    assert abs(res["final"]["netsim"] - e_ref["netsim"]) <= 1e-9 * abs(e_ref["netsim"])
    # Section 3: the result is similar to or better than plain AP on the same S
    Rp, Ap, rp, _ = capi.ap_iterate(Sd, damping=0.9, max_iter=1000, conv_iter=15)
    _, ep = capi.ap_exemplars(Sd, Rp, Ap)
    assert res["final"]["netsim"] >= ep["netsim"] - 0.005 * abs(ep["netsim"])


def test_pap_rejects_bad_partitions():
    S = capi.empty_square(100, "cuda", 0.0)
    for k, part in ((0, None), (4, [0, 10, 20, 30, 99]), (2, [0, 1, 100])):
        with pytest.raises(capi.ApgbError):
            capi.pap_run(S, k, part, max_iter=2, conv_iter=0)
