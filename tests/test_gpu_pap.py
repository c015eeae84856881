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


def _tie_outcomes(S, trials=48):
    """Exemplar sets the oracle converges to from S with every entry scaled by
    (1 + 1e-7 z), z standard normal (seeded): the outcomes rounding can pick
    when the unperturbed problem sits on an exact tie."""
    g = np.random.default_rng(5)
    out = {tuple(oap.exemplars(S, *(lambda r: (r["R"], r["A"]))(
        oap.run(S, lam=0.9, max_iter=1000, convits=15)))["E"])}
    for _ in range(trials):
        P = S * (1.0 + 1e-7 * g.standard_normal(S.shape))
        r = oap.run(P, lam=0.9, max_iter=1000, convits=15)
        out.add(tuple(oap.exemplars(S, r["R"], r["A"])["E"]))
    return out


def test_batched_tiny_and_mixed_sizes_with_clusters_resplit():
    """Sizes from 2 to 1500 in one batch (the launch configuration is the
    largest problem's; the small ones get one cluster each), run to
    convergence with a host check every iteration, so that the clusters are
    re-split between the problems still running many times; every problem
    still matches the oracle, and the batch also matches fixed-iteration
    parity."""
    g = np.random.default_rng(77)
    sizes = [2, 3, 5, 31, 64, 250, 700, 1500]
    mats = []
    for j, n in enumerate(sizes):
        X, _ = synth.gaussian_mixture(n, 4, max(1, min(6, n // 5)), 600 + j, 6.0, 1.0)
        mats.append(s32(X))
    Sa, offs, lds = pack(mats)
    for it, conv in ((9, 0), (1000, 15)):
        Ra = torch.zeros_like(Sa)
        Aa = torch.zeros_like(Sa)
        res, _ = capi.ap_iterate_batched(Sa, Ra, Aa, offs, sizes, lds, damping=0.9, max_iter=it,
                                         conv_iter=conv, check_every=1)
        Rs, As = unpack(Ra, offs, sizes, lds), unpack(Aa, offs, sizes, lds)
        for S, R, A, r in zip(mats, Rs, As, res):
            ref = oap.run(S, lam=0.9, max_iter=it, convits=conv) if conv else \
                oap.run(S, lam=0.9, fixed_iters=it)
            if conv:
                assert r["converged"] == 1
                got = oap.exemplars(S, R, A, dtype=np.float32)
                want = oap.exemplars(S, ref["R"], ref["A"])
                margin = np.abs(np.diag(ref["R"]) + np.diag(ref["A"])).min()
                if margin > 1e-5 * np.abs(S).max():
                    assert np.array_equal(got["idx"], want["idx"])
                else:
                    # an exact tie (n <= 3: the median preference is itself one
                    # of the similarities, so some a + r is exactly 0): rounding
                    # decides the outcome, so the exemplar set must be one the
                    # oracle reaches from S perturbed at float32 rounding level
                    assert np.all(got["idx"][got["E"]] == got["E"])
                    assert tuple(got["E"]) in _tie_outcomes(S)
            else:
                assert r["iters"] == it
                # a vanishing reference (n = 2: both off-diagonal entries are the
                # median, so R and A are exactly 0) is compared on the scale of S
                scale = max(np.abs(ref["R"]).max(), np.abs(ref["A"]).max(), 1e-2 * np.abs(S).max())
                assert np.abs(R - ref["R"]).max() <= TOL * scale
                assert np.abs(A - ref["A"]).max() <= TOL * scale


def test_batched_size_classes_match_oracle():
    """A batch that splits into two size classes (32 problems of 520 points
    and 8 of 1100; each class holds more than 8e6 elements of work, so
    neither merges) runs them one after another with their own launch
    configurations; every problem still matches the oracle after 9 fixed
    iterations, and the converged outcome on a sample of each class."""
    sizes = [520] * 32 + [1100] * 8
    classes = capi.ap_sweep_classes(sizes)
    assert classes == [0] * 32 + [1] * 8
    mats = []
    for j, n in enumerate(sizes):
        X, _ = synth.gaussian_mixture(n, 8, 4 + j % 5, 700 + j, 6.0, 1.0)
        mats.append(s32(X))
    Sa, offs, lds = pack(mats)
    for it, conv in ((9, 0), (1000, 15)):
        Ra = torch.zeros_like(Sa)
        Aa = torch.zeros_like(Sa)
        res, _ = capi.ap_iterate_batched(Sa, Ra, Aa, offs, sizes, lds, damping=0.9, max_iter=it,
                                         conv_iter=conv)
        Rs, As = unpack(Ra, offs, sizes, lds), unpack(Aa, offs, sizes, lds)
        picks = range(len(sizes)) if not conv else (0, 31, 32, 39)
        for j in picks:
            S, R, A, r = mats[j], Rs[j], As[j], res[j]
            if conv:
                ref = oap.run(S, lam=0.9, max_iter=it, convits=conv)
                assert r["converged"] == 1
                got = oap.exemplars(S, R, A, dtype=np.float32)
                want = oap.exemplars(S, ref["R"], ref["A"])
                assert np.array_equal(got["idx"], want["idx"]), j
            else:
                ref = oap.run(S, lam=0.9, fixed_iters=it)
                assert r["iters"] == it
                assert rel_inf(R, ref["R"]) <= TOL and rel_inf(A, ref["A"]) <= TOL, j
