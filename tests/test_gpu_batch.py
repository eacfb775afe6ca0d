"""Batched solve (lsrn_solve_batch): many independent problems phase by phase,
with the preconditioners of all small problems in one launch (one CTA per
problem).  Each result must match the oracle's min-length (or ridge) solution
at the parity tolerance and the same problem solved alone to ~1e-11; the
batched SVD's singular values must match the per-problem path's; problems the
batched kernel does not take (short side > 128, CSR with a TC request, AUTO)
go through the per-problem path in the same call."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")


def _problems():
    """(A for the library, b, dense A for the oracle, lam)"""
    out = []
    rng = np.random.Generator(np.random.PCG64(91))
    shapes = [(3000, 40), (5000, 200), (900, 300), (120, 2500), (64, 700), (4000, 511),
              (2000, 97), (300, 33), (7000, 600), (50, 4000)]
    for k, (m, n) in enumerate(shapes):
        tall = m >= n
        mm, nn = (m, n) if tall else (n, m)
        P = W.dense_householder(mm, nn, rank=max(1, int(0.9 * nn)), cond=1e4, noise=1e-3, seed=100 + k)
        A = P.A if tall else np.ascontiguousarray(P.A.T)
        b = P.b if tall else rng.standard_normal(m)
        out.append((torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), A, b, 0.0))
    C = W.csr_random_density(2500, 60, 0.05, seed=120)
    bc = rng.standard_normal(2500)
    csr = (C.m, C.n, torch.from_numpy(C.row_ptr).cuda(), torch.from_numpy(C.col_idx).cuda(),
           torch.from_numpy(C.values).cuda())
    out.append((csr, torch.from_numpy(bc).cuda(), C.to_dense(), bc, 0.0))
    return out


@pytest.mark.parametrize("solver,sketch", [("lsqr", "tc"), ("cs", "f64")])
def test_batch_matches_oracle_and_single_solves(solver, sketch):
    probs = _problems()
    mode = L.LSRN_SKETCH_TC_SLICED if sketch == "tc" else L.LSRN_SKETCH_F64
    opt = L.default_options(seed=17, sketch_mode=mode)
    xs, infos, stats = L.lsrn_solve_batch([(A, b) for A, b, _, _, _ in probs], opt, solver,
                                          threads=4)
    assert stats == [L.LSRN_OK] * len(probs)
    for (A, b, Ad, bd, lam), x, inf in zip(probs, xs, infos):
        xh = x.cpu().numpy()
        xs_ref, _ = O.minlen_refined(Ad, bd)
        assert O.rel_err(xh, xs_ref) <= 1e-10, (Ad.shape, inf)
        kw = dict(csr=A) if isinstance(A, tuple) else {}
        x1, inf1 = L.solve(None if kw else A, b, solver=solver, seed=17, sketch_mode=mode, **kw)
        assert inf1["rank"] == inf["rank"]
        assert O.rel_err(xh, x1.cpu().numpy()) <= 1e-11
        assert abs(inf1["sigma_max_sketch"] - inf["sigma_max_sketch"]) <= 1e-12 * inf1["sigma_max_sketch"]
        assert abs(inf1["sigma_min_sketch"] - inf["sigma_min_sketch"]) <= 1e-9 * inf1["sigma_min_sketch"]


def test_batch_ridge_and_mixed_iteration_mode():
    rng = np.random.Generator(np.random.PCG64(93))
    probs = []
    for k, (m, n) in enumerate([(2500, 90), (80, 1500), (6000, 300)]):
        P = W.dense_householder(max(m, n), min(m, n), rank=min(m, n), cond=1e3, noise=1e-2, seed=130 + k)
        A = P.A if m >= n else np.ascontiguousarray(P.A.T)
        b = P.b if m >= n else rng.standard_normal(m)
        probs.append((A, b))
    opt = L.default_options(seed=19, lambda_=0.2, sketch_mode=L.LSRN_SKETCH_TC_SLICED,
                            iter_mode=L.LSRN_ITER_F32)
    xs, infos, stats = L.lsrn_solve_batch([(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda())
                                           for A, b in probs], opt, "lsqr")
    assert stats == [L.LSRN_OK] * 3
    for (A, b), x in zip(probs, xs):
        assert O.rel_err(x.cpu().numpy(), O.ridge_closed_form(A, b, 0.2)) <= 1e-10


def test_batch_edge_cases():
    xs, infos, stats = L.lsrn_solve_batch([], None)
    assert xs == [] and stats == []
    A = torch.zeros((300, 20), dtype=torch.float64, device="cuda")     # rank 0: x = 0
    b = torch.ones(300, dtype=torch.float64, device="cuda")
    xs, infos, stats = L.lsrn_solve_batch([(A, b)], None)
    assert stats == [L.LSRN_OK] and infos[0]["rank"] == 0 and float(xs[0].abs().max()) == 0.0


def test_grouped_tensor_core_sketch_is_bit_identical_to_one_at_a_time():
    """lsrn_sketch_group puts the exact tensor-core sketches of small dense
    plans into shared launches; each sketch must be bit for bit the one
    lsrn_sketch gives alone, and plans it does not group (ridge, CSR, FP64
    mode) must still come out right.  The grouped sketch is also checked
    against the oracle's G A (1e-13 of sum |g||a|)."""
    probs = _problems()
    opt_tc = dict(seed=41, sketch_mode=L.LSRN_SKETCH_TC_SLICED)

    def make(k, A, extra=None):
        kw = dict(opt_tc, **(extra or {}))
        if isinstance(A, tuple):
            return L.lsrn_plan(None, L.default_options(**kw), csr=A)
        return L.lsrn_plan(A, L.default_options(**kw))

    extras = [None] * len(probs)
    extras[1] = dict(lambda_=0.05)                    # ridge: sketched alone
    extras[2] = dict(sketch_mode=L.LSRN_SKETCH_F64)   # FP64 mode: sketched alone
    group = [make(k, p[0], extras[k]) for k, p in enumerate(probs)]
    alone = [make(k, p[0], extras[k]) for k, p in enumerate(probs)]
    try:
        sts = L.lsrn_sketch_group(group)
        assert sts == [L.LSRN_OK] * len(group)
        for p in alone:
            L.lsrn_sketch(p)
        for k, (pg, pa) in enumerate(zip(group, alone)):
            Sg, Sa = L.lsrn_plan_get_sketch(pg), L.lsrn_plan_get_sketch(pa)
            assert np.array_equal(Sg, Sa), k
        # one grouped sketch against the oracle: tall 3000 x 40, Gamma^T A
        Sg = L.lsrn_plan_get_sketch(group[0])
        A = probs[0][2]
        Gm = O.sketch_block(41, 0, 0, A.shape[0], Sg.shape[0])
        ref = Gm.T @ A
        bound = 1e-13 * (np.abs(Gm).T @ np.abs(A))
        assert np.all(np.abs(Sg - ref) <= bound + 1e-300)
        # and the grouped plans solve like any other
        x, info = L.lsrn_solve_lsqr(group[3], probs[3][1])
        xs, _ = O.minlen_refined(probs[3][2], probs[3][3])
        assert O.rel_err(x.cpu().numpy(), xs) <= 1e-10
    finally:
        for p in group + alone:
            p.close()
