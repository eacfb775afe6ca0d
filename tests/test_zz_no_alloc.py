"""The allocation-free sketch entry point (lsrn_sketch_f64_noalloc).

For callers that cannot allocate device memory, the FP64 sketch A~ = G A can
run with its split-K partial sums in a fixed device array of the library
instead of allocated workspace.  This test calls that entry point through the C
ABI twice in a row, on two different problems, and checks each result against
the sketch the allocating path (lsrn_plan + lsrn_sketch) computes for the same
A, gamma and seed, within the tolerance of the other sketch tests.  It lives in
a file of its own, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

TOL = 1e-13


def _reference_sketch(A, gamma, seed):
    plan = L.lsrn_plan(A, L.default_options(gamma=gamma, seed=seed))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    plan.close()
    return S


def test_noalloc_sketch_matches_allocating_path_twice():
    cases = [((2000, 100), 2.0, 11), ((777, 37), 2.5, 3)]
    for (m, n), gamma, seed in cases:
        rng = np.random.Generator(np.random.PCG64(m + n))
        A = torch.from_numpy(rng.standard_normal((m, n))).to("cuda")
        s = int(np.ceil(gamma * n))
        out = torch.full((s, n), float("nan"), dtype=torch.float64, device="cuda")
        L.lsrn_sketch_f64_noalloc(A, gamma, seed, out)
        torch.cuda.synchronize()
        ref = _reference_sketch(A, gamma, seed)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)


def test_noalloc_sketch_rejects_sizes_beyond_the_fixed_scratch():
    A = torch.zeros((3000, 1500), dtype=torch.float64, device="cuda")   # s * n = 4.5 Mi > 4 Mi
    out = torch.empty((3000, 1500), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_sketch_f64_noalloc(A, 2.0, 0, out)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
