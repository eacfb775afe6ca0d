"""The allocation-free sketch entry point (lsrn_sketch_f64_noalloc).

For callers that cannot allocate device memory, the FP64 sketch A~ = G A can
run with its split-K partial sums in a fixed device array of the library
instead of allocated workspace.  This test calls that entry point through the C
ABI twice in a row, on two different problems, and checks each result against
the sketch the allocating path (lsrn_plan + lsrn_sketch) computes for the same
A, gamma and seed and against the oracle's G^T A, within the tolerance of the
other sketch tests; one more case sits at the array's capacity, where the
split factor is forced down to one slice.  It lives in a file of its own,
collected last.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

TOL = 1e-13
CAPACITY = 4 << 20          # doubles in the library's fixed scratch array


def _reference_sketch(A, gamma, seed):
    plan = L.lsrn_plan(A, L.default_options(gamma=gamma, seed=seed))
    L.lsrn_sketch(plan)
    S = L.lsrn_plan_get_sketch(plan)
    plan.close()
    return S


def _oracle_sketch(A_host, s, seed):
    # Gamma[i, k] for long-side index i and sketch index k; A~ = Gamma^T A
    return O.sketch_block(seed, 0, 0, A_host.shape[0], s).T @ A_host


def _run(m, n, gamma, seed):
    rng = np.random.Generator(np.random.PCG64(m + n))
    A_host = rng.standard_normal((m, n))
    A = torch.from_numpy(A_host).to("cuda")
    s = int(np.ceil(gamma * n))
    out = torch.full((s, n), float("nan"), dtype=torch.float64, device="cuda")
    L.lsrn_sketch_f64_noalloc(A, gamma, seed, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    return A, A_host, s, got


def test_noalloc_sketch_matches_allocating_path_and_oracle_twice():
    cases = [((2000, 100), 2.0, 11), ((777, 37), 2.5, 3)]
    for (m, n), gamma, seed in cases:
        A, A_host, s, got = _run(m, n, gamma, seed)
        ref = _reference_sketch(A, gamma, seed)
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref)
        orc = _oracle_sketch(A_host, s, seed)
        assert np.linalg.norm(got - orc) <= TOL * np.linalg.norm(orc)


def test_noalloc_sketch_at_the_capacity_edge():
    m, n, gamma, seed = 12000, 1448, 2.0, 5          # s * n = 2896 * 1448 = 4,193,408 <= 4 Mi
    assert 2896 * 1448 <= CAPACITY < 2898 * 1449             # one more column would not fit
    A, A_host, s, got = _run(m, n, gamma, seed)
    orc = _oracle_sketch(A_host, s, seed)
    assert np.linalg.norm(got - orc) <= TOL * np.linalg.norm(orc)


def test_noalloc_sketch_rejects_sizes_beyond_the_fixed_scratch():
    A = torch.zeros((3000, 1500), dtype=torch.float64, device="cuda")   # s * n = 4.5 Mi > 4 Mi
    out = torch.empty((3000, 1500), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LsrnError) as e:
        L.lsrn_sketch_f64_noalloc(A, 2.0, 0, out)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
    with pytest.raises(L.LsrnError) as e:                                # s would overflow int64
        L.lsrn_sketch_f64_noalloc(A, 1e300, 0, out)
    assert e.value.status == L.LSRN_ERR_INVALID_ARG
