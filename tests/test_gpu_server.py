"""GPU tests of the serving boundary (lsrn_server_create / lsrn_submit /
lsrn_poll / lsrn_server_destroy): admitted requests run concurrently on their
own streams, and each result equals what a direct plan + solve of the same
request gives, bit for bit, and the oracle's minimum-length solution within
the parity tolerance."""
import threading
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_1109_5981_gb300")

GiB = 1 << 30


def _wait(srv, ticket, x, limit_s=120.0):
    t0 = time.monotonic()
    while True:
        st, info = L.lsrn_poll(srv, ticket, x)
        if st != L.LSRN_PENDING:
            return st, info
        assert time.monotonic() - t0 < limit_s, "request did not finish"
        time.sleep(0.002)


def _requests():
    """A mix of tall/fat dense, CSR, LSQR/CS and ridge requests."""
    out = []
    for k, (m, n) in enumerate([(3000, 120), (150, 2500), (2500, 90), (4000, 200)]):
        P = W.dense_householder(m, n, rank=min(m, n) - 5, cond=1e4, noise=1e-3, seed=30 + k)
        out.append(dict(A=torch.from_numpy(P.A), b=torch.from_numpy(P.b), solver=k % 2,
                        opt=dict(seed=7 + k), dense=P.A, bnp=P.b, csr=None))
    C = W.csr_random_density(3000, 80, 0.05, seed=41)
    bc = np.random.Generator(np.random.PCG64(42)).standard_normal(3000)
    out.append(dict(A=None, b=torch.from_numpy(bc), solver=0, opt=dict(seed=3), dense=C.to_dense(),
                    bnp=bc, csr=(C.m, C.n, torch.from_numpy(C.row_ptr), torch.from_numpy(C.col_idx),
                                 torch.from_numpy(C.values))))
    P = W.dense_householder(2000, 60, rank=60, cond=1e3, noise=1e-2, seed=50)
    out.append(dict(A=torch.from_numpy(P.A), b=torch.from_numpy(P.b), solver=1,
                    opt=dict(seed=9, lambda_=0.3), dense=P.A, bnp=P.b, csr=None, lam=0.3))
    return out


def _direct(r):
    solver = "cs" if r["solver"] == 1 else "lsqr"
    x, _ = L.solve(r["A"], r["b"], solver=solver, csr=r["csr"], **r["opt"])
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def _expected(r):
    lam = r.get("lam", 0.0)
    if lam > 0:
        return O.ridge_closed_form(r["dense"], r["bnp"], lam)
    # the refined x*: with a nonzero residual the plain FP64 SVD solution is
    # itself ~1e-10 away from x* at cond 1e4 (its error grows like cond^2 * |r|)
    return O.minlen_refined(r["dense"], r["bnp"])[0]


def test_server_results_match_direct_solves_and_oracle():
    reqs = _requests()
    srv = L.lsrn_server_create(64 * GiB, max_slots=3)
    try:
        tickets = [L.lsrn_submit(srv, r["A"], r["b"], L.default_options(**r["opt"]), r["solver"],
                                 csr=r["csr"]) for r in reqs]
        assert len(set(tickets)) == len(tickets)
        outs = []
        for r, t in zip(reqs, tickets):
            x = np.zeros(r["dense"].shape[1])
            st, info = _wait(srv, t, x)
            assert st == L.LSRN_OK, L.status_string(st)
            assert info["n"] == r["dense"].shape[1]
            outs.append(x)
    finally:
        L.lsrn_server_destroy(srv)
    for r, x in zip(reqs, outs):
        assert np.array_equal(x, _direct(r)), "server result differs from a direct solve"
        assert O.rel_err(x, _expected(r)) <= 1e-10


def test_budget_for_one_request_still_serves_all():
    # each of these requests is estimated at ~65-80 MiB (64 MiB of it a fixed
    # allowance), so a 100 MiB budget admits one at a time: the queue drains in order
    reqs = _requests()[:3]
    srv = L.lsrn_server_create(100 << 20, max_slots=4)
    try:
        tickets = [L.lsrn_submit(srv, r["A"], r["b"], L.default_options(**r["opt"]), r["solver"])
                   for r in reqs]
        for r, t in zip(reqs, tickets):
            x = np.zeros(r["dense"].shape[1])
            st, _ = _wait(srv, t, x)
            assert st == L.LSRN_OK
            assert np.array_equal(x, _direct(r))
    finally:
        L.lsrn_server_destroy(srv)


def test_oversize_request_and_bad_tickets_are_rejected():
    r = _requests()[0]
    srv = L.lsrn_server_create(1 << 20, max_slots=1)   # 1 MiB: nothing fits
    try:
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_submit(srv, r["A"], r["b"], None, 0)
        assert e.value.status == L.LSRN_ERR_QUEUE_FULL
        st, _ = L.lsrn_poll(srv, 12345, None)
        assert st == L.LSRN_ERR_INVALID_ARG
    finally:
        L.lsrn_server_destroy(srv)
    srv = L.lsrn_server_create(64 * GiB, max_slots=1)
    try:
        t = L.lsrn_submit(srv, r["A"], r["b"], None, 0)
        x = np.zeros(r["dense"].shape[1])
        assert _wait(srv, t, x)[0] == L.LSRN_OK
        assert L.lsrn_poll(srv, t, x)[0] == L.LSRN_ERR_INVALID_ARG   # already collected
        with pytest.raises(L.LsrnError) as e:
            L.lsrn_submit(srv, r["A"], r["b"], None, 7)                # no such solver
        assert e.value.status == L.LSRN_ERR_INVALID_ARG
    finally:
        L.lsrn_server_destroy(srv)


def test_invalid_request_reports_its_status():
    # gamma <= 1 passes submission and fails in the worker's lsrn_plan
    r = _requests()[0]
    srv = L.lsrn_server_create(64 * GiB, max_slots=2)
    try:
        t = L.lsrn_submit(srv, r["A"], r["b"], L.default_options(gamma=1.0), 0)
        st, _ = _wait(srv, t, None)
        assert st == L.LSRN_ERR_INVALID_ARG
    finally:
        L.lsrn_server_destroy(srv)


def test_concurrent_submitters():
    reqs = _requests()[:4]
    srv = L.lsrn_server_create(64 * GiB, max_slots=4)
    results, errors = {}, []

    def client(i):
        try:
            r = reqs[i]
            for rep in range(2):
                t = L.lsrn_submit(srv, r["A"], r["b"], L.default_options(**r["opt"]), r["solver"])
                x = np.zeros(r["dense"].shape[1])
                st, _ = _wait(srv, t, x)
                assert st == L.LSRN_OK
                results[(i, rep)] = x
        except Exception as exc:   # reported on the main thread
            errors.append(exc)

    threads = [threading.Thread(target=client, args=(i,)) for i in range(4)]
    try:
        for th in threads:
            th.start()
        for th in threads:
            th.join(300)
    finally:
        L.lsrn_server_destroy(srv)
    assert not errors, errors
    for i in range(4):
        assert np.array_equal(results[(i, 0)], results[(i, 1)])
        assert np.array_equal(results[(i, 0)], _direct(reqs[i]))


def test_destroy_with_queued_requests_returns():
    reqs = _requests()
    srv = L.lsrn_server_create(64 * GiB, max_slots=1)
    for r in reqs:
        L.lsrn_submit(srv, r["A"], r["b"], L.default_options(**r["opt"]), r["solver"], csr=r["csr"])
    t0 = time.monotonic()
    L.lsrn_server_destroy(srv)
    assert time.monotonic() - t0 < 60


def test_tc_sketch_result_does_not_depend_on_free_memory():
    """The tensor-core sketch cuts X into row segments (per-column exponents and
    the final FP64 rounding are per segment).  The segment length depends on
    the problem's shape only, so a request gives the same x bit for bit when it
    runs alone and when a neighbour holds nearly all free device memory."""
    P = W.dense_householder(200_000, 512, rank=500, cond=1e4, noise=1e-3, seed=61)
    A = torch.from_numpy(P.A).cuda()
    b = torch.from_numpy(P.b).cuda()
    opt = L.default_options(seed=5, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
    srv = L.lsrn_server_create(64 * GiB, max_slots=1)
    try:
        x_alone = np.zeros(512)
        st, _ = _wait(srv, L.lsrn_submit(srv, A, b, opt, 0), x_alone)
        assert st == L.LSRN_OK
        free, _ = torch.cuda.mem_get_info()
        hog = torch.empty(max(0, free - 8 * GiB), dtype=torch.uint8, device="cuda")
        try:
            x_crowded = np.zeros(512)
            st, _ = _wait(srv, L.lsrn_submit(srv, A, b, opt, 0), x_crowded)
            assert st == L.LSRN_OK
        finally:
            del hog
            torch.cuda.empty_cache()
    finally:
        L.lsrn_server_destroy(srv)
    assert np.array_equal(x_alone, x_crowded)


def test_server_batches_the_preconditioners_of_in_flight_requests():
    """With continuous batching on, requests that reach the preconditioner
    phase together share one batched launch; results still match the oracle
    and, to rounding, the same requests solved directly."""
    reqs = []
    for k, (m, n) in enumerate([(4000, 60), (3000, 120), (110, 2500), (6000, 40), (2500, 90),
                                (5000, 300)]):
        tall = m >= n
        P = W.dense_householder(max(m, n), min(m, n), rank=min(m, n) - 3, cond=1e4, noise=1e-3,
                                seed=170 + k)
        A = P.A if tall else np.ascontiguousarray(P.A.T)
        b = P.b if tall else np.random.Generator(np.random.PCG64(180 + k)).standard_normal(m)
        reqs.append((A, b))
    srv = L.lsrn_server_create(64 * GiB, max_slots=6)
    try:
        L.lsrn_server_set_batching(srv, 128)
        opt = L.default_options(seed=21, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
        tickets = [L.lsrn_submit(srv, torch.from_numpy(A), torch.from_numpy(b), opt, k % 2)
                   for k, (A, b) in enumerate(reqs)]
        xs = []
        for (A, b), t in zip(reqs, tickets):
            x = np.zeros(A.shape[1])
            st, info = _wait(srv, t, x)
            assert st == L.LSRN_OK, L.status_string(st)
            xs.append(x)
        batches, packed = L.lsrn_server_stats(srv)
    finally:
        L.lsrn_server_destroy(srv)
    small = sum(1 for A, _ in reqs if min(A.shape) <= 128)    # the batched kernel's limit
    assert packed == small and 1 <= batches < packed           # at least one launch packed several
    for k, ((A, b), x) in enumerate(zip(reqs, xs)):
        assert O.rel_err(x, O.minlen_refined(A, b)[0]) <= 1e-10
        xd, _ = L.solve(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(),
                        solver="cs" if k % 2 else "lsqr", seed=21, sketch_mode=L.LSRN_SKETCH_TC_SLICED)
        assert O.rel_err(x, xd.cpu().numpy()) <= 1e-11
