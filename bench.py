#!/usr/bin/env python3
"""LSRN benchmark: least-squares solves per second on one GB300.

Workload (N = 1): the dense tall problem A (10^6 x 2000, rank 1800, singular
values log-spaced 1 -> 1e-6, random orthogonal factors from 8 seeded
Householder reflectors), b = A x0 + 1e-4 N(0,1), gamma = 2 (s = 4000), LSQR to
tol 1e-14 plus refinement.  One step = one complete solve through the C ABI:
lsrn_plan + lsrn_sketch + lsrn_precond + lsrn_solve_lsqr (+ destroy), i.e.
Algorithm 1 steps 1-7, on inputs already resident in HBM, in the mixed-precision
configuration (exact tensor-core sketch, double-float passes, FP64 SVD,
recurrences and refinement).  A (16 GB) is larger than L2, so no L2 flush is
needed between steps.  The same problem is solved once more in the FP64-plain
configuration (FP64 sketch and passes) for the "mixed vs FP64 plain" comparison
of the metric, and per-solve latencies give p50/p99.

Each solve's x is checked against the planted-factor closed form
x* = V Sigma^-1 U^T b (computed on the host from the generator's factors, no
oracle call on the GPU leg); the line reports the worst relative error seen.

Under torchrun (N > 1) every rank solves its own independently seeded problem
(no collective on the data path; weak scaling) and value = all solves / max
rank time.

--impl reference times the oracle (plain FP64 CPU LSRN) on bounded samples of
the same workload on this host's cores and extrapolates to one solve with the
paper's cost model (section 4.3); the factors are printed in the line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("LS solves/s at <=1e-10 rel err: mixed precision vs FP64 plain; p50/p99 latency "
          "(dense 1e6x2000 rank 1800)")
UNIT = "solves/s"
M, N, RANK = 1_000_000, 2000, 1800


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solver", default="lsqr", choices=["lsqr", "cs"])
    ap.add_argument("--sketch", default="tc", choices=["f64", "tc", "bf16", "auto"])
    ap.add_argument("--iter", default="x2", choices=["f64", "f32", "x2"])
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--rank", type=int, default=RANK)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-plain", action="store_true",
                    help="skip the FP64-plain comparison solve after the timed region")
    ap.add_argument("--parallel", default="shard", choices=["shard", "replica"],
                    help="N > 1: shard = one problem split by rows over the ranks (section 4.4, "
                         "strong scaling); replica = an independent problem per rank (weak)")
    ap.add_argument("--single-limit", type=int, default=512,
                    help="batch workload: problems solved one at a time for the comparison lines")
    ap.add_argument("--svd", default="f64", choices=["f64", "df"],
                    help="dense workload: FP64 Jacobi sweeps, or double-float pre-sweeps first (df)")
    ap.add_argument("--precond", default="qr", choices=["qr", "svd"],
                    help="c3 workload: N = R^-1 (full-rank ridge) or the SVD preconditioner")
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "serving", "c1", "sketch", "batch", "c3"],
                    help="dense: the 1e6 x 2000 solve; serving: a Poisson stream of mixed-size "
                         "requests through lsrn_submit/lsrn_poll; c1: latency of the 2000 x 100 "
                         "rank-80 FP64 solve")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=0.0, help="arrivals per second (0: all at once)")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--pool", type=int, default=96,
                    help="serving: distinct problems the request stream cycles through")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- #
# clocks during the timed region                                               #
# --------------------------------------------------------------------------- #
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "power_w_max": float(max(power)) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- #
# CPU baseline: the oracle on bounded samples                                  #
# --------------------------------------------------------------------------- #
SAMPLE_ROWS = 10_000          # rows of A in the timed sketch sample (reference arm, per step)
SAMPLE_SVD_N = 480            # columns of the timed Jacobi SVD sample (reference arm, per step)
BASELINE_ROW_FRAC = 0.1       # cpu_baseline (once per run): a tenth of the rows ...
BASELINE_SVD_N = 800          # ... and the Jacobi SVD at 2/5 of the columns (x15.6 by the n^3 law)


def oracle_sampled_solve_seconds(A_host: np.ndarray, b_host: np.ndarray, iters: int,
                                 refine_passes: int, seed: int = 0, rows: int = SAMPLE_ROWS,
                                 svd_n: int = SAMPLE_SVD_N) -> dict:
    """Time the oracle's LSRN stages on bounded samples of the workload and
    extrapolate to one full solve with the paper's cost model (section 4.3, eq.
    lsrn_flops): the sketch (s*m normals + 2smn) is linear in the rows, the SVD
    of the s x n sketch cubic in n, and each iteration one product with A and
    one with A^T.  The stages are the calls oracle.lsrn makes (G from the
    oracle's generator times A with numpy, the oracle's one-sided Jacobi SVD,
    A v and A^T u with numpy).  Returns measured seconds, factors and the
    extrapolated total."""
    import oracle as O
    m, n = A_host.shape
    s = math.ceil(2.0 * n)
    out = {}
    # sketch: G (s x m_s) drawn by the oracle, times A[:m_s]
    m_s = max(1, min(m, rows))
    t = time.perf_counter()
    G = O.sketch_block(seed, 0, 0, m_s, s).T
    At_part = G @ A_host[:m_s]
    t_sk = time.perf_counter() - t
    del G, At_part
    # SVD of a (2 n_s) x n_s matrix with the workload's spectrum shape (log-spaced
    # 1 -> 1e-6 on 90% of the columns) by the oracle's one-sided Jacobi
    n_s = max(1, min(n, svd_n))
    rng = np.random.Generator(np.random.PCG64(1))
    r_s = max(1, int(0.9 * n_s))
    sig = np.zeros(n_s)
    sig[:r_s] = np.logspace(0, -6, r_s)
    U, _ = np.linalg.qr(rng.standard_normal((2 * n_s, n_s)))
    V, _ = np.linalg.qr(rng.standard_normal((n_s, n_s)))
    X = (U * sig) @ V.T
    t = time.perf_counter()
    O.jacobi_svd(X)
    t_svd = time.perf_counter() - t
    # one oracle LSQR-style application of A and A^T on the full matrix
    v = rng.standard_normal(n)
    t = time.perf_counter()
    u = A_host @ v
    w = A_host.T @ u
    t_pass = time.perf_counter() - t
    del u, w
    passes = iters + refine_passes
    f_sk, f_svd = m / m_s, (n / n_s) ** 3
    out["measured_s"] = {"sketch": t_sk, "svd": t_svd, "pass": t_pass}
    out["factors"] = {"sketch": f_sk, "svd": f_svd, "pass": passes}
    out["sketch_s"] = t_sk * f_sk
    out["svd_s"] = t_svd * f_svd
    out["iter_s"] = t_pass * passes
    out["total_s"] = out["sketch_s"] + out["svd_s"] + out["iter_s"]
    out["sample_s"] = t_sk + t_svd + t_pass
    out["sample"] = (f"sketch on {m_s} of {m} rows (x{f_sk:.0f}), Jacobi SVD at "
                     f"{2 * n_s}x{n_s} with the workload's spectrum shape (x(n/{n_s})^3 = "
                     f"x{f_svd:.0f}), one A and one A^T product on the full matrix "
                     f"(x{passes} passes)")
    return out


def kernel_source_hash(src_file: str, name: str) -> str:
    """sha256 (first 16 hex digits) of a kernel's definition in a CUDA source file."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1109_5981_gb300", "csrc", src_file)).read()
    i = src.index(name + "(")
    t, e = src.rfind("template", 0, i), src.rfind("\n}\n", 0, i)
    i = t if t > e else src.rfind("\n", 0, i)
    j = src.index("\n}\n", i)
    return hashlib.sha256(src[i:j + 3].encode()).hexdigest()[:16]


KERNEL_SOURCES = {"row_pass_x2_kernel": "k_iter.cu", "dd_pass_x3_kernel": "k_iter.cu",
                  "sketch_tc_kernel": "k_sketch_tc.cu", "jacobi_pair_kernel": "k_svd.cu",
                  "jacobi_flow_kernel": "k_svd.cu", "qr_coop_kernel": "k_qr_coop.cu"}


# kernels whose body is a device function shared with another launch: hash the body
HASHED_BODY = {"sketch_tc_kernel": "sketch_tc_tile"}


def traffic_per_unit(kernel: str):
    """Bytes per unit from profiles/roofline_traffic.md if the kernel is unchanged, else None."""
    try:
        rows = open(os.path.join(ROOT, "profiles", "roofline_traffic.md")).read().splitlines()
        cur = kernel_source_hash(KERNEL_SOURCES[kernel], HASHED_BODY.get(kernel, kernel))
    except (OSError, KeyError, ValueError):
        return None
    for line in rows:
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 3 and cells[0] == kernel:
            return float(cells[2]) if cells[1] == cur else None
    return None


def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "fallback": True}


def rel_error(x: np.ndarray, xstar: np.ndarray) -> float:
    return float(np.linalg.norm(x - xstar) / np.linalg.norm(xstar))


def max_over_ranks(value: float, dist, device) -> float:
    """Largest `value` over the ranks of the process group (`value` itself alone)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, elapsed_ms: float) -> float:
    """Problems solved by all ranks per second: each rank solves `steps` problems."""
    return world * steps / (elapsed_ms / 1e3)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as W
    t0 = time.perf_counter()
    P = W.c2_problem(seed=0, m=args.m, n=args.n, rank=args.rank)
    gen_s = time.perf_counter() - t0
    iters, refine = 50, 45          # the GPU solve's sweep and refinement passes at this size
    steps = []
    for k in range(args.warmup + args.steps):
        r = oracle_sampled_solve_seconds(P.A, P.b, iters, refine)
        if k >= args.warmup:
            steps.append(r)
    tot = float(np.mean([r["total_s"] for r in steps]))
    sample_ms = float(np.mean([r["sample_s"] for r in steps])) * 1e3
    value = 1.0 / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # each step times a bounded sample; value extrapolates it to one solve
        "ms_per_step": sample_ms, "extrapolated_ms_per_solve": tot * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": f"dense tall {args.m}x{args.n} rank {args.rank}, cond 1e6, "
                               "noise 1e-4, gamma 2, LSQR tol 1e-14",
                   "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": steps[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "stages_s": {k: steps[-1][k] for k in ("sketch_s", "svd_s", "iter_s")},
        "measured_s": steps[-1]["measured_s"], "factors": steps[-1]["factors"],
        "generator_s": gen_s,
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- #
# our implementation                                                           #
# --------------------------------------------------------------------------- #
def _ridge_weights(sigma: np.ndarray, lam: float) -> np.ndarray:
    """sigma / (sigma^2 + lam^2): x*_lam = V diag(.) U^T b for A = U diag(sigma) V^T (section 5)."""
    return sigma / (sigma * sigma + lam * lam)


def _csr_reference(C, b: np.ndarray, lam: float) -> np.ndarray:
    """Min-length (lam = 0) or Tikhonov solution of a full-rank sprandn matrix from the
    normal equations of its short side (well conditioned, so FP64 Cholesky is exact to
    ~1e-15): tall x = (A^T A + lam^2 I)^-1 A^T b, fat x = A^T (A A^T + lam^2 I)^-1 b."""
    import scipy.linalg as sla
    import scipy.sparse as sp
    A = sp.csr_matrix((C.values.astype(np.float64), C.col_idx, C.row_ptr), shape=(C.m, C.n))
    if C.m >= C.n:
        K = (A.T @ A).toarray() + lam * lam * np.eye(C.n)
        return sla.cho_solve(sla.cho_factor(K), A.T @ b)
    K = (A @ A.T).toarray() + lam * lam * np.eye(C.m)
    return A.T @ sla.cho_solve(sla.cho_factor(K), b)


def run_serving(args):
    """A Poisson stream of solve requests through the server (lsrn_submit /
    lsrn_poll): 80% dense problems drawn as in the batched configuration, 20%
    sprandn-like CSR (density 1e-3, short side 32-2000, long side 1e5-2e6),
    lambda in {0, 1e-4, 1e-2}.  A pool of distinct problems is cycled through;
    every result is checked against its reference (planted factors for dense
    problems, the short-side normal equations for CSR).  Mixed precision with
    the preconditioners of in-flight requests batched, against FP64 plain."""
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = "cuda"
    rng = np.random.Generator(np.random.PCG64(11))
    pool_n = max(1, min(args.requests, args.pool))
    pool = []
    for r in W.serving_requests(pool_n, seed=7, device=dev):
        lam = r["lam"]
        if r["kind"] == "dense":
            P = r["P"]
            w = _ridge_weights(P.sigma, lam)
            if r["tall"]:
                A, b = P.A, P.b
                xs = P.apply_V(P.apply_Ut(b.cpu().numpy()) * w)
            else:
                A = P.A.T.contiguous()
                bn = rng.standard_normal(A.shape[0])
                b = torch.from_numpy(bn).to(dev)
                xs = P.apply_U(P.apply_Vt(bn) * w)
            pool.append(dict(A=A, csr=None, b=b, lam=lam, xstar=xs, n=A.shape[1], kind="dense"))
        else:
            C = r["csr"]
            csr = (C.m, C.n, torch.from_numpy(C.row_ptr).to(dev), torch.from_numpy(C.col_idx).to(dev),
                   torch.from_numpy(C.values).to(dev))
            pool.append(dict(A=None, csr=csr, C=C, bnp=r["b"], b=torch.from_numpy(r["b"]).to(dev),
                             lam=lam, xstar=None, n=C.n, kind="csr"))
    solver = 1 if args.solver == "cs" else 0
    order = [k % pool_n for k in range(args.requests)]

    def stream(mode: str):
        mixed = mode == "mixed"
        srv = L.lsrn_server_create(120 << 30, max_slots=args.slots)
        try:
            L.lsrn_server_set_batching(srv, 128 if mixed else 0)
            opts = [L.default_options(seed=99, lambda_=p["lam"],
                                      sketch_mode=L.LSRN_SKETCH_TC_SLICED if mixed else L.LSRN_SKETCH_F64,
                                      iter_mode=L.LSRN_ITER_AUTO if mixed else L.LSRN_ITER_F64)
                    for p in pool]

            def submit(k):
                p = pool[k]
                return L.lsrn_submit(srv, p["A"], p["b"], opts[k], solver, csr=p["csr"])
            for k in range(min(2, pool_n)):                        # warm-up
                t = submit(k)
                while L.lsrn_poll(srv, t, None)[0] == L.LSRN_PENDING:
                    time.sleep(0.001)
            b0, r0 = L.lsrn_server_stats(srv)
            gaps = (rng.exponential(1.0 / args.rate, len(order)) if args.rate > 0
                    else np.zeros(len(order)))
            due = np.cumsum(gaps)
            xs = [np.zeros(pool[k]["n"]) for k in order]
            t_sub = np.zeros(len(order))
            t_done = np.zeros(len(order))
            tickets, statuses = {}, {}
            nxt = 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            while len(statuses) < len(order):
                now = time.perf_counter() - t0
                while nxt < len(order) and due[nxt] <= now:
                    t_sub[nxt] = time.perf_counter() - t0
                    tickets[submit(order[nxt])] = nxt
                    nxt += 1
                progressed = False
                for tk, k in list(tickets.items()):
                    st, _ = L.lsrn_poll(srv, tk, xs[k])
                    if st != L.LSRN_PENDING:
                        t_done[k] = time.perf_counter() - t0
                        statuses[k] = st
                        del tickets[tk]
                        progressed = True
                if not progressed:
                    time.sleep(0.0002)
            elapsed = float(t_done.max())
            b1, r1 = L.lsrn_server_stats(srv)
        finally:
            L.lsrn_server_destroy(srv)
        return dict(xs=xs, lat=(t_done - t_sub) * 1e3, st=statuses, elapsed=elapsed,
                    batches=b1 - b0, batched=r1 - r0)

    runs = {m: stream(m) for m in ("mixed", "fp64")}
    for p in pool:                                                   # references, after the timed runs
        if p["kind"] == "csr":
            p["xstar"] = _csr_reference(p["C"], p["bnp"], p["lam"])

    def summary(res):
        errs = np.array([rel_error(x, pool[k]["xstar"]) for x, k in zip(res["xs"], order)])
        ok = np.array([res["st"][i] == L.LSRN_OK for i in range(len(order))])
        good = int(np.sum(ok & (errs <= 1e-10)))
        lat = res["lat"]
        return {"value": good / res["elapsed"], "solved_within_1e-10": good, "elapsed_s": res["elapsed"],
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "max": float(lat.max())},
                "rel_err": {"max": float(errs.max()), "median": float(np.median(errs))},
                "batched_precond_launches": res["batches"], "batched_requests": res["batched"]}
    mix, f64 = summary(runs["mixed"]), summary(runs["fp64"])
    line = {
        "metric": "LS solves/s at <=1e-10 rel err: mixed batched vs FP64 plain; p50/p99 latency "
                  "(serving mix through lsrn_submit/lsrn_poll)",
        "value": mix["value"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
        "requests": len(order), "distinct_problems": pool_n,
        "mixed": mix, "fp64_plain": f64, "mixed_over_fp64_plain": mix["value"] / max(f64["value"], 1e-30),
        "latency_ms": mix["latency_ms"],
        "dtype": "mixed: bf16 exact-slice sketch, passes by size (f64 below 1 GiB of A), f64 SVD and refinement; "
                 "CSR: f64 sketch and passes",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": f"{len(order)} requests cycling over {pool_n} problems: 80% dense "
                               "(m log-uniform [5e3, 2e5], n log-uniform [32, 512], 70% tall, rank "
                               "0.8-1.0 min(m, n), cond 1e2-1e6), 20% CSR (density 1e-3, short side "
                               "[32, 2000], long side [1e5, 2e6]); lambda in {0, 1e-4, 1e-2}",
                   "arrivals": (f"Poisson {args.rate}/s" if args.rate > 0 else "all at t = 0"),
                   "slots": args.slots, "hbm_budget_gb": 120, "solver": args.solver,
                   "batching": "mixed: preconditioners of in-flight requests packed into shared "
                               "launches; fp64: per request"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_small(args):
    """The 2000 x 100 rank-80 problem (sigma 1 -> 1e-6, Haar factors, noise 1e-3,
    gamma 2, LSQR tol 1e-14, FP64 sketch and passes): latency of one solve,
    plan to destroy, with A and b resident on the device.  A is 1.6 MB and stays
    in L2, so the solve is bound by launch and synchronisation latency, not by
    a roofline."""
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.load_library()
    P = W.c1_problem(seed=0)
    A = torch.from_numpy(np.ascontiguousarray(P.A)).cuda()
    b = torch.from_numpy(P.b).cuda()
    x = torch.empty(P.A.shape[1], dtype=torch.float64, device="cuda")
    xstar = P.apply_V(P.apply_Ut(P.b) / P.sigma)
    opts = L.default_options(seed=3, sketch_mode=L.LSRN_SKETCH_F64, iter_mode=L.LSRN_ITER_F64)
    solve_fn = L.lsrn_solve_lsqr if args.solver == "lsqr" else L.lsrn_solve_cs

    def step():
        plan = L.lsrn_plan(A, opts)
        try:
            _, info = solve_fn(plan, b, x)
        finally:
            plan.close()
        return info

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    steps = max(args.steps, 50)
    lat = []
    launches0 = L.kernel_launches()
    for _ in range(steps):
        t0 = time.perf_counter()
        info = step()
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t0) * 1e3)
    launches = L.kernel_launches() - launches0
    lat = np.array(lat)
    err = rel_error(x.cpu().numpy(), xstar)
    line = {
        "metric": "LS solve latency (dense 2000x100 rank 80, FP64 plain LSRN, plan to destroy)",
        "value": float(np.median(lat)) * 1e3, "unit": "us", "higher_is_better": False,
        "n_gpus": 1, "steps": steps, "warmup": max(args.warmup, 3),
        "latency_us": {"p50": float(np.percentile(lat, 50)) * 1e3,
                       "p99": float(np.percentile(lat, 99)) * 1e3},
        "solves_per_s": float(steps / (lat.sum() * 1e-3)),
        "rel_err": err, "within_1e-10": bool(err <= 1e-10),
        "phases_ms": {"sketch": info["t_sketch_ms"], "precond": info["t_precond_ms"],
                      "iterations": info["t_iter_ms"], "refinement": info["t_refine_ms"]},
        "iterations": info["iterations"], "jacobi_sweeps": info["jacobi_sweeps"],
        "gpu_launches": launches, "dtype": "f64", "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": "dense 2000x100, rank 80, sigma log-spaced 1 -> 1e-6, Haar factors, "
                               "noise 1e-3, gamma 2 (s = 200); A resident in HBM (and L2)",
                   "solver": args.solver, "sketch": "f64", "passes": "f64"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (non-tensor) nominal rate


def phase_rooflines(info_list, args, peaks: dict, fp64_peak: float, m_local: int = 0) -> dict:
    """Roofline of every large phase of a solve, from the library's per-phase
    CUDA-event times averaged over the timed solves.  Work is the method's
    algorithmic work (section 4.3 and the unit counts of the path): the sketch
    2 s m n flop, the QR 2 s n^2 - 2 n^3 / 3 flop, the SVD of the n x n
    triangle 11 n^3 flop, each fused pass 8 m n bytes (A streamed once as its
    two FP32 planes, or once in FP64)."""
    m, n = (m_local or args.m), args.n        # a shard streams its own rows
    s = info_list[-1]["s"]
    mean = lambda k: float(np.mean([i[k] for i in info_list]))
    bf16 = peaks.get("bf16_tflops_sustained", 1707.9)
    hbm = peaks.get("hbm_gbs", 6785.5)
    out = {}
    t_gemm = mean("t_sketch_gemm_ms") if args.sketch == "tc" else mean("t_sketch_ms")
    flops = 2.0 * s * m * n
    if args.sketch == "tc":
        ach = flops / (t_gemm * 1e-3) / 1e12
        out["sketch"] = {"kernel": "sketch_tc_kernel (tcgen05, exact bf16 digit slices)",
                         "ms": t_gemm, "bound": "tensor", "achieved": ach, "peak": bf16,
                         "unit": "TFLOP/s", "frac": ach / bf16,
                         "peak_source": "bf16_tflops_sustained of measured (MEASURED_PEAKS.json)",
                         "work": f"2*s*m*n = {flops:.3e} flop (the method's count)",
                         "slice_products_tflops": 15 * ach,
                         "slice_products_frac": 15 * ach / bf16}
    else:
        ach = flops / (t_gemm * 1e-3) / 1e12
        out["sketch"] = {"kernel": "sketch_f64_kernel", "ms": t_gemm, "bound": "alu",
                         "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": ach / fp64_peak, "work": f"2*s*m*n = {flops:.3e} flop",
                         "peak_source": "FP64 FMA rate probed in this run (lsrn_probe_fp64_fma)"}
    t_qr = mean("t_qr_ms")
    qflops = 2.0 * s * n * n - 2.0 * n ** 3 / 3.0
    ach = qflops / (t_qr * 1e-3) / 1e12 if t_qr > 0 else 0.0
    out["qr"] = {"kernel": "qr_coop_kernel (Householder QR of the sketch in one cooperative launch; "
                           "the per-column hh_* kernels where it does not apply)", "ms": t_qr,
                 "bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                 "frac": ach / fp64_peak, "work": f"2 s n^2 - 2 n^3/3 = {qflops:.3e} flop",
                 "peak_source": "FP64 FMA rate probed in this run (lsrn_probe_fp64_fma)"}
    t_jac = mean("t_jacobi_ms")
    jflops = 11.0 * n ** 3
    ach = jflops / (t_jac * 1e-3) / 1e12 if t_jac > 0 else 0.0
    df = info_list[-1].get("jacobi_sweeps_df", 0)
    kern = ("jacobi_df_flow_kernel (double-float sweeps, FP32 pipe) + df_times_r_kernel + "
            "jacobi_flow_kernel (FP64 sweeps)" if df else "jacobi_flow_kernel (one-sided Jacobi sweeps)")
    out["svd"] = {"kernel": kern, "ms": t_jac,
                  "sweeps": info_list[-1]["jacobi_sweeps"], "sweeps_df": df, "bound": "alu", "achieved": ach,
                  "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                  "work": f"11 n^3 = {jflops:.3e} flop (the SVD count of section 4.3)",
                  "peak_source": "FP64 FMA rate probed in this run (lsrn_probe_fp64_fma)"}
    t_pass_tot = mean("t_pass_ms")
    n_pass = max(1, int(round(mean("n_pass"))))
    t_pass = t_pass_tot / n_pass
    kname = {"x2": "row_pass_x2_kernel (fused A(Nv) and A^T u on two FP32 planes)",
             "f32": "row_pass_kernel<float> (fused A(Nv) and A^T u on FP32 A)",
             "f64": "row_pass_staged_kernel<double> (fused A(Nv) and A^T u, FP64)"}[args.iter]
    streamed = {"x2": 8.0, "f32": 4.0, "f64": 8.0}[args.iter] * m * n
    gbs = 8.0 * m * n / (t_pass * 1e-3) / 1e9
    out["passes"] = {"kernel": kname, "ms": t_pass_tot, "launches": n_pass, "ms_each": t_pass,
                     "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "peak_source": "hbm_gbs of measured (MEASURED_PEAKS.json)",
                     "work": "8*m*n bytes per pass (A read once, FP64-equivalent)",
                     "bytes_streamed_per_pass": streamed}
    return out


def traffic_for(phase: str, args, m_local: int):
    """DRAM bytes per launch of the phase's kernel from profiles/roofline_traffic.md
    (null once the kernel changed since the capture)."""
    if phase == "passes" and args.iter == "x2":
        tpu = traffic_per_unit("row_pass_x2_kernel")
        return None if tpu is None else tpu * m_local * args.n
    if phase == "sketch" and args.sketch == "tc":
        tpu = traffic_per_unit("sketch_tc_kernel")
        return None if tpu is None else tpu * m_local
    if phase == "svd":
        tpu = traffic_per_unit("jacobi_flow_kernel")
        return None if tpu is None else tpu
    if phase == "qr" and args.n == 2000 and math.ceil(2.0 * args.n) == 4000:
        return traffic_per_unit("qr_coop_kernel")   # captured for the 4000 x 2000 sketch
    return None


def sketch_mode_of(L, name: str) -> int:
    return {"f64": L.LSRN_SKETCH_F64, "tc": L.LSRN_SKETCH_TC_SLICED, "bf16": L.LSRN_SKETCH_BF16,
            "auto": L.LSRN_SKETCH_AUTO}[name]


def run_sketch(args):
    """Algorithm 1 steps 2-3 alone on the 10^6 x 2000 matrix: one step = one
    lsrn_sketch (G drawn on the fly and A~ = G A) on a plan made before the
    timed region; the tensor-core GEMM is timed by the library's CUDA events."""
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.load_library()
    P = W.c2_problem(seed=0, device="cuda", m=args.m, n=args.n, rank=args.rank)
    mode = sketch_mode_of(L, args.sketch)
    plan = L.lsrn_plan(P.A, L.default_options(seed=1234, sketch_mode=mode))
    lib = L.load_library()
    s = math.ceil(2.0 * args.n)

    def one():
        L.lsrn_sketch(plan)
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        one()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = L.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gemm_ms = []
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        one()
        # the library accumulates its GEMM events into the plan until lsrn_precond reads them;
        # lsrn_plan_get_sketch does not, so time the GEMM through a precond-free probe below
    ev1.record()
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1)
    launches = L.kernel_launches() - launches0
    clk = clocks.stop()
    # one more sketch + precond to read the GEMM kernel time from lsrn_info
    L.lsrn_sketch(plan)
    L.lsrn_precond(plan)
    _, info = L.lsrn_solve_lsqr(plan, P.b, allow=(L.LSRN_OK, L.LSRN_ERR_NOT_CONVERGED))
    plan.close()
    t_gemm = info["t_sketch_gemm_ms"] if mode in (L.LSRN_SKETCH_TC_SLICED, L.LSRN_SKETCH_BF16) \
        else info["t_sketch_ms"]
    peaks = _measured_peaks()
    bf16 = peaks.get("bf16_tflops_burst", peaks.get("bf16_tflops", 1902.3))
    flops = 2.0 * s * args.m * args.n
    ach = flops / (t_gemm * 1e-3) / 1e12
    work_mult = 15 if mode == L.LSRN_SKETCH_TC_SLICED else 1
    line = {
        "metric": f"sketch A~ = G A per second (dense {args.m}x{args.n}, s = {s}, sketch {args.sketch})",
        "value": args.steps / (elapsed * 1e-3), "unit": "sketches/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": elapsed / args.steps,
        "higher_is_better": True,
        "dtype": {"tc": "bf16 exact digit slices (FP64-accurate)", "bf16": "bf16 operands, f32 accumulate",
                  "f64": "f64", "auto": "bf16 (auto)"}[args.sketch],
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": f"dense tall {args.m}x{args.n} rank {args.rank}, gamma 2",
                   "l2": "inputs larger than L2 (A is 16 GB)"},
        "roofline": {"kernel": {"tc": "sketch_tc_kernel", "bf16": "sketch_bf16_kernel",
                                "auto": "sketch_bf16_kernel", "f64": "sketch_f64_kernel"}[args.sketch],
                     "bound": "tensor" if mode != L.LSRN_SKETCH_F64 else "alu",
                     "ms": t_gemm, "achieved": ach, "unit": "TFLOP/s",
                     "peak": bf16 if mode != L.LSRN_SKETCH_F64 else L.probe_fp64_fma(),
                     "peak_source": "bf16_tflops (burst) of measured (MEASURED_PEAKS.json)"
                     if mode != L.LSRN_SKETCH_F64 else "FP64 FMA rate probed in this run",
                     "work": f"2*s*m*n = {flops:.3e} flop", "mma_work_multiple": work_mult},
        "sketch_ms_total": info["t_sketch_ms"], "gpu_launches": int(launches), "clocks": clk,
    }
    line["roofline"]["frac"] = ach / line["roofline"]["peak"]
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Many independent uneven problems: the batched configuration.  m
    log-uniform in [5e3, 2e5], n log-uniform in [32, 512], 70% tall / 30% fat
    (stored n x m), rank 0.8-1.0 min(m, n), condition 1e2-1e6, noise 1e-4.
    Mixed precision, batched: one lsrn_solve_batch call (exact tensor-core
    sketch, pass precision by size -- LSRN_ITER_AUTO: FP64 below 1 GiB of A --,
    all small preconditioners in one launch).  Compared with the FP64-plain solves (FP64
    sketch and passes) and the same mixed solves, one problem at a time."""
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.load_library()
    rng = np.random.Generator(np.random.PCG64(12))
    count = args.requests
    probs, xstars = [], []
    for P, tall in W.serving_mix(count, seed=1000, device="cuda"):
        if tall:
            A, b = P.A, P.b
            xstars.append(P.apply_V(P.apply_Ut(b.cpu().numpy()) / P.sigma))
        else:
            A = P.A.T.contiguous()
            bn = rng.standard_normal(A.shape[0])
            b = torch.from_numpy(bn).cuda()
            xstars.append(P.apply_U(P.apply_Vt(bn) / P.sigma))
        probs.append((A, b))
    elems = sum(int(A.shape[0]) * int(A.shape[1]) for A, _ in probs)
    mixed = L.default_options(seed=99, sketch_mode=L.LSRN_SKETCH_TC_SLICED, iter_mode=L.LSRN_ITER_AUTO)
    plain = L.default_options(seed=99, sketch_mode=L.LSRN_SKETCH_F64, iter_mode=L.LSRN_ITER_F64)
    solver = args.solver

    def errors(xs):
        return np.array([rel_error(x.cpu().numpy(), xs_) for x, xs_ in zip(xs, xstars)])

    # warm-up on a few problems
    L.lsrn_solve_batch(probs[:8], mixed, solver)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = L.kernel_launches()
    t0 = time.perf_counter()
    xs, infos, stats = L.lsrn_solve_batch(probs, mixed, solver)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    launches = L.kernel_launches() - launches0
    clk = clocks.stop()
    err_b = errors(xs)
    ok_b = int(np.sum((np.array(stats) == L.LSRN_OK) & (err_b <= 1e-10)))
    k1 = min(args.single_limit, count)

    def one_at_a_time(opt):
        out, t = [], time.perf_counter()
        for A, b in probs[:k1]:
            x, _ = L.solve(A, b, solver=solver, allow=(L.LSRN_OK, L.LSRN_ERR_NOT_CONVERGED),
                           **{f: getattr(opt, f) for f, _ in L.lsrn_options._fields_})
            out.append(x)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t
    xs1, t_mixed1 = one_at_a_time(mixed)
    e1 = errors(xs1)[:k1]
    xs64, t_plain = one_at_a_time(plain)
    e64 = np.array([rel_error(x.cpu().numpy(), xs_) for x, xs_ in zip(xs64, xstars[:k1])])
    ok64 = int(np.sum(e64 <= 1e-10))
    line = {
        "metric": "LS solves/s at <=1e-10 rel err: mixed batched vs FP64 plain (batched uneven mix)",
        "value": ok_b / t_batch, "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
        "problems": count, "solved_within_1e-10": ok_b, "batch_s": t_batch,
        "elements_of_A": elems, "gb_of_A_fp64": elems * 8 / 1e9,
        "rel_err": {"max": float(err_b.max()), "median": float(np.median(err_b))},
        "fp64_plain_one_at_a_time": {"value": ok64 / t_plain, "problems": k1, "seconds": t_plain,
                                     "within_1e-10": ok64, "max_rel_err": float(e64.max())},
        "mixed_one_at_a_time": {"value": int(np.sum(e1 <= 1e-10)) / t_mixed1, "problems": k1,
                                "seconds": t_mixed1},
        "batched_over_fp64_plain": (ok_b / t_batch) / max(ok64 / t_plain, 1e-30),
        "batched_precond_ms": float(np.median([i["t_precond_ms"] for i in infos])),
        "per_problem_sums_ms": {k: float(np.sum([i[k] for i in infos]))
                                for k in ("t_sketch_ms", "t_iter_ms", "t_refine_ms")},
        "iterations": {"main_median": float(np.median([i["iterations"] for i in infos])),
                       "refine_median": float(np.median([i["refine_iterations"] for i in infos])),
                       "refine_steps_median": float(np.median([i["refine_steps"] for i in infos]))},
        "dtype": "mixed: bf16 exact-slice sketch, passes by size (f64 below 1 GiB of A), f64 SVD",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": f"{count} problems: m log-uniform [5e3, 2e5], n log-uniform [32, 512], "
                               "70% tall / 30% fat, rank 0.8-1.0 min(m, n), cond 1e2-1e6, noise 1e-4",
                   "solver": solver, "threads": 8},
        "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_c3(args):
    """The sparse under-determined Tikhonov problem: A 10^4 x 10^6 CSR with 2000
    uniform-random columns per row, N(0,1) values, b ~ N(0,1), lambda = 1e-3
    (Algorithm 2 on [A / lambda, I_m], s = 2 * 10^4, G drawn on the fly).  One
    step = plan + sketch + preconditioner + LSQR + refinement; x is checked
    after the timed region against the ridge closed form
    A^T (A A^T + lambda^2 I)^-1 b (sparse product and FP64 Cholesky)."""
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    L.load_library()
    A, b = W.c3_problem(seed=0)
    lam = 1e-3
    csr = (A.m, A.n, torch.from_numpy(A.row_ptr).cuda(), torch.from_numpy(A.col_idx).cuda(),
           torch.from_numpy(A.values).cuda())
    bt = torch.from_numpy(b).cuda()
    x = torch.empty(A.n, dtype=torch.float64, device="cuda")
    mode = L.LSRN_PRECOND_QR if args.precond == "qr" else L.LSRN_PRECOND_SVD
    opt = L.default_options(seed=3, lambda_=lam, precond_mode=mode)
    solve_fn = L.lsrn_solve_lsqr if args.solver == "lsqr" else L.lsrn_solve_cs

    def step():
        plan = L.lsrn_plan(None, opt, csr=csr)
        try:
            _, info = solve_fn(plan, bt, x)
        finally:
            plan.close()
        return info

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = L.kernel_launches()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    ev[0].record()
    infos = []
    for k in range(args.steps):
        infos.append(step())
        ev[k + 1].record()
    torch.cuda.synchronize()
    elapsed = ev[0].elapsed_time(ev[-1])
    launches = L.kernel_launches() - launches0
    clk = clocks.stop()
    import scipy.linalg as sla
    import scipy.sparse as sp
    As = sp.csr_matrix((A.values, A.col_idx, A.row_ptr), shape=(A.m, A.n))
    K = (As @ As.T).toarray() + lam * lam * np.eye(A.m)
    ref = As.T @ sla.cho_solve(sla.cho_factor(K), b)
    err = rel_error(x.cpu().numpy(), ref)
    info = infos[-1]
    mean = lambda k: float(np.mean([i[k] for i in infos]))
    line = {
        "metric": "LS solves/s at <=1e-10 rel err (sparse fat 1e4x1e6 CSR, 2000 nnz/row, ridge 1e-3)",
        "value": args.steps / (elapsed * 1e-3), "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps,
        "higher_is_better": True, "dtype": "f64",
        "data": "synthetic (seeded generator, no dataset)",
        "config": {"workload": "sparse fat 10^4 x 10^6 CSR, 2000 uniform columns per row, N(0,1), "
                               "b ~ N(0,1), lambda 1e-3, gamma 2 (s = 2e4)",
                   "precond": {"qr": "N = R^-1 of the sketch's QR (full rank by the ridge)",
                               "svd": "N = V Sigma^-1 (one-sided Jacobi SVD)"}[args.precond],
                   "solver": args.solver},
        "accuracy": {"rel_err_vs_ridge_closed_form": err, "ok": bool(err <= 1e-10)},
        "phases_ms": {"sketch": mean("t_sketch_ms"), "precond": mean("t_precond_ms"),
                      "precond_qr": mean("t_qr_ms"), "iter": mean("t_iter_ms"),
                      "refine": mean("t_refine_ms")},
        "iterations": info["iterations"], "refine_iterations": info["refine_iterations"],
        "jacobi_sweeps": info["jacobi_sweeps"], "gpu_launches": int(launches), "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_dense(args):
    import torch
    import paper_1109_5981_gb300 as L
    import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl")
        dist = dist_
    L.load_library()
    dev = f"cuda:{local}"
    sharded = world > 1 and args.parallel == "shard"

    if sharded:
        # one problem, rows split over the ranks; every rank ends with the whole x
        off, cnt = L.shard_rows(args.m, world, rank)
        P = W.c2_problem(seed=0, device=dev, m=args.m, n=args.n, rank=args.rank,
                         rows=(off, off + cnt))
        gather = L.torch_allgather()
        sizes = [L.shard_rows(args.m, world, r)[1] for r in range(world)]
        bpad = torch.zeros(max(sizes), dtype=torch.float64, device=dev)
        bpad[:cnt] = P.b
        ball = [torch.empty_like(bpad) for _ in range(world)]
        dist.all_gather(ball, bpad)
        b_full = torch.cat([t[:c] for t, c in zip(ball, sizes)]).cpu().numpy()
    else:
        P = W.c2_problem(seed=rank, device=dev, m=args.m, n=args.n, rank=args.rank)
        b_full = P.b.cpu().numpy()
    A, b = P.A, P.b
    x = torch.empty(args.n, dtype=torch.float64, device=dev)
    # x* = V Sigma^-1 U^T b from the generator's planted factors
    xstar = P.apply_V(P.apply_Ut(b_full) / P.sigma)
    opts = L.default_options(seed=1234 + (0 if sharded else rank),
                             sketch_mode=sketch_mode_of(L, args.sketch),
                             iter_mode={"f32": L.LSRN_ITER_F32, "x2": L.LSRN_ITER_F32X2}.get(
                                 args.iter, L.LSRN_ITER_F64),
                             svd_mode=L.LSRN_SVD_DF if args.svd == "df" else L.LSRN_SVD_F64)
    solve_fn = L.lsrn_solve_lsqr if args.solver == "lsqr" else L.lsrn_solve_cs

    def make_plan(Amat, o):
        if sharded:
            return L.lsrn_plan_sharded(Amat, o, rank, world, off, args.m, gather)
        return L.lsrn_plan(Amat, o)

    def step(o=opts):
        plan = make_plan(A, o)
        try:
            _, info = solve_fn(plan, b, x)
        finally:
            plan.close()
        return info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = L.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    evs[0].record()
    infos = []
    for k in range(args.steps):
        infos.append(step())
        evs[k + 1].record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed_ms = evs[0].elapsed_time(evs[-1])
    per_step = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
    launches = L.kernel_launches() - launches0
    clk = clocks.stop()
    errs = [rel_error(x.cpu().numpy(), xstar)]   # every step solves the same problem
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    # sharded: all ranks together solve one problem per step
    value = job_throughput(1 if sharded else world, args.steps, elapsed_ms)
    info = infos[-1]
    fp64_peak = L.probe_fp64_fma()
    peaks = _measured_peaks()
    phases = phase_rooflines(infos, args, peaks, fp64_peak, int(A.shape[0]))
    dominant = max(phases, key=lambda k: phases[k]["ms"])
    roofline = dict(phases[dominant])
    roofline["phase"] = dominant
    roofline["traffic"] = traffic_for(dominant, args, int(A.shape[0]))
    roofline["selection"] = "largest device time per solve among sketch, qr, svd, passes"

    # FP64 plain: the same problem with the FP64 sketch and FP64 passes (one solve,
    # outside the timed region) -- the comparison point of the metric
    fp64_plain = None
    if not args.no_fp64_plain:
        o64 = L.default_options(seed=1234 + rank, sketch_mode=L.LSRN_SKETCH_F64,
                                iter_mode=L.LSRN_ITER_F64)
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        inf64 = step(o64)
        e1.record()
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        err64 = rel_error(x.cpu().numpy(), xstar)
        fp64_plain = {"value": job_throughput(1 if sharded else world, 1, ms64), "unit": UNIT,
                      "ms_per_solve": ms64,
                      "steps": 1, "rel_err": err64, "within_1e-10": bool(err64 <= 1e-10),
                      "phases_ms": {"sketch": inf64["t_sketch_ms"], "precond": inf64["t_precond_ms"],
                                    "iter": inf64["t_iter_ms"], "refine": inf64["t_refine_ms"]},
                      "config": "FP64 sketch (DFMA), FP64 passes, FP64 SVD and refinement"}

    # end to end through the C ABI with host buffers (pinned A, b in; x out)
    e2e = None
    if not args.no_e2e:
        rows_here = A.shape[0]
        A_h = torch.empty((rows_here, args.n), dtype=torch.float64, pin_memory=True)
        A_h.copy_(A)
        b_h = b.cpu().numpy().copy()
        x_h = np.empty(args.n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            plan = make_plan(A_h, opts)
            solve_fn(plan, b_h, x_h)
            plan.close()
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.e2e_steps
        e2e_s = max_over_ranks(e2e_s * 1e3, dist, dev) / 1e3
        errs.append(rel_error(x_h, xstar))
        e2e = {"value": job_throughput(1 if sharded else world, 1, e2e_s * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(rows_here * args.n * 8 + rows_here * 8),
               "d2h_bytes_per_step": int(args.n * 8)}
        del A_h

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        A_np = A.cpu().numpy()
        r = oracle_sampled_solve_seconds(A_np, b.cpu().numpy(), info["iterations"],
                                         info["refine_iterations"] + 1,
                                         rows=int(BASELINE_ROW_FRAC * A_np.shape[0]),
                                         svd_n=BASELINE_SVD_N)
        cpu = {"value": 1.0 / r["total_s"], "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": r["sample"], "sample_s": r["sample_s"],
               "stages_s": {k: r[k] for k in ("sketch_s", "svd_s", "iter_s")},
               "measured_s": r["measured_s"], "factors": r["factors"]}
        del A_np

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None,
            "dtype": {"x2": "mixed: bf16 exact-slice sketch, f32x2 passes, f32x3 residual, "
                            "f64 SVD/recurrences/refinement",
                      "f32": "mixed: f32 passes, f64 SVD/recurrences/residual",
                      "f64": "f64"}[args.iter],
            "data": "synthetic (seeded generator, no dataset)",
            "config": {"workload": f"dense tall {args.m}x{args.n} rank {args.rank}, cond 1e6, "
                                   f"noise 1e-4, gamma 2, {args.solver.upper()} tol 1e-14 + "
                                   f"refinement, sketch {args.sketch}, passes {args.iter}",
                       "l2": "inputs larger than L2 (A is 16 GB)",
                       "parallelism": (f"one problem row-sharded over {world} GPUs (allgather of "
                                       "n + 1 values per pass)" if sharded
                                       else "independent problem per GPU")},
            "latency_ms": {"p50": float(np.percentile(per_step, 50)),
                           "p99": float(np.percentile(per_step, 99)),
                           "max": float(per_step.max())},
            "fp64_plain": fp64_plain,
            "mixed_over_fp64_plain": (value / fp64_plain["value"]) if fp64_plain else None,
            "accuracy": {"max_rel_err_vs_planted_xstar": max(errs), "target": 1e-10,
                         "ok": bool(max(errs) <= 1e-10)},
            "phases_ms": {"sketch": float(np.mean([i["t_sketch_ms"] for i in infos])),
                          "precond": float(np.mean([i["t_precond_ms"] for i in infos])),
                          "precond_qr": float(np.mean([i["t_qr_ms"] for i in infos])),
                          "precond_jacobi": float(np.mean([i["t_jacobi_ms"] for i in infos])),
                          "iter": float(np.mean([i["t_iter_ms"] for i in infos])),
                          "refine": float(np.mean([i["t_refine_ms"] for i in infos]))},
            "iterations": info["iterations"], "refine_iterations": info["refine_iterations"],
            "jacobi_sweeps": info["jacobi_sweeps"], "jacobi_sweeps_df": info["jacobi_sweeps_df"],
            "refine_steps": info["refine_steps"],
            "rank": info["rank"], "s": info["s"],
            "roofline": roofline,
            "roofline_phases": phases,
            "fp64_peak_tflops": {"probed": fp64_peak, "nominal": FP64_NOMINAL_TFLOPS},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": int(launches),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "c1":
        return run_small(args)
    if args.workload == "sketch":
        return run_sketch(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "c3":
        return run_c3(args)
    return run_dense(args)


if __name__ == "__main__":
    sys.exit(main())
