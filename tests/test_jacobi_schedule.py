"""Host-side checks of the parallel one-sided Jacobi schedule (section 4 of the
paper forms N from the SVD of the sketch; the device computes that SVD by
Jacobi sweeps in round-robin order).

The device sweep for q > 1024 runs the rounds as a dataflow: persistent
workers take the pairs of all rounds in index order (item = round * P/2 + k)
and a pair waits only until its two rows have finished the previous round.
These tests restate the schedule's index rule and check the three facts that
design rests on:
  * every round is a perfect matching of the P players and a sweep meets
    every pair of rows exactly once (so a sweep is a full cyclic sweep);
  * with workers taking items in order, the smallest unfinished item never
    waits, whatever the item durations (no deadlock, any number of workers);
  * executing pairs as soon as their rows are ready gives bit for bit the
    rotations of the round-by-round order."""
import itertools

import numpy as np
import pytest


def round_pairs(P: int, t: int):
    """Pairs of round t for P (even) players: pair 0 = (P-1, t), pair k >= 1 =
    ((t + k) mod (P-1), (t - k + P - 1) mod (P-1))."""
    out = []
    for k in range(P // 2):
        if k == 0:
            out.append((P - 1, t))
        else:
            out.append(((t + k) % (P - 1), (t - k + P - 1) % (P - 1)))
    return out


@pytest.mark.parametrize("Q", [1, 2, 3, 8, 9, 100, 101])
def test_rounds_are_matchings_and_a_sweep_meets_every_pair_once(Q):
    P = Q + (Q & 1)
    seen = set()
    for t in range(P - 1):
        players = [x for pr in round_pairs(P, t) for x in pr]
        assert sorted(players) == list(range(P))          # perfect matching
        for a, b in round_pairs(P, t):
            if a < Q and b < Q:
                key = (min(a, b), max(a, b))
                assert key not in seen
                seen.add(key)
    assert seen == set(itertools.combinations(range(Q), 2))


def _simulate(Q: int, workers: int, seed: int, on_item=None):
    """Event simulation of the persistent sweep: each worker takes the next
    item index, waits until ver[a] >= t and ver[b] >= t, works for a random
    time, then publishes ver = t + 1.  Returns the completion order."""
    P = Q + (Q & 1)
    npairs = P // 2
    total = (P - 1) * npairs
    rng = np.random.Generator(np.random.PCG64(seed))
    ver = [0] * Q
    nxt = 0
    state = []            # per worker: [item or None, remaining work]
    for _ in range(workers):
        state.append([None, 0.0])
    done_order = []
    steps = 0
    while len(done_order) < total:
        steps += 1
        assert steps < 100 * total + 1000, "no progress: the sweep deadlocked"
        progressed = False
        for w in range(workers):
            item, rem = state[w]
            if item is None:
                if nxt >= total:
                    continue
                item, nxt = nxt, nxt + 1
                state[w] = [item, float(rng.exponential(1.0))]
                progressed = True
                continue
            t, k = divmod(item, npairs)
            a, b = round_pairs(P, t)[k]
            ready = (a >= Q or ver[a] >= t) and (b >= Q or ver[b] >= t)
            if not ready:
                continue
            rem -= 1.0
            progressed = True
            if rem > 0:
                state[w][1] = rem
                continue
            if on_item is not None:
                on_item(t, a, b)
            for r in (a, b):
                if r < Q:
                    ver[r] = t + 1
            done_order.append(item)
            state[w] = [None, 0.0]
        # the smallest unfinished item always has its rows ready
        assert progressed or len(done_order) == total
    return done_order


@pytest.mark.parametrize("Q,workers,seed", [(8, 3, 0), (9, 5, 1), (40, 7, 2), (41, 64, 3),
                                            (64, 1, 4), (33, 200, 5)])
def test_dataflow_sweep_never_deadlocks(Q, workers, seed):
    order = _simulate(Q, workers, seed)
    P = Q + (Q & 1)
    assert sorted(order) == list(range((P - 1) * (P // 2)))


def _rotate(W, a, b, tol):
    """One pair step on rows a < b of W, with the Hestenes angle."""
    x, y = W[a].copy(), W[b].copy()
    aa, bb, ab = x @ x, y @ y, x @ y
    if aa == 0.0 or bb == 0.0 or abs(ab) <= tol * np.sqrt(aa) * np.sqrt(bb):
        return
    zeta = (bb - aa) / (2.0 * ab)
    tt = (1.0 if zeta >= 0.0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
    cs = 1.0 / np.sqrt(1.0 + tt * tt)
    sn = cs * tt
    W[a] = cs * x - sn * y
    W[b] = sn * x + cs * y


@pytest.mark.parametrize("Q,workers,seed", [(12, 4, 7), (13, 9, 8)])
def test_dataflow_order_gives_the_round_order_bit_for_bit(Q, workers, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    W0 = np.triu(rng.standard_normal((Q, Q)))
    tol = 2.0 * Q * 2.0 ** -53
    P = Q + (Q & 1)

    ref = W0.copy()
    for t in range(P - 1):
        for a, b in round_pairs(P, t):
            if a < Q and b < Q:
                _rotate(ref, min(a, b), max(a, b), tol)

    flow = W0.copy()

    def on_item(t, a, b):
        if a < Q and b < Q:
            _rotate(flow, min(a, b), max(a, b), tol)

    _simulate(Q, workers, seed, on_item)
    assert np.array_equal(ref, flow)
