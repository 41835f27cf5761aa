"""Serving loop (mx_server_*): results are the same alone and in a mix of requests with
other operators and batched right-hand sides; factorisations are cached and reused across
xi_prob; a small memory budget forces evictions; per-request latency is reported."""
import numpy as np
import pytest

import inputs
from parity import assert_close

pytestmark = pytest.mark.gpu

mx = pytest.importorskip("paper_1711_03789_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _req(s, n, k, xp, xq, seed, nrhs, tol=1e-10, cm=0):
    c, p = inputs.bump_batch(seed, nrhs)
    return mx.mx_server_submit(s, n, k, xp, xq, c, p, core_cells=5, overlap_cells=1, coarse_cells=cm,
                               precision=mx.MX_PLAIN_FP64, tol=tol, restart=0, max_it=300)


def _n_dof(n):
    return 3 * n * (n - 1) ** 2 + 3 * n * n * (n - 1) + n ** 3


def test_same_result_alone_and_in_the_mix():
    s = mx.mx_server_create(8 << 30, workers=3)
    try:
        t = _req(s, 10, 6.0, 6.0, 6.0, seed=5, nrhs=2)
        x_alone, st_alone, tm, rc = mx.mx_server_poll(s, t, _n_dof(10), 2)
        assert rc == mx.MX_OK and all(v["converged"] for v in st_alone) and tm["latency_ms"] > 0
        # the same request among others: same operator (batched with it), other xi_prob
        # (shares the factorisation), and other operators running concurrently
        tickets = [_req(s, 10, 6.0, 6.0, 6.0, seed=7, nrhs=3),
                   _req(s, 10, 6.0, 6.0, 6.0, seed=5, nrhs=2),
                   _req(s, 10, 6.0, 3.0, 6.0, seed=8, nrhs=1),
                   _req(s, 10, 4.0, 4.0, 4.0, seed=9, nrhs=4),
                   _req(s, 10, 6.0, 6.0, 6.0, seed=11, nrhs=5, cm=5)]
        out = {}
        for tk, nr in zip(tickets, [3, 2, 1, 4, 5]):
            out[tk] = mx.mx_server_poll(s, tk, _n_dof(10), nr)
        x_mix = out[tickets[1]][0]
        assert_close(x_mix, x_alone, 1e-7, what="request in the mix against alone")
        info = mx.mx_server_stats(s)
        assert info["completed"] == 6 and info["pending"] == 0
        # three preconditioner keys: (k=6, xi=6, one level), (k=4, xi=4), (k=6, xi=6, coarse 5)
        assert info["factorisations"] == 3, info
    finally:
        mx.mx_server_destroy(s)


def test_budget_forces_eviction():
    # measure what one operator holds, then give the server room for one and a half
    s0 = mx.mx_server_create(8 << 30, workers=1)
    try:
        mx.mx_server_poll(s0, _req(s0, 10, 6.0, 6.0, 6.0, seed=1, nrhs=1, tol=1e-8), _n_dof(10), 1)
        one = mx.mx_server_stats(s0)["cached_bytes"]
    finally:
        mx.mx_server_destroy(s0)
    s = mx.mx_server_create(int(1.5 * one), workers=1)
    try:
        t1 = _req(s, 10, 6.0, 6.0, 6.0, seed=1, nrhs=1, tol=1e-8)
        mx.mx_server_poll(s, t1, _n_dof(10), 1)
        t2 = _req(s, 10, 4.0, 4.0, 4.0, seed=2, nrhs=1, tol=1e-8)
        mx.mx_server_poll(s, t2, _n_dof(10), 1)
        t3 = _req(s, 10, 6.0, 6.0, 6.0, seed=3, nrhs=1, tol=1e-8)
        x, st, tm, rc = mx.mx_server_poll(s, t3, _n_dof(10), 1)
        info = mx.mx_server_stats(s)
        assert rc == mx.MX_OK and info["evictions"] >= 1 and info["factorisations"] == 3, info
    finally:
        mx.mx_server_destroy(s)


def test_request_too_large_for_budget_fails_cleanly():
    s = mx.mx_server_create(1 << 20, workers=1)
    try:
        t = _req(s, 10, 6.0, 6.0, 6.0, seed=1, nrhs=1)
        with pytest.raises(mx.MxError) as e:
            mx.mx_server_poll(s, t, _n_dof(10), 1)
        assert e.value.code == mx.MX_ENOMEM
    finally:
        mx.mx_server_destroy(s)


def _mixed_req(s, seed, nrhs, n=20, k=10.0):
    c, p = inputs.bump_batch(seed, nrhs)
    return mx.mx_server_submit(s, n, k, k * k, k * k, c, p, core_cells=5, overlap_cells=1, coarse_cells=4,
                               precision=mx.MX_MIXED, tol=1e-11, restart=10, max_it=600)


def test_request_joins_a_running_batch_with_the_same_result():
    """Continuous batching in the mixed form: a request submitted while a batch of its operator
    is running is admitted into the batch's free slots at the next restart boundary (one
    worker, so it cannot start a batch of its own), and its solution equals the one it gets
    alone, element by element (both to 1e-11; each slot keeps its own arithmetic, so only the
    rounding of the other slots' presence differs)."""
    import time
    n = 20
    nd = 3 * n * (n - 1) ** 2 + 3 * n * n * (n - 1) + n ** 3
    s = mx.mx_server_create(8 << 30, workers=1)
    try:
        x_alone, st_alone, _, rc = mx.mx_server_poll(s, _mixed_req(s, 31, 3), nd, 3)
        assert rc == mx.MX_OK and all(v["converged"] for v in st_alone)
        # a long batch first (GMRES(10) to 1e-11 on its operator), then the same request again
        t_long = _mixed_req(s, 32, 2)
        t0 = time.perf_counter()
        while mx.mx_server_stats(s)["pending"] and time.perf_counter() - t0 < 30:
            time.sleep(0.001)
        t_join = _mixed_req(s, 31, 3)
        x_mix, st_mix, tm, rc = mx.mx_server_poll(s, t_join, nd, 3)
        _, st_long, tm_long, rc_long = mx.mx_server_poll(s, t_long, nd, 2)
        info = mx.mx_server_stats(s)
        assert rc == mx.MX_OK and all(v["converged"] for v in st_mix)
        assert info["joined"] >= 1 and info["batches"] == 2, info  # the first batch, then the one it joined
        # admitted at a restart boundary of the long batch, not after it
        print("queue", tm["queue_ms"], "ms; long batch", tm_long["latency_ms"], "ms")
        assert tm["queue_ms"] < 0.5 * tm_long["latency_ms"], (tm, tm_long)
        assert_close(x_mix, x_alone, 1e-8, what="request joined into a running batch against alone")
        for a, b in zip(st_mix, st_alone):
            assert abs(a["iterations"] - b["iterations"]) <= 1, (st_mix, st_alone)
    finally:
        mx.mx_server_destroy(s)


def test_batch_waiting_for_memory_goes_first():
    """Under a budget that holds one of two operators, a batch of the second waits for memory
    while a long batch of the first runs. While it waits, a request of the first operator does
    not join the running batch (it would keep the memory held). It runs after the waiting batch
    instead, on a new factorisation: three factorisations, two evictions, nothing joined."""
    import time

    def long_req(s, seed, nrhs, max_it):
        # unreachable tolerance: the batch runs its full iteration count
        c, p = inputs.bump_batch(seed, nrhs)
        return mx.mx_server_submit(s, 30, 15.0, 225.0, 225.0, c, p, core_cells=5, overlap_cells=1, coarse_cells=6,
                                   precision=mx.MX_MIXED, tol=1e-15, restart=10, max_it=max_it)

    nd30, nd10 = _n_dof(30), _n_dof(10)
    s0 = mx.mx_server_create(8 << 30, workers=1)
    try:
        mx.mx_server_poll(s0, long_req(s0, 41, 2, 10), nd30, 2)  # same slots and restart: same bytes
        need_a = mx.mx_server_stats(s0)["cached_bytes"]
        x_b, st_b, _, rc = mx.mx_server_poll(s0, _req(s0, 10, 6.0, 6.0, 6.0, seed=42, nrhs=1, tol=1e-8), nd10, 1)
        need_b = mx.mx_server_stats(s0)["cached_bytes"] - need_a
        assert rc == mx.MX_OK and 0 < need_b < need_a, (need_a, need_b)
    finally:
        mx.mx_server_destroy(s0)
    s = mx.mx_server_create(need_a + need_b // 2, workers=3)
    try:
        t_long = long_req(s, 41, 2, 3000)
        # the long batch holds its memory once admitted (taken from the queue is not enough: a
        # request submitted before the admission could still take the memory first)
        t0 = time.perf_counter()
        while mx.mx_server_stats(s)["cached_bytes"] < need_a and time.perf_counter() - t0 < 30:
            time.sleep(0.001)
        assert mx.mx_server_stats(s)["cached_bytes"] == need_a
        t_b = _req(s, 10, 6.0, 6.0, 6.0, seed=42, nrhs=1, tol=1e-8)
        t0 = time.perf_counter()
        while mx.mx_server_stats(s)["waiting_for_memory"] == 0 and time.perf_counter() - t0 < 60:
            time.sleep(0.001)
        assert mx.mx_server_stats(s)["waiting_for_memory"] == 1, "the long batch ended before the second waited"
        t_a2 = long_req(s, 43, 1, 3000)  # same operator and settings as the running batch
        x, st, _, rc = mx.mx_server_poll(s, t_b, nd10, 1)
        assert rc == mx.MX_OK and st[0]["converged"]
        assert_close(x, x_b, 1e-9, what="request that waited for memory against alone")
        _, st_long, _, _ = mx.mx_server_poll(s, t_long, nd30, 2)
        _, st_a2, _, _ = mx.mx_server_poll(s, t_a2, nd30, 1)
        assert all(v["iterations"] == 3000 for v in st_long + st_a2), (st_long, st_a2)
        info = mx.mx_server_stats(s)
        assert info["joined"] == 0 and info["factorisations"] == 3 and info["evictions"] == 2, info
        assert info["waiting_for_memory"] == 0 and info["completed"] == 3 and info["batches"] == 3, info
    finally:
        mx.mx_server_destroy(s)
