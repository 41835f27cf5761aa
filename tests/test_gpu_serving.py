"""Serving loop (mx_server_*): results are the same alone and in a mix of requests with
other operators and batched right-hand sides; factorisations are cached and reused across
xi_prob; a small memory budget forces evictions; per-request latency is reported."""
import numpy as np
import pytest

import inputs

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
        err = np.linalg.norm(x_mix - x_alone) / np.linalg.norm(x_alone)
        assert err <= 1e-7, err
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
