"""Continuous-batching server: requests that arrive while others run are admitted
as slots and memory free up, and each result is the same bit for bit as the
same request solved on its own."""
import numpy as np
import pytest

import rsw_inputs as ri
from _helpers import cuda_or_skip

pytestmark = pytest.mark.gpu


def _requests(serve):
    specs = [(64, 1e-2, 8, 0.5, 1e-3, 16), (32, 2e-2, 4, 0.2, 2e-3, 8), (128, 5e-3, 6, 0.3, 5e-4, 16),
             (64, 1e-2, 5, 0.25, 1e-3, 32), (32, 1e-2, 8, 0.4, 1e-3, 8), (128, 1e-2, 4, 0.2, 1e-3, 16),
             (64, 3e-3, 4, 0.1, 3e-4, 16), (16, 2e-2, 3, 0.15, 2e-3, 8)]
    reqs = []
    for i, (n, eps, S, T, dt, M) in enumerate(specs):
        u0 = ri.random_spectrum(n, min(8, (n - 1) // 3), 16.0, 700 + i) * 4.0
        reqs.append(serve.Request(n, eps, 1e-4, S, T, dt, M, u0, k_max=3 + i % 3, tol=1e-12 if i % 2 else 0.0))
    return reqs


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_served_results_equal_solo_results(precision):
    cuda_or_skip()
    from paper_1303_6615_gb300 import binding as b
    from paper_1303_6615_gb300 import serve
    reqs = _requests(serve)
    biggest = max(b.arp_query_bytes(r.n_grid, r.slices, r.m_quad, precision) for r in reqs)
    # at most 3 requests in flight, and memory for about 2.5 of the largest; every
    # step one batched level (a lone request's one-call solve has its own test)
    server = serve.Server(memory_budget=int(2.5 * biggest), max_active=3, precision=precision, lone_solve=False)
    try:
        trace = [(0.002 * i, r) for i, r in enumerate(reqs)]
        done = serve.replay(server, trace)
    finally:
        server.close()
    assert sorted(r.rid for r in done) == list(range(len(reqs)))
    # continuous batching: some request was admitted while an earlier one was still running
    overlap = any(a.admitted > c.admitted and a.admitted < c.finished for a in done for c in done if a is not c)
    assert overlap
    for r in done:
        assert r.latency >= 0 and r.levels <= r.k_max
        alone = serve.solve_alone(r, precision)
        np.testing.assert_array_equal(r.result, alone)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_lone_request_solve_equals_batched_levels(precision):
    # requests spaced out so that each runs alone for part of its life: finishing a
    # lone request in one arp_parareal_solve (pipelined where it applies) gives the
    # slices, level and change of the batched levels
    cuda_or_skip()
    from paper_1303_6615_gb300 import serve
    got = {}
    for lone in (True, False):
        reqs = _requests(serve)[:4]
        server = serve.Server(memory_budget=1 << 30, max_active=4, precision=precision, lone_solve=lone)
        try:
            done = serve.replay(server, [(0.03 * i, r) for i, r in enumerate(reqs)])
        finally:
            server.close()
        got[lone] = {r.rid: r for r in done}
    assert sorted(got[True]) == sorted(got[False]) == list(range(4))
    for rid, r in got[True].items():
        q = got[False][rid]
        assert (r.levels, r.change) == (q.levels, q.change)
        np.testing.assert_array_equal(r.result, q.result)
        np.testing.assert_array_equal(r.result, serve.solve_alone(r, precision))
    # one request alone from the start: served by the one-call solve
    r = _requests(serve)[2]
    server = serve.Server(memory_budget=1 << 30, max_active=4, precision=precision)
    try:
        server.submit(r)
        server.step()
        assert not server.active and server.done == [r]
        assert r.levels == r.k_max or r.change <= r.tol
    finally:
        server.close()
    np.testing.assert_array_equal(r.result, serve.solve_alone(r, precision))
