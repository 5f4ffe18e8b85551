"""Serving loop: each result is the same alone and in a mix of concurrent
requests (continuous batching, two workers, shared operator cache); a request
refused by HBM admission fails alone without disturbing its neighbours."""
import numpy as np
import pytest

from workloads import icosphere, cube

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")


def _requests():
    sv, st = icosphere(1, 0.2)
    cv, ct = cube(0.3, 3)
    L1 = np.diag([0.6, 0.6, 1.0])
    L2 = np.diag([0.5, 0.5, 0.5])
    reqs = []
    rng = np.random.default_rng(9)
    for i in range(10):
        if i % 3 == 2:
            mesh, counts, L, k = (cv, ct), (3, 2, 1), L2, [3.0, 5.0][i % 2]
        else:
            mesh, counts, L, k = (sv, st), (4, 3, 1), L1, [2.0, 4.0][i % 2]
        R = 1 + i % 3
        d = rng.normal(size=(R, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        reqs.append((mesh, counts, L, k, d))
    return reqs


def test_results_are_the_same_alone_and_in_the_mix():
    reqs = _requests()
    alone = []
    with gb.Server(max_batch_rhs=16, tol=1e-10, restart=60) as srv:
        for mesh, counts, L, k, d in reqs:
            tk = srv.submit(mesh[0], mesh[1], counts, L, k, d)
            res, p = srv.wait(tk)
            assert res["status_name"] == "FMPB_OK", res
            alone.append(p.copy())
    with gb.Server(max_batch_rhs=16, tol=1e-10, restart=60) as srv:
        tickets = [srv.submit(m[0], m[1], c, L, k, d) for m, c, L, k, d in reqs]
        mixed = []
        batched = []
        for tk in tickets:
            res, p = srv.wait(tk)
            assert res["status_name"] == "FMPB_OK", res
            assert res["relres_true_max"] < 1e-9
            mixed.append(p.copy())
            batched.append(res["batched_with"])
        st = srv.stats()
    assert max(batched) > 1                       # some requests really shared a solve
    for a, b in zip(alone, mixed):
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] and st["cache_hits"] >= 1


def test_admission_refusal_is_isolated():
    sv, st = icosphere(1, 0.2)
    big_counts = (12, 12, 1)     # PBEM spectrum 23 x 23 x 80^2 x 16 B = 54 MB, above the budget
    with gb.Server(hbm_budget_bytes=40 << 20, max_batch_rhs=4, tol=1e-10, restart=40) as srv:
        small = srv.submit(sv, st, (3, 1, 1), np.eye(3) * 0.6, 2.0, [[1.0, 0, 0]], form=gb.FORM_PBEM)
        big = srv.submit(sv, st, big_counts, np.eye(3) * 0.5, 2.0, [[1.0, 0, 0]], form=gb.FORM_PBEM)
        small2 = srv.submit(sv, st, (3, 1, 1), np.eye(3) * 0.6, 3.0, [[0.0, 1.0, 0]], form=gb.FORM_PBEM)
        r1, _ = srv.wait(small)
        rb, _ = srv.wait(big)
        r2, p2 = srv.wait(small2)
    assert r1["status_name"] == "FMPB_OK" and r2["status_name"] == "FMPB_OK"
    assert rb["status_name"] == "FMPB_ENOMEM"
    assert np.isfinite(p2).all() and np.abs(p2).max() > 0
