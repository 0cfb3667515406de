"""The request server (continuous batching of solves on one GPU): results
are the same alone and in a concurrent mix, admission follows the HBM
budget, warm starts reuse resident eigenvectors, and failures (bad or
over-budget requests, NaN input, time-outs, cancellation) are reported as
statuses.  Faults are made on the host side only."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2006_08498_gb300 as pkg  # noqa: E402


@pytest.fixture
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_08498_gb300 import build
    build.build()
    c = pkg.Context(0)
    yield c
    c.close()


GB = 1 << 30


def test_alone_equals_mix(ctx):
    ctx.server_create(64 * GB, 4)
    R = dict(seed=7, Nk=63, Nv=4, Nc=4, nev=20, nex=10)          # N = 1008
    alone = ctx.wait(ctx.submit(**R))
    assert alone["status"] == pkg.BSE_OK
    mix = [dict(seed=11 + i, Nk=63 + 40 * i, Nv=4, Nc=4, nev=10 + 7 * i, nex=10)
           for i in range(5)]
    tickets = [ctx.submit(**r) for r in mix[:3]] + [ctx.submit(**R)] + \
        [ctx.submit(**r) for r in mix[3:]]
    res = [ctx.wait(t) for t in tickets]
    assert all(r["status"] == pkg.BSE_OK for r in res)
    again = res[3]
    assert np.array_equal(again["evals"], alone["evals"])
    assert np.array_equal(again["resid"], alone["resid"])
    assert again["stats"]["iters"] == alone["stats"]["iters"]
    # the requests' device work overlapped in time
    iv = sorted((r["t_start"], r["t_end"]) for r in res)
    assert any(iv[i + 1][0] < iv[i][1] for i in range(len(iv) - 1))
    ctx.server_destroy()


def test_batched_products_share_launches_and_change_nothing(ctx):
    """Product batching: with a window of 5 ms, the products of concurrent
    solves run several to a launch (launch statistics), and every request's
    result is bit for bit the one of the same server with batching off."""
    reqs = [dict(seed=21 + i, Nk=63 + 17 * i, Nv=4, Nc=4, nev=12 + 5 * i, nex=10)
            for i in range(6)]
    ctx.server_create(64 * GB, 6)
    assert ctx.server_batch_stats()["launches"] == 0              # off by default
    ctx.server_batching(True, 5e-3)
    res_b = [ctx.wait(t) for t in [ctx.submit(**r) for r in reqs]]
    st = ctx.server_batch_stats()
    ctx.server_batching(False)
    res_u = [ctx.wait(t) for t in [ctx.submit(**r) for r in reqs]]
    assert ctx.server_batch_stats()["launches"] == 0
    ctx.server_destroy()
    assert all(r["status"] == pkg.BSE_OK for r in res_b + res_u)
    assert st["max_products"] >= 2 and st["products"] > st["launches"]
    for a, b in zip(res_b, res_u):
        assert np.array_equal(a["evals"], b["evals"])
        assert np.array_equal(a["resid"], b["resid"])
        assert a["stats"]["iters"] == b["stats"]["iters"]


def test_server_result_equals_direct_solve(ctx):
    Hd = ctx.build_hamiltonian(3, 63, 4, 4)
    e, V, r, st = ctx.solve(Hd, 20, 10, seed=3)
    ctx.server_create(16 * GB, 2)
    t = ctx.submit(seed=3, Nk=63, Nv=4, Nc=4, nev=20, nex=10)
    res = ctx.wait(t)
    assert np.array_equal(res["evals"], e)
    V2 = ctx.fetch_evecs(t, Hd.shape[0], 20)
    assert torch.equal(V2, V)
    ctx.server_destroy()


def test_server_storage_options_equal_direct_solves(ctx):
    """Requests without the stored H (h_free) and on half storage: bit for
    bit the direct solves of the same kind (chase_solve_bse, chase_opts.
    half_storage); a smaller budget estimate admits the H-free request where
    the stored one is refused; invalid combinations are rejected."""
    Hd = ctx.build_hamiltonian(3, 63, 4, 4)
    eh, Vh, _, _ = ctx.solve(Hd, 20, 10, seed=3, half_storage=True)
    ef, Vf, _, _ = ctx.solve_bse(3, 63, 4, 4, 20, 10, seed_start=3)
    eb, Vb, _, _ = ctx.solve_bse(3, 63, 4, 4, 20, 10, seed_start=3, half_storage=True)
    N = Hd.shape[0]
    del Hd
    ctx.server_create(16 * GB, 3)
    tickets = [ctx.submit(seed=3, Nk=63, Nv=4, Nc=4, nev=20, nex=10, half_storage=True),
               ctx.submit(seed=3, Nk=63, Nv=4, Nc=4, nev=20, nex=10, h_free=True),
               ctx.submit(seed=3, Nk=63, Nv=4, Nc=4, nev=20, nex=10, h_free=True,
                          half_storage=True)]
    for t, (e, V) in zip(tickets, ((eh, Vh), (ef, Vf), (eb, Vb))):
        res = ctx.wait(t)
        assert res["status"] == pkg.BSE_OK
        assert np.array_equal(res["evals"], e)
        assert torch.equal(ctx.fetch_evecs(t, N, 20), V)
    for bad in (dict(h_free=True, precision=pkg.CHASE_FP64_DFMA),
                dict(half_storage=True, precision=pkg.CHASE_FP64_DFMA),
                dict(h_free=True, H=pkg.colmajor_empty(N, N).zero_())):
        with pytest.raises(pkg.BseError) as ei:
            ctx.submit(seed=3, Nk=63, Nv=4, Nc=4, nev=20, nex=10, **bad)
        assert ei.value.status == pkg.BSE_EINVAL
    ctx.server_destroy()
    # N = 8000: the stored H alone is 1 GB; a budget between the two estimates
    ctx.server_create(int(2.0 * GB), 1)
    with pytest.raises(pkg.BseError) as ei:
        ctx.submit(seed=1, Nk=500, Nv=4, Nc=4, nev=20, nex=10)
    assert ei.value.status == pkg.BSE_ENOMEM
    t = ctx.submit(seed=1, Nk=500, Nv=4, Nc=4, nev=20, nex=10, h_free=True, half_storage=True)
    assert ctx.wait(t)["status"] == pkg.BSE_OK
    ctx.server_destroy()


def test_admission_by_budget(ctx):
    # one N = 2000 request is estimated at ~0.19 GB (H 64 MB, slices of H
    # 100 MB, search space and workspace): a 0.3 GB budget admits one at a time
    budget = int(0.3 * GB)
    ctx.server_create(budget, 4)
    reqs = [ctx.submit(seed=s, Nk=125, Nv=4, Nc=4, nev=30, nex=15) for s in range(3)]
    seen_running = 0
    while any(ctx.poll(t) is None for t in reqs):
        info = ctx.server_info()
        seen_running = max(seen_running, info["running"])
        assert info["held_bytes"] <= budget
    assert seen_running <= 1
    res = [ctx.wait(t) for t in reqs]
    assert all(r["status"] == pkg.BSE_OK for r in res)
    # strictly sequential execution
    iv = sorted((r["t_start"], r["t_end"]) for r in res)
    assert all(iv[i + 1][0] >= iv[i][1] for i in range(len(iv) - 1))
    with pytest.raises(pkg.BseError) as ei:
        ctx.submit(seed=1, Nk=500, Nv=4, Nc=4, nev=30, nex=15)   # N = 8000: 1 GB for H alone
    assert ei.value.status == pkg.BSE_ENOMEM
    ctx.server_destroy()


def test_warm_start_from_resident_eigenvectors(ctx):
    ctx.server_create(32 * GB, 2)
    a = ctx.submit(seed=5, Nk=80, Nv=4, Nc=4, nev=30, nex=15)
    ra = ctx.wait(a)
    b = ctx.submit(seed=5, Nk=80, Nv=4, Nc=4, nev=30, nex=15, warm_ticket=a)
    rb = ctx.wait(b)
    assert rb["status"] == pkg.BSE_OK
    assert rb["stats"]["iters"] < ra["stats"]["iters"]
    assert np.allclose(rb["evals"], ra["evals"], rtol=1e-11, atol=0)
    # a neighbour: slightly different screening strength
    c = ctx.submit(seed=5, Nk=80, Nv=4, Nc=4, nev=30, nex=15, warm_ticket=a,
                   model=dict(w0=0.3 * 1.01))
    rc = ctx.wait(c)
    assert rc["status"] == pkg.BSE_OK and np.max(rc["resid"]) <= 1e-10
    ctx.server_destroy()


def test_timeout_cancel_and_bad_requests(ctx):
    ctx.server_create(int(0.45 * GB), 1)
    t1 = ctx.submit(seed=1, Nk=125, Nv=4, Nc=4, nev=40, nex=20)
    t2 = ctx.submit(seed=2, Nk=125, Nv=4, Nc=4, nev=40, nex=20)     # queued behind t1
    with pytest.raises(pkg.BseError) as ei:
        ctx.wait(t1, timeout_s=1e-4)
    assert ei.value.status == pkg.BSE_ETIMEOUT
    assert ctx.release(t2) == pkg.BSE_OK                              # cancel while queued
    r2 = ctx.wait(t2)
    assert r2["status"] == pkg.BSE_EINVAL and r2["evals"] is None
    assert ctx.wait(t1)["status"] == pkg.BSE_OK
    for bad in (dict(nev=0, nex=5), dict(nev=40, nex=600), dict(nev=10, nex=5, tol=-1.0),
                dict(nev=10, nex=5, precision=9), dict(nev=10, nex=5, degree_group=-2)):
        kw = dict(seed=1, Nk=16, Nv=4, Nc=4)
        kw.update(bad)
        with pytest.raises(pkg.BseError) as ei:
            ctx.submit(**kw)
        assert ei.value.status == pkg.BSE_EINVAL
    ctx.server_destroy()


def test_nan_request_is_reported(ctx):
    ctx.server_create(16 * GB, 2)
    t = ctx.submit(seed=1, Nk=40, Nv=4, Nc=4, nev=10, nex=5, model=dict(w0=math.nan))
    good = ctx.submit(seed=1, Nk=40, Nv=4, Nc=4, nev=10, nex=5)
    assert ctx.wait(t)["status"] == pkg.BSE_ENONFINITE
    assert ctx.wait(good)["status"] == pkg.BSE_OK                  # the server keeps serving
    ctx.server_destroy()


def test_concurrent_mixed_sizes_all_ok(ctx):
    """Sixteen requests of growing search-space size (m = nev + nex from 20
    to 150) in flight on eight slots at once: every one converges.  The
    clustered small kernels set their launch attributes once per process,
    for the largest size, so no solver thread launches against a limit that
    another thread is still raising."""
    ctx.server_create(64 * GB, 8)
    reqs = [dict(seed=100 + i, Nk=63 + 8 * (i % 5), Nv=4, Nc=4, nev=10 + 6 * i,
                 nex=max(10, math.ceil((10 + 6 * i) / 2))) for i in range(16)]
    tickets = [ctx.submit(**r) for r in reqs]
    res = [ctx.wait(t) for t in tickets]
    assert [r["status"] for r in res] == [pkg.BSE_OK] * len(reqs)
    for r, q in zip(res, reqs):
        assert r["nev"] == q["nev"]
        assert np.max(r["resid"]) <= 1e-10
    ctx.server_destroy()


def test_serving_sizes_match_exact_eigenvalues(ctx):
    """Requests of the serving mix's sizes (N = 1008 .. 4000, nev 10 .. 100,
    one warm neighbour with w0 scaled by 1.01) against the exact eigenvalues
    of the same synthetic Hamiltonians (structured oracle)."""
    import oracle
    reqs = [dict(seed=31, Nk=63, nev=10, nex=10), dict(seed=32, Nk=125, nev=50, nex=25),
            dict(seed=33, Nk=250, nev=100, nex=50), dict(seed=31, Nk=63, nev=10, nex=10,
                                                        model=dict(w0=0.303))]
    ctx.server_create(64 * GB, 4)
    t0 = ctx.submit(Nv=4, Nc=4, **reqs[0])
    ts = [t0] + [ctx.submit(Nv=4, Nc=4, **r) for r in reqs[1:3]]
    ts.append(ctx.submit(Nv=4, Nc=4, warm_ticket=t0, **reqs[3]))
    res = [ctx.wait(t) for t in ts]
    ctx.server_destroy()
    for r, q in zip(res, reqs):
        assert r["status"] == pkg.BSE_OK and np.max(r["resid"]) <= 1e-10
        lam = oracle.structured.lowest_eigenvalues(
            oracle.structured.bse_blocks(q["seed"], q["Nk"], 4, 4, q.get("model")), q["nev"])
        assert np.max(np.abs(r["evals"] - lam) / np.abs(lam)) <= 1e-10


def test_request_with_caller_hamiltonian(ctx):
    """A request may carry the caller's device matrix instead of the
    generator's parameters: a seeded Hermitian matrix with a known spectrum
    (N = 600 = 150 x 2 x 2), against its eigenvalues and the dense oracle."""
    import oracle
    from inputs import hermitian
    A, lam = hermitian(600, 41)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().T
    ctx.server_create(16 * GB, 2)
    t = ctx.submit(seed=0, Nk=150, Nv=2, Nc=2, nev=30, nex=15, H=Ad)
    r = ctx.wait(t)
    ctx.server_destroy()
    assert r["status"] == pkg.BSE_OK and r["N"] == 600
    w, _ = oracle.eigh(A, 0)
    assert np.max(np.abs(r["evals"] - w[:30]) / np.abs(w[:30])) <= 1e-10
    assert np.max(np.abs(r["evals"] - lam[:30]) / lam[:30]) <= 1e-10
