"""The request server: continuous batching keeps every result identical to the
same request run alone, admits against the memory budget, cancels, and
reports failures per request without disturbing the others."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


def _alone(P, r):
    lat = P.Lattice(r["L"], r["T"], seed=r["seed"], init="hot")
    M, E = lat.sweep(r["nsweeps"], r["record_every"], collect=True)
    d = lat.measure()
    s = lat.spins()
    lat.close()
    return M, E, d, s


def test_results_equal_alone_under_rotation_and_small_budget(P):
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(40):
        L = int(rng.choice([64, 128, 256, 512, 1024]))
        reqs.append(dict(L=L, T=float(rng.uniform(1.5, 3.5)),
                         nsweeps=int(round(10 ** rng.uniform(1.0, 2.5))),
                         seed=int(rng.integers(0, 2 ** 63)), record_every=int(rng.choice([1, 3, 7]))))
    # a budget that holds only a few lattices, few lattices per launch, short epochs
    with P.Server(hbm_budget_bytes=600_000, epoch_sweeps=17, max_active=5, keep_samples=True) as srv:
        ids = [srv.submit(r["L"], r["T"], r["nsweeps"], seed=r["seed"], record_every=r["record_every"],
                          tag=i) for i, r in enumerate(reqs)]
        got = {}
        while len(got) < len(reqs):
            for res in srv.poll(wait_s=1.0):
                got[res["tag"]] = res
        st = srv.stats()
        assert st["completed"] == len(reqs) and st["peak_mem"] <= 600_000
        for i, r in enumerate(reqs):
            res = got[i]
            assert res["status"] == P.OK and res["id"] == ids[i]
            assert res["t_submit"] <= res["t_admit"] <= res["t_first_run"] <= res["t_finish"]
            M, E = srv.samples(ids[i])
            Ma, Ea, da, _ = _alone(P, r)
            assert np.array_equal(M, Ma) and np.array_equal(E, Ea), i
            assert res["obs"] == da, i
        # the budget forced admission waits and the launch cap forced several launches
        assert st["epochs"] > len(reqs) // 5


def test_budget_cancel_and_failure_isolation(P):
    with P.Server(hbm_budget_bytes=200_000, epoch_sweeps=10) as srv:
        big = srv.submit(2048, 2.0, 10, seed=1)            # 512 KiB > budget
        keep = srv.submit(256, 2.0, 30, seed=2, record_every=1)
        victim = srv.submit(512, 2.0, 100000, seed=3)
        srv.cancel(victim)
        res = {}
        while len(res) < 3:
            for r in srv.poll(wait_s=1.0):
                res[r["id"]] = r
        assert res[big]["status"] == P.ERR_OOM
        assert res[victim]["status"] == P.ERR_CANCELLED
        assert res[keep]["status"] == P.OK
        a = P.Lattice(256, 2.0, seed=2, init="hot")
        a.sweep(30, 1)
        assert res[keep]["obs"] == a.measure()
        st = srv.stats()
        assert st["failed"] == 1 and st["cancelled"] == 1 and st["completed"] == 1


def test_poisson_stream_smoke(P):
    from paper_1007_3726_gb300 import serve

    reqs = serve.poisson_requests(rate=40, duration=1.0, Ls=(64, 128, 256, 512),
                                  log10_sweeps=(1.0, 2.5))
    with P.Server(epoch_sweeps=50) as srv:
        out = serve.run_stream(srv, reqs, drain_s=30.0)
    assert out["completed"] == len(reqs) and out["failed"] == 0
    assert out["p50_s"] <= out["p99_s"]


def test_served_requests_equal_the_oracle(P, orc):
    """Six requests of mixed L and T, served together (small epochs, at most three
    resident, so that they share launches and start at different epochs): every
    sample and the moments against the oracle run of the same request."""
    rng = np.random.default_rng(29)
    reqs = []
    for i, L in enumerate((64, 128, 256, 512, 128, 320)):
        reqs.append(dict(L=L, T=float(rng.uniform(1.5, 3.5)), nsweeps=int(rng.integers(40, 120)),
                         seed=int(rng.integers(0, 2 ** 63)), stream_id=int(rng.integers(0, 2 ** 31)),
                         record_every=int(rng.choice([1, 4, 5]))))
    with P.Server(epoch_sweeps=13, max_active=3, keep_samples=True) as srv:
        ids = [srv.submit(r["L"], r["T"], r["nsweeps"], seed=r["seed"], stream_id=r["stream_id"],
                          record_every=r["record_every"], tag=i) for i, r in enumerate(reqs)]
        got = {}
        while len(got) < len(reqs):
            for res in srv.poll(wait_s=1.0):
                got[res["tag"]] = res
        for i, r in enumerate(reqs):
            res = got[i]
            assert res["status"] == P.OK
            M, E = srv.samples(ids[i])
            thr4, thr8 = orc.thresholds(r["T"])
            s = orc.init_hot(r["L"], r["seed"], r["stream_id"])
            Mo, Eo = orc.run(s, r["nsweeps"], r["seed"], r["stream_id"], thr4, thr8)
            k = r["record_every"]
            assert np.array_equal(M, Mo[k - 1::k]) and np.array_equal(E, Eo[k - 1::k]), i
            obs = res["obs"]
            assert (obs["M"], obs["E"]) == (Mo[-1], Eo[-1]), i
            ref = orc.moments(Mo[k - 1::k], Eo[k - 1::k], N=r["L"] ** 2, T=r["T"])
            for key in ("mean_abs_m", "mean_m2", "mean_m4", "U4", "chi"):
                assert abs(obs[key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key])), (i, key)
