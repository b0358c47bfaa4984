"""Physics pin of the finite-size-scaling batch (Sec. 3, Eq. 2): the Binder
cumulants of L = 256 and L = 512 cross between T = 2.25 and T = 2.29, around
Onsager's T_c = 2/ln(1 + sqrt 2) = 2.269185.

Below T_c the larger lattice is closer to the ordered value 2/3, above T_c
closer to the disordered value 0, so U4(512) - U4(256) changes sign in
between.  The 10^4 sweeps of the 128-lattice batch are far shorter than the
Metropolis relaxation time at these sizes (about L^2.17 sweeps at T_c), so this
pin uses longer runs and replicas (independent Philox streams) of the same two
sizes, at the two temperatures only, all in persistent batch launches:

  T = 2.25: cold start (no coarsening from a random start), 64 replicas per L,
            2 x 10^5 sweeps;
  T = 2.29: hot start, 256 replicas per L, 2.5 x 10^5 sweeps;

a sample every 100 sweeps, the first 20 % dropped.  The moments of each
lattice come from ising_measure_from (FP64 sums in sample order); the replicas'
<m^2> and <m^4> are averaged (equal sample counts) before U4 is formed.  The
margin of each sign is required to exceed four standard errors estimated from
the spread of the replicas.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_1007_3726_gb300 as P

    P.build()
    P.load()
    return P


def _replicas(P, L, T, init, replicas, stream0):
    return [P.Lattice(L, T, seed=3, stream_id=stream0 + r, init=init) for r in range(replicas)]


def _pooled(lats, burn):
    m2 = np.array([lat.measure(first_sample=burn)["mean_m2"] for lat in lats])
    m4 = np.array([lat.measure(first_sample=burn)["mean_m4"] for lat in lats])
    u4 = 1.0 - m4.mean() / (3.0 * m2.mean() ** 2)
    # jackknife over replicas
    n = len(lats)
    jk = np.array([1.0 - (m4.sum() - m4[i]) / (n - 1) / (3.0 * ((m2.sum() - m2[i]) / (n - 1)) ** 2)
                   for i in range(n)])
    err = np.sqrt((n - 1) / n * np.sum((jk - jk.mean()) ** 2))
    return u4, err


@pytest.mark.parametrize("T,init,replicas,sweeps,sign", [(2.25, "cold_up", 64, 200000, +1),
                                                         (2.29, "hot", 256, 250000, -1)])
def test_binder_cumulants_of_L256_and_L512_cross_near_tc(P, T, init, replicas, sweeps, sign):
    rec = 100
    burn = sweeps // rec // 5
    runs = {}
    all_lats = []
    for i, L in enumerate((256, 512)):
        runs[L] = (_replicas(P, L, T, init, replicas, stream0=100000 * (i + 1)), burn)
        all_lats += runs[L][0]
    with P.Batch(all_lats, [sweeps] * len(all_lats), rec) as b:
        b.run(1)
    (u256, e256), (u512, e512) = (_pooled(*runs[256]), _pooled(*runs[512]))
    diff = u512 - u256
    err = float(np.hypot(e256, e512))
    msg = "T=%.2f: U4(256)=%.5f+-%.5f U4(512)=%.5f+-%.5f" % (T, u256, e256, u512, e512)
    print(msg)
    assert sign * diff > 4.0 * err, msg
    for lat in all_lats:
        lat.close()
