"""Command-line runner: one lattice through the C ABI, observables as JSON.

    python -m paper_1007_3726_gb300 --L 32768 --T 2.269185 --seed 7 --init hot \
        --sweeps 1000 --record-every 1 [--word-bits 32] [--H 0.1] [--time]
    python -m paper_1007_3726_gb300 fss-batch --sweeps 10000   (128 lattices, one launch)
"""
import argparse
import json
import sys
import time


def fss_batch(argv):
    """The 128-lattice finite-size-scaling batch in one persistent launch."""
    ap = argparse.ArgumentParser(prog="python -m paper_1007_3726_gb300 fss-batch")
    ap.add_argument("--sweeps", type=int, default=10000)
    ap.add_argument("--record-every", type=int, default=10)
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--ctas-per-sm", type=int, default=4)
    ap.add_argument("--rows-per-item", type=int, default=4)
    a = ap.parse_args(argv)

    import paper_1007_3726_gb300 as P
    from paper_1007_3726_gb300 import workloads as WL

    P.load()
    specs = WL.fss_batch(sweeps=a.sweeps, record_every=a.record_every)
    lats = [P.Lattice(**WL.lattice_kwargs(sp)) for sp in specs]
    t0 = time.perf_counter()
    with P.Batch(lats, [a.sweeps] * len(lats), a.record_every, block=a.block, ctas_per_sm=a.ctas_per_sm,
                 rows_per_item=a.rows_per_item) as b:
        info = b.info()
        b.run(1)
    el = time.perf_counter() - t0
    N = sum(sp["L"] ** 2 for sp in specs)
    print(json.dumps({"lattices": len(lats), "sweeps": a.sweeps, "plan": info, "seconds": el,
                      "attempts_per_ns": N * a.sweeps / el / 1e9}))
    return 0


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if argv and argv[0] == "fss-batch":
        return fss_batch(argv[1:])
    ap = argparse.ArgumentParser(prog="python -m paper_1007_3726_gb300")
    ap.add_argument("--L", type=int, default=1024)
    ap.add_argument("--T", type=float, default=2.269185)
    ap.add_argument("--H", type=float, default=0.0, help="external field (Eq. 1)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--stream-id", type=int, default=0)
    ap.add_argument("--init", default="hot", choices=["hot", "cold_up", "cold_down"])
    ap.add_argument("--sweeps", type=int, default=100)
    ap.add_argument("--record-every", type=int, default=1)
    ap.add_argument("--word-bits", type=int, default=0)
    ap.add_argument("--time", action="store_true", help="report wall time of the sweeps")
    ap.add_argument("--autotune", action="store_true", help="pick the launch configuration first")
    ap.add_argument("--launch", default=None,
                    help="launch configuration proc_bits,regcap,block,rows_per_item[,grid[,insert[,persistent]]]")
    a = ap.parse_args(argv)

    import paper_1007_3726_gb300 as P

    P.load()
    lat = P.Lattice(a.L, a.T, seed=a.seed, stream_id=a.stream_id, init=a.init, word_bits=a.word_bits,
                    H=a.H)
    if a.autotune:
        cfg, _ = lat.autotune()
    if a.launch:
        v = [int(x) for x in a.launch.split(",")]
        keys = ["proc_bits", "regcap", "block", "rows_per_item", "grid", "insert", "persistent"]
        lat.set_launch(**dict(zip(keys, v)))
    t0 = time.perf_counter()
    lat.sweep(a.sweeps, a.record_every)
    d = lat.measure()
    el = time.perf_counter() - t0
    d["L"], d["T"], d["H"], d["word_bits"] = a.L, a.T, a.H, lat.word_bits
    d["launch"] = lat.launch
    if a.time:
        d["seconds"] = el
        d["attempts_per_ns"] = a.L * a.L * a.sweeps / el / 1e9
    lat.close()
    print(json.dumps(d))
    return 0


if __name__ == "__main__":
    sys.exit(main())
