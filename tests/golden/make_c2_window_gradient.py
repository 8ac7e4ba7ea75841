"""Writes c2_window_gradient.txt: the FP64 oracle's objective and tangent-linear gradient of
the 96^3 periodic array of 27 fixed spheres (r = 4, body force 1e-5 along +x, tau 0.6) over a
window of 500 steps from rest: J = sum over the steps of x . (sum over spheres of the
momentum-exchange force) (Eqs. netforce, momentum_transfer), dJ/dtau and dJ/dg (x, y, z).
Calls only the oracle (and the seeded workload placement); each direction runs in a process
of its own.  Takes about 7 minutes on 4 cores."""
import os
import sys
from concurrent.futures import ProcessPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

STEPS = 500
DIRS = {"tau": (1.0, (0.0, 0.0, 0.0)), "gx": (0.0, (1.0, 0.0, 0.0)), "gy": (0.0, (0.0, 1.0, 0.0)),
        "gz": (0.0, (0.0, 0.0, 1.0))}


def _one(name):
    import oracle
    from paper_1712_07028_gb300 import workloads as W
    oracle.build()
    o = oracle.Sim(W.periodic_array_c2())
    dtau, dg = DIRS[name]
    J, dJ = o.tangent_window(STEPS, dtau=dtau, dg=dg, jdir=(1.0, 0.0, 0.0))
    return name, J, dJ


def main():
    import multiprocessing as mp
    with ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as ex:
        res = {n: (J, dJ) for n, J, dJ in ex.map(_one, list(DIRS))}
    Js = {round(v[0], 12) for v in res.values()}
    assert len(Js) == 1, Js   # the same forward window in every process
    J = res["tau"][0]
    with open(os.path.join(HERE, "c2_window_gradient.txt"), "w") as f:
        f.write("# FP64 oracle, tangent-linear window: 96^3 periodic, 27 fixed spheres r=4 (seed 2), tau 0.6,\n"
                "# g = (1e-5, 0, 0), from rest, %d steps; J = sum_t x . sum_P F_P(t).\n"
                "# written by tests/golden/make_c2_window_gradient.py (oracle only)\n" % STEPS)
        f.write("J %.17g\n" % J)
        for n in ("tau", "gx", "gy", "gz"):
            f.write("dJ_d%s %.17g\n" % (n, res[n][1]))


if __name__ == "__main__":
    main()
