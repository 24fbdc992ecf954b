"""Writes equilibrated liquid snapshots for the parity tests, using only the
FP64 oracle and the seeded input generators.

Each workload starts on its seeded lattice (random orientations), is relaxed by
oracle NVT leapfrog steps with isokinetic scaling (short time step first, then
the workload's own), and the final (R, q, v, L) is stored as <name>.npz next to
this script.  Run:  python tests/golden/make_snapshots.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import Oracle  # noqa: E402
from paper_1507_07548_gb300 import workloads as W  # noqa: E402

# name -> (workload factory, [(dt, steps, kmax override or None), ...])
RECIPES = {
    "water_N1000": (lambda: W.water_box(N=1000, rc=14.0, seed=2), [(0.5, 200, None), (2.0, 600, None)]),
    "water_N216": (lambda: W.water_box(N=216, rc=9.0, seed=9), [(0.5, 200, None), (2.0, 600, None)]),
    # ragged tiles: N = 1003 is no multiple of any tile or block size
    "water_N1003": (lambda: W.water_box(N=1003, rc=13.0, seed=5), [(0.5, 200, None), (2.0, 400, None)]),
    "ionic_N1040": (lambda: W.ionic_solution(seed=3), [(0.5, 150, (4, 4, 4)), (2.0, 350, (4, 4, 4))]),
    "stockmayer_N500": (lambda: W.stockmayer_fluid(N=500, seed=4), [(1.0, 200, None), (2.0, 400, None)]),
    # two models (species numbering): 800 water + 200 argon-like atoms
    "water_argon_N1000": (lambda: W.water_argon(n_water=800, n_argon=200, rc=14.0, seed=6),
                          [(0.5, 200, None), (2.0, 400, None)]),
}


def make(name):
    factory, stages = RECIPES[name]
    wl = factory()
    R, q, v, L = wl.R, wl.q, wl.v, wl.Lang
    t0 = time.time()
    for dt, n, kmax in stages:
        kw = {} if kmax is None else dict(kmax=kmax)
        o = Oracle.from_workload(wl, **kw)
        R, q, v, L, th, _ = o.run_leapfrog(R, q, v, L, dt, n, T0=wl.T)
        print("%s: dt=%g %d steps, U=%.1f K, T=%.1f K" % (name, dt, n, th[-1, 0],
                                                         2 * (th[-1, 2] + th[-1, 3]) / o.ndof()))
    np.savez_compressed(os.path.join(HERE, name + ".npz"), R=R, q=q, v=v, Lang=L)
    print("%s written in %.0f s" % (name, time.time() - t0))


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(RECIPES)):
        make(n)
