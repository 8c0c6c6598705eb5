"""Write the FP64 oracle's 100-step trajectories used by the precision report
(tests/precision_report.py): the state of a seeded sample of particles after
100 steps of the Sod tube (1,072,476 particles) and of the Sedov blast.

Every value is computed by `oracle/` alone, from the seeded inputs of
`sph_inputs`.  A step is the oracle's composition: density with 5 Newton
steps on h, EOS, force, kick/drift (symplectic Euler, dt fixed); the next
step starts from the new x, v, u and the converged h.  The Sedov blast runs
on the 128 x 128 x 64 lattice (1,048,576 particles): the FP64 oracle takes
about 20 s per million-particle step on 8 host cores, and 100 steps of the
8,388,608-particle lattice would take hours; its 1-step errors are measured
at full size on sampled targets instead.

Run from the repository root:
    OMP_NUM_THREADS=8 python tests/golden/make_trajectories.py [sod|sedov ...]
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import sph_inputs  # noqa: E402

STEPS = 100
N_SAMPLE = 1024
OUT = os.path.dirname(os.path.abspath(__file__))


def workload(name):
    if name == "sod":
        return sph_inputs.sod()
    if name == "sedov":
        return sph_inputs.sedov(128, 128, 64)
    raise ValueError(name)


def sample(wl, seed):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(wl.n, N_SAMPLE, replace=False).tolist())
    if wl.name == "sedov":
        idx.update(int(i) for i in wl.meta["hot"])       # the blast itself
    return np.array(sorted(idx), dtype=np.int64)


def run(name):
    wl = workload(name)
    tgt = sample(wl, 7 if name == "sod" else 8)
    t0 = time.time()
    for k in range(STEPS):
        o = oracle.step(wl)
        wl.col("x")[:] = o["x_new"]
        wl.col("v")[:] = o["v_new"]
        wl.col("u")[:] = o["u_new"]
        wl.col("h")[:] = o["h"]
        wl.col("rho")[:] = o["rho"]
        wl.col("P")[:] = o["P"]
        wl.col("a")[:] = o["a"]
        if k % 10 == 9:
            print(f"{name}: step {k + 1}/{STEPS}  {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(OUT, f"trajectory_{name}.npz")
    np.savez_compressed(
        path, name=name, n=wl.n, steps=STEPS, dt=wl.dt, targets=tgt,
        x=wl.col("x")[tgt], v=wl.col("v")[tgt], u=wl.col("u")[tgt], h=wl.col("h")[tgt],
        rho=wl.col("rho")[tgt], P=wl.col("P")[tgt], a=wl.col("a")[tgt],
        flags=o["flags"][tgt])
    print("wrote", path, flush=True)


if __name__ == "__main__":
    for nm in (sys.argv[1:] or ["sod", "sedov"]):
        run(nm)
