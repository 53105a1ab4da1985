"""Write the converged oracle solutions that the reduced-precision convergence tests compare with.

Every stored number comes from the FP64 CPU oracle (``oracle/``) run to Err < 1e-10 (Eq. 15,
checked every 100 iterations); the inputs come from the seeded generators in
``paper_1712_01132_gb300/inputs.py``.  Nothing here touches the CUDA library.

    python tests/golden/make_convergence_golden.py [case ...]

For each case: ``convergence_<case>.npz`` with the fields (rho minus its fluid mean, u; float32,
enough for the 1e-3 max-norm bound of the tests) and ``convergence_<case>.json`` with k, G_p, the
iteration count and Err, and the k of the first checks (iterations 100, 200, ...) for reference.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1712_01132_gb300 import inputs  # noqa: E402

TOL = 1e-10


def cases():
    """name -> (mask, Kn, velocities per axis, description)."""
    d192 = inputs.random_discs(192, 192, seed=5)
    c3a = inputs.disc_batch(1, seed0=1000, nmin=96, nmax=160)[0]
    c3b = inputs.disc_batch(1, seed0=1004, nmin=96, nmax=160)[0]
    rock = inputs.gaussian_rock(24, seed=3, corr_len=3.0, porosity=0.35)
    return {
        "discs192_kn0.01": (d192, 0.01, 32, "random_discs(192, 192, seed=5), 32^2 velocities, Kn 0.01"),
        "discs192_kn10": (d192, 10.0, 32, "random_discs(192, 192, seed=5), 32^2 velocities, Kn 10"),
        "c3_seed1000": (c3a[0], c3a[1], 24, "disc_batch(1, seed0=1000, nmin=96, nmax=160), 24^2 velocities"),
        "c3_seed1004": (c3b[0], c3b[1], 24, "disc_batch(1, seed0=1004, nmin=96, nmax=160), 24^2 velocities"),
        "rock24_kn0.5": (rock, 0.5, 16, "gaussian_rock(24, seed=3, corr_len=3, porosity=0.35), 16^3 velocities, Kn 0.5"),
    }


def write(name, mask, kn, n_axis, desc, max_iter=60000, max_seconds=5400.0):
    v, w = oracle.velocity_grid(mask.ndim, n_axis)
    o = oracle.Oracle(mask, kn, v, w, lateral="periodic")
    t0 = time.perf_counter()
    while True:   # Eq. 15 checks every 100 iterations, reported every 1000
        it, k, err = o.run(TOL, min(max_iter, o.iterations + 1000))
        dt = time.perf_counter() - t0
        print("  %s: %d iterations, Err %.3e, k %.12e, %.0f s" % (name, it, err, k, dt), flush=True)
        if err < TOL or it >= max_iter or dt > max_seconds:
            break
    rho, u = o.moments()
    fl = ~mask
    rho = (rho - rho[fl].mean()) * fl
    np.savez_compressed(os.path.join(HERE, "convergence_%s.npz" % name), rho=rho.astype(np.float32),
                        u=u.astype(np.float32))
    hist = o.k_history
    meta = {"case": name, "description": desc, "kn": kn, "velocities_per_axis": n_axis,
            "lateral": "periodic", "shape": list(mask.shape), "fluid_points": int(fl.sum()),
            "oracle_tol": TOL, "iterations": it, "err": err, "k": k,
            "gp": float(u[0].sum() / u[0].size), "oracle_seconds": round(dt, 1),
            "k_at_checks": [hist[i - 1] for i in range(100, len(hist) + 1, 100)][:200]}
    with open(os.path.join(HERE, "convergence_%s.json" % name), "w") as f:
        json.dump(meta, f, indent=1)
    print(name, "iterations", it, "k", k, "err", err, "%.0f s" % dt, flush=True)


def main():
    cs = cases()
    for name in sys.argv[1:] or list(cs):
        mask, kn, n_axis, desc = cs[name]
        write(name, mask, kn, n_axis, desc)


if __name__ == "__main__":
    main()
