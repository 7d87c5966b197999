"""Writes the stored oracle results of the full-size GPU parity tests (tests/golden/oracle_*.npz).

Calls only the CPU oracle (``oracle/``) and the seeded input generator (``synthetic_inputs``); no
value comes from the GPU library.  The oracle's whole solves at these sizes take minutes (P4/P3 on
16 -> 64) to tens of minutes (P2/P1 on 32 -> 512), too long to repeat inside every GPU test run, so
they are computed once here and read back by the tests.

    python tests/golden/make_golden.py [case ...]      (default: every case)

Each file holds: the problem (N_coarse, nlevels, k, seed, rtol), the oracle's Chebyshev eigenvalue
estimates per level, the FGMRES iteration count and residual history (modified Gram-Schmidt; for
cases with ``cgs2`` also the history of the oracle's classical Gram-Schmidt-twice run, which marks the
entries the method determines), and the solution: all of it, or (``stride``) every stride-th entry
with their indices and the norm of the whole vector.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import solver  # noqa: E402
import synthetic_inputs as si  # noqa: E402

CASES = {
    # P4/P3, 16 -> 64 (3 levels): composite vertex / edge / cell patches of Sec. 3.1, 169,347 DoFs
    "p4_16to64": dict(Nc=16, L=3, k=4, seed=0, rtol=1e-8, cgs2=True, stride=None),
    # P2/P1, 32 -> 512 (5 levels): 2,364,419 DoFs, every 37th solution entry kept
    "p2_32to512": dict(Nc=32, L=5, k=2, seed=0, rtol=1e-8, cgs2=False, stride=37),
}


def path_of(name):
    return os.path.join(HERE, f"oracle_{name}.npz")


def make(name):
    c = CASES[name]
    t0 = time.time()
    H = solver.Hierarchy(c["Nc"], c["L"], c["k"])
    t_setup = time.time() - t0
    n = H.finest.space.ndof
    b = si.rhs_normal(n, c["seed"])
    t0 = time.time()
    res = solver.solve(H, b, c["rtol"], 100)
    t_solve = time.time() - t0
    out = dict(Nc=c["Nc"], L=c["L"], k=c["k"], seed=c["seed"], rtol=c["rtol"], ndof=n,
               lambdas=np.array([0.0] + [H.levels[l].lam for l in range(1, c["L"])]),
               iterations=res.iters, converged=res.converged, hist=np.array(res.hist),
               true_res=res.true_res, x_norm=np.linalg.norm(res.x))
    if c["cgs2"]:
        r2 = solver.solve(H, b, c["rtol"], 100, orth="cgs2")
        out["hist_cgs2"] = np.array(r2.hist)
        out["iterations_cgs2"] = r2.iters
    if c["stride"]:
        idx = np.arange(0, n, c["stride"], dtype=np.int64)
        out["x_idx"] = idx
        out["x_val"] = res.x[idx]
    else:
        out["x"] = res.x
    np.savez_compressed(path_of(name), **out)
    print(f"{name}: ndof {n}, {res.iters} iterations, setup {t_setup:.0f} s, solve {t_solve:.0f} s", flush=True)


def load(name):
    """The stored arrays of one case as a dict (None if the file has not been written)."""
    p = path_of(name)
    if not os.path.exists(p):
        return None
    with np.load(p) as z:
        return {k: z[k] for k in z.files}


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        make(name)
