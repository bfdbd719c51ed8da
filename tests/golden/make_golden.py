"""Writes the stored expected values used by the full-size GPU parity tests and by the
benchmark's CPU-baseline extrapolation.  Calls only the CPU oracle (and the seeded input
generators).  Run from the repository root:

    python tests/golden/make_golden.py [name ...]

Each case stores the oracle's Newton/GMRES counts, residual history and the potential
phi sampled at fixed grid points (every case lists its exact parameters).
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import ot_inputs as I  # noqa: E402

CASES = {
    "blob256": dict(kind="blob_pair", N=256, M=256, seed=1000, tau=4.0, tol=1e-10, eta=1e-1),
    "noise1024": dict(kind="noise_blob_pair", N=1024, M=1024, seed=3000, tau=1.0, tol=1e-8,
                      eta=1e-2, symbols=1),
    "noise2048": dict(kind="noise_blob_pair", N=2048, M=2048, seed=3000, tau=1.0, tol=1e-8,
                      eta=1e-1),
}


def sample_indices(N, M, count=512):
    rng = I.SplitMix64(12345)
    r = rng.uniform(2 * count).reshape(count, 2)
    return (r[:, 0] * N).astype(int), (r[:, 1] * M).astype(int)


def inputs(case):
    gen = {"blob_pair": I.blob_pair, "noise_blob_pair": I.noise_blob_pair}[case["kind"]]
    return gen(case["N"], case["M"], s=case["seed"])


def run(name):
    case = CASES[name]
    f, g = inputs(case)
    t = time.time()
    # symbols: 0 the spectral derivative symbols of Sec. 4.2, 1 those of the stencils
    with O.fd_symbols(case.get("symbols", 0)):
        u, st, hres, hgm = O.solve(f, g, tau=case["tau"], tol=case["tol"], eta=case["eta"],
                                   max_newton=300)
    secs = time.time() - t
    ii, jj = sample_indices(case["N"], case["M"])
    out = dict(case=case, oracle_seconds=secs, stats=st, res_history=hres.tolist(),
               gmres_history=hgm.tolist(), sample_i=ii.tolist(), sample_j=jj.tolist(),
               phi_samples=u[ii, jj].tolist(), phi_absmax=float(np.abs(u).max()),
               command="python tests/golden/make_golden.py " + name)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + ".json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print(name, st, "%.1fs" % secs, flush=True)


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["noise1024", "blob256"]):
        run(n)
