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
                      eta=1e-2, symbols=1),
}
# pairs of the batched workload (ot_inputs.batch_workload(512)): the first pair of each size
# and the two 512^2 pairs that lose convexity at tau = 1; the batched solver's settings
# (stencil symbols, tau = 1, eta = 0.1, tol 1e-8), a diverged solve repeated with twice tau
# up to twice (the remedy of Sec. 3.2 / Sec. 5.3)
for _k in (0, 2, 5, 7, 9, 200, 297):
    CASES["batch%d" % _k] = dict(kind="blob_pair", batch_index=_k, seed=4000 + _k, tau=1.0,
                                 tol=1e-8, eta=1e-1, symbols=1, tau_retry=2, max_newton=1000)


def sample_indices(N, M, count=512):
    rng = I.SplitMix64(12345)
    r = rng.uniform(2 * count).reshape(count, 2)
    return (r[:, 0] * N).astype(int), (r[:, 1] * M).astype(int)


def inputs(case):
    if "batch_index" in case:
        n, s = I.batch_workload(512)[case["batch_index"]]
        assert s == case["seed"]
        case["N"] = case["M"] = n
    gen = {"blob_pair": I.blob_pair, "noise_blob_pair": I.noise_blob_pair}[case["kind"]]
    return gen(case["N"], case["M"], s=case["seed"])


def run(name):
    case = CASES[name]
    f, g = inputs(case)
    t = time.time()
    # symbols: 0 the spectral derivative symbols of Sec. 4.2, 1 those of the stencils
    tau = case["tau"]
    attempts = []
    with O.fd_symbols(case.get("symbols", 0)):
        for _ in range(1 + case.get("tau_retry", 0)):
            u, st, hres, hgm = O.solve(f, g, tau=tau, tol=case["tol"], eta=case["eta"],
                                       max_newton=case.get("max_newton", 300))
            attempts.append(dict(tau=tau, stats=st))
            if st["status"] != O.ORC_EDIVERGED:
                break
            tau *= 2.0
    secs = time.time() - t
    ii, jj = sample_indices(case["N"], case["M"])
    out = dict(case=case, oracle_seconds=secs, stats=st, attempts=attempts,
               res_history=hres.tolist(),
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
