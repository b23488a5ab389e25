"""Iteration counts of the oracle's plain Jacobi-PCG (``fe.solve_pcg``) on the
benchmark workloads, written to ``oracle/reference_iterations.json``.

The CPU baseline of ``bench.py`` times a bounded sample of these iterations
on the host and scales by the stored count (the full oracle solve of the
128x64x64 workload takes tens of minutes).  Calls only ``oracle/`` and the
input generators.

    python -m oracle.reference_iterations
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import fe  # noqa: E402
from synthetic import cantilever_128x64x64_voids  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "reference_iterations.json")


def main():
    w = cantilever_128x64x64_voids()
    t0 = time.perf_counter()
    K = fe.assemble(w.nx, w.ny, w.nz, w.E)
    t1 = time.perf_counter()
    u, it = fe.solve_pcg(K, w.f[0], w.fixed, rtol=w.tol, maxiter=200000)
    t2 = time.perf_counter()
    rel = fe.relative_residual(K, u, w.f[0], w.fixed)
    rec = {w.name: {"rtol": w.tol, "iterations": it, "final_rel_residual": rel,
                    "assembly_s": t1 - t0, "solve_s": t2 - t1, "nnz": int(K.nnz)}}
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data.update(rec)
    json.dump(data, open(OUT, "w"), indent=1, sort_keys=True)
    print(rec)


if __name__ == "__main__":
    main()
