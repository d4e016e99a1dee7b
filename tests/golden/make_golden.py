"""Write stored oracle values used by the GPU parity tests.

Calls only ``oracle`` and the seeded input generators; nothing here touches the
CUDA library.  Usage (from the repository root)::

    python tests/golden/make_golden.py rod256   # 256x256 rod crystal, 31-point path
    python tests/golden/make_golden.py rod64    # 64x64 rod crystal, 31-point path

Output: one line per Bloch vector ``k1 k2 lambda_1 ... lambda_8`` (%.17e).
"""
import os
import sys
from multiprocessing import get_context

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import fem, eigen  # noqa: E402
import pbs_inputs as gi  # noqa: E402

CASES = {
    # name: (n, nk, bands, radius, eps_rod)
    "rod256": (256, 31, 8, 0.2, 8.9),
    "rod64": (64, 31, 8, 0.2, 8.9),
}


def _one(args):
    n, k, bands, radius, eps_rod = args
    eps = gi.rod_eps(n, n, radius=radius, eps_rod=eps_rod)
    ops = fem.assemble(fem.Mesh(1.0, 1.0, n, n), eps, k)
    lam, _ = eigen.eigs_sparse(ops, bands)
    return lam


def main(name, procs=4):
    n, nk, bands, radius, eps_rod = CASES[name]
    ks = gi.gxmg_path(nk)
    with get_context("spawn").Pool(procs) as pool:
        vals = pool.map(_one, [(n, tuple(k), bands, radius, eps_rod) for k in ks])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_path{nk}.txt")
    with open(path, "w") as f:
        f.write(f"# oracle.eigen.eigs_sparse: rod eps={eps_rod} r={radius}a, {n}x{n}, a=b=1, "
                f"Gamma-X-M-Gamma {nk} points, {bands} smallest non-zero eigenvalues\n")
        for k, lam in zip(ks, vals):
            f.write(" ".join(f"{v:.17e}" for v in list(k) + list(lam)) + "\n")
    print("wrote", path)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 4)
