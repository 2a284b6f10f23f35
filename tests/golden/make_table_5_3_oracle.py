"""Writes table_5_3_oracle.txt: the oracle's PCG iteration counts for the workload of Table 5.3
(Sec. 5.2: u = exp(-2 pi^2 t) sin(pi x) sin(pi y), g = 0, eps = 1e-6 absolute in the K_X-norm
of Eq. 3.3) at the paper's space level K = 9 (N_x = 261121), with

* the multigrid of this project's reading (2 V-cycles, 3 + 3 three-colour Gauss-Seidel sweeps,
  Sec. 5.1), which the GPU must reproduce, and
* the direct inverses K_j = (alpha A_x + 2^j M_x)^-1, K_x = A_x^-1 of Sec. 5.1, which show how far
  the printed counts are from the method with exact spatial solves.

Calls only oracle/ (and the seeded input generator).  Slow: about an hour on 8 cores.
Usage: python tests/golden/make_table_5_3_oracle.py [J ...]   (default J = 3 4 5)
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import schur  # noqa: E402
from paper_2009_08875_gb300 import inputs  # noqa: E402

K = 9
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table_5_3_oracle.txt")


def count(J, inverses):
    p = schur.Problem(K, J, inverses=inverses)
    g, u0, _ = inputs.decaying(K, J)
    _, _, info = schur.solve(p, g, u0, tol=1e-6, tol_mode="abs", maxit=60)
    return info["iters"], info["rho"][-2] ** 0.5, info["rho"][-1] ** 0.5


def main():
    Js = [int(a) for a in sys.argv[1:]] or [3, 4, 5]
    rows = []
    for J in Js:
        t0 = time.time()
        mg = count(J, "mg")
        di = count(J, "direct")
        rows.append((2 ** J + 1, mg, di))
        print(f"N_t={2 ** J + 1}: multigrid {mg[0]}, direct {di[0]} ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT, "w") as fh:
        fh.write("# Oracle PCG iteration counts, workload of Table 5.3 (Sec. 5.2): u = exp(-2 pi^2 t) sin(pi x)\n"
                 "# sin(pi y), g = 0, eps = 1e-6 absolute (Eq. 3.3), K = 9 (N_x = 261121).  Written by\n"
                 "# make_table_5_3_oracle.py from oracle/ only.  Columns: N_t, iterations with the multigrid\n"
                 "# reading (2 V-cycles, 3 + 3 three-colour sweeps), sqrt(r^T K_X r) at the last two iterates,\n"
                 "# iterations with direct inverses, the same two norms.\n")
        for Nt, mg, di in rows:
            fh.write(f"{Nt} {mg[0]} {mg[1]:.6e} {mg[2]:.6e} {di[0]} {di[1]:.6e} {di[2]:.6e}\n")


if __name__ == "__main__":
    main()
