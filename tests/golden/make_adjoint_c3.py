"""Write tests/golden/adjoint_c3_oracle.txt: the oracle's gradient of the breakdown
integral on the adjoint configuration (the 1,280-triangle sphere at V0 = 1, 256
Fibonacci lines, h = 1e-3, r_max = 10, alpha_eff with c = 1e-2, E0 = 0.5, d = 0.1;
J = sum of K over all lines), with respect to all 1,926 vertex coordinates, V0 and the
permittivities.  Calls only the oracle (oracle.Problem: dense assembly, LU, tracer and
its hand-written reverse pass) and the seeded mesh generator.  About 15 minutes on 8
cores.

    python tests/golden/make_adjoint_c3.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2003_12663_gb300 import meshgen as mg  # noqa: E402

OUT = os.path.join(HERE, "adjoint_c3_oracle.txt")


def main():
    mesh = mg.sphere_mesh(3)
    seeds = mg.fibonacci_seeds(256)
    P = O.Problem(mesh, eta=4.0, g=3)
    A = P.assemble()
    u = np.linalg.solve(A, P.rhs())
    w = np.ones(len(seeds))
    K, gX, gV0, geps = P.adjoint(u, seeds, w, O.TraceParams(h=1e-3, r_max=10.0, c=1e-2, E0=0.5, d=0.1), A=A)
    with open(OUT, "w") as f:
        f.write("# oracle gradient of J = sum_l K_l (Eq. Breakdowncrit along 256 field lines)\n")
        f.write("# mesh: sphere_mesh(3) (1280 triangles, 642 vertices), V0 = 1; seeds: fibonacci_seeds(256)\n")
        f.write("# h = 1e-3, r_max = 10, c = 1e-2, E0 = 0.5, d = 0.1; eta = 4, far rule 3x3\n")
        f.write("# written by tests/golden/make_adjoint_c3.py (oracle only)\n")
        f.write(f"J {float(K.sum()):.17e}\n")
        f.write(f"dJ_dV0 {gV0[0]:.17e}\n")
        f.write(f"dJ_deps {geps[0, 0]:.17e} {geps[0, 1]:.17e}\n")
        for k in range(len(K)):
            f.write(f"K {k} {K[k]:.17e}\n")
        for v in range(len(gX)):
            f.write(f"gX {v} {gX[v, 0]:.17e} {gX[v, 1]:.17e} {gX[v, 2]:.17e}\n")
    print(OUT)


if __name__ == "__main__":
    main()
