"""Write the FP64 oracle's expected values for the curved-mesh (flow past a sphere) DIRK parity
test.

Output: tests/golden/dirk_sphere_2x1_p2.npz with
  u0, q0, uh0  the initial state: the free stream (rho = 1, v = (0.3, 0, 0), T = 1) with the
               velocity blended to zero inside r = 0.6 at the nodes, uhat = the trace of the
               face's first owner, q the lifted gradient (R_Q = 0 with the per-macro mass
               matrix M_J of the curved macros);
  u1, q1, uh1  the state after one step of Alexander's DIRK3 (Sec. 2.4, eq. C242), every stage
               solved by Newton to |R_F| <= 1e-12 |R_F^0| with direct trace solves.
Problem: cubed-sphere shell 0.5 <= r <= 2, 6 panels x 2 x 2 cells x 1 layer of curved hexes,
m = 1, p = 2, isothermal wall at T = 1 on the sphere, characteristic far field at r = 2,
Mach 0.3, Re = 100 on the diameter (Re_c = 100 / 0.3), SUPG on; dt = 0.05 (acoustic units).

Calls only oracle/ and workloads/ (test infrastructure); run from the repository root:
  python tests/golden/make_dirk_sphere.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import solve  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dirk_sphere_2x1_p2.npz")
DT = 0.05


def problem():
    return W.sphere(nq=2, nr=1, m=1, p=2, r0=0.5, r1=2.0)


def main():
    P = solve.Problem(problem())
    u0, q0, uh0 = solve.initial_state(P, lift=True)
    u1, q1, uh1, stats = solve.dirk_step(P, u0, q0, uh0, dt=DT, rtol=1e-12, atol=0.0, precond="direct")
    np.savez_compressed(OUT, u0=u0, q0=q0, uh0=uh0, u1=u1, q1=q1, uh1=uh1, dt=DT,
                        newton=np.array([s["newton"] for s in stats]))
    print("wrote", OUT, [(s["newton"], s["RF"] / s["RF0"]) for s in stats])


if __name__ == "__main__":
    main()
