"""Write the FP64 oracle's expected values for the 3D DIRK parity test.

Output: tests/golden/dirk3d_tgv_2cubed_p2.npz with
  u0, q0, uh0  the initial state of the 3D Taylor-Green vortex (Sec. 5.3, eq. TGV0):
               u = the closed-form conserved state at the nodes, uhat = the trace of the
               face's first owner, q the lifted gradient (the solution of R_Q = 0,
               linear in q with A_qq = I (x) M);
  u1, q1, uh1  the state after one step of Alexander's DIRK3 (Sec. 2.4, eq. C242),
               every stage solved by Newton to |R_F| <= 1e-12 |R_F^0| (the round-off floor of
               this problem is near 1e-13 |R_F^0|) with direct
               trace solves.
Problem: periodic [0, 2 pi]^3, 2^3 macro-elements of 2^3 hexes, p = 2, Re = 1600, M0 = 0.1
(Re_c = 16000), dt = 0.05 t_c = 0.5 in acoustic time units.

Calls only oracle/ and workloads/ (test infrastructure); run from the repository root:
  python tests/golden/make_dirk3d_tgv.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import assemble as asm  # noqa: E402
from oracle import fields, solve  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dirk3d_tgv_2cubed_p2.npz")
DT = 0.5


def problem():
    return W.tgv(nmac=2, m=2, p=2)


def initial_state(P, pr):
    u = np.zeros((P.E, P.ns, P.Np))
    for e in range(P.E):
        u[e] = fields.tgv_u(P.geometry(e).xn, pr["field_par"][0], pr["gamma"])
    uh = np.zeros(P.F * P.ns * P.Nfn)
    idx = np.arange(P.Np).reshape([P.mesh.n1] * P.d)      # [.., i1, i0], axis 0 fastest
    for f, own in enumerate(P.mesh.face_owners()):
        e, fl = own[0]
        k, side = fl // 2, fl % 2
        sl = [slice(None)] * P.d
        sl[P.d - 1 - k] = -1 if side else 0
        fn = idx[tuple(sl)].reshape(-1)
        for s in range(P.ns):
            uh[(f * P.ns + s) * P.Nfn:(f * P.ns + s + 1) * P.Nfn] = u[e, s, fn]
    q = np.zeros((P.E, P.d, P.ns, P.Np))
    for e in range(P.E):
        geo = P.geometry(e)
        blk = asm.assemble_macro(geo, P.phys, u[e], q[e], P.local_trace(e, uh), None, P.source(geo),
                                 P.bfaces(e, geo), want_jac=True)
        RQ = blk["RQ"].reshape(P.d * P.ns, P.Np)
        q[e] = -np.linalg.solve(blk["M"], RQ.T).T.reshape(P.d, P.ns, P.Np)
    return u, q, uh


def main():
    pr = problem()
    P = solve.Problem(pr)
    u0, q0, uh0 = initial_state(P, pr)
    u1, q1, uh1, stats = solve.dirk_step(P, u0, q0, uh0, dt=DT, rtol=1e-12, precond="direct")
    np.savez_compressed(OUT, u0=u0, q0=q0, uh0=uh0, u1=u1, q1=q1, uh1=uh1, dt=DT,
                        newton=np.array([s["newton"] for s in stats]))
    print("wrote", OUT, [(s["newton"], s["RF"] / s["RF0"]) for s in stats])


if __name__ == "__main__":
    main()
