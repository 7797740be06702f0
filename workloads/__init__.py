"""Problem descriptions and seeded synthetic inputs.

This module holds no arithmetic of the method: only the parameters of each
workload (mesh sizes, physical constants, boundary kinds) and seeded random
arrays.  Both the oracle (through the tests) and the CUDA library binding read
from it; neither side imports the other.

Workloads (all synthetic, generated from closed forms; no mesh or dataset files):
  couette2d  -- [0,1]^2 periodic in x, isothermal walls, upper wall moving at
                Mach 0.15, Re = 100 (Re_c = Re / 0.15), Pr = 0.72, gamma = 1.4,
                4x4 macro-elements of 2x2 quads, p = 2
  mms3d      -- unit cube, Dirichlet on all faces from the manufactured solution
                rho = 1 + 0.1 sin sin sin, v = 0.3 (sin, cos, sin)(2 pi x),
                P = 1/gamma + 0.05 cos(pi (x+y+z)), Re_c = 100, 8^3 macros of
                2^3 hexes, p = 2
  tgv        -- periodic [0, 2pi]^3, Re = 1600 at Mach 0.1 (Re_c = 16000),
                16^3 macros of 2^3 hexes, p = 2, DIRK3 dt = 0.05 t_c
  batched    -- 256 manufactured-solution problems with seeded m, p, amplitudes
  sphere     -- flow past a sphere of diameter 1: cubed-sphere O-grid of the shell
                0.5 <= r <= 10, 6 panels x 8 x 8 cells x 16 layers (layer thickness
                ratio 1.15) of 2^3 curved hexes, p = 2; isothermal no-slip wall at
                T = 1 on the sphere, characteristic far field at r = 10; free stream
                rho = 1, v = (0.3, 0, 0), T = 1 (Mach 0.3), Re = 100 on the diameter
                (Re_c = 100 / 0.3); initial state the free stream with the velocity
                blended to zero inside r = 0.6 (smooth step over 0.6 <= r <= 1)
"""
import numpy as np

BC_NONE, BC_DIRICHLET, BC_WALL, BC_FARFIELD = 0, 1, 2, 3
FIELD_NONE, FIELD_MMS, FIELD_UNIFORM, FIELD_TGV, FIELD_SPHERE, FIELD_COUETTE3D = 0, 1, 2, 3, 4, 5
MESH_BOX, MESH_SHELL, MESH_SIMPLEX = 0, 1, 2


def _base(dim, nmac, lo, hi, periodic, m, p, Re_c, Pr=0.72, gamma=1.4, supg=1):
    return dict(dim=dim, nmac=list(nmac) + [1] * (3 - len(nmac)), lo=list(lo) + [0.0] * (3 - len(lo)),
                hi=list(hi) + [1.0] * (3 - len(hi)), periodic=list(periodic) + [0] * (3 - len(periodic)),
                bc=[BC_NONE] * 6, wall_T=[1.0] * 6, wall_v=[[0.0, 0.0, 0.0] for _ in range(6)],
                m=m, p=p, gamma=gamma, Re=Re_c, Pr=Pr, supg=supg, field=FIELD_NONE,
                field_par=[0.0] * 8)


def couette2d(nmac=4, m=2, p=2, Re=100.0, Mw=0.15, supg=1):
    """Config 1: steady 2D Couette flow (periodic x, isothermal walls at T = 1)."""
    pr = _base(2, [nmac, nmac], [0, 0], [1, 1], [1, 0], m, p, Re / Mw, supg=supg)
    pr["bc"][2] = BC_WALL            # y = 0, at rest
    pr["bc"][3] = BC_WALL            # y = 1, moving
    pr["wall_v"][3] = [Mw, 0.0, 0.0]
    pr["field"] = FIELD_UNIFORM
    pr["field_par"] = [1.0, 0.0, 0.0, 0.0, 1.0, 0, 0, 0]   # rho, v1..v3, T of the rest state
    pr["name"] = "couette2d"
    pr["Mw"] = Mw
    return pr


def mms(dim=3, nmac=8, m=2, p=2, Re_c=100.0, amp=0.1, vel=0.3, pamp=0.05, supg=1):
    """Config 2 (dim=3) and its 2D analogue: manufactured solution, Dirichlet everywhere."""
    pr = _base(dim, [nmac] * dim, [0] * dim, [1] * dim, [0] * dim, m, p, Re_c, supg=supg)
    for s in range(2 * dim):
        pr["bc"][s] = BC_DIRICHLET
    pr["field"] = FIELD_MMS
    pr["field_par"] = [amp, vel, pamp, 0, 0, 0, 0, 0]
    pr["name"] = "mms%dd" % dim
    return pr


def tgv(nmac=16, m=2, p=2, Re=1600.0, M0=0.1, supg=1):
    """Config 5: Taylor-Green vortex, periodic cube [0, 2 pi]^3."""
    L = 2 * np.pi
    pr = _base(3, [nmac] * 3, [0] * 3, [L] * 3, [1, 1, 1], m, p, Re / M0, supg=supg)
    pr["field"] = FIELD_TGV
    pr["field_par"] = [M0, 0, 0, 0, 0, 0, 0, 0]
    pr["name"] = "tgv"
    return pr


def periodic_uniform(dim=3, nmac=2, m=2, p=2, rho=1.2, v=(0.2, -0.1, 0.05), T=0.9, Re_c=100.0, supg=1):
    """Periodic box with a uniform state (free-stream preservation)."""
    pr = _base(dim, [nmac] * dim, [0] * dim, [1] * dim, [1] * dim, m, p, Re_c, supg=supg)
    pr["field"] = FIELD_UNIFORM
    pr["field_par"] = [rho, v[0], v[1] if dim > 1 else 0, v[2] if dim > 2 else 0, T, 0, 0, 0]
    pr["name"] = "uniform%dd" % dim
    return pr


def sphere(nq=8, nr=16, m=2, p=2, r0=0.5, r1=10.0, ratio=1.15, Re=100.0, Mach=0.3, supg=1,
           inner=BC_WALL, outer=BC_FARFIELD):
    """Config 4: flow past a sphere on the cubed-sphere shell mesh (module docstring)."""
    pr = _base(3, [1, 1, 1], [0.0] * 3, [1.0] * 3, [0, 0, 0], m, p, Re / Mach, supg=supg)
    pr["mesh_kind"] = MESH_SHELL
    pr["shell_n"] = [nq, nr]
    pr["shell_r"] = [r0, r1, ratio]
    pr["bc"] = [inner, outer, BC_NONE, BC_NONE, BC_NONE, BC_NONE]
    pr["wall_T"] = [1.0] * 6
    pr["field"] = FIELD_SPHERE
    pr["field_par"] = [1.0, Mach, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    pr["name"] = "sphere"
    return pr


def couette3d(nmac=2, m=2, p=2, Mach=0.15, Re=1.0, Pr=0.71, alpha=0.8, beta=0.85, supg=1):
    """Compressible Couette flow with a source term on the unit cube (the paper's Sec. 5.1
    case), Dirichlet data from the closed form on every side; Re on the unit length, so
    Re_c = Re / Mach; viscous-heating coefficient K = (gamma - 1) Pr Mach^2 / 2."""
    gamma = 1.4
    pr = _base(3, [nmac] * 3, [0.0] * 3, [1.0] * 3, [0, 0, 0], m, p, Re / Mach, Pr=Pr, gamma=gamma, supg=supg)
    pr["bc"] = [BC_DIRICHLET] * 6
    pr["field"] = FIELD_COUETTE3D
    pr["field_par"] = [Mach, alpha, beta, 0.5 * (gamma - 1.0) * Pr * Mach * Mach, 0.0, 0.0, 0.0, 0.0]
    pr["name"] = "couette3d"
    return pr


def sizes(prob):
    """Node and trace counts implied by the discrete spaces (used for array shapes)."""
    d, m, p = prob["dim"], prob["m"], prob["p"]
    n1 = m * p + 1
    Np, Nfn = n1 ** d, n1 ** (d - 1)
    if prob.get("mesh_kind", MESH_BOX) == MESH_SIMPLEX:
        # d! simplicial macros per box cell; d + 1 faces each, shared by two except on the
        # non-periodic boundary planes ((d-1)! simplicial faces per boundary cell face)
        from math import comb, factorial
        n = m * p
        ncell = int(np.prod(prob["nmac"][:d]))
        E = ncell * factorial(d)
        B = 0
        for k in range(d):
            if not prob["periodic"][k]:
                B += 2 * factorial(d - 1) * int(np.prod([prob["nmac"][j] for j in range(d) if j != k]))
        Nfn = comb(n + d - 1, d - 1)
        return dict(d=d, ns=d + 2, Np=comb(n + d, d), Nfn=Nfn, Nth=(d + 1) * Nfn, E=E, F=((d + 1) * E + B) // 2)
    if prob.get("mesh_kind", MESH_BOX) == MESH_SHELL:
        nq, nr = prob["shell_n"]
        E = 6 * nq * nq * nr
        F = 6 * nq * nq * (nr + 1) + 12 * nq * nq * nr
        return dict(d=d, ns=d + 2, Np=Np, Nfn=Nfn, Nth=2 * d * Nfn, E=E, F=F)
    E = int(np.prod(prob["nmac"][:d]))
    F = 0
    for k in range(d):
        npos = prob["nmac"][k] if prob["periodic"][k] else prob["nmac"][k] + 1
        F += npos * int(np.prod([prob["nmac"][j] for j in range(d) if j != k]))
    return dict(d=d, ns=d + 2, Np=Np, Nfn=Nfn, Nth=2 * d * Nfn, E=E, F=F)


def random_state(prob, seed, du=0.05, dq=0.2):
    """Seeded state around a smooth-flow-like constant: u [E,ns,Np], q [E,d,ns,Np], uhat [F*ns*Nfn].

    Base conserved state (rho, rho v, rho E) = (1, 0.1, -0.05, 0.08, 2.0) (first d
    momenta used, energy adjusted to keep the pressure positive) plus U(-du, du)
    per entry; q entries U(-dq, dq); uhat = base + U(-du, du).
    """
    z = sizes(prob)
    rng = np.random.default_rng(seed)
    d, ns = z["d"], z["ns"]
    base = np.array([1.0] + [0.1, -0.05, 0.08][:d] + [2.0])
    u = base[None, :, None] + rng.uniform(-du, du, size=(z["E"], ns, z["Np"]))
    q = rng.uniform(-dq, dq, size=(z["E"], d, ns, z["Np"]))
    uh = (base[None, :, None] + rng.uniform(-du, du, size=(z["F"], ns, z["Nfn"]))).reshape(-1)
    return u, q, uh


def perturbation(prob, seed, amp=1e-3):
    """U(-amp, amp) per nodal value of u and of uhat (Couette/MMS initial perturbation)."""
    z = sizes(prob)
    rng = np.random.default_rng(seed)
    du = rng.uniform(-amp, amp, size=(z["E"], z["ns"], z["Np"]))
    duh = rng.uniform(-amp, amp, size=(z["F"] * z["ns"] * z["Nfn"],))
    return du, duh


def random_vector(n, seed, scale=1.0):
    return np.random.default_rng(seed).uniform(-scale, scale, size=n)


def batched_problems(count=256, seed0=1000):
    """Config 3 draws: per problem k with seed 1000+k: m_c in {2..6}, p in {1,2,3},
    density amplitude in [0.05, 0.15], Mach (velocity amplitude) in [0.1, 0.3],
    Re in [50, 200] (used as Re_c), pressure amplitude 0.05 * amp / 0.1."""
    out = []
    for k in range(count):
        r = np.random.default_rng(seed0 + k)
        mc = int(r.integers(2, 7))
        p = int(r.integers(1, 4))
        amp = float(r.uniform(0.05, 0.15))
        mach = float(r.uniform(0.1, 0.3))
        Re = float(r.uniform(50, 200))
        out.append(mms(3, mc, 2, p, Re_c=Re, amp=amp, vel=mach, pamp=0.05 * amp / 0.1))
    return out
