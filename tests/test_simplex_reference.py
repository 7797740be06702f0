"""The library's simplicial reference tables (csrc/simplex.cu, host code, no GPU needed) against
the oracle's (oracle/simplex.py): the two are written independently; the same node lattice, the
same quadrature points and weights (as sets), bases that reproduce P_p, and the same face node
lists and face rules.  The GPU kernels of simplicial meshes read exactly these tables."""
import numpy as np
import pytest

from oracle import simplex as sx


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2402_11361_gb300 as m
    return m


def _sorted_rows(pts, w):
    rows = np.hstack([np.round(pts, 12), np.round(w, 14)[:, None]])
    return rows[np.lexsort(rows.T[::-1])]


@pytest.mark.parametrize("d,m,p", [(2, 1, 1), (2, 2, 2), (2, 3, 3), (3, 1, 2), (3, 2, 1), (3, 2, 2), (3, 2, 3)])
def test_simplex_tables_match_the_oracle(pkg, d, m, p):
    T = pkg.simplex_reference(d, m, p)
    K = sx.KuhnMacro(d, m, p)
    c = T["counts"]
    assert (c["Np"], c["Nfn"], c["nel"]) == (K.Np, K.Nfn, len(K.subs))
    assert np.array_equal(T["lattice"], K.lat)
    # volume rule: the same points and weights
    assert np.allclose(_sorted_rows(T["vxi"], T["vw"]), _sorted_rows(K.xq.T, K.wq), atol=1e-12)
    # the basis at each point reproduces a random polynomial of degree p and its gradient
    rng = np.random.default_rng(d * 100 + m * 10 + p)
    coef = {a: rng.uniform(-1, 1) for a in sx.monomials(d, p)}

    def poly(x):
        v = np.zeros(len(x))
        g = np.zeros((len(x), d))
        for a, cc in coef.items():
            v += cc * np.prod(x ** np.array(a), axis=1)
            for l in range(d):
                if a[l]:
                    b = np.array(a)
                    b[l] -= 1
                    g[:, l] += cc * a[l] * np.prod(x ** b, axis=1)
        return v, g

    nodal, _ = poly(K.xn)
    v, g = poly(T["vxi"])
    ng = c["ng"]
    for pt in range(len(v)):
        el = pt // ng
        vals = nodal[T["vnode"][el]]
        assert abs(T["vtab"][pt, :, 0] @ vals - v[pt]) < 1e-11
        assert np.abs(T["vtab"][pt, :, 1:].T @ vals - g[pt]).max() < 1e-10
    # faces: node lists, points and weights
    for fl in range(d + 1):
        fc = K.faces[fl]
        assert np.array_equal(T["fnodes"][fl], fc["nodes"])
        assert np.allclose(_sorted_rows(T["fxi"][fl], T["fwt"][fl]), _sorted_rows(fc["xi"].T, fc["wt"]), atol=1e-12)


def test_simplex_reference_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.MehdgError):
        pkg.simplex_reference(4, 1, 1)
    with pytest.raises(pkg.MehdgError):
        pkg.simplex_reference(3, 2, 4)


@pytest.mark.parametrize("case", ["2d_dirichlet_p2", "2d_periodic_p1_m3", "2d_wall_p2_m3", "3d_dirichlet_p1",
                                  "3d_periodic_p2_m1", "3d_periodic_x_p3_m1"])
def test_simplex_mesh_maps_and_operators_match_the_oracle(pkg, case):
    """The library's simplicial mesh (host code) against the oracle's: the same macro and face
    numbering, gather maps (node by node), owners, boundary sides and node positions, and the
    per-macro mass, lifting and face matrices M, G_k, Gh_k of every macro within 1e-12."""
    import workloads as W
    from oracle import assemble as asm
    from oracle import solve
    d = int(case[0])
    if case == "2d_dirichlet_p2":
        pr = W.mms(dim=2, nmac=2, m=2, p=2)
    elif case == "2d_periodic_p1_m3":
        pr = W.periodic_uniform(dim=2, nmac=2, m=3, p=1)
    elif case == "2d_wall_p2_m3":
        pr = W.couette2d(nmac=2, m=3, p=2)
    elif case == "3d_dirichlet_p1":
        pr = W.mms(dim=3, nmac=1, m=2, p=1)
    elif case == "3d_periodic_x_p3_m1":
        pr = W.mms(dim=3, nmac=2, m=1, p=3)
        pr["periodic"] = [1, 0, 0]
        pr["bc"][0] = pr["bc"][1] = W.BC_NONE
    else:
        pr = W.periodic_uniform(dim=3, nmac=2, m=1, p=2)
    pr["mesh_kind"] = W.MESH_SIMPLEX
    T = pkg.simplex_mesh(pr)
    P = solve.Problem(pr)
    assert (T["E"], T["F"], T["Np"], T["Nfn"]) == (P.E, P.F, P.Np, P.Nfn)
    own = P.mesh.face_owners()
    for f in range(P.F):
        exp = [e * (d + 1) + fl for e, fl in own[f]] + [-1] * (2 - len(own[f]))
        assert list(T["owner"][f]) == exp
    u0 = np.zeros((P.ns, P.Np))
    for e in range(P.E):
        assert np.array_equal(T["gather"][e], P.maps[e].reshape(-1))
        assert [b for _, b in P.mesh.macro_faces(e)] == list(T["bside"][e])
        geo = P.geometry(e)
        assert np.abs(T["xnode"][e] - geo.xn).max() < 1e-13
        with np.errstate(all="ignore"):
            b = asm.assemble_macro(geo, P.phys, u0 + 1.0, np.zeros((d, P.ns, P.Np)), np.ones((P.ns, P.Nth)),
                                   want_jac=False)
        assert np.abs(T["M"][e] - b["M"]).max() < 1e-12 * np.abs(b["M"]).max()
        for k in range(d):
            assert np.abs(T["Gk"][e, k] - b["Gk"][k]).max() < 1e-12 * np.abs(b["Gk"][k]).max()
            assert np.abs(T["Ghk"][e, k] - b["Ghk"][k]).max() < 1e-12 * np.abs(b["Ghk"][k]).max()
