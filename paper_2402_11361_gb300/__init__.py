"""Python binding of libmehdg (GB300 matrix-free macro-element HDG, arXiv 2402.11361).

Argument marshalling only: every step of the solver runs in the CUDA library
declared in ``include/mehdg.h``.  PyTorch supplies device memory and the stream.
Importing works without a GPU; creating a ``Context`` needs the built library
and a CUDA device and raises otherwise (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmehdg.so")

c_int, c_double, c_void_p, c_longlong = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_longlong

PREC_FP64, PREC_MIXED = 0, 1

EXPORTS = ["mehdg_mesh", "mehdg_query", "mehdg_init_state", "mehdg_assemble_local", "mehdg_condense_factor",
           "mehdg_apply_trace", "mehdg_precondition", "mehdg_linear_solve", "mehdg_recover", "mehdg_dirk_stage",
           "mehdg_get_block", "mehdg_phase_times", "mehdg_phase_stats", "mehdg_launch_count", "mehdg_mlp_setup", "mehdg_mlp_params",
           "mehdg_mlp_record", "mehdg_mlp_set_recording", "mehdg_mlp_gradient", "mehdg_mlp_train",
           "mehdg_stage_begin", "mehdg_newton_step", "mehdg_stage_end", "mehdg_set_precond", "mehdg_tc_gemm_tf32", "mehdg_tc_gemm_nt", "mehdg_lu_batched", "mehdg_apply_trace_noalloc", "mehdg_lu_queue", "mehdg_graph_replays", "mehdg_batch_create",
           "mehdg_batch_size", "mehdg_batch_context", "mehdg_batch_steady_solve", "mehdg_batch_tiles",
           "mehdg_batch_graph_replays", "mehdg_batch_last_error", "mehdg_batch_destroy", "mehdg_flow_integrals",
           "mehdg_simplex_reference", "mehdg_simplex_mesh", "mehdg_destroy",
           "mehdg_last_error"]

ERRORS = {0: "OK", -1: "ARG", -2: "CUDA", -3: "OOM", -4: "SINGULAR", -5: "NOT_CONVERGED", -6: "TIMEOUT", -7: "NAN"}


class Problem(ctypes.Structure):
    _fields_ = [("dim", c_int), ("m", c_int), ("p", c_int), ("nmac", c_int * 3), ("lo", c_double * 3),
                ("hi", c_double * 3), ("periodic", c_int * 3), ("bc", c_int * 6), ("wall_T", c_double * 6),
                ("wall_v", (c_double * 3) * 6), ("gamma", c_double), ("Re", c_double), ("Pr", c_double),
                ("supg", c_int), ("field", c_int), ("field_par", c_double * 8), ("mesh_kind", c_int),
                ("shell_n", c_int * 2), ("shell_r", c_double * 3)]


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int), ("precond", c_int), ("restart", c_int), ("max_iters", c_int),
                ("lin_rtol", c_double), ("lin_atol", c_double), ("inner_iters", c_int),
                ("newton_rtol", c_double), ("newton_atol", c_double), ("max_newton", c_int),
                ("tau_init", c_double), ("tau_max", c_double), ("refine_iters", c_int), ("apply_mode", c_int),
                ("tc_mode", c_int), ("precond_bf16", c_int), ("solver", c_int),
                ("condense_layers", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("dim", c_int), ("ns", c_int), ("Np", c_int), ("Nfn", c_int), ("Nth", c_int), ("Nu", c_int),
                ("Nq", c_int), ("Nt", c_int), ("n_macro", c_int), ("n_face", c_int), ("n_trace", c_longlong),
                ("bytes_device", c_longlong)]


class TimeTerm(ctypes.Structure):
    _fields_ = [("coef", c_double), ("hist", c_void_p), ("supg_time", c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("newton_steps", c_int), ("fgmres_iters", c_int), ("res0", c_double), ("res", c_double),
                ("t_assemble", c_double), ("t_condense", c_double), ("t_krylov", c_double),
                ("t_recover", c_double), ("status", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


DEFAULT_OPTIONS = dict(precision=PREC_FP64, precond=0, restart=30, max_iters=2000, lin_rtol=1e-6, lin_atol=0.0,
                       inner_iters=5, newton_rtol=1e-8, newton_atol=1e-14, max_newton=100, tau_init=1.0,
                       tau_max=1e8, refine_iters=2, apply_mode=0, tc_mode=0,
                       precond_bf16=0, solver=0, condense_layers=2)

_lib = None


def load_library(path=LIB_PATH):
    """Load libmehdg.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libmehdg.so not found at %s; run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    P, I = ctypes.POINTER, c_int
    lib.mehdg_mesh.argtypes = [P(c_void_p), P(Problem), I, P(Options), c_void_p]
    lib.mehdg_query.argtypes = [c_void_p, P(Info)]
    lib.mehdg_init_state.argtypes = [c_void_p, c_void_p, c_void_p, I, c_void_p, c_void_p, c_void_p]
    lib.mehdg_assemble_local.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, P(TimeTerm), P(c_double)]
    lib.mehdg_condense_factor.argtypes = [c_void_p, c_double, c_void_p]
    lib.mehdg_apply_trace.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.mehdg_precondition.argtypes = [c_void_p, I, c_void_p, c_void_p]
    lib.mehdg_linear_solve.argtypes = [c_void_p, c_void_p, c_void_p, P(SolveStats)]
    lib.mehdg_recover.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    lib.mehdg_dirk_stage.argtypes = [c_void_p, I, c_double, c_void_p, c_void_p, c_void_p, P(SolveStats)]
    lib.mehdg_stage_begin.argtypes = [c_void_p, I, c_double, c_void_p, c_void_p, c_void_p, P(SolveStats)]
    lib.mehdg_newton_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, P(SolveStats)]
    lib.mehdg_stage_end.argtypes = [c_void_p, c_void_p]
    lib.mehdg_get_block.argtypes = [c_void_p, I, I, c_void_p, P(c_longlong)]
    lib.mehdg_phase_times.argtypes = [c_void_p, P(c_double), I]
    lib.mehdg_phase_stats.argtypes = [c_void_p, P(c_double), P(c_longlong), I, I]
    lib.mehdg_launch_count.argtypes = [c_void_p, P(c_longlong)]
    lib.mehdg_graph_replays.argtypes = [c_void_p, P(c_longlong)]
    lib.mehdg_mlp_setup.argtypes = [c_void_p, I, ctypes.c_ulonglong, I, I]
    lib.mehdg_mlp_params.argtypes = [c_void_p, I, c_void_p, P(c_longlong)]
    lib.mehdg_mlp_record.argtypes = [c_void_p, c_void_p, c_void_p]
    lib.mehdg_mlp_set_recording.argtypes = [c_void_p, I, P(c_int)]
    lib.mehdg_mlp_gradient.argtypes = [c_void_p, c_void_p, c_void_p, I, c_void_p, P(c_double)]
    lib.mehdg_mlp_train.argtypes = [c_void_p, I, I, c_double, P(c_double)]
    lib.mehdg_set_precond.argtypes = [c_void_p, I]
    lib.mehdg_lu_batched.argtypes = [I, I, c_void_p, c_void_p, I, c_void_p, c_void_p]
    L, F = c_longlong, ctypes.c_float
    lib.mehdg_tc_gemm_nt.argtypes = [I, I, I, c_void_p, L, L, c_void_p, L, L, c_void_p, L, L, F, F, I, c_void_p,
                                     c_void_p]
    lib.mehdg_lu_queue.argtypes = [I, P(c_int), P(c_void_p), P(c_void_p), I, I, c_void_p, c_void_p]
    lib.mehdg_batch_create.argtypes = [P(c_void_p), P(Problem), I, P(Options), c_void_p]
    lib.mehdg_batch_size.argtypes = [c_void_p]
    lib.mehdg_batch_context.argtypes = [c_void_p, I]
    lib.mehdg_batch_steady_solve.argtypes = [c_void_p, P(c_void_p), P(c_void_p), P(c_void_p), P(SolveStats),
                                             P(c_int)]
    lib.mehdg_batch_tiles.argtypes = [c_void_p, I, P(c_int), P(c_int), P(c_int), P(c_double)]
    lib.mehdg_batch_graph_replays.argtypes = [c_void_p]
    lib.mehdg_batch_last_error.argtypes = [c_void_p]
    lib.mehdg_batch_destroy.argtypes = [c_void_p]
    lib.mehdg_destroy.argtypes = [c_void_p]
    lib.mehdg_destroy.restype = None
    lib.mehdg_last_error.argtypes = [c_void_p]
    lib.mehdg_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if not hasattr(lib, name):
            raise RuntimeError("libmehdg.so lacks %s" % name)
        if name not in ("mehdg_destroy", "mehdg_last_error"):
            getattr(lib, name).restype = c_int
    lib.mehdg_batch_context.restype = c_void_p
    lib.mehdg_batch_graph_replays.restype = c_longlong
    lib.mehdg_batch_last_error.restype = ctypes.c_char_p
    lib.mehdg_batch_destroy.restype = None
    _lib = lib
    return lib


def problem_struct(prob):
    s = Problem()
    s.dim, s.m, s.p = prob["dim"], prob["m"], prob["p"]
    for k in range(3):
        s.nmac[k] = int(prob["nmac"][k])
        s.lo[k] = float(prob["lo"][k])
        s.hi[k] = float(prob["hi"][k])
        s.periodic[k] = int(prob["periodic"][k])
    for i in range(6):
        s.bc[i] = int(prob["bc"][i])
        s.wall_T[i] = float(prob["wall_T"][i])
        for k in range(3):
            s.wall_v[i][k] = float(prob["wall_v"][i][k])
    s.gamma, s.Re, s.Pr = prob["gamma"], prob["Re"], prob["Pr"]
    s.supg, s.field = int(prob.get("supg", 0)), int(prob["field"])
    for i in range(8):
        s.field_par[i] = float(prob["field_par"][i])
    s.mesh_kind = int(prob.get("mesh_kind", 0))
    if s.mesh_kind == 1:
        for i in range(2):
            s.shell_n[i] = int(prob["shell_n"][i])
        for i in range(3):
            s.shell_r[i] = float(prob["shell_r"][i])
    return s


def options_struct(opts=None):
    o = dict(DEFAULT_OPTIONS)
    o.update(opts or {})
    s = Options()
    for k, _ in Options._fields_:
        setattr(s, k, o[k])
    return s


class MehdgError(RuntimeError):
    pass


def tc_gemm_nt(A, Bt, C, alpha=1.0, beta=0.0):
    """C_b = alpha A_b Bt_b^T + beta C_b on tcgen05 (split TF32) for contiguous CUDA float32
    tensors A [batch, M, K], Bt [batch, N, K], C [batch, M, N] (mehdg_tc_gemm_nt).  Returns the
    error word (nonzero: a wait timed out and C is invalid)."""
    import torch
    lib = load_library()
    batch, M, K = A.shape
    N = Bt.shape[1]
    assert Bt.shape == (batch, N, K) and C.shape == (batch, M, N)
    for t in (A, Bt, C):
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    P = c_void_p
    rc = lib.mehdg_tc_gemm_nt(M, N, K, P(A.data_ptr()), K, M * K, P(Bt.data_ptr()), K, N * K, P(C.data_ptr()), N,
                              M * N, ctypes.c_float(alpha), ctypes.c_float(beta), batch, P(err.data_ptr()),
                              P(torch.cuda.current_stream(A.device).cuda_stream))
    if rc != 0:
        raise MehdgError("mehdg_tc_gemm_nt failed (%s)" % ERRORS.get(rc, rc))
    return int(err.item())


def lu_batched(A, perm=None):
    """P A_b = L_b U_b in place for a contiguous CUDA tensor A [batch, n, n] (float64 or
    float32) through mehdg_lu_batched; returns perm [batch, n] (int32).  Raises MehdgError
    (SINGULAR) on an exactly zero pivot."""
    import torch
    lib = load_library()
    assert A.is_cuda and A.is_contiguous() and A.dim() == 3 and A.shape[1] == A.shape[2]
    assert A.dtype in (torch.float64, torch.float32)
    batch, n = A.shape[0], A.shape[1]
    if perm is None:
        perm = torch.empty(batch, n, dtype=torch.int32, device=A.device)
    flag = torch.zeros(2, dtype=torch.int32, device=A.device)
    rc = lib.mehdg_lu_batched(n, batch, c_void_p(A.data_ptr()), c_void_p(perm.data_ptr()),
                              int(A.dtype == torch.float32), c_void_p(flag.data_ptr()),
                              c_void_p(torch.cuda.current_stream(A.device).cuda_stream))
    if rc != 0:
        raise MehdgError("mehdg_lu_batched failed (%s)" % ERRORS.get(rc, rc))
    return perm


def lu_queue(mats, nb=16, perms=None):
    """P A_i = L_i U_i in place for a list of square contiguous CUDA tensors of uneven size (all
    float64 or all float32) in ONE persistent work-queue launch (mehdg_lu_queue) with panel
    width nb (8, 16 or 32); returns the pivot vectors (int32)."""
    import torch
    lib = load_library()
    n = len(mats)
    fp32 = int(mats[0].dtype == torch.float32)
    if perms is None:
        perms = [torch.empty(a.shape[0], dtype=torch.int32, device=a.device) for a in mats]
    for a in mats:
        assert a.is_cuda and a.is_contiguous() and a.dim() == 2 and a.shape[0] == a.shape[1]
        assert a.dtype == (torch.float32 if fp32 else torch.float64)
    ns = (c_int * n)(*[a.shape[0] for a in mats])
    As = (c_void_p * n)(*[a.data_ptr() for a in mats])
    Ps = (c_void_p * n)(*[p.data_ptr() for p in perms])
    flag = torch.zeros(2, dtype=torch.int32, device=mats[0].device)
    rc = lib.mehdg_lu_queue(n, ns, As, Ps, fp32, int(nb), c_void_p(flag.data_ptr()),
                            c_void_p(torch.cuda.current_stream(mats[0].device).cuda_stream))
    if rc != 0:
        raise MehdgError("mehdg_lu_queue failed (%s)" % ERRORS.get(rc, rc))
    return perms


def simplex_reference(d, m, p):
    """The simplicial reference macro-element's tables (mehdg_simplex_reference; host only)."""
    import ctypes as C
    lib = load_library()
    cnt = (C.c_int * 8)()
    rc = lib.mehdg_simplex_reference(d, m, p, cnt, None, None, None, None, None, None, None, None)
    if rc != 0:
        raise MehdgError("mehdg_simplex_reference failed (%s)" % ERRORS.get(rc, rc))
    Np, Nfn, nel, ng, nloc, nsf, nfp, nfs = list(cnt)
    lat = np.zeros((Np, d), dtype=np.int32)
    vxi = np.zeros((nel * ng, d))
    vw = np.zeros(nel * ng)
    vtab = np.zeros((nel * ng, nloc, d + 1))
    vnode = np.zeros((nel, nloc), dtype=np.int32)
    fnodes = np.zeros((d + 1, Nfn), dtype=np.int32)
    fxi = np.zeros((d + 1, nsf * nfp, d))
    fwt = np.zeros((d + 1, nsf * nfp))
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = lib.mehdg_simplex_reference(d, m, p, cnt, ptr(lat), ptr(vxi), ptr(vw), ptr(vtab), ptr(vnode), ptr(fnodes),
                                     ptr(fxi), ptr(fwt))
    if rc != 0:
        raise MehdgError("mehdg_simplex_reference failed (%s)" % ERRORS.get(rc, rc))
    return dict(counts=dict(Np=Np, Nfn=Nfn, nel=nel, ng=ng, nloc=nloc, nsf=nsf, nfp=nfp, nfs=nfs), lattice=lat,
                vxi=vxi, vw=vw, vtab=vtab, vnode=vnode, fnodes=fnodes, fxi=fxi, fwt=fwt)


def simplex_mesh(prob):
    """Maps and per-macro operators of a simplicial mesh (mehdg_simplex_mesh; host only)."""
    import ctypes as C
    lib = load_library()
    ps = problem_struct(prob)
    cnt = (C.c_int * 5)()
    z = [None] * 7
    rc = lib.mehdg_simplex_mesh(C.byref(ps), cnt, *z)
    if rc != 0:
        raise MehdgError("mehdg_simplex_mesh failed (%s)" % ERRORS.get(rc, rc))
    E, F, Np, Nfn, Nth = list(cnt)
    d, ns = prob["dim"], prob["dim"] + 2
    out = dict(E=E, F=F, Np=Np, Nfn=Nfn, Nth=Nth, gather=np.zeros((E, ns * Nth), dtype=np.int32),
               owner=np.zeros((F, 2), dtype=np.int32), bside=np.zeros((E, d + 1), dtype=np.int32),
               M=np.zeros((E, Np, Np)), Gk=np.zeros((E, d, Np, Np)), Ghk=np.zeros((E, d, Np, Nth)),
               xnode=np.zeros((E, d, Np)))
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    rc = lib.mehdg_simplex_mesh(C.byref(ps), cnt, ptr(out["gather"]), ptr(out["owner"]), ptr(out["bside"]),
                                ptr(out["M"]), ptr(out["Gk"]), ptr(out["Ghk"]), ptr(out["xnode"]))
    if rc != 0:
        raise MehdgError("mehdg_simplex_mesh failed (%s)" % ERRORS.get(rc, rc))
    return out


class Context:
    """One problem on one GPU; owns the library context (all blocks and workspaces)."""

    def __init__(self, prob, options=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise MehdgError("mehdg needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda:0")
        torch.cuda.set_device(self.device)
        self.stream = torch.cuda.current_stream(self.device)
        self.prob = dict(prob)
        self.options = dict(DEFAULT_OPTIONS)
        self.options.update(options or {})
        self._p = problem_struct(prob)
        self._o = options_struct(self.options)
        h = c_void_p()
        rc = self.lib.mehdg_mesh(ctypes.byref(h), ctypes.byref(self._p), 1, ctypes.byref(self._o),
                                 c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise MehdgError("mehdg_mesh failed (%s)" % ERRORS.get(rc, rc))
        self.h = h
        inf = Info()
        self._check(self.lib.mehdg_query(self.h, ctypes.byref(inf)), "query")
        self.info = {k: getattr(inf, k) for k, _ in Info._fields_}

    # -- helpers
    def _check(self, rc, what, allow=()):
        if rc != 0 and rc not in allow:
            msg = self.lib.mehdg_last_error(self.h).decode() if self.h else ""
            raise MehdgError("%s failed (%s): %s" % (what, ERRORS.get(rc, rc), msg))
        return rc

    def _ptr(self, t):
        if t is None:
            return None
        assert t.is_cuda and t.dtype == self.torch.float64 and t.is_contiguous(), "need contiguous cuda float64"
        return c_void_p(t.data_ptr())

    def empty(self, *shape):
        return self.torch.empty(*shape, dtype=self.torch.float64, device=self.device)

    def zeros(self, *shape):
        return self.torch.zeros(*shape, dtype=self.torch.float64, device=self.device)

    def state_shapes(self):
        i = self.info
        return (i["n_macro"], i["ns"], i["Np"]), (i["n_macro"], i["dim"], i["ns"], i["Np"]), (i["n_trace"],)

    def new_state(self):
        su, sq, sh = self.state_shapes()
        return self.zeros(*su), self.zeros(*sq), self.zeros(*sh)

    # -- the C ABI
    def init_state(self, du=None, duh=None, lift=False):
        u, q, uh = self.new_state()
        self._check(self.lib.mehdg_init_state(self.h, self._ptr(du), self._ptr(duh), int(lift), self._ptr(u),
                                              self._ptr(q), self._ptr(uh)), "init_state")
        return u, q, uh

    def flow_integrals(self, u, q):
        """(int rho |v|^2 / 2, int rho |curl v|^2 / 2, int 1) of the state (mehdg_flow_integrals)."""
        out = (c_double * 3)()
        self._check(self.lib.mehdg_flow_integrals(self.h, self._ptr(u), self._ptr(q), out), "flow_integrals")
        return tuple(out)

    def tgv_diagnostics(self, u, q, V0):
        """Kinetic energy per unit volume and the dissipation rate of eq. C5321 in the Taylor-Green
        scaling (rho_0 = L = 1): E_k / V0^2 and eps / (V0^3 / L), with mu = 1 / Re of the problem."""
        K, Z, V = self.flow_integrals(u, q)
        mu = 1.0 / self.prob["Re"]
        return K / V / V0 ** 2, 2.0 * mu * Z / V / V0 ** 3

    def assemble(self, u, q, uh, coef=0.0, hist=None, supg_time=0):
        norms = (c_double * 4)()
        tt = TimeTerm(float(coef), None if hist is None else hist.data_ptr(), int(supg_time))
        self._check(self.lib.mehdg_assemble_local(self.h, self._ptr(u), self._ptr(q), self._ptr(uh),
                                                  ctypes.byref(tt), norms), "assemble_local")
        return np.array(list(norms))

    def condense(self, shift=0.0, bhat=None):
        if bhat is None:
            bhat = self.empty(self.info["n_trace"])
        self._check(self.lib.mehdg_condense_factor(self.h, float(shift), self._ptr(bhat)), "condense_factor")
        return bhat

    def apply(self, x, y=None):
        y = self.empty(self.info["n_trace"]) if y is None else y
        self._check(self.lib.mehdg_apply_trace(self.h, self._ptr(x), self._ptr(y)), "apply_trace")
        return y

    def precondition(self, kind, r, z=None):
        z = self.empty(self.info["n_trace"]) if z is None else z
        self._check(self.lib.mehdg_precondition(self.h, int(kind), self._ptr(r), self._ptr(z)), "precondition")
        return z

    def linear_solve(self, b, x=None, allow_not_converged=False):
        x = self.empty(self.info["n_trace"]) if x is None else x
        st = SolveStats()
        allow = (-5,) if allow_not_converged else ()
        self._check(self.lib.mehdg_linear_solve(self.h, self._ptr(b), self._ptr(x), ctypes.byref(st)),
                    "linear_solve", allow)
        return x, st.as_dict()

    def recover(self, duh):
        su, sq, _ = self.state_shapes()
        du, dq = self.empty(*su), self.empty(*sq)
        self._check(self.lib.mehdg_recover(self.h, self._ptr(duh), self._ptr(du), self._ptr(dq)), "recover")
        return du, dq

    def dirk_stage(self, stage, dt, u, q, uh, allow_not_converged=False):
        st = SolveStats()
        allow = (-5,) if allow_not_converged else ()
        self._check(self.lib.mehdg_dirk_stage(self.h, int(stage), float(dt), self._ptr(u), self._ptr(q),
                                              self._ptr(uh), ctypes.byref(st)), "dirk_stage", allow)
        return st.as_dict()

    def stage_begin(self, stage, dt, u, q, uh):
        st = SolveStats()
        self._check(self.lib.mehdg_stage_begin(self.h, int(stage), float(dt), self._ptr(u), self._ptr(q),
                                               self._ptr(uh), ctypes.byref(st)), "stage_begin")
        d = st.as_dict()
        d["converged"] = bool(st.status & 2)
        return d

    def newton_step(self, u, q, uh):
        st = SolveStats()
        self._check(self.lib.mehdg_newton_step(self.h, self._ptr(u), self._ptr(q), self._ptr(uh),
                                               ctypes.byref(st)), "newton_step")
        d = st.as_dict()
        d["converged"] = bool(st.status & 2)
        return d

    def stage_end(self, u):
        self._check(self.lib.mehdg_stage_end(self.h, self._ptr(u)), "stage_end")

    def get_block(self, which, macro):
        n = c_longlong()
        self._check(self.lib.mehdg_get_block(self.h, int(which), int(macro), None, ctypes.byref(n)), "get_block")
        out = np.empty(n.value, dtype=np.float64)
        self._check(self.lib.mehdg_get_block(self.h, int(which), int(macro), out.ctypes.data_as(c_void_p), None),
                    "get_block")
        return out

    PHASES = ["vol_point", "vol_contract", "faces", "condense", "lu", "face_lu", "bhat", "apply", "recover",
              "precond", "form_local", "apply_bf16", "cond_gemm", "trsm"]

    def phase_times(self):
        """Device milliseconds of the last run of each internal phase (dict)."""
        out = (c_double * 16)()
        self._check(self.lib.mehdg_phase_times(self.h, out, 16), "phase_times")
        return {k: out[i] for i, k in enumerate(self.PHASES)}

    # -- learned preconditioner correction (kind 2)
    def phase_stats(self, reset=False):
        """Cumulative device milliseconds and execution counts of each internal phase since
        the context was made or the last reset: {name: (ms, count)}."""
        ms, cnt = (c_double * 16)(), (c_longlong * 16)()
        self._check(self.lib.mehdg_phase_stats(self.h, ms, cnt, 16, int(reset)), "phase_stats")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.PHASES)}

    def set_precond(self, kind):
        self._check(self.lib.mehdg_set_precond(self.h, int(kind)), "set_precond")
        self.options["precond"] = int(kind)

    def mlp_setup(self, hidden=256, seed=0, max_pairs=400, neighbors=0):
        self._check(self.lib.mehdg_mlp_setup(self.h, int(hidden), int(seed), int(max_pairs), int(neighbors)),
                    "mlp_setup")
        n = c_longlong()
        self._check(self.lib.mehdg_mlp_params(self.h, 0, None, ctypes.byref(n)), "mlp_params")
        self.mlp_nparams = n.value
        self.mlp_nout = ((self.info["ns"] * self.info["Nfn"] + 31) // 32) * 32
        nf = self.info["Nth"] // self.info["Nfn"]          # faces per macro-element
        self.mlp_nin = (2 + (2 * (nf - 1) if neighbors else 0)) * self.mlp_nout
        self.mlp_hidden = int(hidden)

    def mlp_params(self, values=None):
        """Get (values None) or set the packed FP32 master parameters (numpy float32)."""
        if values is None:
            out = np.empty(self.mlp_nparams, dtype=np.float32)
            self._check(self.lib.mehdg_mlp_params(self.h, 0, out.ctypes.data_as(c_void_p), None), "mlp_params")
            return out
        v = np.ascontiguousarray(values, dtype=np.float32)
        self._check(self.lib.mehdg_mlp_params(self.h, 1, v.ctypes.data_as(c_void_p), None), "mlp_params")

    def mlp_record(self, r, e):
        self._check(self.lib.mehdg_mlp_record(self.h, self._ptr(r), self._ptr(e)), "mlp_record")

    def mlp_set_recording(self, on):
        n = c_int()
        self._check(self.lib.mehdg_mlp_set_recording(self.h, int(bool(on)), ctypes.byref(n)), "mlp_set_recording")
        return n.value

    def mlp_gradient(self, X, T):
        """Loss and gradient for device float32 tensors X [n][n_in], T [n][n_out]."""
        assert X.dtype == self.torch.float32 and T.dtype == self.torch.float32 and X.is_contiguous()
        g = np.empty(self.mlp_nparams, dtype=np.float32)
        loss = c_double()
        self._check(self.lib.mehdg_mlp_gradient(self.h, c_void_p(X.data_ptr()), c_void_p(T.data_ptr()),
                                                int(X.shape[0]), g.ctypes.data_as(c_void_p), ctypes.byref(loss)),
                    "mlp_gradient")
        return loss.value, g

    def mlp_train(self, epochs=200, batch=4096, lr=1e-3):
        out = (c_double * 2)()
        self._check(self.lib.mehdg_mlp_train(self.h, int(epochs), int(batch), float(lr), out), "mlp_train")
        return out[0], out[1]

    def graph_replays(self):
        """Replays of the inner-GMRES CUDA graph (0 on the legacy default stream: no capture)."""
        n = c_longlong(0)
        self._check(self.lib.mehdg_graph_replays(self.h, ctypes.byref(n)), "graph_replays")
        return n.value

    def launch_count(self):
        n = c_longlong()
        self._check(self.lib.mehdg_launch_count(self.h, ctypes.byref(n)), "launch_count")
        return n.value

    @classmethod
    def _borrow(cls, handle, prob, options, device):
        """A Context view of a context owned by a Batch (not destroyed by close())."""
        import torch
        self = cls.__new__(cls)
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device(device or "cuda:0")
        self.stream = torch.cuda.current_stream(self.device)
        self.prob = dict(prob)
        self.options = dict(DEFAULT_OPTIONS)
        self.options.update(options or {})
        self.h = c_void_p(handle)
        self.owned = False
        inf = Info()
        self._check(self.lib.mehdg_query(self.h, ctypes.byref(inf)), "query")
        self.info = {k: getattr(inf, k) for k, _ in Info._fields_}
        return self

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "owned", True):
                self.lib.mehdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent problems of uneven size solved together on one GPU (mehdg_batch_*): one
    context per problem (reachable as .contexts[i]), lockstep steady Newton rounds whose
    assembly and condensation run as CUDA-graph replays, the local LU of all problems in one
    persistent work-queue launch with autotuned panel widths."""

    def __init__(self, probs, options=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise MehdgError("mehdg needs a CUDA device (no CPU fallback)")
        self.lib = load_library()
        self.device = torch.device(device or "cuda:0")
        torch.cuda.set_device(self.device)
        self.stream = torch.cuda.current_stream(self.device)
        n = len(probs)
        opts = options if isinstance(options, (list, tuple)) else [options] * n
        self._opts = [dict(DEFAULT_OPTIONS, **(o or {})) for o in opts]
        self._p = (Problem * n)(*[problem_struct(p) for p in probs])
        self._o = (Options * n)(*[options_struct(o) for o in self._opts])
        h = c_void_p()
        rc = self.lib.mehdg_batch_create(ctypes.byref(h), self._p, n, self._o, c_void_p(self.stream.cuda_stream))
        if rc != 0:
            raise MehdgError("mehdg_batch_create failed (%s)" % ERRORS.get(rc, rc))
        self.h = h
        self.contexts = [Context._borrow(self.lib.mehdg_batch_context(self.h, i), probs[i], self._opts[i],
                                         self.device) for i in range(n)]

    def steady_solve(self, states, allow_not_converged=False):
        """states: list of (u, q, uh) CUDA float64 tensors, updated in place.  Returns (per-problem
        statistics, lockstep rounds).  allow_not_converged: return the statistics (each with its
        'converged' flag) instead of raising when some problem did not converge."""
        n = len(self.contexts)
        U = (c_void_p * n)(*[s[0].data_ptr() for s in states])
        Q = (c_void_p * n)(*[s[1].data_ptr() for s in states])
        H = (c_void_p * n)(*[s[2].data_ptr() for s in states])
        st = (SolveStats * n)()
        rounds = c_int(0)
        rc = self.lib.mehdg_batch_steady_solve(self.h, U, Q, H, st, ctypes.byref(rounds))
        if rc != 0 and not (allow_not_converged and rc == -5):
            raise MehdgError("mehdg_batch_steady_solve failed (%s): %s"
                             % (ERRORS.get(rc, rc), self.lib.mehdg_batch_last_error(self.h).decode()))
        out = []
        for s in st:
            d = s.as_dict()
            d["converged"] = bool(s.status & 2)
            out.append(d)
        return out, rounds.value

    def tiles(self):
        """The autotuner's record: [(n, fp64, chosen panel width, {width: sample ms})]."""
        k = self.lib.mehdg_batch_tiles(self.h, 0, None, None, None, None)
        n_, f_, nb_ = (c_int * k)(), (c_int * k)(), (c_int * k)()
        ms = (c_double * (3 * k))()
        self.lib.mehdg_batch_tiles(self.h, k, n_, f_, nb_, ms)
        return [(n_[i], bool(f_[i]), nb_[i], {w: ms[3 * i + j] for j, w in enumerate((8, 16, 32)) if ms[3 * i + j] >= 0})
                for i in range(k)]

    def graph_replays(self):
        return int(self.lib.mehdg_batch_graph_replays(self.h))

    def close(self):
        if getattr(self, "h", None):
            for c in self.contexts:
                c.h = None
            self.lib.mehdg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
