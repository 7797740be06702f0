/*
 * mehdg.h -- C ABI of the GB300 matrix-free macro-element HDG solver for the
 * compressible Navier-Stokes equations (Badrkhani, ten Eikelder, Hiemstra,
 * Schillinger, arXiv 2402.11361).
 *
 * Conventions for every call
 *  - Return value: MEHDG_OK (0) or a negative MEHDG_ERR_* code; the message of the
 *    last failure is kept in the context (mehdg_last_error).  No call aborts.
 *  - Pointers named u, q, uhat, x, y, r, z, bhat, du, dq, duhat, hist are DEVICE
 *    pointers owned by the caller, contiguous FP64, in the layouts below.
 *    Pointers documented as "host" are host memory.
 *  - The context owns every internal block and workspace (allocated once in
 *    mehdg_mesh, released by mehdg_destroy).
 *  - All calls are ordered on the CUDA stream given to mehdg_mesh.  Calls that
 *    return scalars to the host (norms, statistics) synchronise that stream.
 *
 * Data layout (one problem; E macro-elements, F macro-faces, d = dim, ns = d+2):
 *  - box meshes (mesh_kind MEHDG_MESH_BOX): macro-elements are boxes; macro
 *    e = ix + nx (iy + ny iz); the shell mesh is described at MEHDG_MESH_SHELL;
 *  - Np = (m p + 1)^d C0 nodes per macro-element, lexicographic, x fastest;
 *  - Nfn = (m p + 1)^(d-1) nodes per macro-face, Nth = 2 d Nfn per macro-element;
 *  - u     [E][ns][Np]       conserved variables (rho, rho v, rho E)
 *  - q     [E][d][ns][Np]    gradient, q[e][k][s] = d u_s / d x_k
 *  - uhat  [F][ns][Nfn]      trace (hybrid) variable; this is also the layout of
 *                            every global trace vector (x, y, r, z, bhat, duhat)
 *  - faces: all x-normal, then y-normal, then z-normal macro-faces; within the
 *    k-normal group index = pos + npos_k * (tangential macro index, lower axis
 *    fastest), npos_k = n_k (periodic) or n_k + 1; face nodes lexicographic in
 *    the tangential axes, lower axis fastest;
 *  - local faces of a macro-element are ordered (-x, +x, -y, +y, -z, +z); a
 *    macro's local trace vector is species-major [ns][(local face, face node)].
 *  - simplicial meshes (MEHDG_MESH_SIMPLEX, the paper's element type, Sec. 2.2): every box
 *    cell is split into d! macro-elements x = C + H P_sigma xi over the Kuhn simplex
 *    K = {1 >= xi_1 >= ... >= xi_d >= 0}, macro e = cell d! + (rank of the axis order sigma in
 *    lexicographic order), cell index x fastest; each macro is refined m times into m^d
 *    sub-simplices carrying P_p; Np = C(m p + d, d) nodes a / (m p), m p >= a_1 >= ... >= a_d
 *    >= 0 (lexicographic, a_d fastest); d + 1 local faces xi_1 = 1, xi_k = xi_{k+1},
 *    xi_d = 0, Nfn = C(m p + d - 1, d - 1) nodes each (the face's lattice points), Nth =
 *    (d + 1) Nfn; faces numbered in order of first appearance over (macro, local face), a
 *    face's nodes in its first owner's order.  Supported with precision FP64, apply_mode 0,
 *    tc_mode 0, condense_layers 2 and m p <= 6.
 */
#ifndef MEHDG_H
#define MEHDG_H

#ifdef __cplusplus
extern "C" {
#endif

#define MEHDG_OK 0
#define MEHDG_ERR_ARG (-1)
#define MEHDG_ERR_CUDA (-2)
#define MEHDG_ERR_OOM (-3)
#define MEHDG_ERR_SINGULAR (-4)
#define MEHDG_ERR_NOT_CONVERGED (-5)
#define MEHDG_ERR_TIMEOUT (-6)
#define MEHDG_ERR_NAN (-7)
#define MEHDG_ERR_TOO_LARGE (-8)

/* boundary kinds per domain side (-x, +x, -y, +y, -z, +z) */
#define MEHDG_BC_NONE 0      /* periodic direction (or unused) */
#define MEHDG_BC_DIRICHLET 1 /* B^ = uhat - u_D, u_D from the problem's field */
#define MEHDG_BC_WALL 2      /* isothermal no-slip wall at wall_T moving at wall_v */
#define MEHDG_BC_FARFIELD 3  /* characteristic far field: B^ = A_n^+(uhat)(u - uhat) - A_n^-(uhat)
                                (u_inf - uhat), A_n^+- = (A_n +- |A_n|_delta) / 2 with the
                                eigenvalue magnitudes smoothed as sqrt(lambda^2 + (0.05 c)^2);
                                u_inf is the uniform state of field_par (rho, v1, v2, v3, T).
                                The paper's boundary operator of Sec. 2.3 leaves B^ open; this
                                is the characteristic reading */

/* closed-form fields (Dirichlet data, source term, initial state) */
#define MEHDG_FIELD_NONE 0
#define MEHDG_FIELD_MMS 1     /* par: rho amplitude, velocity amplitude, pressure amplitude */
#define MEHDG_FIELD_UNIFORM 2 /* par: rho, v1, v2, v3, T */
#define MEHDG_FIELD_TGV 3     /* par: V0 (Mach of the vortex) */
#define MEHDG_FIELD_COUETTE3D 5 /* compressible Couette flow with a source term (Sec. 5.1, eq. CF0), in acoustic
                                 units: v_1 = M x_2 log(1 + x_2), v_2 = v_3 = 0, T = a + x_2 (b - a)
                                 + K x_2 (1 - x_2), P = 1/gamma (rho = 1/T); par: M, a, b, K; the
                                 source term is the divergence of the fluxes of this state */
#define MEHDG_FIELD_SPHERE 4  /* par as UNIFORM (the free stream, also the Dirichlet and far-field
                                 state); initial state: the free stream with the velocity times
                                 3 s^2 - 2 s^3, s = clamp((|x| - 0.6) / 0.4, 0, 1) */

/* mesh kinds */
#define MEHDG_MESH_BOX 0      /* nmac, lo, hi, periodic: a box of box macro-elements */
#define MEHDG_MESH_SIMPLEX 2  /* nmac, lo, hi, periodic: each box cell split into d! simplicial
    macro-elements (the Kuhn triangulation), each refined m times into m^d sub-simplices with P_p
    (the data-layout notes above give the numbering).  Boundary sides as on box meshes (the planes
    x_k = lo_k, hi_k).  SUPG length h = min_k (hi_k - lo_k) / nmac_k / m.  Supported with precision
    FP64, apply_mode 0, tc_mode 0, condense_layers 2 and m p <= 6; mehdg_flow_integrals refuses
    these meshes. */
#define MEHDG_MESH_SHELL 1    /* dim 3: cubed-sphere O-grid of the shell r0 <= |x| <= r1 (flow past a
    sphere).  E = 6 nq^2 nr curved macro-elements; macro e = ((panel nr + k) nq + j) nq + i for the
    cube panels (+x, -x, +y, -y, +z, -z) with frames (e_n, e_1, e_2) = (x, y, z), (-x, z, y),
    (y, z, x), (-y, x, z), (z, x, y), (-z, y, x); macro reference axes xi_0 along e_1, xi_1 along
    e_2, xi_2 outward.  The macro node with macro-lattice coordinates t in [0, 1]^3 sits at
    R(k + t_2) dir / |dir|, dir = e_n + tan(a) e_1 + tan(b) e_2, a = -pi/4 + (i + t_0) pi / (2 nq),
    b = -pi/4 + (j + t_1) pi / (2 nq), R(s) = r0 + (r1 - r0) (ratio^s - 1) / (ratio^nr - 1)
    (linear when ratio == 1); the geometry inside each macro is the isoparametric interpolant of
    its nodes (per-point Jacobians, per-macro mass matrix M_J).  Faces are numbered in order of
    first appearance over (macro, local face); a face's node order is its first owner's
    (lexicographic in that owner's tangential axes); the gather map of the second owner carries
    the permutation found by matching node positions.  Boundary sides: bc[0], wall_T[0],
    wall_v[0] for the inner sphere, bc[1] for the outer sphere.  SUPG length h = min(R(1) - r0,
    r0 pi / (2 nq)) / m.  Supported with condense_layers 2, tc_mode 0, 1, 4 or 5 and m p <= 4. */

#define MEHDG_PREC_FP64 0   /* every block and solve in FP64 */
#define MEHDG_PREC_MIXED 1  /* FP32 blocks, TF32 tensor-core condensation and LU,
                               FP64 residuals, Krylov vectors and refinement */

typedef struct mehdg_problem {
  int dim;            /* 2 or 3 */
  int m, p;           /* sub-elements per macro edge, polynomial degree */
  int nmac[3];        /* macro-elements per direction */
  double lo[3], hi[3];
  int periodic[3];
  int bc[6];
  double wall_T[6];
  double wall_v[6][3];
  double gamma, Re, Pr; /* Re is the acoustic Reynolds number Re_c (Sec. 2.1) */
  int supg;           /* 1: SUPG term of eq. C38b on */
  int field;          /* MEHDG_FIELD_* */
  double field_par[8];
  int mesh_kind;      /* MEHDG_MESH_* (0: box) */
  int shell_n[2];     /* shell: nq cells per cube-panel edge, nr radial layers */
  double shell_r[3];  /* shell: inner radius r0, outer radius r1, layer thickness ratio */
} mehdg_problem;

typedef struct mehdg_options {
  int precision;      /* MEHDG_PREC_* */
  int precond;        /* 0 block-Jacobi (A_uhuh)^-1, 1 multi-level (inner GMRES + block-Jacobi),
                         2 block-Jacobi + learned MLP correction */
  int restart;        /* FGMRES restart length */
  int max_iters;      /* FGMRES iteration cap per linear solve */
  double lin_rtol, lin_atol;
  int inner_iters;    /* inner GMRES iterations of precond 1 */
  double newton_rtol, newton_atol;
  int max_newton;
  double tau_init, tau_max; /* pseudo-time SER parameters (eq. C31222) */
  int refine_iters;   /* FP64 refinement sweeps of each local S solve (mixed precision) */
  int apply_mode;     /* 0: Algorithm 2 (C, S^-1, B, D per apply); 1: the local operator
                         A^T_i = B S^-1 C + D is formed once after factorisation (it
                         replaces D in place) and each apply is one product per macro */
  int tc_mode;        /* mixed precision dense local work: 0 FP32 SIMT; 1 batched LU of S
                         with tcgen05 trailing updates in split TF32 (3 products, about
                         FP32 accuracy); 2 also the condensation products and forming
                         A^T_i in split TF32; 3 as 2 with plain TF32; 4 forming A^T_i =
                         D + B (S^-1 C) on tcgen05 with operands staged K-major in the
                         128-byte-swizzled layout (split TF32), LU and substitutions SIMT;
                         5 as 0 with the dense (not sum-factorised) volume contraction */
  int precond_bf16;   /* apply_mode 1 with precond 1: the inner GMRES of the multi-level
                         preconditioner applies a BF16 copy of A^T_i (half the bytes of
                         the FP32 operator; FGMRES allows the inexact preconditioner),
                         the outer FGMRES keeps the FP32/FP64 operator.  In the mixed
                         path the face-block inverses get a BF16 copy too, and the
                         inner block-Jacobi product reads the apply's per-macro results
                         directly (the face sum is done inside it) */
  int solver;         /* 0: FGMRES right-preconditioned by the option precond (flexible,
                         Sec. 4.2); 1: GMRES left-preconditioned by the macro-face
                         block-Jacobi (A_uhuh)^-1, the paper's baseline of Sec. 4.2 (Table 2);
                         its tolerance applies to the preconditioned residual |M^-1 r| */
  int condense_layers; /* 2 (or 0): second-layer static condensation, eqs. AP12 and ASC2 (the
                         paper's method); 1: one-layer condensation of eqs. C46-C47, the whole
                         local matrix [A_qq A_qu; A_uq A_uu] factored per macro-element, for
                         comparison (paper's Table 4); needs precision FP64, apply_mode 1 and
                         32 (d + 1) Nu doubles of shared memory (2D and 3D p = 1) */
} mehdg_options;

typedef struct mehdg_info {
  int dim, ns, Np, Nfn, Nth, Nu, Nq, Nt;
  int n_macro, n_face;
  long long n_trace;        /* F * ns * Nfn */
  long long bytes_device;   /* bytes held by the context */
} mehdg_info;

typedef struct mehdg_time_term {
  double coef;         /* d_ii / dt for a DIRK stage (eq. C242), 0 for steady */
  const double* hist;  /* device [E][ns][Np] nodal history term or NULL */
  int supg_time;       /* 1: the time term enters the SUPG strong residual */
} mehdg_time_term;

typedef struct mehdg_solve_stats {
  int newton_steps;
  int fgmres_iters;     /* summed over the Newton steps of the call */
  double res0, res;     /* |R_F| at entry and exit */
  double t_assemble, t_condense, t_krylov, t_recover; /* seconds (device events) */
  int status;
} mehdg_solve_stats;

typedef struct mehdg_ctx mehdg_ctx;

/* a0 -- macro-element mesh, DOF maps and reference operators (Sec. 2.2; the
 * gather map eps of Algorithm 2 "Extract global DOF indices on dT_i").
 * prob: host array of nprob problem descriptions (nprob == 1 in this version).
 * opt: host, may be NULL for defaults.  stream: cudaStream_t or NULL.
 * On success *ctx owns all device memory of the problem.  Errors: ARG for an
 * invalid description, OOM when device memory is short, CUDA otherwise. */
int mehdg_mesh(mehdg_ctx** ctx, const mehdg_problem* prob, int nprob,
               const mehdg_options* opt, void* stream);

/* sizes of the discrete spaces; info is host memory */
int mehdg_query(const mehdg_ctx* ctx, mehdg_info* info);

/* Initial state: u = closed-form field at the nodes + du_pert, q = 0 (or the
 * lifted gradient when lift != 0, i.e. q solving R_Q = 0), uhat = trace of the
 * owning macro-element's u + duh_pert.  du_pert [E][ns][Np] and duh_pert
 * [F][ns][Nfn] are device pointers or NULL. */
int mehdg_init_state(mehdg_ctx* ctx, const double* du_pert, const double* duh_pert,
                     int lift, double* u, double* q, double* uhat);

/* Inspection of the simplicial reference macro-element (Sec. 2.2), host only (no device
 * needed): the tables of the m-refined Kuhn simplex with P_p sub-elements that simplicial
 * meshes use.  counts (host int[8], required): Np, Nfn, nel (sub-simplices), ng (points per
 * sub-simplex), nloc (nodes per sub-simplex), nsf (sub-faces per face), nfp (points per
 * sub-face), nfs (nodes per sub-face).  The other host arrays may be NULL: lattice [Np][d]
 * integer node coordinates (spacing 1 / (m p)); vxi [nel ng][d] volume points in K and vw
 * [nel ng] their weights; vtab [nel ng][nloc][d + 1] values and d/dxi of the point's
 * sub-simplex basis; vnode [nel][nloc] their macro nodes; fnodes [d + 1][Nfn] macro node of
 * each face node; fxi [d + 1][nsf nfp][d] face points in K and fwt [d + 1][nsf nfp] their
 * weights in face coordinates.  Errors: ARG (d not 2 or 3, p not 1..3, m p > 12). */
int mehdg_simplex_reference(int d, int m, int p, int* counts, int* lattice, double* vxi, double* vw,
                            double* vtab, int* vnode, int* fnodes, double* fxi, double* fwt);

/* Inspection of a simplicial mesh, host only (no device needed): prob a MEHDG_MESH_SIMPLEX
 * description.  counts (host int[5], required): E, F, Np, Nfn, Nth.  The other host arrays may
 * be NULL: gather [E][Nt] (the map eps of Algorithm 2), owner [F][2] (e (d + 1) + local face,
 * -1 for none; the first owner orders the face's nodes), bside [E][d + 1] (boundary side or
 * -1), the per-macro mass and lifting matrices M [E][Np][Np], Gk [E][d][Np][Np], Ghk
 * [E][d][Np][Nth] (A_qq, A_qu, A_quh per species, Sec. 3.3) and xnode [E][d][Np] node
 * positions.  Errors: ARG (invalid description, m p > 6). */
int mehdg_simplex_mesh(const mehdg_problem* prob, int* counts, int* gather, int* owner, int* bside, double* M,
                       double* Gk, double* Ghk, double* xnode);

/* Taylor-Green diagnostics (Sec. 5.3, eq. C5321) of a state, by the volume quadrature of the
 * method (the Gauss points of every sub-element; the curved weights on shell meshes):
 * out[0] = int rho |v|^2 / 2, out[1] = int rho (omega . omega) / 2, out[2] = int 1, with
 * v = m / rho and omega = curl v (2D: the scalar d_1 v_2 - d_2 v_1) taken from the HDG
 * gradient, d_j v_i = (q_{j,1+i} - v_i q_{j,0}) / rho.  The dissipation rate of eq. C5321 is
 * eps = 2 mu out[1] / out[2] (mu = 1 / Re in the problem's units), the kinetic energy per
 * unit volume out[0] / out[2].  u [E][ns][Np] and q [E][d][ns][Np]: device state (FP64 in
 * both precisions), read only; out: host double[3].  The sums run in a fixed order (the
 * same state gives the same bits).  Synchronises the context's stream.  Errors: ARG (null
 * pointer), CUDA. */
int mehdg_flow_integrals(mehdg_ctx* ctx, const double* u, const double* q, double* out);

/* a1-a2 -- residuals R_Q, R_U, R_Uhat (eq. C31221 from C38 / C242) and the Newton
 * blocks of eq. C312 of every macro-element at (u, q, uhat).  tt may be NULL
 * (steady).  res_norms: host double[4] = |R_Q|, |R_U|, |R_Uhat|, |R_F| (global
 * l2 norms; R_Uhat summed over both sides of each face) or NULL. */
int mehdg_assemble_local(mehdg_ctx* ctx, const double* u, const double* q,
                         const double* uhat, const mehdg_time_term* tt,
                         double* res_norms);

/* a3-a6 -- second-layer static condensation (eqs. AP12, ASC2): S, B, C, D of every
 * macro-element, LU factorisation of S with partial pivoting (Remark, Sec. 3.3),
 * and the condensed right-hand side b^ = sum_i eps_i^T (h_i - B_i S_i^{-1} g_i)
 * (Algorithm 1, lines 2-5) written to bhat (device, global trace layout).
 * shift adds shift * (I (x) M) to A_uu (pseudo-time term).  Also factors the
 * macro-face blocks of A_uhuh used by mehdg_precondition.
 * Errors: SINGULAR when a pivot is exactly zero (message names the macro). */
int mehdg_condense_factor(mehdg_ctx* ctx, double shift, double* bhat);

/* a7 -- matrix-free y = A^ x (Algorithm 2): per macro-element gather x on dT_i,
 * y1 = C x, y2 = S^{-1} y1, y3 = B y2, y4 = y3 + D x, then the face reduction
 * (step 4).  x and y are global trace vectors (device), x != y. */
int mehdg_apply_trace(mehdg_ctx* ctx, const double* x, double* y);

/* a9 -- z = P^{-1} r (Sec. 4.2): kind 0 block-Jacobi with the macro-face blocks of
 * A_uhuh, kind 1 inner GMRES on A^ left-preconditioned by kind 0 (multi-level),
 * kind 2 kind 0 plus the learned correction.  r != z. */
int mehdg_precondition(mehdg_ctx* ctx, int kind, const double* r, double* z);

/* a8 -- FGMRES (right, flexible) on A^ duhat = bhat with the options' preconditioner,
 * CGS2 orthogonalisation in FP64 (Sec. 4.2).  stats: host or NULL.
 * Returns NOT_CONVERGED when the iteration cap is reached (duhat holds the last iterate). */
int mehdg_linear_solve(mehdg_ctx* ctx, const double* bhat, double* duhat,
                       mehdg_solve_stats* stats);

/* a10 -- local recovery (eqs. Csc4a then Csc4b): du = S^{-1}(g + C duhat_i),
 * dq = A_qq^{-1}(-R_Q - A_qu du - A_quh duhat_i). */
int mehdg_recover(mehdg_ctx* ctx, const double* duhat, double* du, double* dq);

/* a11/a12 -- nonlinear solve.  stage 0: steady pseudo-transient Newton with SER
 * (eq. C31222) to the options' tolerance.  stage i = 1..3: stage i of the
 * 3-stage DIRK (eq. C242, Alexander's stiffly accurate scheme) with step dt;
 * stage 1 records u as u^n; after stage 3, u holds u^{n+1}.  u, q, uhat are
 * updated in place (device).  stats: host or NULL. */
int mehdg_dirk_stage(mehdg_ctx* ctx, int stage, double dt, double* u, double* q,
                     double* uhat, mehdg_solve_stats* stats);

/* a11/a12 one Newton step at a time: the three calls mehdg_dirk_stage is made of, for
 * callers that drive, interleave or time the nonlinear iteration step by step (Sec. 3.1:
 * each Newton step is the linear solve of eq. C312 by Algorithm 1 plus the state update).
 * mehdg_stage_begin: start the system of stage i = 1..3 of the DIRK step (eq. C242; stage 1
 *   records u as u^n, later stages use the stage values stored by mehdg_stage_end) or, for
 *   stage 0, the steady pseudo-transient system (dtau = tau_init); assembles at (u, q, uhat).
 *   stats->res0 = stats->res = |R_F| there.
 * mehdg_newton_step: one Newton step of the begun stage: condensation and LU, FGMRES,
 *   recovery, the update of u, q, uhat in place and the assembly at the new state (and, for
 *   stage 0, the SER update of dtau).  stats: fgmres_iters of this step, res = the new |R_F|.
 * For both, stats->status bit 1 (value 2) is set when |R_F| <= max(newton_rtol |R_F^0|,
 * newton_atol) with R_F^0 the residual at mehdg_stage_begin: the stage has converged.
 * mehdg_stage_end: store u as the stage value u^{n,i} (stage >= 1) and close the stage.
 * All three synchronise the stream.  Errors: ARG (bad arguments, a step or end without a
 * begun stage), NAN (non-finite residual), and those of the phases they run. */
int mehdg_stage_begin(mehdg_ctx* ctx, int stage, double dt, double* u, double* q, double* uhat,
                      mehdg_solve_stats* stats);
int mehdg_newton_step(mehdg_ctx* ctx, double* u, double* q, double* uhat, mehdg_solve_stats* stats);
int mehdg_stage_end(mehdg_ctx* ctx, const double* u);

/* Copy one internal per-macro array to host memory (test access).  which:
 * 0 A_uu/S (after condensation: LU factors), 1..3 A_uq_k, 4 A_uuh/C, 5 A_uhu/B,
 * 6..8 A_uhq_k, 9 A_uhuh/D, 10 R_Q, 11 R_U, 12 R_Uhat (local), 13 g, 14 h,
 * 15 pivots (as doubles), 16 bhat_local, 17 the unfactored S kept for the FP64
 * refinement of the local solves (mixed precision with refine_iters > 0).  Returns
 * the element count in *count. */
int mehdg_get_block(mehdg_ctx* ctx, int which, int macro, double* host_out,
                    long long* count);

/* Trace apply for callers that cannot allocate device memory.  No counterpart in
 * the paper: it is the a7 apply (same kernels, same result as mehdg_apply_trace)
 * with every array supplied by the caller and the one scratch array it needs
 * (one result slot of Nt doubles per macro-element, summed per face afterwards)
 * taken from a fixed array compiled into this library.
 *
 * Who needs it: code that runs inside a host application that owns all device
 * memory through its own pool or arena and gives a solver plugin a fixed budget,
 * and loops that must not call cudaMalloc, which can stall or implicitly
 * synchronise the device.  This call allocates nothing: no cudaMalloc, no cudaFree,
 * no allocating library routine.
 *
 * Arguments (device pointers unless stated): dim 2 or 3 (ns = dim + 2,
 * Nth = 2 dim Nfn, Nt = ns Nth); n_macro, n_face, Nu = ns Np, Nfn as in mehdg_info;
 * S_lu [n_macro][Nu][Nu] LU factors of S with unit lower L (row-major) and perm
 * [n_macro][Nu] the row permutation (row i of P S is row perm[i] of S); B
 * [n_macro][Nt][Nu], C [n_macro][Nu][Nt], D [n_macro][Nt][Nt]; gather [n_macro][Nt]
 * global trace index of each local trace entry; owner [n_face][2] the touching
 * (macro * 2 dim + local face) or -1; x, y global trace vectors (n_face ns Nfn),
 * x != y; stream a cudaStream_t or NULL.  All in the layouts of this header.  The
 * face sum reads both owners' entries in the face's node order, so it serves meshes
 * whose two owners of a face order its nodes alike (the box meshes); on the shell
 * mesh use mehdg_apply_trace.
 *
 * Limits and sharing: n_macro * Nt must not exceed 4194304 (2^22) doubles, the size
 * of the fixed scratch array (32 MiB, held on every GPU that loads the library
 * until the process exits); larger sizes return MEHDG_ERR_TOO_LARGE with a message
 * on stderr.  Every call on a device uses the same array and leaves its contents
 * behind; each call overwrites every entry it reads, so nothing has to start at
 * zero.  Calls that overlap on the GPU (other streams, other threads) race on the
 * array: order them on one stream.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress with that device current); make that
 * first call before any stream capture begins.  The looked-up address is kept for the
 * life of the process and does not survive cudaDeviceReset of that device.  Shared memory:
 * Nt + 2 Nu doubles per block plus the kernel's static part must fit the device's
 * per-block limit (ARG otherwise).  Errors: ARG for invalid sizes or
 * pointers, TOO_LARGE as above, CUDA for a failed lookup or launch. */
int mehdg_apply_trace_noalloc(int dim, int n_macro, int n_face, int Nu, int Nfn,
                              const double* S_lu, const int* perm, const double* B,
                              const double* C, const double* D, const int* gather,
                              const int* owner, const double* x, double* y, void* stream);

/* Learned preconditioner correction (preconditioner kind 2).  No counterpart in the
 * paper (spec addition): FGMRES tolerates a variable preconditioner (Sec. 4.2),
 * so the block-Jacobi output z0 is corrected face by face,
 *   z_f = z0_f + |z0_f| MLP(r_f/|r_f|, z0_f/|z0_f| [, z0_g/|z0_f| for the other faces g of
 *                                                   the face's owner macro-elements]),
 * by a network n_in -> hidden (ReLU) -> hidden (ReLU) -> n_out (n_out = ns Nfn rounded up
 * to 32, n_in = 2 n_out, or (2 + 2 (2d - 1)) n_out with neighbors != 0; absent neighbours
 * of boundary faces are zeros) with BF16 weights, FP32 biases and FP32 accumulation.
 * mehdg_mlp_setup: allocate with seeded weights and room for max_pairs pairs.
 * mehdg_mlp_params: copy the FP32 master parameters to (set = 0) or from (set = 1)
 *   host memory, packed [W1 (h x n_in), b1, W2 (h x h), b2, W3 (n_out x h), b3];
 *   *count receives the length.
 * mehdg_mlp_record: store one (residual r, error e) pair of global trace vectors as
 *   one sample per face (inputs as above, target (e_f - z0_f)/|z0_f|).  mehdg_mlp_set_recording(on): FGMRES then records up to 8
 *   pairs per converged solve (iterates of its last cycle against its solution).
 * mehdg_mlp_gradient: mean-squared loss and gradient (host float[count]) for n rows
 *   of device inputs X [n][n_in] and targets T [n][n_out].
 * mehdg_mlp_train: epochs of Adam over the recorded samples in minibatches; losses
 *   (host double[2]) receives the mean loss of the first and last epoch.
 * In kind-2 solves FGMRES falls back to kind 1 when its residual falls by less than
 * 10x over 20 iterations (stats->status bit 0). */
/* Switch the preconditioner kind (0, 1, 2 as in mehdg_precondition) used by later
 * mehdg_linear_solve / mehdg_dirk_stage calls of this context, e.g. to compare the
 * learned correction with the multi-level preconditioner on one resident problem.
 * Kind 2 needs mehdg_mlp_setup first.  Returns MEHDG_ERR_ARG otherwise. */
int mehdg_set_precond(mehdg_ctx* ctx, int kind);
int mehdg_mlp_setup(mehdg_ctx* ctx, int hidden, unsigned long long seed, int max_pairs, int neighbors);
int mehdg_mlp_params(mehdg_ctx* ctx, int set, float* host, long long* count);
int mehdg_mlp_record(mehdg_ctx* ctx, const double* r, const double* e);
int mehdg_mlp_set_recording(mehdg_ctx* ctx, int on, int* n_samples);
int mehdg_mlp_gradient(mehdg_ctx* ctx, const float* X, const float* T, int n, float* grad,
                       double* loss);
int mehdg_mlp_train(mehdg_ctx* ctx, int epochs, int batch, double lr, double* losses);

/* Batched dense product on the tcgen05 tensor cores (TF32 inputs, FP32 accumulation),
 * the kernel used by the mixed-precision path for its local GEMMs (forming A^T_i,
 * condensation products):  C_b = alpha A_b B_b + beta C_b for b < batch, with
 * A_b = A + b sA [M x K], B_b = B + b sB [K x N], C_b = C + b sC [M x N], all
 * row-major FP32 device arrays with the given leading dimensions (no alignment
 * requirement).  split != 0: each operand is split into a TF32 part and a TF32
 * remainder and three products are accumulated (close to FP32 accuracy, three
 * times the tensor work).  err: device int set to 1 if an internal wait timed out
 * (the result is then invalid).  Asynchronous on stream.  Errors: ARG, CUDA. */
int mehdg_tc_gemm_tf32(int M, int N, int K, const float* A, long long lda, long long sA,
                       const float* B, long long ldb, long long sB, float* C, long long ldc,
                       long long sC, float alpha, float beta, int batch, int split, int* err,
                       void* stream);

/* Batched dense LU with partial pivoting (Remark, Sec. 3.3: the factorisation of the local
 * Schur complements S), the kernel mehdg_condense_factor runs, for caller-owned matrices:
 * P A_b = L_b U_b for b < batch.  A: device, batch row-major n x n matrices, contiguous,
 * FP64 (fp32 = 0) or FP32 (fp32 != 0), overwritten by the factors (unit lower L below the
 * diagonal, U on and above it); perm: device int [batch][n], row i of P A is row perm[i] of
 * A (first row of largest magnitude wins ties); dflag: device int[2] of scratch owned by the
 * caller.  Synchronises stream.  Errors: ARG, SINGULAR when a pivot is exactly zero (the
 * message on stderr names the first such matrix; the other matrices are factored), CUDA. */
int mehdg_lu_batched(int n, int batch, void* A, int* perm, int fp32, int* dflag, void* stream);

/* The same factorisation for matrices of UNEVEN size in one persistent launch (the batching
 * of independent problems): matrix i is n[i] x n[i] at the device address A[i] with pivot
 * vector perm[i] (device int[n[i]]); n, A, perm are host arrays of nmat entries.  The CTAs of
 * one grid sized to the GPU take the matrices from a device counter, largest first; nb is the
 * panel width (8, 16 or 32), whose panel of n[i] x (nb + 1) entries must fit in shared memory
 * (TOO_LARGE otherwise).  fp32 selects FP32 matrices.  dflag: device int[2] scratch.
 * Synchronises stream.  Errors: ARG, TOO_LARGE, SINGULAR (first matrix named on stderr), CUDA. */
int mehdg_lu_queue(int nmat, const int* n, void* const* A, int* const* perm, int fp32, int nb,
                   int* dflag, void* stream);

/* a13 -- a batch of independent problems of uneven size on one GPU (the benchmark spec's batching
 * form; the paper solves one problem at a time).  mehdg_batch_create builds one context per
 * problem (probs[i] with options opts[i], or defaults when opts is NULL), all on stream, and
 * autotunes the panel width of the batched LU for every (precision, local size Nu) class of the
 * batch: each width whose panel fits in shared memory is timed on sample matrices of that size.
 * Each problem's context is reachable by mehdg_batch_context (for mehdg_init_state and every
 * per-problem call) and is owned by the batch.  condense_layers must be 2 (default).  With
 * stream NULL (the legacy default stream, on which CUDA graphs cannot be captured) the batch
 * creates a blocking stream of its own, ordered with the default stream.
 * Errors: ARG, OOM, CUDA. */
typedef struct mehdg_batch mehdg_batch;
int mehdg_batch_create(mehdg_batch** batch, const mehdg_problem* probs, int nprob,
                       const mehdg_options* opts, void* stream);
int mehdg_batch_size(const mehdg_batch* batch);
mehdg_ctx* mehdg_batch_context(mehdg_batch* batch, int i);

/* Steady solve of every problem of the batch (pseudo-transient Newton of Sec. 3.1 with the
 * SER update, as mehdg_dirk_stage with stage 0, to each problem's newton_rtol), in lockstep
 * rounds: per round one CUDA-graph replay assembles every unconverged problem and reduces its
 * residual norms on the device; one replay condenses every such problem, factors all their
 * local matrices S in ONE persistent work-queue launch (the autotuned panel widths) and forms
 * their b^ (and explicit local operators); then each problem's FGMRES, recovery and update
 * run.  The graphs are captured for the current set of unconverged problems and captured
 * again when it changes; when capture is not possible the same work is launched directly.
 * u, q, uh: host arrays of nprob device pointers to each problem's state (in/out, layouts as
 * for one problem); st: host array of nprob statistics (newton_steps, fgmres_iters, res0,
 * res; status bit 1 = converged, bit 2 (value 4) = a step was retried); rounds (host, or
 * NULL): lockstep rounds run.  A step that leaves the physical states (non-finite residual at
 * the new state: negative pressure or density somewhere) or more than doubles |R_F| is undone
 * and retried with a ten times smaller pseudo-time step (not in the paper, whose SER update
 * has no such safeguard);
 * a problem gives up after 20 retries or max_newton steps.  Errors: ARG, NAN (at the initial
 * state), SINGULAR, NOT_CONVERGED (some problem did not converge; the others are solved),
 * CUDA; the message names the problem (mehdg_batch_last_error). */
int mehdg_batch_steady_solve(mehdg_batch* batch, double* const* u, double* const* q,
                             double* const* uh, mehdg_solve_stats* st, int* rounds);

/* The autotuner's record, one entry per (local size, precision) class, up to cap entries:
 * n[i], fp64[i], the chosen panel width nb[i] and ms[3 i + j] the sample time of widths 8,
 * 16, 32 (-1 where the panel does not fit).  Host arrays (or NULL).  Returns the number of
 * classes, or a negative MEHDG_ERR_*. */
int mehdg_batch_tiles(const mehdg_batch* batch, int cap, int* n, int* fp64, int* nb, double* ms);

/* CUDA-graph replays of the last solves (-1 if capture was not possible and the work was
 * launched directly). */
long long mehdg_batch_graph_replays(const mehdg_batch* batch);
const char* mehdg_batch_last_error(const mehdg_batch* batch);
void mehdg_batch_destroy(mehdg_batch* batch);

/* The product with a transposed right operand on the tcgen05 tensor cores (kind::tf32, each
 * operand split into a TF32 part and a TF32 remainder, three products: close to FP32
 * accuracy), the kernel of tc_mode 4:  C_b = alpha A_b Bt_b^T + beta C_b for b < batch, A_b =
 * A + b sA [M x K], Bt_b = Bt + b sB [N x K], C_b = C + b sC [M x N], row-major FP32 device
 * arrays with the given leading dimensions (4-byte alignment only).  err: device int set to 1
 * if an internal wait timed out (the result is then invalid).  Asynchronous on stream.
 * Errors: ARG, CUDA. */
int mehdg_tc_gemm_nt(int M, int N, int K, const float* A, long long lda, long long sA, const float* Bt,
                     long long ldb, long long sB, float* C, long long ldc, long long sC, float alpha,
                     float beta, int batch, int* err, void* stream);

/* Device time in milliseconds of the most recent execution of each internal phase
 * (CUDA events on the context stream; -1 for phases not run since mehdg_mesh):
 * 0 volume pointwise Jacobians, 1 volume contraction, 2 faces + R_Q, 3 condensation
 * products, 4 batched LU of S, 5 LU of the face blocks, 6 condensed rhs, 7 trace
 * apply kernel, 8 recovery, 9 block-Jacobi, 10 forming A^T_i (apply_mode 1),
 * 11 BF16 trace apply of the inner GMRES (precond_bf16; timed inside its CUDA graph),
 * 12 the two fused condensation GEMM launches, 13 the multi-right-hand-side S^-1 C
 * substitutions of forming A^T_i.
 * ms: host double[n], n <= 16.
 * Synchronises the stream. */
int mehdg_phase_times(mehdg_ctx* ctx, double* ms, int n);

/* Cumulative device time of the internal phases (numbered as in mehdg_phase_times): for
 * each phase p < n, sum_ms[p] (host double[n], or NULL) receives the milliseconds summed over
 * every execution since mehdg_mesh or the last reset, and count[p] (host long long[n], or
 * NULL) the number of executions.  Executions inside the inner-GMRES CUDA graph (phase 11)
 * are counted per replay at the duration of the latest one.  reset != 0 zeroes both after
 * reading.  Synchronises the stream. */
int mehdg_phase_stats(mehdg_ctx* ctx, double* sum_ms, long long* count, int n, int reset);

/* Number of CUDA kernels this context has launched since mehdg_mesh (host counter;
 * count is host memory). */
int mehdg_launch_count(const mehdg_ctx* ctx, long long* count);

/* Replays of the inner-GMRES CUDA graph (multi-level preconditioner) since mehdg_mesh (host).
 * The graph is captured at the first preconditioner call when the context's stream is not the
 * legacy default stream, on which CUDA graphs cannot be captured; there (count 0) the same
 * kernels are launched directly. */
int mehdg_graph_replays(const mehdg_ctx* ctx, long long* count);

void mehdg_destroy(mehdg_ctx* ctx);
const char* mehdg_last_error(const mehdg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
