// Internal state of a mehdg context and helpers shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/mehdg.h"

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return ctx_fail(ctx, e_ == cudaErrorMemoryAllocation ? MEHDG_ERR_OOM : MEHDG_ERR_CUDA, \
                      std::string(#call) + ": " + cudaGetErrorString(e_));              \
    }                                                                                   \
  } while (0)

#define CKL()                                                                           \
  do {                                                                                  \
    ++ctx->launches;                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess)                                                              \
      return ctx_fail(ctx, MEHDG_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

// a row-compressed operator of one macro-element type: row r of macro e holds val[e * nnz + k]
// at column col[k] for off[r] <= k < off[r + 1] (pattern shared by all macro-elements)
struct SpOp {
  const int* off = nullptr;
  const int* col = nullptr;
  double* val = nullptr;
  long long nnz = 0;
};

template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct mehdg_ctx {
  mehdg_problem prob;
  mehdg_options opt;
  cudaStream_t stream = nullptr;
  std::string err;

  // sizes
  int d, ns, m, p, n1, Np, Nfn, Nth, Nu, Nq, Nt, E, F;
  long long ntr;          // global trace length F * ns * Nfn
  int nel, nloc, ng1, Ng; // sub-elements per macro, nodes per sub-element, Gauss points
  int nsf, nfs, nfp;      // sub-faces per macro face, nodes per sub-face, points per sub-face
  int ndir_v, ndir_f;     // Jacobian input directions (volume, face)
  double hm[3], he[3];    // macro and sub-element sizes
  double h_supg;
  long long bytes = 0;

  // host tables
  std::vector<double> b1, db1, gw;   // [ng1][p+1] reference basis at Gauss points, weights
  std::vector<int> facenode;         // [nf][Nfn] macro node of each face node (nf faces per macro)
  std::vector<int> h_gather;         // [E][Nt]
  std::vector<int> h_owner;          // [F][2] (e * 2d + fl) or -1
  std::vector<int> h_bkind;          // [E][nf]
  std::vector<int> h_bside;          // [E][nf] domain side or -1

  // device: maps and reference data
  int* gather = nullptr;     // [E][Nt]
  int* owner = nullptr;      // [F][2]
  int* bkind = nullptr;      // [E][nf]
  int* bside = nullptr;      // [E][nf]
  int* fnode = nullptr;      // [nf][Nfn]
  double* tab = nullptr;     // b1, db1, gw packed
  double* Mref = nullptr;    // [Np][Np]
  double* Minv = nullptr;    // [Np][Np]
  double* Gk = nullptr;      // [d][Np][Np]
  double* Ghk = nullptr;     // [d][Np][Nth]
  double* Wk = nullptr;      // [d][Np][Np]   M^-1 G_k
  double* Whk = nullptr;     // [d][Np][Nth]  M^-1 Gh_k
  double* Bcat = nullptr;    // [d*Np][Np+Nth] = [W_k | -Wh_k] stacked over k (fused condensation GEMM)
  float* Bcat32 = nullptr;   // FP32 copy (mixed precision)
  // Kronecker factors of the liftings on affine box macros (null when the mesh is not of that
  // kind): [d][n1][n1] with W_k[a][b] = klift[k][a_k][b_k] when a and b agree off axis k, then
  // [2d][n1] with Wh_k[a][(f, i)] = klift[f][a_k] when face f is normal to k and a lies on the
  // line through face node i
  double* klift = nullptr;
  // curved (mapped) macro-elements of the shell mesh: per-point geometry, per-macro operators.
  // Mref, Minv, Gk, Ghk, Wk, Whk and Bcat then hold one copy per macro-element at the strides
  // below (0: one copy shared by all macro-elements, the box meshes)
  // batches of problems: the pseudo-time shift read from device memory (so that a captured
  // condensation can be replayed with new shifts), phase timers off inside batch graphs
  const double* dshift = nullptr;
  bool no_phase = false;
  bool mapped = false;
  double* vgeo = nullptr;    // [E][nel][Ng][d*d + 1]: (J^-1)[j][k] = dxi_j/dx_k (xi the macro reference coordinates), weight
  double* fgeo = nullptr;    // [E][nf][nsf][nfp][d + 1]: unit outward normal, weight
  double* xnode = nullptr;   // [E][d][Np] node positions
  int* ofn = nullptr;        // [F][2][Nfn] owner's local face node of each face node (null: same order)
  std::vector<int> h_ofn;
  size_t sM = 0, sG = 0, sGh = 0, sB = 0;
  double* src = nullptr;     // [E][nel][Ng][ns] or null
  double* uD = nullptr;      // [E][nf][nsf][nfp][ns] or null

  // device: blocks (FP64)
  double *Auu = nullptr, *Auq = nullptr, *Auh = nullptr, *Ahu = nullptr, *Ahq = nullptr, *Ahh = nullptr;
  int* perm = nullptr;       // [E][Nu]
  double *RQ = nullptr, *RU = nullptr, *RUh = nullptr, *gv = nullptr, *hv = nullptr, *MinvRQ = nullptr,
         *bloc = nullptr, *slot = nullptr;
  double *Kvol = nullptr, *rvol = nullptr, *Kface = nullptr, *rface = nullptr;
  double* fblk = nullptr;    // [F][nfb][nfb]
  int* fperm = nullptr;      // [F][nfb]
  int nfb = 0;
  int* dflag = nullptr;      // device status words
  double* dred = nullptr;    // reduction scratch
  double* ddiag = nullptr;   // per-macro partial sums of mehdg_flow_integrals, [E][3] + 4
  // simplicial macro-elements (mesh_kind MEHDG_MESH_SIMPLEX): reference tables on the device
  int simplex = 0;
  int nf = 0;                  // faces per macro-element: 2 d (boxes, shell), d + 1 (simplices)
  double* sx_vtab = nullptr;   // [nel][Ng][nloc][d + 1]: phi, d phi / d xi_j of the sub-simplex's nodes
  int* sx_vnode = nullptr;     // [nel][nloc] macro node of each sub-simplex node
  double* sx_ftab = nullptr;   // [nf][nsf][nfp][nfs]: trace basis of the sub-face's nodes at its points
  int* sx_fsub = nullptr;      // [nf][nsf][nfs] face node of each sub-face node
  double* hred = nullptr;    // pinned host mirror

  float *Wk32 = nullptr, *Whk32 = nullptr;   // FP32 copies of W_k, Wh_k (mixed precision)
  int* dtcerr = nullptr;                       // tensor-core kernel error word
  bool use_tc_condense = false, use_tc_form = false, use_tc_lu = false, tc_split = true, use_tc_nt = false;
  float* finv32 = nullptr;   // explicit FP32 inverses of the face blocks (mixed precision block-Jacobi)
  // mixed precision: FP32 copies of the state, history, 1D tables and source for the FP32
  // Jacobian pass of the assembly
  float *u32 = nullptr, *q32 = nullptr, *h32 = nullptr, *tab32 = nullptr, *src32 = nullptr;
  float *uD32 = nullptr, *uh32 = nullptr;
  double* Xbuf = nullptr;     // S^-1 C of every macro (apply_mode 1), storage type of the blocks
  unsigned short* Ahat16 = nullptr;   // BF16 copy of A^T_i for the inner GMRES (precond_bf16)
  int ld16 = 0;                       // its row stride: Nt rounded up to 4 (8-byte rows), zero-padded
  bool lowp_apply = false;            // set while the inner GMRES runs: apply the BF16 copy
  int apply_grid = 0, apply_grid16 = 0;   // persistent grids of the explicit apply kernels
  int bj_grid = 0, bj_grid16 = 0;         // ... and of the block-Jacobi product
  unsigned short* finv16 = nullptr;       // BF16 copy of the face-block inverses (precond_bf16)
  int ldf16 = 0;                          // its row stride: nfb rounded up to 32, zero-padded
  // mixed precision: S before its factorisation, for the FP64 refinement of local solves
  float* S32 = nullptr;
  // apply_mode 2: row-compressed B, C, D (FP64), their patterns and the row of each entry
  SpOp spB, spC, spD;
  int *spB_row = nullptr, *spC_row = nullptr, *spD_row = nullptr;
  bool sp_pending = false;
  // one-layer condensation (condense_layers 1): A_local [E][NL][NL] (factored in place), its
  // pivots, the right-hand sides [A_quh; A_uuh | R] [E][NL][Nt + 1] and X = A_local^-1 of them
  double *Aloc = nullptr, *Rloc = nullptr, *Xloc = nullptr;
  int* permL = nullptr;

  // Krylov workspace
  int restart = 30;
  double *V = nullptr, *Zk = nullptr, *wv = nullptr, *tv = nullptr, *tv2 = nullptr, *rv = nullptr;
  double *iV = nullptr, *iw = nullptr;    // inner GMRES
  double* xstart = nullptr;               // FGMRES iterate at the start of the current cycle
  double* dHo = nullptr;                  // device Hessenberg, rotations, rhs of the outer FGMRES
  double* dHi = nullptr;                  // the same for the inner GMRES
  double *gin = nullptr, *gout = nullptr; // fixed in/out vectors of the captured inner GMRES
  cudaGraphExec_t ig_exec = nullptr;      // inner GMRES as one CUDA graph
  long long ig_nodes = 0;                 // kernels per replay of that graph
  bool ig_failed = false, capturing = false;
  // Newton / DIRK
  double *un = nullptr, *ustage = nullptr, *hist = nullptr, *du = nullptr, *dq = nullptr, *duh = nullptr,
         *bhat = nullptr;
  int lu_status = 0;
  bool condensed = false;
  // nonlinear iteration state of the current stage (mehdg_stage_begin / mehdg_newton_step)
  int cur_stage = -1;         // -1: no stage begun
  double stage_dt = 0.0, stage_R0 = 0.0, stage_dtau = 1.0;
  double stage_norms[4] = {};
  int stage_newton = 0;
  mehdg_time_term stage_tt{};
  // MLP preconditioner correction (kind 2)
  void* mlp = nullptr;
  // phase timers (CUDA events on the context stream).  Outside graph capture every execution
  // of a phase records its own event pair from a per-phase pool; completed pairs are summed
  // (ph_sum, ph_cnt) at the library's synchronisation points.  Phases captured into the inner
  // GMRES graph keep one external pair, re-recorded by each replay (ev, ph_graph executions
  // per replay).
  cudaEvent_t ev[2 * 16] = {};
  long long launches = 0;   // kernels launched by this context
  bool ev_rec[16] = {};
  std::vector<cudaEvent_t> ring_b[16], ring_e[16];
  int ring_n[16] = {};
  double ph_sum[16] = {}, ph_last[16] = {};
  long long ph_cnt[16] = {};
  int ph_graph[16] = {};
  long long ig_replays = 0;   // inner-GMRES graph replays not yet added to the sums
  long long ig_total = 0;     // inner-GMRES graph replays since mehdg_mesh
};

enum Phase {
  PH_VOL_POINT = 0, PH_VOL_CONTRACT = 1, PH_FACES = 2, PH_CONDENSE = 3, PH_LU = 4, PH_FACE_LU = 5,
  PH_BHAT = 6, PH_APPLY = 7, PH_RECOVER = 8, PH_PRECOND = 9, PH_FORM = 10, PH_APPLY_BF16 = 11,
  PH_COND_GEMM = 12, PH_TRSM = 13, PH_COUNT = 16
};
void phase_begin(mehdg_ctx* ctx, int p);
void phase_end(mehdg_ctx* ctx, int p);
// add every completed phase execution to the sums (call after a stream synchronisation)
void phase_harvest(mehdg_ctx* ctx);

int ctx_fail(mehdg_ctx* ctx, int code, const std::string& msg);

// geometry helpers usable on the device
struct Geo {
  int d, ns, m, p, n1, Np, Nfn, Nth, Nu, Nt, nel, nloc, ng1, Ng, nsf, nfs, nfp;
  int nf;   // faces per macro-element
  double he[3];
};

// reference tables of the m-refined Kuhn simplex (csrc/simplex.cu)
struct SxRef {
  int d = 0, m = 0, p = 0, Np = 0, Nfn = 0, nel = 0, ng = 0, nloc = 0, nsf = 0, nfp = 0, nfs = 0;
  std::vector<int> lat;        // [Np][d] integer node coordinates (spacing 1 / (m p))
  std::vector<double> vxi;     // [nel ng][d] volume points in K
  std::vector<double> vw;      // [nel ng] their weights
  std::vector<double> vtab;    // [nel ng][nloc][d + 1]
  std::vector<int> vnode;      // [nel][nloc]
  std::vector<int> fnodes;     // [d + 1][Nfn] macro node of each face node
  std::vector<double> nref;    // [d + 1][d] unit outward normals in K
  std::vector<double> fM;      // [d + 1][d][d - 1] face vertex differences (xi = W0 + M t)
  std::vector<double> fxi;     // [d + 1][nsf nfp][d] face points in K
  std::vector<double> fwt;     // [d + 1][nsf nfp] their weights in face coordinates t
  std::vector<double> ftab;    // [d + 1][nsf nfp][nfs]
  std::vector<int> fsub;       // [d + 1][nsf][nfs]
};
// host geometry of a simplicial mesh, uploaded by setup()
struct SxHost {
  std::vector<double> vgeo, fgeo, xnode, xq, xf, M, Minv, Gk, Ghk, Wk, Whk, Bcat;
};
int sx_reference(int d, int m, int p, SxRef& R);
int sx_maps(mehdg_ctx* ctx, SxRef& R, SxHost& H);
int sx_source(mehdg_ctx* ctx, const double* xq, long long n, double* src);
int sx_bdata(mehdg_ctx* ctx, const double* xf, long long n, int per_f, double* uD);
int sx_init_state(mehdg_ctx* ctx, const double* du, double* u);
void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w);
void invert(std::vector<double>& A, int n);
Geo make_geo(const mehdg_ctx* c);

// launch helpers implemented in the .cu files
int assemble_all(mehdg_ctx* ctx, const double* u, const double* q, const double* uh,
                 const mehdg_time_term* tt, double* norms);
int condense_all(mehdg_ctx* ctx, double shift, double* bhat);
// the condensation in parts (1: up to the LU of S, 2: from the face blocks' LU on, no status
// read) and the status read that ends it
int condense_part(mehdg_ctx* ctx, double shift, double* bhat, int part);
int condense_status(mehdg_ctx* ctx);
int apply_trace_impl(mehdg_ctx* ctx, const double* x, double* y);
bool apply_bf16_slots_available(const mehdg_ctx* ctx);
int apply_bf16_slots(mehdg_ctx* ctx, const double* x);
int recover_impl(mehdg_ctx* ctx, const double* duh, double* du, double* dq);
int precond_impl(mehdg_ctx* ctx, int kind, const double* r, double* z);
int linear_solve_impl(mehdg_ctx* ctx, const double* b, double* x, mehdg_solve_stats* st);
int face_reduce(mehdg_ctx* ctx, const double* slot, double* y);
int condense_one(mehdg_ctx* ctx, double shift, double* bhat);
int recover_one(mehdg_ctx* ctx, const double* duh, double* du, double* dq);
// shell mesh (curved macro-elements): host maps, device geometry, boundary data, initial state
int shell_maps(mehdg_ctx* ctx, const std::vector<double>& t, std::vector<double>& xnode);
int shell_geometry(mehdg_ctx* ctx, const double* dend);
int shell_bdata(mehdg_ctx* ctx);
int shell_init_state(mehdg_ctx* ctx, const double* du, double* u);
int sparse_setup(mehdg_ctx* ctx);
int sparse_pack(mehdg_ctx* ctx);
int apply_sparse(mehdg_ctx* ctx, const double* x, double* y);
void sparse_destroy(mehdg_ctx* ctx);
int vec_dot(mehdg_ctx* ctx, const double* a, const double* b, long long n, double* out_host);
int vec_axpy(mehdg_ctx* ctx, long long n, double a, const double* x, double* y);
int vec_scal(mehdg_ctx* ctx, long long n, double a, double* x);
int vec_copy(mehdg_ctx* ctx, long long n, const double* x, double* y);
int vec_lincomb(mehdg_ctx* ctx, long long n, double a, const double* x, double b, const double* y, double* z);
int batched_lu(mehdg_ctx* ctx, double* A, int* perm, int n, int batch, int* flag);
int to_float(mehdg_ctx* ctx, const double* x, float* y, long long n);
int mlp_apply(mehdg_ctx* ctx, const double* r, double* z);
bool mlp_recording(const mehdg_ctx* ctx);
int mlp_record_pair(mehdg_ctx* ctx, const double* r, const double* e);
void mlp_destroy(mehdg_ctx* ctx);
struct TcArgs;
cudaError_t tc_gemm_launch(const TcArgs& a, int batch, cudaStream_t st, bool split);
struct TcNT;
cudaError_t tc_gemm_nt_launch(const TcNT& a, int batch, cudaStream_t st);
