// a13: batches of independent problems of uneven size (many problems on one GPU at once).
//
// A batch owns one context per problem, all on the batch's stream, and solves them in lockstep
// rounds of the steady Newton / pseudo-transient iteration (Sec. 3.1; the same iteration as
// mehdg_dirk_stage with stage 0).  One round of every unconverged problem is
//   1. one CUDA-graph replay: the assembly of every problem and its residual norms (device
//      reductions into one array, read back with one copy);
//   2. one CUDA-graph replay: the condensation of every problem up to the LU of S, then ONE
//      persistent work-queue launch (k_lu_queue) that factors the local matrices S of all
//      problems -- items of uneven size n = ns (mp + 1)^3, sorted largest first, taken by the
//      CTAs from a device counter -- then the face blocks' LU, b^ and the explicit local
//      operators of every problem; the pseudo-time shifts are read from device memory, so
//      the captured graph is replayed with new shifts every round;
//   3. per problem: FGMRES on its trace system (host-driven, as for a single problem),
//      recovery and the state update.
// The graphs are captured once per set of active problems (again when a problem converges).
// The panel width of the queued LU is chosen per (precision, n) by an autotuner that times
// every width whose panel fits in shared memory on sample matrices of that size when the
// batch is created.
#include <algorithm>
#include <cmath>
#include <map>

#include "internal.cuh"
#include "lu_panel.cuh"

namespace {

constexpr size_t kSmemLimit = 227 * 1024 - 2048;   // dynamic shared memory per CTA, static part kept free
constexpr int kNormBlocks = 256;

// uniform [-1, 1) values from a counter hash (splitmix64 finaliser), for the autotuner's matrices
template <class T>
__global__ void k_fill_uniform(T* A, long long n, unsigned long long seed) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  A[i] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// deterministic sum of squares: per-block partial sums, then one block adds them in order
__global__ void k_sumsq_part(const double* __restrict__ x, long long n, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += x[i] * x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_sumsq_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

template <class T>
size_t queue_smem(int n, int nb) {
  if (nb == 8) return lu_panel_smem<T, false, 8>(n);
  if (nb == 16) return lu_panel_smem<T, false, 16>(n);
  return lu_panel_smem<T, false, 32>(n);
}

struct Queue {
  LuItem* items = nullptr;   // device
  int n = 0;
  size_t smem = 0;
  int grid = 0;
};

struct TuneRec {
  int n, fp64, nb;
  double ms[3];   // time of widths 8, 16, 32 on the sample (-1: the panel does not fit)
  int sample;
};

}  // namespace

struct mehdg_batch {
  std::vector<mehdg_ctx*> ctx;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  std::string err;
  std::vector<TuneRec> tune;
  std::map<long long, int> nb_of;   // key n * 2 + fp64
  Queue q[2];                       // [0] FP32 matrices, [1] FP64
  int* counter = nullptr;           // [2] device queue counters
  double* dshift = nullptr;         // [nprob]
  double* dnorm = nullptr;          // [nprob][4]: |R_Q|^2, |R_U|^2, |R_Uh|^2
  double* dpart = nullptr;          // reduction scratch [nprob][3][kNormBlocks]
  double* hnorm = nullptr;          // pinned [nprob][4]
  int* hflag = nullptr;             // pinned [nprob][5]
  double* hshift = nullptr;         // pinned [nprob]
  cudaGraphExec_t gasm = nullptr, gcond = nullptr;
  std::vector<char> sig_asm, sig_cond;
  std::vector<double*> prev;          // per problem: u, q, uh before the last update (retries)
  cudaStream_t own = nullptr;         // the batch's stream when the caller passed the legacy default stream
  bool graphs = true;
  long long replays = 0;
};

namespace {

int bfail(mehdg_batch* b, int code, const std::string& msg) {
  b->err = msg;
  return code;
}
#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? MEHDG_ERR_OOM : MEHDG_ERR_CUDA,           \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)
#define BRC(call)                                                                                 \
  do {                                                                                            \
    int r_ = (call);                                                                              \
    if (r_) return r_;                                                                            \
  } while (0)

bool is_fp64(const mehdg_ctx* c) { return c->opt.precision != MEHDG_PREC_MIXED; }

template <class T>
int launch_queue(mehdg_batch* b, const Queue& q, int* counter) {
  if (q.n == 0) return MEHDG_OK;
  BCK(cudaMemsetAsync(counter, 0, sizeof(int), b->stream));
  k_lu_queue<T><<<q.grid, LP_NT, q.smem, b->stream>>>(q.items, q.n, counter);
  BCK(cudaGetLastError());
  return MEHDG_OK;
}

// queue of the given items: device copy, shared memory of the largest panel, persistent grid
template <class T>
int make_queue(mehdg_batch* b, Queue& q, std::vector<LuItem>& it) {
  std::stable_sort(it.begin(), it.end(), [](const LuItem& x, const LuItem& y) { return x.n > y.n; });
  if (q.items) cudaFree(q.items);
  q = Queue{};
  q.n = (int)it.size();
  if (q.n == 0) return MEHDG_OK;
  for (const LuItem& w : it) q.smem = std::max(q.smem, queue_smem<T>(w.n, w.nb));
  BCK(cudaMalloc(&q.items, sizeof(LuItem) * it.size()));
  BCK(cudaMemcpyAsync(q.items, it.data(), sizeof(LuItem) * it.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaFuncSetAttribute(k_lu_queue<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q.smem));
  int per = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lu_queue<T>, LP_NT, q.smem));
  q.grid = std::min(q.n, b->nsm * std::max(per, 1));
  BCK(cudaStreamSynchronize(b->stream));   // the host item array goes out of scope
  return MEHDG_OK;
}

// autotuner: time every panel width that fits on `count` sample matrices of size n
template <class T>
int tune_class(mehdg_batch* b, int n, int count) {
  const int fp64 = sizeof(T) == 8;
  TuneRec rec{n, fp64, 0, {-1.0, -1.0, -1.0}, 0};
  const size_t bytes_one = sizeof(T) * (size_t)n * n;
  int K = std::min(count, 2 * b->nsm);
  K = (int)std::max<size_t>(1, std::min<size_t>((size_t)K, ((size_t)2 << 30) / bytes_one));
  rec.sample = K;
  T* A = nullptr;
  int *perm = nullptr, *flag = nullptr;
  BCK(cudaMalloc(&A, bytes_one * K));
  BCK(cudaMalloc(&perm, sizeof(int) * (size_t)n * K));
  BCK(cudaMalloc(&flag, sizeof(int) * 2));
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  const int widths[3] = {8, 16, 32};
  double best = 1e300;
  int rc = MEHDG_OK;
  for (int wi = 0; wi < 3 && !rc; ++wi) {
    const int nb = widths[wi];
    if (queue_smem<T>(n, nb) > kSmemLimit) continue;
    std::vector<LuItem> it(K);
    for (int k = 0; k < K; ++k)
      it[k] = LuItem{A + (size_t)k * n * n, perm + (size_t)k * n, flag, n, nb, k + 1, 0};
    Queue q;
    if ((rc = make_queue<T>(b, q, it))) break;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && !rc; ++rep) {   // first run warms up, second is timed
      const long long tot = (long long)K * n * n;
      k_fill_uniform<T><<<(unsigned)((tot + 255) / 256), 256, 0, b->stream>>>(A, tot, 12345ull + rep);
      cudaEventRecord(e0, b->stream);
      rc = launch_queue<T>(b, q, b->counter);
      cudaEventRecord(e1, b->stream);
    }
    if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
      rec.ms[wi] = ms;
      if (ms < best) { best = ms; rec.nb = nb; }
    }
    cudaFree(q.items);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(perm);
  cudaFree(flag);
  if (rc) return rc;
  if (rec.nb == 0) return bfail(b, MEHDG_ERR_ARG, "batch: no panel width fits n = " + std::to_string(n));
  b->tune.push_back(rec);
  b->nb_of[(long long)n * 2 + fp64] = rec.nb;
  return MEHDG_OK;
}

// assembly and residual norms of every active problem (graph body)
int record_asm(mehdg_batch* b, const std::vector<char>& active, double* const* u, double* const* q,
               double* const* uh) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (!active[i]) continue;
    mehdg_ctx* c = b->ctx[i];
    BRC(assemble_all(c, u[i], q[i], uh[i], nullptr, nullptr));
    BRC(face_reduce(c, c->RUh, c->tv2));
    const double* vec[3] = {c->RQ, c->RU, c->tv2};
    const long long len[3] = {(long long)c->E * c->Nq, (long long)c->E * c->Nu, c->ntr};
    for (int k = 0; k < 3; ++k) {
      double* part = b->dpart + ((size_t)i * 3 + k) * kNormBlocks;
      k_sumsq_part<<<kNormBlocks, 256, 0, b->stream>>>(vec[k], len[k], part);
      k_sumsq_final<<<1, 256, 0, b->stream>>>(part, kNormBlocks, b->dnorm + (size_t)i * 4 + k);
    }
    BCK(cudaGetLastError());
  }
  return MEHDG_OK;
}

// condensation up to the LU, the queued LU of every S, then the rest of the condensation
int record_cond(mehdg_batch* b, const std::vector<char>& active) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (!active[i]) continue;
    mehdg_ctx* c = b->ctx[i];
    c->dshift = b->dshift + i;
    BCK(cudaMemsetAsync(c->dflag, 0, sizeof(int) * 16, b->stream));
    BRC(condense_part(c, 0.0, c->bhat, 1));
  }
  BRC(launch_queue<float>(b, b->q[0], b->counter));
  BRC(launch_queue<double>(b, b->q[1], b->counter + 1));
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (!active[i]) continue;
    BRC(condense_part(b->ctx[i], 0.0, b->ctx[i]->bhat, 2));
  }
  return MEHDG_OK;
}

int build_queues(mehdg_batch* b, const std::vector<char>& active) {
  std::vector<LuItem> it[2];
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (!active[i]) continue;
    mehdg_ctx* c = b->ctx[i];
    const int f = is_fp64(c) ? 1 : 0;
    const size_t esz = f ? 8 : 4;
    const int nb = b->nb_of[(long long)c->Nu * 2 + f];
    for (int e = 0; e < c->E; ++e)
      it[f].push_back(LuItem{reinterpret_cast<char*>(c->Auu) + esz * (size_t)e * c->Nu * c->Nu,
                             c->perm + (size_t)e * c->Nu, c->dflag, c->Nu, nb, e + 1, 0});
  }
  BRC(make_queue<float>(b, b->q[0], it[0]));
  BRC(make_queue<double>(b, b->q[1], it[1]));
  return MEHDG_OK;
}

// run `rec` as a graph captured for this active set (captured again when the set changes), or
// directly when capture is not possible
template <class F>
int run_graph(mehdg_batch* b, cudaGraphExec_t& exec, std::vector<char>& sig, const std::vector<char>& active, F rec) {
  if (b->graphs && (!exec || sig != active)) {
    if (exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      const int rc = rec();
      cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
      if (rc == MEHDG_OK && ec == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        sig = active;
      } else {
        exec = nullptr;
        b->graphs = false;   // fall back to direct launches from now on
      }
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
    } else {
      b->graphs = false;
      cudaGetLastError();
    }
  }
  if (b->graphs && exec) {
    BCK(cudaGraphLaunch(exec, b->stream));
    ++b->replays;
    return MEHDG_OK;
  }
  return rec();
}

}  // namespace

extern "C" int mehdg_batch_create(mehdg_batch** out, const mehdg_problem* probs, int nprob, const mehdg_options* opts,
                                  void* stream) {
  if (!out || !probs || nprob < 1) return MEHDG_ERR_ARG;
  *out = nullptr;
  mehdg_batch* b = new mehdg_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  if (!b->stream) {
    // CUDA graphs cannot be captured on the legacy default stream: the batch runs on a stream
    // of its own, created blocking, so that it stays ordered with work on the default stream
    if (cudaStreamCreate(&b->own) != cudaSuccess) {
      delete b;
      return MEHDG_ERR_CUDA;
    }
    b->stream = b->own;
    stream = b->own;
  }
  int rc = MEHDG_OK;
  auto fail = [&](int code) {
    fprintf(stderr, "mehdg_batch_create: %s\n", b->err.c_str());
    mehdg_batch_destroy(b);
    return code;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    b->err = "no CUDA device";
    return fail(MEHDG_ERR_CUDA);
  }
  for (int i = 0; i < nprob; ++i) {
    mehdg_ctx* c = nullptr;
    rc = mehdg_mesh(&c, probs + i, 1, opts ? opts + i : nullptr, stream);
    if (rc) {
      b->err = "problem " + std::to_string(i) + ": mehdg_mesh failed";
      return fail(rc);
    }
    if (c->opt.condense_layers == 1) {
      mehdg_destroy(c);
      b->err = "problem " + std::to_string(i) + ": batches use the second-layer condensation";
      return fail(MEHDG_ERR_ARG);
    }
    c->no_phase = true;
    b->ctx.push_back(c);
  }
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && !rc) {
      b->err = cudaGetErrorString(e);
      rc = e == cudaErrorMemoryAllocation ? MEHDG_ERR_OOM : MEHDG_ERR_CUDA;
    }
  };
  ck(cudaMalloc(&b->counter, sizeof(int) * 2));
  ck(cudaMalloc(&b->dshift, sizeof(double) * nprob));
  ck(cudaMalloc(&b->dnorm, sizeof(double) * 4 * nprob));
  ck(cudaMalloc(&b->dpart, sizeof(double) * 3 * kNormBlocks * nprob));
  ck(cudaMallocHost(&b->hnorm, sizeof(double) * 4 * nprob));
  ck(cudaMallocHost(&b->hflag, sizeof(int) * 5 * nprob));
  ck(cudaMallocHost(&b->hshift, sizeof(double) * nprob));
  for (mehdg_ctx* c : b->ctx) {
    double* pv = nullptr;
    ck(cudaMalloc(&pv, sizeof(double) * ((size_t)c->E * c->Nu * (1 + c->d) + (size_t)c->ntr)));
    b->prev.push_back(pv);
  }
  if (rc) return fail(rc);
  // autotune the panel width of every (precision, n) class of the batch
  std::map<long long, int> count;
  for (mehdg_ctx* c : b->ctx) count[(long long)c->Nu * 2 + (is_fp64(c) ? 1 : 0)] += c->E;
  for (const auto& kv : count) {
    const int n = (int)(kv.first / 2);
    rc = (kv.first % 2) ? tune_class<double>(b, n, kv.second) : tune_class<float>(b, n, kv.second);
    if (rc) return fail(rc);
  }
  *out = b;
  return MEHDG_OK;
}

extern "C" int mehdg_batch_size(const mehdg_batch* b) { return b ? (int)b->ctx.size() : 0; }

extern "C" mehdg_ctx* mehdg_batch_context(mehdg_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

extern "C" int mehdg_batch_tiles(const mehdg_batch* b, int cap, int* n, int* fp64, int* nb, double* ms) {
  if (!b || cap < 0) return MEHDG_ERR_ARG;
  const int k = std::min(cap, (int)b->tune.size());
  for (int i = 0; i < k; ++i) {
    if (n) n[i] = b->tune[i].n;
    if (fp64) fp64[i] = b->tune[i].fp64;
    if (nb) nb[i] = b->tune[i].nb;
    if (ms)
      for (int j = 0; j < 3; ++j) ms[3 * i + j] = b->tune[i].ms[j];
  }
  return (int)b->tune.size();
}

extern "C" long long mehdg_batch_graph_replays(const mehdg_batch* b) { return b ? (b->graphs ? b->replays : -1) : -1; }

extern "C" const char* mehdg_batch_last_error(const mehdg_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int mehdg_batch_steady_solve(mehdg_batch* b, double* const* u, double* const* q, double* const* uh,
                                        mehdg_solve_stats* st, int* rounds) {
  if (!b || !u || !q || !uh || !st) return MEHDG_ERR_ARG;
  const int N = (int)b->ctx.size();
  for (int i = 0; i < N; ++i)
    if (!u[i] || !q[i] || !uh[i]) return MEHDG_ERR_ARG;
  std::vector<char> active(N, 1);
  std::vector<double> R0(N), RU(N), dtau(N), RF(N);
  std::vector<int> retries(N, 0);
  for (int i = 0; i < N; ++i) {
    st[i] = mehdg_solve_stats{};
    dtau[i] = b->ctx[i]->opt.tau_init;
  }
  auto read_norms = [&]() -> int {
    BCK(cudaMemcpyAsync(b->hnorm, b->dnorm, sizeof(double) * 4 * N, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < N; ++i) {
      double* h = b->hnorm + 4 * i;
      h[3] = std::sqrt(h[0] + h[1] + h[2]);
    }
    return MEHDG_OK;
  };
  auto conv = [&](int i) {
    const mehdg_ctx* c = b->ctx[i];
    return b->hnorm[4 * i + 3] <= std::max(c->opt.newton_rtol * R0[i], c->opt.newton_atol);
  };
  auto assemble = [&]() -> int {
    BRC(run_graph(b, b->gasm, b->sig_asm, active, [&]() { return record_asm(b, active, u, q, uh); }));
    return read_norms();
  };
  BRC(assemble());
  int max_newton = 0;
  for (int i = 0; i < N; ++i) {
    R0[i] = b->hnorm[4 * i + 3];
    if (!std::isfinite(R0[i])) return bfail(b, MEHDG_ERR_NAN, "problem " + std::to_string(i) + ": non-finite residual");
    RU[i] = std::sqrt(b->hnorm[4 * i + 1]);
    RF[i] = R0[i];
    st[i].res0 = st[i].res = R0[i];
    if (conv(i)) {
      active[i] = 0;
      st[i].status |= 2;
    }
    max_newton = std::max(max_newton, b->ctx[i]->opt.max_newton);
  }
  int r = 0;
  while (r < 2 * max_newton && std::count(active.begin(), active.end(), 1) > 0) {
    // condensation and factorisation of every active problem
    for (int i = 0; i < N; ++i) b->hshift[i] = 1.0 / dtau[i];
    BCK(cudaMemcpyAsync(b->dshift, b->hshift, sizeof(double) * N, cudaMemcpyHostToDevice, b->stream));
    if (b->sig_cond != active || !b->graphs || !b->gcond) BRC(build_queues(b, active));
    BRC(run_graph(b, b->gcond, b->sig_cond, active, [&]() { return record_cond(b, active); }));
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      BCK(cudaMemcpyAsync(b->hflag + 5 * i, b->ctx[i]->dflag, sizeof(int) * 4, cudaMemcpyDeviceToHost, b->stream));
      BCK(cudaMemcpyAsync(b->hflag + 5 * i + 4, b->ctx[i]->dtcerr, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      const int* f = b->hflag + 5 * i;
      if (f[4]) return bfail(b, MEHDG_ERR_TIMEOUT, "problem " + std::to_string(i) + ": tensor-core wait timed out");
      if (f[0] || f[2])
        return bfail(b, MEHDG_ERR_SINGULAR, "problem " + std::to_string(i) + ": zero pivot in the local factors");
      b->ctx[i]->condensed = true;
    }
    // trace systems, recovery and updates (the state before the update is kept for a retry)
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      mehdg_ctx* c = b->ctx[i];
      const long long nu = (long long)c->E * c->Nu;
      int rc;
      double* pv = b->prev[i];
      if ((rc = vec_copy(c, nu, u[i], pv)) || (rc = vec_copy(c, nu * c->d, q[i], pv + nu)) ||
          (rc = vec_copy(c, c->ntr, uh[i], pv + nu * (1 + c->d))))
        return bfail(b, rc, c->err);
      mehdg_solve_stats ls{};
      rc = linear_solve_impl(c, c->bhat, c->duh, &ls);
      if (rc && rc != MEHDG_ERR_NOT_CONVERGED) return bfail(b, rc, "problem " + std::to_string(i) + ": " + c->err);
      st[i].fgmres_iters += ls.fgmres_iters;
      st[i].status |= ls.status & 1;
      if ((rc = recover_impl(c, c->duh, c->du, c->dq))) return bfail(b, rc, c->err);
      if ((rc = vec_axpy(c, nu, 1.0, c->du, u[i]))) return bfail(b, rc, c->err);
      if ((rc = vec_axpy(c, nu * c->d, 1.0, c->dq, q[i]))) return bfail(b, rc, c->err);
      if ((rc = vec_axpy(c, c->ntr, 1.0, c->duh, uh[i]))) return bfail(b, rc, c->err);
      ++st[i].newton_steps;
    }
    BRC(assemble());
    bool again = false;
    for (int i = 0; i < N; ++i) {
      if (!active[i]) continue;
      mehdg_ctx* c = b->ctx[i];
      const double rf = b->hnorm[4 * i + 3];
      if (!std::isfinite(rf) || rf > 2.0 * RF[i]) {
        // the step left the physical states (a non-finite residual) or more than doubled the
        // residual: back to the previous state with a ten times smaller pseudo-time step
        const long long nu = (long long)c->E * c->Nu;
        const double* pv = b->prev[i];
        int rc;
        if ((rc = vec_copy(c, nu, pv, u[i])) || (rc = vec_copy(c, nu * c->d, pv + nu, q[i])) ||
            (rc = vec_copy(c, c->ntr, pv + nu * (1 + c->d), uh[i])))
          return bfail(b, rc, c->err);
        dtau[i] = std::max(dtau[i] * 0.1, 1e-8);
        st[i].status |= 4;
        again = true;
        if (++retries[i] > 20) active[i] = 0;   // given up: reported as not converged
        continue;
      }
      const double ru = std::sqrt(b->hnorm[4 * i + 1]);
      dtau[i] = std::min(std::max(dtau[i] * RU[i] / std::max(ru, 1e-300), c->opt.tau_init), c->opt.tau_max);
      RU[i] = ru;
      RF[i] = rf;
      st[i].res = rf;
      if (conv(i)) {
        active[i] = 0;
        st[i].status |= 2;
      } else if (st[i].newton_steps >= c->opt.max_newton) {
        active[i] = 0;
      }
    }
    if (again) BRC(assemble());   // the restored states, assembled again for the next round
    ++r;
  }
  if (rounds) *rounds = r;
  for (int i = 0; i < N; ++i)
    if (!(st[i].status & 2))
      return bfail(b, MEHDG_ERR_NOT_CONVERGED, "problem " + std::to_string(i) + ": not converged");
  return MEHDG_OK;
}

extern "C" void mehdg_batch_destroy(mehdg_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gasm) cudaGraphExecDestroy(b->gasm);
  if (b->gcond) cudaGraphExecDestroy(b->gcond);
  for (Queue& q : b->q)
    if (q.items) cudaFree(q.items);
  for (void* p : {(void*)b->counter, (void*)b->dshift, (void*)b->dnorm, (void*)b->dpart})
    if (p) cudaFree(p);
  if (b->hnorm) cudaFreeHost(b->hnorm);
  if (b->hflag) cudaFreeHost(b->hflag);
  if (b->hshift) cudaFreeHost(b->hshift);
  for (double* pv : b->prev)
    if (pv) cudaFree(pv);
  for (mehdg_ctx* c : b->ctx) mehdg_destroy(c);
  if (b->own) cudaStreamDestroy(b->own);
  delete b;
}

// the queued LU on caller matrices of uneven size: one persistent launch
extern "C" int mehdg_lu_queue(int nmat, const int* n, void* const* A, int* const* perm, int fp32, int nb, int* dflag,
                              void* stream) {
  if (nmat < 0 || (nmat > 0 && (!n || !A || !perm || !dflag)) || !(nb == 8 || nb == 16 || nb == 32)) return MEHDG_ERR_ARG;
  mehdg_batch tmp;
  mehdg_batch* b = &tmp;
  b->stream = static_cast<cudaStream_t>(stream);
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev));
  std::vector<LuItem> it(nmat);
  for (int i = 0; i < nmat; ++i) {
    if (n[i] < 1 || !A[i] || !perm[i]) return MEHDG_ERR_ARG;
    if ((fp32 ? queue_smem<float>(n[i], nb) : queue_smem<double>(n[i], nb)) > kSmemLimit) {
      fprintf(stderr, "mehdg_lu_queue: n = %d with panel width %d does not fit in shared memory\n", n[i], nb);
      return MEHDG_ERR_TOO_LARGE;
    }
    it[i] = LuItem{A[i], perm[i], dflag, n[i], nb, i + 1, 0};
  }
  BCK(cudaMemsetAsync(dflag, 0, sizeof(int) * 2, b->stream));
  Queue q;
  int* counter = nullptr;
  BCK(cudaMalloc(&counter, sizeof(int)));
  int rc = fp32 ? make_queue<float>(b, q, it) : make_queue<double>(b, q, it);
  if (!rc) rc = fp32 ? launch_queue<float>(b, q, counter) : launch_queue<double>(b, q, counter);
  int h[2] = {0, 0};
  if (!rc) {
    BCK(cudaMemcpyAsync(h, dflag, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
  }
  if (q.items) cudaFree(q.items);
  cudaFree(counter);
  if (rc) {
    fprintf(stderr, "mehdg_lu_queue: %s\n", b->err.c_str());
    return rc;
  }
  if (h[0]) {
    fprintf(stderr, "mehdg_lu_queue: zero pivot in matrix %d\n", h[1] - 1);
    return MEHDG_ERR_SINGULAR;
  }
  return MEHDG_OK;
}
