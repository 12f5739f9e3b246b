// C ABI of libpsp (include/psp.h): handle, workspace, captured restart cycles and the host
// loop of one implicit-Euler step (Eq. 4) solved by Algorithm 1 with the progressive
// preconditioner of Algorithm 2.
//
// One restart cycle of Algorithm 1 is captured once as a CUDA graph: the FP64 restart
// residual, then for k = 1..m the preconditioner solve (or a scaled copy when N = I), the
// stencil matvec and the three Gram-Schmidt passes whose last CTA runs the Givens step,
// then the update Z = V Q, X = X_0 + N^{-1} Z and a copy of the cycle summary to pinned
// host memory.  Kernels after the finish test see DevState::active == 0 and return at
// once, so the host waits once per cycle, not once per iteration.  Three graphs exist:
// N = I and one per factor slot (the adopted N and a freshly fitted candidate).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <type_traits>
#include <atomic>
#include <mutex>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "band_solve.cuh"
#include "onchip.cuh"

namespace {

thread_local std::string g_last_error;

// A host-side NVTX range for the scope (a step, a segment of restart cycles, a fit, a batch):
// a profiler's timeline shows the library's phases; without a tool attached a range costs a
// branch.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

psp_status fail(psp_status s, const std::string &msg) {
  g_last_error = msg;
  return s;
}

#define PSP_CUDA(call)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(PSP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
  } while (0)

// Finite-difference weights of the derivatives 0..M at z on the nodes x[0..n-1]
// (Fornberg's recursion, Math. Comp. 51 (1988) 699-706), c[j*(M+1) + m].
void fornberg(int M, long double z, const std::vector<long double> &x, std::vector<long double> &c) {
  const int n = (int)x.size();
  c.assign((size_t)n * (M + 1), 0.0L);
  long double c1 = 1.0L, c4 = x[0] - z;
  c[0] = 1.0L;
  for (int i = 1; i < n; ++i) {
    const int mn = std::min(i, M);
    long double c2 = 1.0L;
    const long double c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      const long double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k)
          c[(size_t)i * (M + 1) + k] = c1 * (k * c[(size_t)(i - 1) * (M + 1) + k - 1] -
                                             c5 * c[(size_t)(i - 1) * (M + 1) + k]) / c2;
        c[(size_t)i * (M + 1)] = -c1 * c5 * c[(size_t)(i - 1) * (M + 1)] / c2;
      }
      for (int k = mn; k >= 1; --k)
        c[(size_t)j * (M + 1) + k] = (c4 * c[(size_t)j * (M + 1) + k] - k * c[(size_t)j * (M + 1) + k - 1]) / c3;
      c[(size_t)j * (M + 1)] = c4 * c[(size_t)j * (M + 1)] / c3;
    }
    c1 = c2;
  }
}

// Central weights w_{-r..r} for d^k/dx^k of even accuracy order p, r = (k-1)/2 + p/2.
std::vector<double> central_weights(int k, int p) {
  const int r = (k - 1) / 2 + p / 2;
  std::vector<long double> x;
  for (int j = -r; j <= r; ++j) x.push_back((long double)j);
  std::vector<long double> c;
  fornberg(k, 0.0L, x, c);
  std::vector<double> w(2 * r + 1);
  for (int j = 0; j < 2 * r + 1; ++j) w[j] = (double)c[(size_t)j * (k + 1) + k];
  return w;
}

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

}  // namespace

namespace psp {
// Lets other translation units of the library report through psp_last_error().
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace psp

using namespace psp;

constexpr int kProfileEvery = 4;   // profiling samples iterations 1, 5, 9, ...

struct psp_ctx {
  Geometry geo{};
  double h[3] = {0, 0, 0};
  double wdir[3][2 * kMaxR + 1] = {};   // stencil of L per direction (no dt)
  int order = 0, b = 0, m = 0;
  psp_opts opts{};
  bool mixed = false;
  bool fused = false;                // matvec folded into the first Gram-Schmidt pass
  cudaStream_t stream = nullptr;     // caller's stream
  cudaStream_t cap = nullptr;        // internal capture stream
  int64_t ld = 0;                    // leading dimension of every n-vector column
  int mmax = 0;

  // device workspace
  void *V = nullptr, *Px = nullptr, *Py = nullptr, *Z = nullptr;   // Krylov precision
  double *X = nullptr, *B = nullptr;                               // FP64 solution / rhs
  double *partial = nullptr;
  DevState *st = nullptr;
  DevState *api_st = nullptr;        // coefficients for psp_matvec
  double *moments = nullptr;
  double *band_adopted = nullptr, *band_cand = nullptr;
  int *dev_int = nullptr;            // [0] factor failure, [1] singular rows
  void *slot_mem[BandSolver::kSlots] = {nullptr, nullptr, nullptr};
  double *band_T = nullptr;          // N^T of the adopted N (transposed solve)
  double *Ab = nullptr;              // explicit banded operator (psp_create_banded), FP64
  float *Ab32 = nullptr;             // ... and its FP32 copy
  int adopted_version = 0;           // bumped whenever the adopted N changes
  int t_version = -1;                // adopted_version that slot 2 (N^T) was factored for
  // per-term stencils of L (unit alpha, h^-k folded in), for psp_apply_L
  std::vector<std::pair<int, std::vector<double>>> term_w;
  std::vector<double> term_alpha;    // alpha of each term (psp_adjoint_grads)
  double *grad_dev = nullptr;        // kMaxTerms per-term dot products (psp_adjoint_grads)
  void *apply_mem = nullptr;
  BandSolver bs;

  // host mirrors
  CycleSummary *sum_host = nullptr;  // pinned
  DevState *st_host = nullptr;       // pinned staging for parameter uploads
  int *int_host = nullptr;           // pinned

  // preconditioner state
  int adopted = -1;      // slot of the adopted N, -1: N = I
  int cand = -1;         // slot of an untried candidate, -1: none
  double rate_ref = -1;  // reference per-iteration residual reduction
  int wait = 0, wait_len = 1;
  double hist_dt = NAN;
  double api_dt = NAN;   // dt of the coefficients in api_st (psp_matvec)
  int last_singular = 0;

  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // [0] N = I, [1] slot 0, [2] slot 1
  int graph_kernels[3] = {0, 0, 0};                          // kernel nodes per graph
  // segment graphs: the cycle graph's body in a WHILE node, the restart loop on the device
  cudaGraphExec_t seg_graph[3] = {nullptr, nullptr, nullptr};
  int seg_kernels[3] = {0, 0, 0};    // kernel nodes of one cycle of the body
  bool seg_ok = true;                // false once building a segment graph failed (per-cycle graphs then)
  SegSummary *seg_dev = nullptr;     // device
  SegSummary *seg_host = nullptr;    // pinned: [0] the launch's initial state, [1] the result
  bool profiling = false;
  bool restart_df_ok = false;        // the mixed cycle graphs hold the double-float restart
  double last_batch_s = 0.0;         // wall time of its last step on psp_step_batch's graph path
  cudaEvent_t ev[3][kMaxM][6] = {};                          // profiling events per graph
  psp_profile prof{};
  double *hostbuf = nullptr;   // pinned staging for psp_step_host
  double *dev_un = nullptr, *dev_unp1 = nullptr;
  // host waits of psp_step: a stream synchronisation (the CUDA runtime spin-waits), or with
  // blocking_wait a blocking-sync event, on which the thread sleeps -- set by psp_step_batch
  // when it runs more threads than the host has cores
  bool blocking_wait = false;
  cudaEvent_t wait_ev = nullptr;
  // psp_step_batch's graph path steps the handle on a stream of its own host thread; this
  // event orders that work after the work already on the handle's stream, and later work on
  // the handle's stream after it
  cudaEvent_t join_ev = nullptr;
  // integrators (psp_step_bdf2, psp_step_sdirk2): right-hand side and first-stage vectors
  double *int_rhs = nullptr, *int_u1 = nullptr;
  int hist_count_host = 0;   // history columns at the end of the last step (0 after a clear)
  // the history length a rolled-back segment reached (a broken trial, a step with a
  // non-finite residual): ring slots [count, hist_poison) mod mmax hold its pairs until
  // later pairs overwrite them (0 after a clear)
  int hist_poison = 0;
  // on-chip path (one CTA runs all cycles of a step): its descriptor and result
  bool onchip = false;
  int oc_threads = 256;        // CTA size of this system's on-chip launches
  int oc_ctas_per_sm = 2;      // resident CTAs per SM of a batched launch
  OnChipDesc *oc_desc = nullptr, *oc_desc_host = nullptr;
  OnChipResult *oc_res = nullptr, *oc_res_host = nullptr;
};

namespace {

// Wait for everything enqueued on s so far (see psp_ctx::blocking_wait).
// History pairs valid at history length `count`: the last min(count, mmax), less the ring
// slots that still hold the pairs of a rolled-back segment.  Those lie inside the ring's
// valid window only once the ring has wrapped past them (hist_poison > mmax).
int hist_valid(const psp_ctx *h, int count) {
  int c = std::min(count, h->mmax);
  if (h->hist_poison > h->mmax) c = std::min(c, std::max(0, count + h->mmax - h->hist_poison));
  return c;
}

cudaError_t host_wait(psp_ctx *h, cudaStream_t s) {
  if (h->blocking_wait && h->wait_ev) {
    cudaError_t e = cudaEventRecord(h->wait_ev, s);
    return e != cudaSuccess ? e : cudaEventSynchronize(h->wait_ev);
  }
  return cudaStreamSynchronize(s);
}

void set_coef(const psp_ctx *h, double dt, double (*coef)[2 * kMaxR + 1]) {
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 2 * kMaxR + 1; ++j) coef[d][j] = (d < h->geo.ndim) ? -dt * h->wdir[d][j] : 0.0;
  double centre = 1.0;
  for (int d = 0; d < 3; ++d) {
    centre += coef[d][kMaxR];
    coef[d][kMaxR] = 0.0;
  }
  coef[0][kMaxR] = centre;
}

template <typename T>
void enqueue_cycle(psp_ctx *h, int slot, cudaStream_t s, bool summary_copy = true) {
  T *V = reinterpret_cast<T *>(h->V);
  T *Px = reinterpret_cast<T *>(h->Px);
  T *Py = reinterpret_cast<T *>(h->Py);
  T *Z = reinterpret_cast<T *>(h->Z);
  const Geometry &g = h->geo;
  if constexpr (std::is_same<T, float>::value) {
    // columns 1 and 2 of the basis are free until the first iteration writes v_1
    float *Xh = h->m >= 2 ? V + h->ld : nullptr;
    h->restart_df_ok =
        launch_restart_mixed(g, h->X, h->B, Px, Py, h->ld, V, Xh, Xh ? Xh + h->ld : nullptr, h->st, h->partial, s);
  } else {
    launch_restart<T, T>(g, h->X, h->B, Px, Py, h->ld, V, h->st, h->partial, h->mixed ? 1 : 0, s);
  }
  const int *active = &h->st->active;
  const int which = slot + 1;
  // iteration j: Y_j = N^{-1} v_j -> P_x ring column hist_base+1+j, w_j = A Y_j -> P_y column,
  // then the DCGS2 passes (orthogonalise, complete column j-1, Givens, finish test)
  const bool fused = h->fused;
  for (int j = 0; j < h->m; ++j) {
    // profiling samples one iteration in kProfileEvery
    cudaEvent_t *ev = (h->profiling && j % kProfileEvery == 0) ? h->ev[which][j] : nullptr;
    OutRef<T> pxcol = ring_out<T>(Px, h->ld, &h->st->hist_base, h->mmax, 1 + j);
    OutRef<T> pycol = ring_out<T>(Py, h->ld, &h->st->hist_base, h->mmax, 1 + j);
    if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
    TileMatvec<T> mv{};
    if (slot < 0) {
      // N = I: P_x(:,i) = v_j and P_y(:,i) = A v_j
      if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
      if (fused) mv = TileMatvec<T>{fixed_in<T>(V + (int64_t)j * h->ld), pycol, pxcol, g.nx, g.ny, g.nz, g.ndim, g.R};
      else launch_stencil<T, T, T>(g, fixed_in<T>(V + (int64_t)j * h->ld), pycol, h->st, active, s, pxcol, nullptr);
    } else {
      h->bs.apply<T>(slot, V + (int64_t)j * h->ld, nullptr, active, pxcol, nullptr, 0, s);
      if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
      InRef<T> xin = ring_in<T>(Px, h->ld, &h->st->hist_base, h->mmax, 1 + j);
      if (fused) mv = TileMatvec<T>{xin, pycol, OutRef<T>{nullptr, 0, nullptr, 1, 0}, g.nx, g.ny, g.nz, g.ndim, g.R};
      else launch_stencil<T, T, T>(g, xin, pycol, h->st, active, s);
    }
    if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
    launch_arnoldi<T>(j, 0, g.n, V, h->ld, Py, h->ld, h->st, h->partial, h->mixed ? 1 : 0, s,
                      ev ? ev + 3 : nullptr, fused ? &mv : nullptr);
  }
  // reduction-only step completing column m-1 when the cycle runs to m columns
  launch_arnoldi<T>(h->m, 1, g.n, V, h->ld, Py, h->ld, h->st, h->partial, h->mixed ? 1 : 0, s, nullptr);
  if (slot < 0) {
    launch_update_z<T>(g.n, V, h->ld, Z, h->X, 1, h->st, s);
  } else {
    launch_update_z<T>(g.n, V, h->ld, Z, h->X, 0, h->st, s);
    h->bs.apply<T>(slot, Z, nullptr, &h->st->k_end, fixed_out<T>(nullptr), h->X, 1, s);
  }
  if (summary_copy) cudaMemcpyAsync(h->sum_host, &h->st->sum, sizeof(CycleSummary), cudaMemcpyDeviceToHost, s);
}

// One restart cycle of BiCGSTAB (FP64): the restart (true residual, restart pair), then m
// iterations, each storing its two matvec pairs (scaled by 1/||r||) at ring columns
// hist_base+1+2j and hist_base+2+2j; X is updated every iteration.
void enqueue_bicgstab_cycle(psp_ctx *h, int slot, cudaStream_t s, bool summary_copy = true) {
  double *V = reinterpret_cast<double *>(h->V);
  double *Px = reinterpret_cast<double *>(h->Px);
  double *Py = reinterpret_cast<double *>(h->Py);
  const Geometry &g = h->geo;
  const int64_t n = g.n, ld = h->ld;
  DevState *st = h->st;
  const int *active = &st->active;
  launch_restart<double, double>(g, h->X, h->B, Px, Py, ld, V, st, h->partial, 0, s);
  launch_bi_start(n, V, ld, st, s);
  const OutRef<double> none{nullptr, 0, nullptr, 1, 0};
  for (int j = 0; j < h->m; ++j) {
    const int c1 = 1 + 2 * j, c2 = 2 + 2 * j;   // ring offsets of the iteration's two pairs
    launch_bi_p(j == 0, n, V, ld, ring_in<double>(Py, ld, &st->hist_base, h->mmax, j > 0 ? c1 - 2 : 0),
                slot < 0 ? ring_out<double>(Px, ld, &st->hist_base, h->mmax, c1) : none, st, s);
    if (slot >= 0)
      h->bs.apply<double>(slot, V + 2 * ld, &st->bi[4], active, ring_out<double>(Px, ld, &st->hist_base, h->mmax, c1),
                          nullptr, 0, s);
    launch_stencil<double, double, double>(g, ring_in<double>(Px, ld, &st->hist_base, h->mmax, c1),
                                           ring_out<double>(Py, ld, &st->hist_base, h->mmax, c1), st, active, s);
    launch_bi_alpha(n, V, ld, ring_in<double>(Py, ld, &st->hist_base, h->mmax, c1), st, h->partial, s);
    launch_bi_s(n, V, ld, ring_in<double>(Py, ld, &st->hist_base, h->mmax, c1),
                slot < 0 ? ring_out<double>(Px, ld, &st->hist_base, h->mmax, c2) : none, st, s);
    if (slot >= 0)
      h->bs.apply<double>(slot, V + 3 * ld, &st->bi[4], active, ring_out<double>(Px, ld, &st->hist_base, h->mmax, c2),
                          nullptr, 0, s);
    launch_stencil<double, double, double>(g, ring_in<double>(Px, ld, &st->hist_base, h->mmax, c2),
                                           ring_out<double>(Py, ld, &st->hist_base, h->mmax, c2), st, active, s);
    launch_bi_omega(n, V, ld, ring_in<double>(Py, ld, &st->hist_base, h->mmax, c2), st, h->partial, s);
    launch_bi_xr(j, h->m, n, h->X, V, ld, ring_in<double>(Px, ld, &st->hist_base, h->mmax, c1),
                 ring_in<double>(Px, ld, &st->hist_base, h->mmax, c2),
                 ring_in<double>(Py, ld, &st->hist_base, h->mmax, c2), st, h->partial, s);
  }
  if (summary_copy) cudaMemcpyAsync(h->sum_host, &h->st->sum, sizeof(CycleSummary), cudaMemcpyDeviceToHost, s);
}

psp_status capture(psp_ctx *h, int which) {
  cudaGraph_t graph;
  PSP_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  const int slot = which - 1;
  if (h->opts.solver == PSP_SOLVER_BICGSTAB) enqueue_bicgstab_cycle(h, slot, h->cap);
  else if (h->mixed) enqueue_cycle<float>(h, slot, h->cap);
  else enqueue_cycle<double>(h, slot, h->cap);
  cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
  if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(graph, nodes.data(), &nn);
  int kn = 0;
  for (size_t i = 0; i < nn; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
  }
  h->graph_kernels[which] = kn;
  e = cudaGraphInstantiate(&h->graph[which], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return PSP_OK;
}

psp_status ensure_graph(psp_ctx *h, int which) {
  if (h->graph[which]) return PSP_OK;
  return capture(h, which);
}

// The segment graph of slot `which`: a WHILE conditional node whose body is one restart cycle
// (the cycle graph's kernels, then k_seg_control, which sets the condition), followed by the
// copy of the segment summary to the host.  Returns false (and leaves no graph) when the
// runtime refuses any step of it; the caller then runs the per-cycle graphs.
bool capture_segment(psp_ctx *h, int which) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t loop = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  cudaGraph_t body = nullptr;
  if (ok) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = cond;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    ok = cudaGraphAddNode(&loop, g, nullptr, nullptr, 0, &p) == cudaSuccess;
    if (ok) body = p.conditional.phGraph_out[0];
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      const int slot = which - 1;
      if (h->opts.solver == PSP_SOLVER_BICGSTAB) enqueue_bicgstab_cycle(h, slot, h->cap, false);
      else if (h->mixed) enqueue_cycle<float>(h, slot, h->cap, false);
      else enqueue_cycle<double>(h, slot, h->cap, false);
      launch_seg_control(h->st, h->seg_dev, cond, h->cap);
      cudaGraph_t out = nullptr;
      ok = cudaStreamEndCapture(h->cap, &out) == cudaSuccess;
    }
  }
  if (ok) {
    ok = cudaStreamBeginCaptureToGraph(h->cap, g, &loop, nullptr, 1, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      cudaMemcpyAsync(h->seg_host + 1, h->seg_dev, sizeof(SegSummary), cudaMemcpyDeviceToHost, h->cap);
      cudaGraph_t out = nullptr;
      ok = cudaStreamEndCapture(h->cap, &out) == cudaSuccess;
    }
  }
  if (ok) {
    size_t nn = 0;
    cudaGraphGetNodes(body, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(body, nodes.data(), &nn);
    int kn = 0;
    for (size_t i = 0; i < nn; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kn;
    }
    h->seg_kernels[which] = kn;
    ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  }
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();   // a refused step must not surface as a later launch error
    if (exec) cudaGraphExecDestroy(exec);
    return false;
  }
  h->seg_graph[which] = exec;
  return true;
}

// Factor band (device) into `slot`; returns PSP_ERR_NUMERIC on a failed pivot.
psp_status factor_into(psp_ctx *h, int slot, const double *band) {
  PSP_CUDA(cudaMemsetAsync(h->dev_int, 0, sizeof(int), h->stream));
  h->bs.factor(slot, band, h->dev_int, h->stream);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("band factorisation launch: ") + cudaGetErrorString(e));
  }
  PSP_CUDA(cudaMemcpyAsync(h->int_host, h->dev_int, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PSP_CUDA(host_wait(h, h->stream));
  if (h->int_host[0]) return fail(PSP_ERR_NUMERIC, "band factorisation: zero or non-finite pivot");
  // cyclic band: the corner columns' solves and the capacitance matrix of the slot
  if (h->bs.cyclic && !h->bs.prepare_cyclic(slot, band, h->stream)) {
    cudaGetLastError();
    return fail(PSP_ERR_NUMERIC, "cyclic band: singular capacitance matrix");
  }
  return PSP_OK;
}

template <typename TH>
psp_status fit_into(psp_ctx *h, const TH *Px, const TH *Py, int64_t ld, int M, double *band, int *singular) {
  PSP_CUDA(cudaMemsetAsync(h->dev_int + 1, 0, sizeof(int), h->stream));
  launch_fit<TH>(h->b, h->opts.intercept, h->geo.n, M, Px, Py, ld, h->moments, band, h->dev_int + 1, h->stream,
                 h->opts.cyclic);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("band fit launch: ") + cudaGetErrorString(e));
  }
  PSP_CUDA(cudaMemcpyAsync(h->int_host + 1, h->dev_int + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PSP_CUDA(host_wait(h, h->stream));
  if (singular) *singular = h->int_host[1];
  return PSP_OK;
}

// Algorithm 2's fit of the candidate band (into band_cand) from the first M history columns
// and its factorisation into slot `slot`, with one host synchronisation for both outcomes:
// *singular = the fit's degenerate rows; PSP_ERR_NUMERIC if a pivot (or the cyclic band's
// capacitance matrix) failed.
template <typename TH>
psp_status fit_and_factor(psp_ctx *h, const TH *Px, const TH *Py, int M, int slot, int *singular) {
  NvtxRange range("psp_fit");
  PSP_CUDA(cudaMemsetAsync(h->dev_int, 0, 2 * sizeof(int), h->stream));
  launch_fit<TH>(h->b, h->opts.intercept, h->geo.n, M, Px, Py, h->ld, h->moments, h->band_cand, h->dev_int + 1,
                 h->stream, h->opts.cyclic);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("band fit launch: ") + cudaGetErrorString(e));
  }
  h->bs.factor(slot, h->band_cand, h->dev_int, h->stream);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PSP_ERR_CUDA, std::string("band factorisation launch: ") + cudaGetErrorString(e));
  }
  PSP_CUDA(cudaMemcpyAsync(h->int_host, h->dev_int, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PSP_CUDA(host_wait(h, h->stream));
  *singular = h->int_host[1];
  if (h->int_host[0]) return fail(PSP_ERR_NUMERIC, "band factorisation: zero or non-finite pivot");
  if (h->bs.cyclic && !h->bs.prepare_cyclic(slot, h->band_cand, h->stream)) {
    cudaGetLastError();
    return fail(PSP_ERR_NUMERIC, "cyclic band: singular capacitance matrix");
  }
  return PSP_OK;
}

// Add the device time of the sampled iterations among 1..k_end of the last replay of graph
// `which`.
void accumulate_profile(psp_ctx *h, int which, int k_end) {
  const double s = h->mixed ? 4.0 : 8.0;
  const double n = (double)h->geo.n;
  for (int k = 1; k <= k_end && k <= h->m; k += kProfileEvery) {
    cudaEvent_t *ev = h->ev[which][k - 1];
    float ms[5];
    for (int c = 0; c < 5; ++c)
      if (cudaEventElapsedTime(&ms[c], ev[c], ev[c + 1]) != cudaSuccess) {
        ms[c] = 0.0f;
        cudaGetLastError();   // a failed query must not surface as a later launch error
      }
    // N = I: the stencil reads V(:,k) and writes the P_x and P_y columns (class 1; class 0
    // is then empty).  DCGS2 at iteration j = k-1: pass A reads V(:,0..j) and w_j (k+1
    // vectors), pass B reads the same and writes q_j and v_{j+1} (class 3 is empty).  With
    // the matvec folded into pass A, class 1 is empty and pass A moves V(:,0..j) and the
    // matvec's input in, w_j (and the P_x copy) out: k+2 vectors.
    const double st_bytes = h->fused ? 0.0 : (which == 0 ? 3.0 : 2.0) * s * n;
    const double dots_bytes = (h->fused ? k + 2.0 : k + 1.0) * s * n;
    const double bytes[5] = {(which == 0 ? 0.0 : (2.0 * h->b + 3.0)) * s * n, st_bytes, dots_bytes, 0.0,
                             (k + 3.0) * s * n};
    for (int c = 0; c < 5; ++c) {
      if (bytes[c] == 0.0) continue;
      h->prof.ms[c] += ms[c];
      h->prof.bytes[c] += bytes[c];
      h->prof.launches[c] += 1;
    }
  }
}

double rate_of(double R_end, double beta, int k) {
  if (k <= 0 || !(beta > 0.0)) return 1.0;
  return std::pow(std::max(R_end, 1e-300) / beta, 1.0 / k);
}

// Slot 2 holds the factors of N^T for the adopted N (made on first use after a change).
psp_status ensure_transposed(psp_ctx *h) {
  if (h->t_version == h->adopted_version) return PSP_OK;
  launch_transpose_band(h->band_adopted, h->band_T, h->geo.n, h->b, h->stream, h->bs.cyclic);
  PSP_CUDA(cudaGetLastError());
  psp_status s = factor_into(h, 2, h->band_T);
  if (s != PSP_OK) return s;
  h->t_version = h->adopted_version;
  return PSP_OK;
}

// Coefficients of L (term < 0) or of one term's derivative with unit alpha (term >= 0), in
// the stencil kernels' layout (centres folded into direction 0), without dt or identity.
void set_L_coef(const psp_ctx *h, int term, double (*coef)[2 * kMaxR + 1]) {
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 2 * kMaxR + 1; ++j) coef[d][j] = 0.0;
  if (term < 0) {
    for (int d = 0; d < h->geo.ndim; ++d)
      for (int j = 0; j < 2 * kMaxR + 1; ++j) coef[d][j] = h->wdir[d][j];
  } else {
    const auto &tw = h->term_w[term];
    for (int j = 0; j < 2 * kMaxR + 1; ++j) coef[tw.first][j] = tw.second[j];
  }
  double centre = 0.0;
  for (int d = 0; d < 3; ++d) {
    centre += coef[d][kMaxR];
    coef[d][kMaxR] = 0.0;
  }
  coef[0][kMaxR] = centre;
}

// Coefficients of A for psp_matvec, uploaded only when dt differs from the last call's.
psp_status upload_api_coef(psp_ctx *h, double dt) {
  if (h->api_dt == dt) return PSP_OK;
  set_coef(h, dt, h->st_host->coef);
  PSP_CUDA(cudaMemcpyAsync(h->api_st->coef, h->st_host->coef, sizeof(h->st_host->coef), cudaMemcpyHostToDevice,
                           h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));   // the pinned staging is reused by psp_step
  h->api_dt = dt;
  return PSP_OK;
}

}  // namespace

extern "C" {

const char *psp_last_error(void) { return g_last_error.c_str(); }

psp_status psp_default_opts(psp_opts *o) {
  if (!o) return fail(PSP_ERR_ARG, "opts is NULL");
  o->precision = PSP_FP64;
  o->intercept = 1;
  o->max_restarts = 200;
  o->max_hist_cols = 0;
  o->inner_tol = 1e-5;
  o->accept_rule = 1;
  o->fuse_matvec = 1;
  o->adjoint = 0;
  o->cyclic = 0;
  o->solver = PSP_SOLVER_GMRES;
  o->onchip = -1;
  o->cycle_loop = 0;
  return PSP_OK;
}

psp_status psp_create_banded(int64_t n, const double *A_band, int w, int b, int m, const psp_opts *opts,
                             void *cuda_stream, psp_handle *out) {
  if (!A_band || !out) return fail(PSP_ERR_ARG, "NULL argument");
  if (w < 1 || w > 64) return fail(PSP_ERR_ARG, "band half-width w must be in 1..64");
  if (n < 3 || n < 2 * (int64_t)w + 1) return fail(PSP_ERR_ARG, "need n >= max(3, 2w+1)");
  psp_opts o;
  psp_default_opts(&o);
  if (opts) o = *opts;
  if (o.cyclic) return fail(PSP_ERR_ARG, "a cyclic band needs a periodic grid (psp_create, ndim = 1)");
  const int adjoint = o.adjoint;
  o.adjoint = 0;
  o.fuse_matvec = 0;
  // a 1D handle whose placeholder stencil (a zero-coefficient second difference) the banded
  // operator replaces: the solver, history, fit and preconditioner are the same
  psp_grid g{};
  g.ndim = 1;
  g.n[0] = n;
  g.n[1] = g.n[2] = 1;
  g.length[0] = g.length[1] = g.length[2] = 1.0;
  psp_term t{2, 0, 0.0};
  psp_handle h = nullptr;
  psp_status s = psp_create(&g, 2, &t, 1, b, m, &o, cuda_stream, &h);
  if (s != PSP_OK) return s;
  h->opts.adjoint = adjoint;
  const int64_t cnt = n * (2 * w + 1);
  if (cudaMalloc((void **)&h->Ab, cnt * 8) != cudaSuccess || cudaMalloc((void **)&h->Ab32, cnt * 4) != cudaSuccess) {
    cudaGetLastError();
    psp_destroy(h);
    return fail(PSP_ERR_OOM, "banded operator storage");
  }
  if (adjoint) launch_transpose_band(A_band, h->Ab, n, w, h->stream);
  else cudaMemcpyAsync(h->Ab, A_band, cnt * 8, cudaMemcpyDeviceToDevice, h->stream);
  launch_to_f32(h->Ab, h->Ab32, cnt, h->stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) {
    psp_destroy(h);
    return fail(PSP_ERR_CUDA, "banded operator upload");
  }
  h->geo.band_w = w;
  h->geo.Ab = h->Ab;
  h->geo.Ab32 = h->Ab32;
  h->fused = false;
  *out = h;
  return PSP_OK;
}

psp_status psp_destroy(psp_handle h) {
  if (!h) return PSP_OK;
  for (auto &g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : h->seg_graph)
    if (g) cudaGraphExecDestroy(g);
  for (auto &a : h->ev)
    for (auto &b : a)
      for (auto &e : b)
        if (e) cudaEventDestroy(e);
  void *dev[] = {h->V, h->Px, h->Py, h->Z, h->X, h->B, h->partial, h->st, h->api_st, h->moments,
                 h->band_adopted, h->band_cand, h->dev_int, h->slot_mem[0], h->slot_mem[1], h->slot_mem[2],
                 h->band_T, h->Ab, h->Ab32, h->apply_mem, h->grad_dev,
                 h->dev_un, h->dev_unp1, h->int_rhs, h->int_u1, h->oc_desc, h->oc_res, h->seg_dev};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (h->oc_desc_host) cudaFreeHost(h->oc_desc_host);
  if (h->oc_res_host) cudaFreeHost(h->oc_res_host);
  if (h->sum_host) cudaFreeHost(h->sum_host);
  if (h->seg_host) cudaFreeHost(h->seg_host);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->int_host) cudaFreeHost(h->int_host);
  if (h->hostbuf) cudaFreeHost(h->hostbuf);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->wait_ev) cudaEventDestroy(h->wait_ev);
  if (h->join_ev) cudaEventDestroy(h->join_ev);
  delete h;
  return PSP_OK;
}

psp_status psp_create(const psp_grid *grid, int order, const psp_term *terms, int nterms, int b, int m,
                      const psp_opts *opts, void *cuda_stream, psp_handle *out) {
  if (!grid || !terms || !out) return fail(PSP_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (grid->ndim < 1 || grid->ndim > 3) return fail(PSP_ERR_ARG, "ndim must be 1, 2 or 3");
  if (order != 2 && order != 4 && order != 6 && order != 8) return fail(PSP_ERR_ARG, "order must be 2, 4, 6 or 8");
  if (b < 1 || b > kMaxB) return fail(PSP_ERR_ARG, "band half-width b must be in 1..4");
  if (m < 1 || m > kMaxM) return fail(PSP_ERR_ARG, "restart length m must be in 1..64");
  if (nterms < 1) return fail(PSP_ERR_ARG, "need at least one term");
  psp_opts o;
  psp_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != PSP_FP64 && o.precision != PSP_MIXED) return fail(PSP_ERR_ARG, "bad precision");
  if (o.max_restarts < 1) return fail(PSP_ERR_ARG, "max_restarts must be >= 1");
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return fail(PSP_ERR_ARG, "inner_tol must be in (0, 1)");
  if (o.solver != PSP_SOLVER_GMRES && o.solver != PSP_SOLVER_BICGSTAB) return fail(PSP_ERR_ARG, "bad solver");
  if (o.solver == PSP_SOLVER_BICGSTAB && (o.precision != PSP_FP64 || m < 3))   // V columns r, rh, p, s
    return fail(PSP_ERR_ARG, "the BiCGSTAB solver runs in FP64 with m >= 3");

  psp_ctx *h = new psp_ctx();
  h->order = order;
  h->b = b;
  h->m = m;
  h->opts = o;
  h->mixed = (o.precision == PSP_MIXED);
  h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  int64_t nn[3] = {1, 1, 1};
  for (int d = 0; d < grid->ndim; ++d) {
    if (grid->n[d] < 1 || !(grid->length[d] > 0.0)) {
      delete h;
      return fail(PSP_ERR_ARG, "grid sizes and lengths must be positive");
    }
    nn[d] = grid->n[d];
    h->h[d] = grid->length[d] / (double)grid->n[d];
  }
  const int64_t n = nn[0] * nn[1] * nn[2];
  if (n > (int64_t)1 << 31) { delete h; return fail(PSP_ERR_ARG, "at most 2^31 unknowns"); }
  if (n < 2 * b + 1) { delete h; return fail(PSP_ERR_ARG, "need n >= 2b+1"); }
  if (o.cyclic && (grid->ndim != 1 || n < 4 * b + 2)) {
    delete h;
    return fail(PSP_ERR_ARG, "a cyclic band needs a 1D grid with n >= 4b+2");
  }
  int R = 1;
  for (int t = 0; t < nterms; ++t) {
    const psp_term &tm = terms[t];
    if (tm.k < 1 || tm.k > 4 || tm.dir < 0 || tm.dir >= grid->ndim) {
      delete h;
      return fail(PSP_ERR_ARG, "term needs k in 1..4 and 0 <= dir < ndim");
    }
    const int r = (tm.k - 1) / 2 + order / 2;
    const std::vector<double> w = central_weights(tm.k, order);
    const double hk = std::pow(h->h[tm.dir], -(double)tm.k);
    const double sc = tm.alpha * hk;
    std::vector<double> tw(2 * kMaxR + 1, 0.0);
    for (int j = -r; j <= r; ++j) {
      h->wdir[tm.dir][kMaxR + j] += sc * w[j + r];
      tw[kMaxR + j] = hk * w[j + r];
    }
    h->term_w.emplace_back(tm.dir, std::move(tw));
    h->term_alpha.push_back(tm.alpha);
    R = std::max(R, r);
  }
  if (o.adjoint) {
    // A^T = I - dt L^T: on a periodic grid L^T applies every stencil mirrored, w_j -> w_-j
    for (int d = 0; d < 3; ++d)
      for (int j = 1; j <= kMaxR; ++j) std::swap(h->wdir[d][kMaxR + j], h->wdir[d][kMaxR - j]);
    for (auto &tw : h->term_w)
      for (int j = 1; j <= kMaxR; ++j) std::swap(tw.second[kMaxR + j], tw.second[kMaxR - j]);
  }
  for (int d = 0; d < grid->ndim; ++d)
    if (2 * R + 1 > nn[d]) { delete h; return fail(PSP_ERR_ARG, "every direction needs n >= 2R+1 (R: widest stencil radius)"); }
  h->geo.ndim = grid->ndim;
  h->geo.nx = (int)nn[0];
  h->geo.ny = (int)nn[1];
  h->geo.nz = (int)nn[2];
  h->geo.n = n;
  h->geo.R = R;
  h->fused = o.fuse_matvec != 0 && fused_matvec_ok(h->geo, h->mixed ? 4 : 8);
  // the on-chip path: one CTA runs all the cycles of a step (GMRES only); by default for the
  // systems small enough that launch latency, not bandwidth, bounds the cycle graphs
  h->onchip = o.solver == PSP_SOLVER_GMRES && n <= kOnChipMaxN &&
              (o.onchip > 0 || (o.onchip < 0 && n <= kOnChipAutoN));
  h->oc_threads = onchip_threads_for(n);
  h->ld = round_up(n, 512);   // every column starts on a 2 KB boundary (16-byte vector loads)
  h->mmax = o.max_hist_cols > 0 ? o.max_hist_cols : 2 * (m + 1);
  if (h->mmax < m + 1) h->mmax = m + 1;
  const size_t es = h->mixed ? sizeof(float) : sizeof(double);
  arnoldi_setup();

  auto dalloc = [&](void **p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    return cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  bool ok = true;
  ok = ok && dalloc(&h->V, (size_t)h->ld * (m + 1) * es);
  ok = ok && dalloc(&h->Px, (size_t)h->ld * h->mmax * es);
  ok = ok && dalloc(&h->Py, (size_t)h->ld * h->mmax * es);
  ok = ok && dalloc(&h->Z, (size_t)h->ld * es);
  ok = ok && dalloc((void **)&h->X, (size_t)h->ld * 8);
  ok = ok && dalloc((void **)&h->B, (size_t)h->ld * 8);
  ok = ok && dalloc((void **)&h->partial, (size_t)3 * (kMaxM + 2) * kMaxCta * 8);   // three pass regions
  ok = ok && dalloc((void **)&h->st, sizeof(DevState));
  ok = ok && dalloc((void **)&h->api_st, sizeof(DevState));
  ok = ok && dalloc((void **)&h->moments, (size_t)n * (4 * b + 4) * 8);
  ok = ok && dalloc((void **)&h->band_adopted, (size_t)n * (2 * b + 1) * 8);
  ok = ok && dalloc((void **)&h->band_cand, (size_t)n * (2 * b + 1) * 8);
  ok = ok && dalloc((void **)&h->band_T, (size_t)n * (2 * b + 1) * 8);
  ok = ok && dalloc((void **)&h->dev_int, 64);
  ok = ok && dalloc((void **)&h->grad_dev, kMaxTerms * sizeof(double));
  ok = ok && dalloc((void **)&h->oc_desc, sizeof(OnChipDesc));
  ok = ok && dalloc((void **)&h->oc_res, sizeof(OnChipResult));
  ok = ok && cudaMallocHost((void **)&h->oc_desc_host, sizeof(OnChipDesc)) == cudaSuccess;
  ok = ok && cudaMallocHost((void **)&h->oc_res_host, sizeof(OnChipResult)) == cudaSuccess;
  if (ok) {
    h->bs.cyclic = o.cyclic != 0;
    h->bs.plan(n, b);
    for (int s = 0; s < BandSolver::kSlots && ok; ++s) {
      ok = dalloc(&h->slot_mem[s], h->bs.slot_bytes());
      if (ok) h->bs.bind(h->slot_mem[s], s);
    }
    ok = ok && dalloc(&h->apply_mem, h->bs.apply_bytes());
    if (ok) h->bs.bind_apply(h->apply_mem);
  }
  ok = ok && cudaMallocHost((void **)&h->sum_host, sizeof(CycleSummary)) == cudaSuccess;
  ok = ok && cudaMallocHost((void **)&h->seg_host, 2 * sizeof(SegSummary)) == cudaSuccess;
  ok = ok && dalloc((void **)&h->seg_dev, sizeof(SegSummary));
  ok = ok && cudaMallocHost((void **)&h->st_host, sizeof(DevState)) == cudaSuccess;
  ok = ok && cudaMallocHost((void **)&h->int_host, 64) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    psp_destroy(h);
    return fail(PSP_ERR_OOM, "device or pinned allocation failed");
  }
  std::memset(h->st_host, 0, sizeof(DevState));
  h->st_host->mmax = h->mmax;
  h->st_host->m = m;
  h->st_host->inner_tol = o.inner_tol;
  if (cudaMemcpy(h->st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->api_st, h->st_host, sizeof(DevState), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    psp_destroy(h);
    return fail(PSP_ERR_CUDA, "state upload failed");
  }
  *out = h;
  return PSP_OK;
}

}  // extern "C"

namespace {

// One launch's worth of restart cycles (one cycle graph, or an on-chip launch of up to
// max_cycles cycles) as the step's host logic sees it.
struct Segment {
  int cycles = 0, iters = 0, k_last = 0, status = 0, error = 0;
  bool df_restart = false;   // the cycle's restart ran in double-float
  int hist_count = 0;        // DevState::hist_count after the segment
  double beta_first = 0.0, beta_last = 0.0, R_last = 0.0, bnorm = 0.0;
};

// The host state of one psp_step between its segments.
struct StepRun {
  const double *u_n = nullptr;
  double *u_np1 = nullptr;
  double dt = 0.0, tol = 0.0;
  int iters = 0, cycles = 0, flags = 0, launches = 0, c = 0;
  bool converged = false, numeric = false, done = false;
  double last_R = 0.0, bnorm = 0.0;
  bool try_cand = false;
  int cur = -1;
  double trial_beta = -1.0, trial_R = 0.0, main_beta = -1.0, main_R = 0.0;
  int trial_iters = 0, main_iters = 0;
  int hist_before_trial = 0, prev_adopted = -1;
  int hist_count = 0;        // DevState::hist_count as of the last segment (or the rollback)
  bool adopted_now = false;
  psp_status status = PSP_OK;
};

// Parameters of the step, the back-off bookkeeping and the choice of the first cycle's N.
psp_status step_begin(psp_ctx *h, StepRun &r, const double *u_n, double *u_np1, double dt, double tol) {
  const int64_t n = h->geo.n;
  cudaStream_t s = h->stream;
  r = StepRun{};
  r.u_n = u_n;
  r.u_np1 = u_np1;
  r.dt = dt;
  r.tol = tol;
  if (!(h->hist_dt == dt)) {   // A changed: the history no longer describes it
    h->hist_dt = dt;
    h->cand = -1;
    h->rate_ref = -1.0;
    h->wait = 0;
    h->wait_len = 1;
    h->hist_count_host = 0;
    h->hist_poison = 0;
    PSP_CUDA(cudaMemsetAsync(&h->st->hist_count, 0, sizeof(int), s));
  }
  set_coef(h, dt, h->st_host->coef);
  h->st_host->tol = tol;
  h->st_host->first = 1;
  // the mixed form's restart residual in double-float (about 2^-45 sum|c| |x| of rounding)
  // when tol is well above it, else in FP64
  double csum = 0.0;
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 2 * kMaxR + 1; ++j) csum += std::fabs(h->st_host->coef[d][j]);
  h->st_host->restart_df = (h->mixed && tol >= std::ldexp(csum, -42)) ? 1 : 0;
  PSP_CUDA(cudaMemcpyAsync(&h->st->restart_df, &h->st_host->restart_df, sizeof(int), cudaMemcpyHostToDevice, s));
  PSP_CUDA(cudaMemcpyAsync(h->st->coef, h->st_host->coef, sizeof(h->st_host->coef), cudaMemcpyHostToDevice, s));
  PSP_CUDA(cudaMemcpyAsync(&h->st->tol, &h->st_host->tol, sizeof(double), cudaMemcpyHostToDevice, s));
  PSP_CUDA(cudaMemcpyAsync(&h->st->first, &h->st_host->first, sizeof(int), cudaMemcpyHostToDevice, s));
  PSP_CUDA(cudaMemcpyAsync(h->B, u_n, n * 8, cudaMemcpyDeviceToDevice, s));
  PSP_CUDA(cudaMemcpyAsync(h->X, u_n, n * 8, cudaMemcpyDeviceToDevice, s));
  // the first cycle may try the candidate (the acceptance rule: a fresh candidate runs the
  // step's first cycle and is adopted if that cycle converges or reduces the residual per
  // iteration at least as fast as the last step's cycles did; else it is dropped and the
  // next fit waits a number of steps that doubles with every rejection)
  r.try_cand = (h->cand >= 0 && h->wait == 0);
  if (!r.try_cand && h->wait > 0) h->wait -= 1;
  r.cur = r.try_cand ? h->cand : h->adopted;
  r.prev_adopted = h->adopted;
  r.hist_before_trial = h->hist_count_host;   // the history length to restore if the trial breaks
  r.hist_count = h->hist_count_host;
  return PSP_OK;
}

// Cycles the next segment may run: the candidate's trial cycle alone, else the rest.
int step_next_cycles(const psp_ctx *h, const StepRun &r) {
  return (r.c == 0 && r.try_cand) ? 1 : std::max(1, h->opts.max_restarts - r.c);
}

// Which cycle graph / factor slot the next segment uses (0: N = I, 1 + slot).
int step_which(const StepRun &r) { return r.cur < 0 ? 0 : r.cur + 1; }

// The host logic after a segment (Algorithm 1's restart loop with the acceptance rule).
psp_status step_after_segment(psp_ctx *h, StepRun &r, const Segment &sg, int launches) {
  const int64_t n = h->geo.n;
  cudaStream_t s = h->stream;
  const bool trial_now = (r.c == 0 && r.try_cand);
  r.cycles += sg.cycles;
  r.iters += sg.iters;
  r.launches += launches;
  r.c += sg.cycles;
  r.bnorm = sg.bnorm;
  r.hist_count = sg.hist_count;
  if (sg.df_restart) r.flags |= PSP_FLAG_DF_RESTART;
  if (sg.error) {
    r.done = true;
    return fail(PSP_ERR_DEVICE, "device error flag " + std::to_string(sg.error) +
                                    " (a bounded wait expired or a launch was misconfigured)");
  }
  const bool broken = (sg.status & kStNumeric) || !std::isfinite(sg.R_last) || !std::isfinite(sg.beta_last);
  if (broken && (trial_now || r.adopted_now)) {
    // the fresh candidate broke a cycle of this step (in the mixed form an ill-conditioned
    // N can overflow the FP32 solve): it is rejected like a slow one and the step restarts
    // from u^n with the previous N -- X back to u^n, the pairs of the cycles run with the
    // candidate dropped from the history
    r.flags |= PSP_FLAG_CANDIDATE_TRIED;
    r.flags &= ~PSP_FLAG_CANDIDATE_ACCEPTED;
    PSP_CUDA(cudaMemcpyAsync(h->X, r.u_n, n * 8, cudaMemcpyDeviceToDevice, s));
    h->hist_poison = std::max(h->hist_poison, r.hist_count);
    h->int_host[3] = r.hist_before_trial;
    PSP_CUDA(cudaMemcpyAsync(&h->st->hist_count, h->int_host + 3, sizeof(int), cudaMemcpyHostToDevice, s));
    PSP_CUDA(host_wait(h, s));
    r.hist_count = r.hist_before_trial;
    if (r.adopted_now) {
      h->adopted = r.prev_adopted;
      h->adopted_version += 1;
      r.adopted_now = false;
      h->wait_len = std::max(h->wait_len, 1);
    }
    h->wait = h->wait_len;
    h->wait_len *= 2;
    r.cur = h->adopted;
    h->cand = -1;
    r.main_beta = -1.0;
    r.main_iters = 0;
    if (r.c == 0) r.c = 1;   // the trial's cycle counts against max_restarts
    r.try_cand = false;
    r.done = r.c >= h->opts.max_restarts;
    return PSP_OK;
  }
  if (sg.status & kStNumeric) {
    r.numeric = true;
    r.done = true;
    return PSP_OK;
  }
  if (sg.status & kStBreakdown) r.flags |= PSP_FLAG_BREAKDOWN;
  // residual at the end of the segment: the FP64 true residual of a converged restart
  // (mixed form) or the Givens estimate R(k_end)
  const double R_now = (h->mixed && sg.k_last == 0) ? sg.beta_last : sg.R_last;
  r.last_R = h->mixed ? sg.beta_last : sg.R_last;
  if (sg.status & kStConverged) r.converged = true;
  if (trial_now) {
    r.trial_beta = sg.beta_first;
    r.trial_iters = sg.iters;
    r.trial_R = R_now;
    r.flags |= PSP_FLAG_CANDIDATE_TRIED;
    const double r1 = rate_of(sg.R_last, sg.beta_first, sg.iters);
    const bool cycle_done = r.converged || (sg.R_last <= r.tol * sg.bnorm);
    if (!h->opts.accept_rule || cycle_done || h->rate_ref < 0.0 || r1 <= h->rate_ref) {
      h->adopted = h->cand;
      h->adopted_version += 1;
      h->wait_len = 1;
      r.flags |= PSP_FLAG_CANDIDATE_ACCEPTED;
      r.adopted_now = true;
    } else {
      h->wait = h->wait_len;
      h->wait_len *= 2;
    }
    r.cur = h->adopted;
    h->cand = -1;
  } else {
    if (r.main_beta < 0.0) r.main_beta = sg.beta_first;
    r.main_iters += sg.iters;
    r.main_R = R_now;
  }
  r.done = r.converged || r.c >= h->opts.max_restarts;
  return PSP_OK;
}

// After the last segment: the reference rate, the adopted band, u^{n+1}, and the
// Algorithm 2 fit of the next candidate (when the next step tries one).
psp_status step_finish(psp_ctx *h, StepRun &r, psp_step_info *info) {
  const int64_t n = h->geo.n;
  cudaStream_t s = h->stream;
  if (r.numeric) {
    // a step that ended with a non-finite residual keeps none of its matvec pairs (they would
    // enter the next fit: the history length goes back to the one the step started with) and
    // leaves the acceptance rule's reference rate as it was
    if (r.hist_count != r.hist_before_trial) {
      h->hist_poison = std::max(h->hist_poison, r.hist_count);
      h->int_host[3] = r.hist_before_trial;
      PSP_CUDA(cudaMemcpyAsync(&h->st->hist_count, h->int_host + 3, sizeof(int), cudaMemcpyHostToDevice, s));
      r.hist_count = r.hist_before_trial;
    }
  } else if (r.main_iters > 0 && r.main_beta > 0.0) {
    h->rate_ref = rate_of(r.main_R, r.main_beta, r.main_iters);
  } else if (r.trial_iters > 0 && r.trial_beta > 0.0) {
    h->rate_ref = rate_of(r.trial_R, r.trial_beta, r.trial_iters);
  }

  if (r.adopted_now)
    PSP_CUDA(cudaMemcpyAsync(h->band_adopted, h->band_cand, (size_t)n * (2 * h->b + 1) * 8,
                             cudaMemcpyDeviceToDevice, s));
  psp_status result = PSP_OK;
  if (r.numeric) result = fail(PSP_ERR_NUMERIC, "non-finite residual");
  else if (!r.converged) result = fail(PSP_ERR_NOCONV, "max_restarts reached");
  PSP_CUDA(cudaMemcpyAsync(r.u_np1, h->X, n * 8, cudaMemcpyDeviceToDevice, s));

  // progressive fit of the candidate for the next step (Algorithm 2); the history length is
  // the one the last segment's summary reported
  h->hist_count_host = r.hist_count;
  const int hist = std::min(r.hist_count, h->mmax);
  const int need = 2 * h->b + (h->opts.intercept ? 2 : 1);
  int singular = 0;
  // a fit is only worth making when the next step tries it: while the acceptance rule's
  // back-off still runs (wait > 0) the next step keeps the adopted N, and the step after
  // it fits afresh from the longer history, so the skipped fit could never be used
  // (the fit reads ring slots [0, hist): none may still hold a rolled-back segment's pairs)
  if (!r.numeric && hist >= need && h->wait == 0 && hist_valid(h, r.hist_count) == hist) {
    const int slot = (h->adopted == 0) ? 1 : 0;
    psp_status f2 = h->mixed ? fit_and_factor<float>(h, (const float *)h->Px, (const float *)h->Py, hist, slot,
                                                     &singular)
                             : fit_and_factor<double>(h, (const double *)h->Px, (const double *)h->Py, hist, slot,
                                                      &singular);
    if (f2 != PSP_OK && f2 != PSP_ERR_NUMERIC) return f2;
    r.flags |= PSP_FLAG_FITTED;
    if (singular) r.flags |= PSP_FLAG_SINGULAR_FIT;
    r.launches += 2 + 2 * (int)h->bs.levels.size() - 1;   // fit + factor/assemble per level
    if (f2 == PSP_OK) h->cand = slot;
    else { r.flags |= PSP_FLAG_FACTOR_FAILED; h->cand = -1; }
  } else {
    PSP_CUDA(host_wait(h, s));   // u_np1 is complete when psp_step returns (the fit's wait covers it)
  }
  h->last_singular = singular;
  if (info) {
    info->iters = r.iters;
    info->cycles = r.cycles;
    info->status = result;
    info->flags = r.flags;
    info->rel_res = r.bnorm > 0.0 ? r.last_R / r.bnorm : 0.0;
    info->hist_cols = hist;
    info->singular_rows = singular;
    info->launches = r.launches;
  }
  return result;
}

// The on-chip descriptor of handle h for a segment with slot `which` and max_cycles cycles.
OnChipDesc onchip_desc(psp_ctx *h, int which, int max_cycles, OnChipResult *res_dev) {
  OnChipDesc d{};
  const Geometry &g = h->geo;
  d.ndim = g.ndim;
  d.nx = g.nx;
  d.ny = g.ny;
  d.nz = g.nz;
  d.R = g.R;
  d.n = (int)g.n;
  d.band_w = g.band_w;
  d.b = h->b;
  d.Ab = g.Ab;
  d.Ab32 = g.Ab32;
  d.X = h->X;
  d.Bv = h->B;
  d.V = h->V;
  d.Px = h->Px;
  d.Py = h->Py;
  d.Z = h->Z;
  d.ld = h->ld;
  d.m = h->m;
  d.mmax = h->mmax;
  d.st = h->st;
  const int slot = which - 1;
  if (slot >= 0) {
    d.lev = h->mixed ? (const void *)h->bs.dev_app32[slot] : (const void *)h->bs.dev_app64[slot];
    d.nlev = (int)h->bs.levels.size();
    d.cyclic = h->bs.cyclic ? 1 : 0;
    if (d.cyclic) {
      const BandSolver::Slot &S = h->bs.slots[slot];
      d.smwZ = h->mixed ? (const void *)S.Z32 : (const void *)S.Z64;
      d.smwK = h->mixed ? (const void *)S.K32 : (const void *)S.K64;
      d.tmp = h->bs.cyc_y;
    }
  }
  d.max_cycles = max_cycles;
  d.res = res_dev;
  return d;
}

// Dynamic shared memory of the on-chip factor cache for h's factor slots (every array of every
// level rounded up to 16 bytes, as the kernel copies them), or 0 when it exceeds the cache.
int onchip_cache_bytes(const psp_ctx *h) {
  const size_t es = h->mixed ? 4 : 8;
  const size_t BB = (size_t)h->b * h->b;
  size_t total = 0;
  if (h->bs.levels.size() > 16) return 0;
  for (const LevelShape &l : h->bs.levels) {
    const size_t gq = (size_t)l.G * l.q * BB * es, gs = (size_t)l.G * BB * es;
    total += 5 * ((gq + 15) / 16 * 16) + 2 * ((gs + 15) / 16 * 16);
  }
  return total <= (size_t)kOnChipCacheMax ? (int)total : 0;
}

Segment segment_of(const OnChipResult &o) {
  Segment sg;
  sg.cycles = o.cycles;
  sg.iters = o.iters;
  sg.k_last = o.k_last;
  sg.status = o.status;
  sg.error = o.error;
  sg.beta_first = o.first_beta;
  sg.beta_last = o.last_beta;
  sg.R_last = o.last_R;
  sg.bnorm = o.bnorm;
  sg.hist_count = o.hist_count;
  return sg;
}

// One segment of handle h's step with slot `which`: one captured cycle graph, or an on-chip
// launch of up to max_cycles cycles.  Returns the kernels launched in *launches.
psp_status run_segment(psp_ctx *h, int which, int max_cycles, Segment *out, int *launches) {
  NvtxRange range("psp_segment");
  cudaStream_t s = h->stream;
  if (h->onchip) {
    *h->oc_desc_host = onchip_desc(h, which, max_cycles, h->oc_res);
    // a single system's launch caches its factors in shared memory when they fit
    const int cache = which > 0 ? onchip_cache_bytes(h) : 0;
    h->oc_desc_host->cache_bytes = cache;
    PSP_CUDA(cudaMemcpyAsync(h->oc_desc, h->oc_desc_host, sizeof(OnChipDesc), cudaMemcpyHostToDevice, s));
    if (h->mixed) launch_onchip<float>(h->oc_desc, 1, h->dev_int + 8, h->oc_threads, 1, s, cache);
    else launch_onchip<double>(h->oc_desc, 1, h->dev_int + 8, h->oc_threads, 1, s, cache);
    PSP_CUDA(cudaGetLastError());
    PSP_CUDA(cudaMemcpyAsync(h->oc_res_host, h->oc_res, sizeof(OnChipResult), cudaMemcpyDeviceToHost, s));
    PSP_CUDA(host_wait(h, s));
    *out = segment_of(*h->oc_res_host);
    *launches = 1;
    return PSP_OK;
  }
  if (h->opts.cycle_loop && h->seg_ok && !h->profiling) {
    // the restart loop on the device: up to max_cycles cycles in one launch
    if (!h->seg_graph[which] && !capture_segment(h, which)) h->seg_ok = false;
    if (h->seg_ok) {
      SegSummary init{};
      init.max_cycles = max_cycles;
      h->seg_host[0] = init;
      PSP_CUDA(cudaMemcpyAsync(h->seg_dev, h->seg_host, sizeof(SegSummary), cudaMemcpyHostToDevice, s));
      PSP_CUDA(cudaGraphLaunch(h->seg_graph[which], s));
      PSP_CUDA(host_wait(h, s));
      const SegSummary g = h->seg_host[1];
      Segment sg;
      sg.cycles = g.cycles;
      sg.iters = g.iters;
      sg.k_last = g.k_last;
      sg.status = g.status;
      sg.error = g.error;
      sg.beta_first = g.first_beta;
      sg.beta_last = g.last_beta;
      sg.R_last = g.last_R;
      sg.bnorm = g.bnorm;
      sg.hist_count = g.hist_count;
      sg.df_restart = h->mixed && h->restart_df_ok && h->st_host->restart_df;
      *out = sg;
      *launches = h->seg_kernels[which] * std::max(1, g.cycles);
      return PSP_OK;
    }
  }
  psp_status ps = ensure_graph(h, which);
  if (ps != PSP_OK) return ps;
  PSP_CUDA(cudaGraphLaunch(h->graph[which], s));
  PSP_CUDA(host_wait(h, s));
  const CycleSummary sm = *h->sum_host;
  if (h->profiling && h->opts.solver == PSP_SOLVER_GMRES) accumulate_profile(h, which, sm.k_end);
  Segment sg;
  sg.cycles = 1;
  sg.iters = sm.k_end;
  sg.k_last = sm.k_end;
  sg.status = sm.status;
  sg.error = sm.error;
  sg.beta_first = sg.beta_last = sm.beta;
  sg.R_last = sm.R_end;
  sg.bnorm = sm.bnorm;
  sg.hist_count = sm.hist_count;
  sg.df_restart = h->mixed && h->restart_df_ok && h->st_host->restart_df;
  *out = sg;
  *launches = h->graph_kernels[which];
  return PSP_OK;
}

// The batch autotuner (psp_batch_tuner): per size class (floor(log2 n)) it tries, on the
// first calls of psp_step_batch, every execution of a step -- the captured cycle graphs, and
// the on-chip path with CTAs of 128, 256 and 512 threads (tile shapes of 4 rows per thread
// at these sizes and up) -- one candidate per call for all instances of the class, and keeps
// the one whose calls had the least wall time per Arnoldi iteration of the whole batch.  The
// classes share the GPU during a call, so one instance's own time (device time on the
// on-chip path, host wall time on the graph path) does not show what its execution costs
// the batch; the call's wall time does.
constexpr int kTuneCands = 4;                      // graphs, on-chip 128 / 256 / 512
constexpr int kTuneThreads[kTuneCands] = {0, 128, 256, 512};
struct TuneClass {
  double t[kTuneCands] = {0, 0, 0, 0};   // summed seconds
  double it[kTuneCands] = {0, 0, 0, 0};  // summed iterations
  int cnt[kTuneCands] = {0, 0, 0, 0};
  int choice = -1;                       // decided candidate
};
struct BatchTuner {
  bool on = false;
  int calls = 0;
  TuneClass cls[32];
};
std::mutex g_tune_mu;
BatchTuner g_tune;

int size_class(int64_t n) {
  int c = 0;
  while (c < 31 && ((int64_t)1 << (c + 1)) <= n) ++c;
  return c;
}
// The tuner tries the on-chip path up to 2^16 unknowns: one CTA streams a system's Krylov
// basis at a fraction of the bandwidth the grid-wide passes reach, so larger systems take the
// cycle graphs without being tried.
constexpr int64_t kTuneOnChipMaxN = (int64_t)1 << 16;
bool onchip_capable(const psp_ctx *h) { return h->opts.solver == PSP_SOLVER_GMRES && h->geo.n <= kTuneOnChipMaxN; }

// Device and pinned buffers of the batched on-chip launches, made on the first batched call
// (and grown when a larger batch comes); one set per process, used under a mutex.
struct BatchBuffers {
  int cap = 0;
  OnChipDesc *desc = nullptr, *desc_host = nullptr;
  OnChipResult *res = nullptr, *res_host = nullptr;
  int *counter = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int sms = 0;
};
std::mutex g_batch_mu;
BatchBuffers g_batch;

psp_status batch_buffers(int count) {
  BatchBuffers &b = g_batch;
  if (!b.stream) {
    PSP_CUDA(cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking));
    PSP_CUDA(cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming));
    PSP_CUDA(cudaMalloc((void **)&b.counter, 256));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b.sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (count > b.cap) {
    if (b.desc) cudaFree(b.desc);
    if (b.res) cudaFree(b.res);
    if (b.desc_host) cudaFreeHost(b.desc_host);
    if (b.res_host) cudaFreeHost(b.res_host);
    b.desc = nullptr; b.res = nullptr; b.desc_host = nullptr; b.res_host = nullptr; b.cap = 0;
    const int cap = std::max(count, 64);
    if (cudaMalloc((void **)&b.desc, cap * sizeof(OnChipDesc)) != cudaSuccess ||
        cudaMalloc((void **)&b.res, cap * sizeof(OnChipResult)) != cudaSuccess ||
        cudaMallocHost((void **)&b.desc_host, cap * sizeof(OnChipDesc)) != cudaSuccess ||
        cudaMallocHost((void **)&b.res_host, cap * sizeof(OnChipResult)) != cudaSuccess) {
      cudaGetLastError();
      return fail(PSP_ERR_OOM, "batch buffers");
    }
    b.cap = cap;
  }
  return PSP_OK;
}

// The batched form on the on-chip path: the segments of every instance's step run in shared
// persistent launches (one CTA per system at a time, systems taken largest first from a
// counter), the host logic between them per instance; the fits and factorisations that end
// the steps run from nthreads host threads, each instance on its own stream.
psp_status step_batch_onchip(psp_ctx **hs, int count, const double *const *u_n, double *const *u_np1, const double *dt,
                             double tol, int nthreads, psp_step_info *infos, double *seconds, psp_status *statuses) {
  NvtxRange range("psp_batch_onchip");
  std::lock_guard<std::mutex> lock(g_batch_mu);
  psp_status bs = batch_buffers(count);
  if (bs != PSP_OK) return bs;
  BatchBuffers &B = g_batch;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<StepRun> runs(count);
  std::vector<double> dev_ns(count, 0.0);
  for (int i = 0; i < count; ++i) {
    psp_ctx *h = hs[i];
    const int64_t n = h->geo.n;
    if ((u_n[i] < u_np1[i] + n) && (u_np1[i] < u_n[i] + n)) return fail(PSP_ERR_ARG, "u_n and u_np1 overlap");
    if (!std::isfinite(dt[i])) return fail(PSP_ERR_ARG, "dt must be finite");
    psp_status st = step_begin(h, runs[i], u_n[i], u_np1[i], dt[i], tol);
    if (st != PSP_OK) return st;
    PSP_CUDA(cudaEventRecord(B.ev, h->stream));
    PSP_CUDA(cudaStreamWaitEvent(B.stream, B.ev, 0));
  }
  // largest systems first: they bound the launch, the small ones fill the SMs behind them
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hs[a]->geo.n > hs[b]->geo.n; });
  const bool mixed = hs[0]->mixed;
  for (int round = 0;; ++round) {
    // systems still stepping, grouped by CTA size (a system's CTA size is fixed at create, so
    // its arithmetic, reductions included, is the same batched or alone); one persistent
    // launch per group, back to back on the batch stream
    std::vector<int> live;
    for (int i : order)
      if (!runs[i].done) live.push_back(i);
    if (live.empty()) break;
    std::stable_sort(live.begin(), live.end(), [&](int a, int b) { return hs[a]->oc_threads > hs[b]->oc_threads; });
    for (size_t k = 0; k < live.size(); ++k) {
      const int i = live[k];
      B.desc_host[k] = onchip_desc(hs[i], step_which(runs[i]), step_next_cycles(hs[i], runs[i]), B.res + k);
    }
    const int cnt = (int)live.size();
    PSP_CUDA(cudaMemcpyAsync(B.desc, B.desc_host, cnt * sizeof(OnChipDesc), cudaMemcpyHostToDevice, B.stream));
    for (int k0 = 0, grp = 0; k0 < cnt; ++grp) {
      const int threads = hs[live[k0]]->oc_threads;
      int k1 = k0;
      while (k1 < cnt && hs[live[k1]]->oc_threads == threads) ++k1;
      const int per_sm = std::max(1, hs[live[k0]]->oc_ctas_per_sm);
      const int grid = std::min(k1 - k0, std::max(1, B.sms) * per_sm);
      if (mixed) launch_onchip<float>(B.desc + k0, k1 - k0, B.counter + grp, threads, grid, B.stream);
      else launch_onchip<double>(B.desc + k0, k1 - k0, B.counter + grp, threads, grid, B.stream);
      PSP_CUDA(cudaGetLastError());
      k0 = k1;
    }
    PSP_CUDA(cudaMemcpyAsync(B.res_host, B.res, cnt * sizeof(OnChipResult), cudaMemcpyDeviceToHost, B.stream));
    PSP_CUDA(cudaStreamSynchronize(B.stream));
    for (int k = 0; k < cnt; ++k) {
      const int i = live[k];
      dev_ns[i] += (double)(B.res_host[k].t_end - B.res_host[k].t_begin);
      psp_status st = step_after_segment(hs[i], runs[i], segment_of(B.res_host[k]), 1);
      if (st != PSP_OK) {
        runs[i].done = true;
        runs[i].status = st;
      }
    }
  }
  const double t_cycles = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  (void)t_cycles;
  // the ends of the steps (u^{n+1}, fits, factorisations) from a pool of host threads
  int dev = 0;
  cudaGetDevice(&dev);
  const int nt = std::max(1, std::min(nthreads < 1 ? 1 : nthreads, count));
  std::atomic<int> next{0};
  std::atomic<int> first_err{(int)PSP_OK};
  std::atomic<bool> noconv{false};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= count) break;
      const auto tf = std::chrono::steady_clock::now();
      psp_step_info info{};
      psp_status st = runs[i].status;
      if (st == PSP_OK) st = step_finish(hs[i], runs[i], &info);
      const double fin = std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
      if (infos) infos[i] = info;
      if (seconds) seconds[i] = dev_ns[i] * 1e-9 + fin;
      if (statuses) statuses[i] = st;
      if (st == PSP_ERR_NOCONV) {
        noconv = true;
      } else if (st != PSP_OK) {
        int expected = (int)PSP_OK;
        first_err.compare_exchange_strong(expected, (int)st);
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto &th : pool) th.join();
  if (first_err.load() != (int)PSP_OK)
    return fail((psp_status)first_err.load(), "at least one instance of the batch failed (see statuses)");
  return noconv.load() ? fail(PSP_ERR_NOCONV, "an instance reached max_restarts") : PSP_OK;
}

}  // namespace

extern "C" {

psp_status psp_step(psp_handle h, const double *u_n, double *u_np1, double dt, double tol, psp_step_info *info) {
  if (!h || !u_n || !u_np1) return fail(PSP_ERR_ARG, "NULL argument");
  if (!(tol > 0.0) || !std::isfinite(dt)) return fail(PSP_ERR_ARG, "tol must be > 0 and dt finite");
  const int64_t n = h->geo.n;
  if ((u_n < u_np1 + n) && (u_np1 < u_n + n)) return fail(PSP_ERR_ARG, "u_n and u_np1 overlap");
  NvtxRange range("psp_step");
  StepRun r;
  psp_status st = step_begin(h, r, u_n, u_np1, dt, tol);
  if (st != PSP_OK) return st;
  while (!r.done) {
    Segment sg;
    int launches = 0;
    st = run_segment(h, step_which(r), step_next_cycles(h, r), &sg, &launches);
    if (st != PSP_OK) return st;
    st = step_after_segment(h, r, sg, launches);
    if (st != PSP_OK) return st;
  }
  return step_finish(h, r, info);
}

}  // extern "C"

namespace {

// Streams of psp_step_batch's host threads, one per thread and device, created on first use
// and kept for the process: instances stepped at the same time never share a stream, whatever
// streams their handles were given (a framework's pooled streams are often shared by many
// handles, and instances on one stream would run one after another).
bool batch_streams(int dev, int nt, std::vector<cudaStream_t> &out) {
  static std::mutex mu;
  static std::vector<std::vector<cudaStream_t>> per_dev;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0) return false;
  if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1);
  std::vector<cudaStream_t> &v = per_dev[dev];
  while ((int)v.size() < nt) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
    v.push_back(s);
  }
  out.assign(v.begin(), v.begin() + nt);
  return true;
}

// The graph-path instances of a batch: nthreads host threads take them in order, each stepping
// one handle at a time on the thread's own stream (joined to the handle's stream by the
// handle's event at both ends), so the GPU runs nthreads instances' cycle graphs concurrently
// while each thread waits for its instance's cycle summaries.
void step_batch_graphs(psp_ctx **hs, const std::vector<int> &idx, const double *const *u_n, double *const *u_np1,
                       const double *dt, double tol, int nthreads, psp_step_info *infos, double *seconds,
                       psp_status *statuses, std::atomic<int> &first_err, std::atomic<bool> &noconv) {
  const int count = (int)idx.size();
  if (count == 0) return;
  int dev = 0;
  cudaGetDevice(&dev);
  const int nt = std::max(1, std::min(nthreads < 1 ? 1 : nthreads, count));
  std::vector<cudaStream_t> ts;
  bool ok = batch_streams(dev, nt, ts);
  // the batch's work on a handle follows the work already enqueued on the handle's stream
  for (int i : idx) {
    ok = ok && (hs[i]->join_ev || cudaEventCreateWithFlags(&hs[i]->join_ev, cudaEventDisableTiming) == cudaSuccess);
    ok = ok && cudaEventRecord(hs[i]->join_ev, hs[i]->stream) == cudaSuccess;
  }
  if (!ok) {
    int expected = (int)PSP_OK;
    first_err.compare_exchange_strong(expected, (int)PSP_ERR_CUDA);
    return;
  }
  // more threads than cores: the threads wait on blocking-sync events instead of spinning
  const unsigned cores = std::thread::hardware_concurrency();
  const bool block = cores > 0 && (unsigned)nt > cores;
  for (int i : idx) {
    if (block && !hs[i]->wait_ev &&
        cudaEventCreateWithFlags(&hs[i]->wait_ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
      int expected = (int)PSP_OK;
      first_err.compare_exchange_strong(expected, (int)PSP_ERR_CUDA);
      return;
    }
    hs[i]->blocking_wait = block;
  }
  std::atomic<int> next{0};
  auto work = [&](int t) {
    cudaSetDevice(dev);
    const cudaStream_t s = ts[t];
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= count) break;
      const int i = idx[k];
      psp_ctx *h = hs[i];
      const auto t0 = std::chrono::steady_clock::now();
      psp_step_info info{};
      psp_status st = PSP_ERR_CUDA;
      if (cudaStreamWaitEvent(s, h->join_ev, 0) == cudaSuccess) {
        const cudaStream_t own = h->stream;
        h->stream = s;
        st = psp_step(h, u_n[i], u_np1[i], dt[i], tol, &info);
        h->stream = own;
        if (cudaEventRecord(h->join_ev, s) != cudaSuccess && (st == PSP_OK || st == PSP_ERR_NOCONV))
          st = fail(PSP_ERR_CUDA, "psp_step_batch: cudaEventRecord failed");
      } else {
        st = fail(PSP_ERR_CUDA, "psp_step_batch: cudaStreamWaitEvent failed");
      }
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      hs[i]->last_batch_s = sec;
      if (infos) infos[i] = info;
      if (seconds) seconds[i] = sec;
      if (statuses) statuses[i] = st;
      if (st == PSP_ERR_NOCONV) {
        noconv = true;
      } else if (st != PSP_OK) {
        int expected = (int)PSP_OK;
        first_err.compare_exchange_strong(expected, (int)st);
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work, t);
  work(0);
  for (auto &th : pool) th.join();
  for (int i : idx) {
    hs[i]->blocking_wait = false;
    // later work on the handle's stream follows the batch's
    if (cudaStreamWaitEvent(hs[i]->stream, hs[i]->join_ev, 0) != cudaSuccess) {
      int expected = (int)PSP_OK;
      first_err.compare_exchange_strong(expected, (int)PSP_ERR_CUDA);
    }
  }
}

}  // namespace

extern "C" {

psp_status psp_step_batch(psp_handle *hs, int count, const double *const *u_n, double *const *u_np1,
                          const double *dt, double tol, int nthreads, psp_step_info *infos, double *seconds,
                          psp_status *statuses) {
  if (!hs || !u_n || !u_np1 || !dt || count < 0) return fail(PSP_ERR_ARG, "NULL argument or negative count");
  if (!(tol > 0.0)) return fail(PSP_ERR_ARG, "tol must be > 0");
  for (int i = 0; i < count; ++i)
    if (!hs[i]) return fail(PSP_ERR_ARG, "NULL handle in the batch");
  {  // two threads must never step one handle (its stream and workspace are not shared)
    std::vector<psp_handle> sorted(hs, hs + count);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
      return fail(PSP_ERR_ARG, "a handle appears twice in the batch");
  }
  if (count == 0) return PSP_OK;
  NvtxRange range("psp_step_batch");
  // per-instance times and iterations are needed by the tuner even when the caller does not
  // ask for them
  std::vector<double> secs(count, 0.0);
  std::vector<psp_step_info> inf(count);
  std::vector<psp_status> sts(count, PSP_OK);
  // the tuner's plan for this call: every instance of a size class runs the class's candidate
  std::vector<int> cand(count, -1);
  const auto t_call = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_tune.on) {
      for (int i = 0; i < count; ++i) {
        TuneClass &tc = g_tune.cls[size_class(hs[i]->geo.n)];
        int c = tc.choice;
        if (c < 0) c = g_tune.calls % kTuneCands;
        if (c > 0 && !onchip_capable(hs[i])) c = 0;
        cand[i] = c;
        hs[i]->onchip = c > 0;
        if (c > 0) hs[i]->oc_threads = kTuneThreads[c];
      }
    }
  }
  // the on-chip group (one precision) runs in shared persistent launches driven by one host
  // thread, concurrently with the graph group's host threads
  std::vector<int> oc, gr;
  int oc_mixed = -1;
  for (int i = 0; i < count; ++i) {
    if (hs[i]->onchip && (oc_mixed < 0 || (int)hs[i]->mixed == oc_mixed)) {
      oc_mixed = hs[i]->mixed ? 1 : 0;
      oc.push_back(i);
    } else {
      gr.push_back(i);
    }
  }
  // longest first (its last step's wall time, else its size): the host threads take the
  // instances from a shared counter, so the long ones no longer start last and stretch the call
  std::stable_sort(gr.begin(), gr.end(), [&](int a, int b) {
    const double ka = hs[a]->last_batch_s > 0.0 ? hs[a]->last_batch_s : 1e-9 * (double)hs[a]->geo.n;
    const double kb = hs[b]->last_batch_s > 0.0 ? hs[b]->last_batch_s : 1e-9 * (double)hs[b]->geo.n;
    return ka > kb;
  });
  std::atomic<int> first_err{(int)PSP_OK};
  std::atomic<bool> noconv{false};
  psp_status oc_status = PSP_OK;
  std::string oc_msg;
  std::thread oc_thread;
  if (!oc.empty()) {
    int dev = 0;
    cudaGetDevice(&dev);
    const int fin_threads = gr.empty() ? nthreads : std::max(1, nthreads / 4);
    oc_thread = std::thread([&, dev, fin_threads]() {
      cudaSetDevice(dev);
      std::vector<psp_ctx *> hv;
      std::vector<const double *> ui;
      std::vector<double *> uo;
      std::vector<double> dv;
      for (int i : oc) {
        hv.push_back(hs[i]);
        ui.push_back(u_n[i]);
        uo.push_back(u_np1[i]);
        dv.push_back(dt[i]);
      }
      const int k = (int)oc.size();
      std::vector<psp_step_info> oi(k);
      std::vector<double> os(k);
      std::vector<psp_status> ost(k, PSP_OK);
      oc_status = step_batch_onchip(hv.data(), k, ui.data(), uo.data(), dv.data(), tol, fin_threads, oi.data(),
                                    os.data(), ost.data());
      if (oc_status != PSP_OK && oc_status != PSP_ERR_NOCONV) oc_msg = g_last_error;
      for (int j = 0; j < k; ++j) {
        inf[oc[j]] = oi[j];
        secs[oc[j]] = os[j];
        sts[oc[j]] = ost[j];
      }
    });
  }
  step_batch_graphs(hs, gr, u_n, u_np1, dt, tol, nthreads, inf.data(), secs.data(), sts.data(), first_err, noconv);
  if (oc_thread.joinable()) oc_thread.join();
  if (oc_status == PSP_ERR_NOCONV) noconv = true;
  else if (oc_status != PSP_OK) {
    int expected = (int)PSP_OK;
    first_err.compare_exchange_strong(expected, (int)oc_status);
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    if (g_tune.on) {
      // the call's wall time per Arnoldi iteration of all its instances, credited once to
      // every class with the candidate it ran (a call with a failed instance is not counted)
      const double wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_call).count();
      double iters = 0.0;
      bool all_ok = true;
      for (int i = 0; i < count; ++i) {
        iters += std::max(1, inf[i].iters);
        all_ok = all_ok && (sts[i] == PSP_OK || sts[i] == PSP_ERR_NOCONV);
      }
      std::vector<int> seen(32, -1);
      for (int i = 0; i < count && all_ok; ++i) {
        if (cand[i] < 0) continue;
        const int c = size_class(hs[i]->geo.n);
        if (seen[c] == cand[i]) continue;
        seen[c] = cand[i];
        TuneClass &tc = g_tune.cls[c];
        tc.t[cand[i]] += wall;
        tc.it[cand[i]] += iters;
        tc.cnt[cand[i]] += 1;
      }
      g_tune.calls += 1;
      for (int c = 0; c < 32; ++c) {   // decide the classes whose every possible candidate was measured
        TuneClass &tc = g_tune.cls[c];
        if (tc.choice >= 0 || tc.cnt[0] == 0) continue;
        const bool oc_ok = ((int64_t)1 << c) <= kTuneOnChipMaxN;
        bool all = true;
        for (int k = 1; k < kTuneCands && oc_ok; ++k) all = all && tc.cnt[k] > 0;
        if (!all && g_tune.calls < 2 * kTuneCands) continue;
        int best = -1;
        double bv = 0.0;
        for (int k = 0; k < kTuneCands; ++k) {
          if (tc.cnt[k] == 0) continue;
          const double v = tc.t[k] / tc.it[k];
          if (best < 0 || v < bv) { best = k; bv = v; }
        }
        tc.choice = best;
      }
    }
  }
  for (int i = 0; i < count; ++i) {
    if (infos) infos[i] = inf[i];
    if (seconds) seconds[i] = secs[i];
    if (statuses) statuses[i] = sts[i];
  }
  if (first_err.load() != (int)PSP_OK)
    return fail((psp_status)first_err.load(),
                oc_msg.empty() ? "at least one instance of the batch failed (see statuses)" : oc_msg);
  return noconv.load() ? fail(PSP_ERR_NOCONV, "an instance reached max_restarts") : PSP_OK;
}

psp_status psp_batch_tuner(int mode, psp_tuning_class *classes, int max_classes, int *nclasses) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (mode == 1) {
    g_tune = BatchTuner{};
    g_tune.on = true;
  } else if (mode == 0) {
    g_tune.on = false;
  } else if (mode != -1) {
    return fail(PSP_ERR_ARG, "mode must be 1, 0 or -1");
  }
  int k = 0;
  for (int c = 0; c < 32; ++c) {
    const TuneClass &tc = g_tune.cls[c];
    bool seen = false;
    for (int j = 0; j < kTuneCands; ++j) seen = seen || tc.cnt[j] > 0;
    if (!seen) continue;
    if (classes && k < max_classes) {
      psp_tuning_class &o = classes[k];
      o.log2_n = c;
      o.choice = tc.choice < 0 ? -1 : kTuneThreads[tc.choice];
      for (int j = 0; j < kTuneCands; ++j) {
        o.samples[j] = tc.cnt[j];
        o.us_per_iter[j] = tc.cnt[j] > 0 ? 1e6 * tc.t[j] / tc.it[j] : 0.0;
      }
    }
    ++k;
  }
  if (nclasses) *nclasses = k;
  return PSP_OK;
}

namespace {
psp_status integrator_buffers(psp_ctx *h) {
  if (h->geo.band_w > 0) return fail(PSP_ERR_ARG, "the integrators need a PDE handle (psp_create): dt scales L");
  const size_t bytes = (size_t)h->geo.n * 8;
  if (!h->int_rhs && cudaMalloc((void **)&h->int_rhs, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(PSP_ERR_OOM, "integrator buffers");
  }
  if (!h->int_u1 && cudaMalloc((void **)&h->int_u1, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(PSP_ERR_OOM, "integrator buffers");
  }
  return PSP_OK;
}
}  // namespace

psp_status psp_step_bdf2(psp_handle h, const double *u_nm1, const double *u_n, double *u_np1, double dt, double tol,
                         psp_step_info *info) {
  if (!h || !u_nm1 || !u_n || !u_np1) return fail(PSP_ERR_ARG, "NULL argument");
  if (!(dt > 0.0)) return fail(PSP_ERR_ARG, "dt must be > 0");
  psp_status bs = integrator_buffers(h);
  if (bs != PSP_OK) return bs;
  // (I - 2/3 dt L) u^{n+1} = (4 u^n - u^{n-1}) / 3
  launch_axpby(h->geo.n, 4.0 / 3.0, u_n, -1.0 / 3.0, u_nm1, h->int_rhs, h->stream);
  PSP_CUDA(cudaGetLastError());
  psp_status st = psp_step(h, h->int_rhs, u_np1, 2.0 * dt / 3.0, tol, info);
  if (info) info->launches += 1;
  return st;
}

psp_status psp_step_sdirk2(psp_handle h, const double *u_n, double *u_np1, double dt, double tol,
                           psp_step_info *info) {
  if (!h || !u_n || !u_np1) return fail(PSP_ERR_ARG, "NULL argument");
  if (!(dt > 0.0)) return fail(PSP_ERR_ARG, "dt must be > 0");
  psp_status bs = integrator_buffers(h);
  if (bs != PSP_OK) return bs;
  const double g = 1.0 - 1.0 / std::sqrt(2.0);
  psp_step_info i1{}, i2{};
  // stage 1: (I - gamma dt L) U1 = u^n
  psp_status s1 = psp_step(h, u_n, h->int_u1, g * dt, tol, &i1);
  if (s1 != PSP_OK && s1 != PSP_ERR_NOCONV) return s1;
  // stage 2: (I - gamma dt L) u^{n+1} = u^n + (1 - gamma) dt L U1
  psp_status sl = psp_apply_L(h, -1, h->int_u1, h->int_rhs);
  if (sl != PSP_OK) return sl;
  launch_axpby(h->geo.n, 1.0, u_n, (1.0 - g) * dt, h->int_rhs, h->int_rhs, h->stream);
  PSP_CUDA(cudaGetLastError());
  psp_status s2 = psp_step(h, h->int_rhs, u_np1, g * dt, tol, &i2);
  if (info) {
    *info = i2;
    info->iters = i1.iters + i2.iters;
    info->cycles = i1.cycles + i2.cycles;
    info->flags = i1.flags | i2.flags;
    info->rel_res = std::max(i1.rel_res, i2.rel_res);
    info->launches = i1.launches + i2.launches + 2;
    info->status = (s2 != PSP_OK) ? s2 : s1;
  }
  if (s2 != PSP_OK) return s2;
  return s1 == PSP_OK ? PSP_OK : fail(s1, "SDIRK2 stage 1 reached max_restarts");
}

psp_status psp_step_host(psp_handle h, const double *u_n_host, double *u_np1_host, double dt, double tol,
                         psp_step_info *info) {
  if (!h || !u_n_host || !u_np1_host) return fail(PSP_ERR_ARG, "NULL argument");
  NvtxRange range("psp_step_host");
  const int64_t n = h->geo.n;
  if (!h->dev_un) {
    if (cudaMalloc((void **)&h->dev_un, n * 8) != cudaSuccess || cudaMalloc((void **)&h->dev_unp1, n * 8) != cudaSuccess)
      return fail(PSP_ERR_OOM, "host-step buffers");
  }
  PSP_CUDA(cudaMemcpyAsync(h->dev_un, u_n_host, n * 8, cudaMemcpyHostToDevice, h->stream));
  psp_status st = psp_step(h, h->dev_un, h->dev_unp1, dt, tol, info);
  if (st != PSP_OK && st != PSP_ERR_NOCONV) return st;
  PSP_CUDA(cudaMemcpyAsync(u_np1_host, h->dev_unp1, n * 8, cudaMemcpyDeviceToHost, h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return st;
}

psp_status psp_matvec(psp_handle h, const double *x, double *y, double dt) {
  if (!h || !x || !y) return fail(PSP_ERR_ARG, "NULL argument");
  psp_status cs = upload_api_coef(h, dt);
  if (cs != PSP_OK) return cs;
  launch_stencil<double, double, double>(h->geo, fixed_in<double>(x), fixed_out<double>(y), h->api_st, nullptr, h->stream);
  PSP_CUDA(cudaGetLastError());
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

psp_status psp_matvec_f32(psp_handle h, const float *x, float *y, double dt) {
  if (!h || !x || !y) return fail(PSP_ERR_ARG, "NULL argument");
  psp_status cs = upload_api_coef(h, dt);
  if (cs != PSP_OK) return cs;
  launch_stencil<float, float, float>(h->geo, fixed_in<float>(x), fixed_out<float>(y), h->api_st, nullptr, h->stream);
  PSP_CUDA(cudaGetLastError());
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

psp_status psp_apply_L(psp_handle h, int term, const double *x, double *y) {
  if (!h || !x || !y) return fail(PSP_ERR_ARG, "NULL argument");
  if (h->geo.band_w > 0) return fail(PSP_ERR_ARG, "an explicit banded operator has no L");
  if (term >= (int)h->term_w.size()) return fail(PSP_ERR_ARG, "term index out of range");
  set_L_coef(h, term, h->st_host->coef);
  PSP_CUDA(cudaMemcpyAsync(h->api_st->coef, h->st_host->coef, sizeof(h->st_host->coef), cudaMemcpyHostToDevice,
                           h->stream));
  h->api_dt = NAN;   // api_st no longer holds A's coefficients
  launch_stencil<double, double, double>(h->geo, fixed_in<double>(x), fixed_out<double>(y), h->api_st, nullptr, h->stream);
  PSP_CUDA(cudaGetLastError());
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

psp_status psp_adjoint_grads(psp_handle h, const double *lam, const double *u, double dt, double *grads_host) {
  if (!h || !lam || !u || !grads_host) return fail(PSP_ERR_ARG, "NULL argument");
  if (h->geo.band_w > 0) return fail(PSP_ERR_ARG, "an explicit banded operator has no L");
  if (h->opts.adjoint) return fail(PSP_ERR_ARG, "the gradients need the forward handle (opts.adjoint = 0)");
  const int nt = (int)h->term_w.size();
  std::vector<double> d(nt, 0.0);
  for (int t0 = 0; t0 < nt; t0 += kMaxTerms) {
    TermStencils ts{};
    ts.nt = std::min(kMaxTerms, nt - t0);
    ts.R = h->geo.R;
    for (int t = 0; t < ts.nt; ++t) {
      ts.dir[t] = h->term_w[t0 + t].first;
      for (int j = 0; j < 2 * kMaxR + 1; ++j) ts.w[t][j] = h->term_w[t0 + t].second[j];
    }
    launch_term_dots(h->geo, lam, u, ts, h->partial, &h->api_st->counter[2], h->grad_dev, h->stream);
    PSP_CUDA(cudaGetLastError());
    PSP_CUDA(cudaMemcpyAsync(d.data() + t0, h->grad_dev, ts.nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    PSP_CUDA(cudaStreamSynchronize(h->stream));
  }
  double dl = 0.0;
  for (int t = 0; t < nt; ++t) dl += h->term_alpha[t] * d[t];
  grads_host[0] = dl;
  for (int t = 0; t < nt; ++t) grads_host[1 + t] = dt * d[t];
  return PSP_OK;
}

psp_status psp_set_band_from(psp_handle dst, psp_handle src, int transpose) {
  if (!dst || !src) return fail(PSP_ERR_ARG, "NULL argument");
  if (dst->geo.n != src->geo.n || dst->b != src->b || dst->bs.cyclic != src->bs.cyclic)
    return fail(PSP_ERR_ARG, "the handles need the same n, band half-width and cyclic option");
  const int64_t n = src->geo.n;
  const int W = 2 * src->b + 1;
  PSP_CUDA(cudaStreamSynchronize(src->stream));
  if (src->adopted < 0) {   // N = I (its own transpose)
    std::vector<double> id((size_t)n * W, 0.0);
    for (int64_t i = 0; i < n; ++i) id[(size_t)i * W + src->b] = 1.0;
    PSP_CUDA(cudaMemcpy(dst->band_T, id.data(), id.size() * 8, cudaMemcpyHostToDevice));
  } else if (transpose) {
    launch_transpose_band(src->band_adopted, dst->band_T, n, src->b, dst->stream, dst->bs.cyclic);
    PSP_CUDA(cudaGetLastError());
  } else {
    PSP_CUDA(cudaMemcpyAsync(dst->band_T, src->band_adopted, (size_t)n * W * 8, cudaMemcpyDeviceToDevice,
                             dst->stream));
  }
  // band_T is dst's scratch for its own N^T: the adoption below bumps adopted_version, so
  // that N^T is made afresh before dst's next transposed solve
  return psp_set_band(dst, dst->band_T);
}

psp_status psp_fit_band(psp_handle h, const double *Px, const double *Py, int64_t ld, int M, double *N_band,
                        int *singular_rows) {
  if (!h || !Px || !Py || !N_band) return fail(PSP_ERR_ARG, "NULL argument");
  if (M < 1 || ld < h->geo.n) return fail(PSP_ERR_ARG, "need M >= 1 and ld >= n");
  return fit_into<double>(h, Px, Py, ld, M, N_band, singular_rows);
}

psp_status psp_fit_band_f32(psp_handle h, const float *Px, const float *Py, int64_t ld, int M, double *N_band,
                            int *singular_rows) {
  if (!h || !Px || !Py || !N_band) return fail(PSP_ERR_ARG, "NULL argument");
  if (M < 1 || ld < h->geo.n) return fail(PSP_ERR_ARG, "need M >= 1 and ld >= n");
  return fit_into<float>(h, Px, Py, ld, M, N_band, singular_rows);
}

psp_status psp_get_history(psp_handle h, double *Px, double *Py, int64_t ld, int max_cols, int *cols) {
  if (!h || !cols) return fail(PSP_ERR_ARG, "NULL argument");
  PSP_CUDA(cudaMemcpyAsync(h->int_host + 4, &h->st->hist_count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  const int count = h->int_host[4];
  const int c = hist_valid(h, count);
  *cols = c;
  if (!Px || !Py) return PSP_OK;   // query only
  if (ld < h->geo.n || max_cols < c) return fail(PSP_ERR_ARG, "need ld >= n and max_cols >= the valid columns");
  const int first = ((count - c) % h->mmax + h->mmax) % h->mmax;
  if (h->mixed)
    launch_history_copy<float>(h->geo.n, c, first, h->mmax, (const float *)h->Px, (const float *)h->Py, h->ld, Px, Py,
                               ld, h->stream);
  else
    launch_history_copy<double>(h->geo.n, c, first, h->mmax, (const double *)h->Px, (const double *)h->Py, h->ld, Px,
                                Py, ld, h->stream);
  PSP_CUDA(cudaGetLastError());
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

psp_status psp_set_band(psp_handle h, const double *N_band) {
  if (!h || !N_band) return fail(PSP_ERR_ARG, "NULL argument");
  const size_t bytes = (size_t)h->geo.n * (2 * h->b + 1) * 8;
  const int slot = (h->adopted == 0) ? 1 : 0;
  psp_status s = factor_into(h, slot, N_band);
  if (s != PSP_OK) return s;
  PSP_CUDA(cudaMemcpyAsync(h->band_adopted, N_band, bytes, cudaMemcpyDeviceToDevice, h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  h->adopted = slot;
  h->adopted_version += 1;
  if (h->cand == slot) h->cand = -1;
  return PSP_OK;
}

psp_status psp_get_band(psp_handle h, double *N_band) {
  if (!h || !N_band) return fail(PSP_ERR_ARG, "NULL argument");
  const int64_t n = h->geo.n;
  const int W = 2 * h->b + 1;
  if (h->adopted < 0) {
    std::vector<double> id((size_t)n * W, 0.0);
    for (int64_t i = 0; i < n; ++i) id[(size_t)i * W + h->b] = 1.0;
    PSP_CUDA(cudaMemcpy(N_band, id.data(), id.size() * 8, cudaMemcpyHostToDevice));
    return PSP_OK;
  }
  PSP_CUDA(cudaMemcpyAsync(N_band, h->band_adopted, (size_t)n * W * 8, cudaMemcpyDeviceToDevice, h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

psp_status psp_apply_precond(psp_handle h, const double *v, double *y, int transpose) {
  if (!h || !v || !y) return fail(PSP_ERR_ARG, "NULL argument");
  if (h->adopted < 0) {
    if (v != y) PSP_CUDA(cudaMemcpyAsync(y, v, h->geo.n * 8, cudaMemcpyDeviceToDevice, h->stream));
    return PSP_OK;
  }
  int slot = h->adopted;
  if (transpose) {
    psp_status ts = ensure_transposed(h);
    if (ts != PSP_OK) return ts;
    slot = 2;
  }
  h->bs.apply<double>(slot, v, nullptr, nullptr, fixed_out<double>(y), nullptr, 0, h->stream);
  PSP_CUDA(cudaGetLastError());
  return PSP_OK;
}

psp_status psp_apply_precond_f32(psp_handle h, const float *v, float *y, int transpose) {
  if (!h || !v || !y) return fail(PSP_ERR_ARG, "NULL argument");
  if (h->adopted < 0) {
    if (v != y) PSP_CUDA(cudaMemcpyAsync(y, v, h->geo.n * 4, cudaMemcpyDeviceToDevice, h->stream));
    return PSP_OK;
  }
  int slot = h->adopted;
  if (transpose) {
    psp_status ts = ensure_transposed(h);
    if (ts != PSP_OK) return ts;
    slot = 2;
  }
  h->bs.apply<float>(slot, v, nullptr, nullptr, fixed_out<float>(y), nullptr, 0, h->stream);
  PSP_CUDA(cudaGetLastError());
  return PSP_OK;
}

psp_status psp_get_stencil(psp_handle h, double *w_host, int *radius) {
  if (!h || !radius) return fail(PSP_ERR_ARG, "NULL argument");
  const int R = h->geo.R;
  *radius = R;
  if (w_host)
    for (int d = 0; d < 3; ++d)
      for (int j = -R; j <= R; ++j) w_host[d * (2 * R + 1) + j + R] = (d < h->geo.ndim) ? h->wdir[d][kMaxR + j] : 0.0;
  return PSP_OK;
}

psp_status psp_set_profiling(psp_handle h, int enable) {
  if (!h) return fail(PSP_ERR_ARG, "NULL argument");
  const bool on = enable != 0;
  if (on == h->profiling) return PSP_OK;
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  for (int w = 0; w < 3; ++w) {
    if (h->graph[w]) { cudaGraphExecDestroy(h->graph[w]); h->graph[w] = nullptr; }
  }
  if (on && !h->ev[0][0][0]) {
    for (int w = 0; w < 3; ++w)
      for (int k = 0; k < h->m; ++k)
        for (int c = 0; c < 6; ++c) PSP_CUDA(cudaEventCreate(&h->ev[w][k][c]));
  }
  h->profiling = on;
  return PSP_OK;
}

psp_status psp_last_cycle_residuals(psp_handle h, double *R_host, int maxk, int *k_end) {
  if (!h || !R_host || !k_end) return fail(PSP_ERR_ARG, "NULL argument");
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  int k = 0;
  PSP_CUDA(cudaMemcpy(&k, &h->st->k_end, sizeof(int), cudaMemcpyDeviceToHost));
  *k_end = k;
  if (k > maxk) k = maxk;
  if (k > 0) PSP_CUDA(cudaMemcpy(R_host, h->st->R, k * sizeof(double), cudaMemcpyDeviceToHost));
  return PSP_OK;
}

psp_status psp_get_profile(psp_handle h, psp_profile *out, int reset) {
  if (!h || !out) return fail(PSP_ERR_ARG, "NULL argument");
  *out = h->prof;
  if (reset) h->prof = psp_profile{};
  return PSP_OK;
}

psp_status psp_reset(psp_handle h) {
  if (!h) return fail(PSP_ERR_ARG, "NULL argument");
  h->adopted = -1;
  h->adopted_version += 1;
  h->cand = -1;
  h->rate_ref = -1.0;
  h->wait = 0;
  h->wait_len = 1;
  h->hist_dt = NAN;
  h->hist_count_host = 0;
  h->hist_poison = 0;
  PSP_CUDA(cudaMemsetAsync(&h->st->hist_count, 0, sizeof(int), h->stream));
  PSP_CUDA(cudaStreamSynchronize(h->stream));
  return PSP_OK;
}

}  // extern "C"
