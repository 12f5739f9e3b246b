// Arnoldi step of Algorithm 1 (Gram-Schmidt, H(:,k), V(:,k+1)), the Givens update of the
// Hessenberg least-squares problem with the residual R(k) = |G(k+1)| and the finish test,
// and the cycle update Z = sum_j Q(j) V(:,j) with Q = H^{-1} G.
//
// Gram-Schmidt is classical Gram-Schmidt applied twice (CGS2), equal in exact arithmetic
// to the modified Gram-Schmidt loop of the paper and as stable in practice, in three
// streaming passes over the basis:
//   pass 1: h1 = V^T U                                   (and ||U||^2 for the breakdown test)
//   pass 2: U' = U - V h1 formed on the fly, h2 = V^T U'
//   pass 3: V~(:,k+1) = U - V (h1 + h2), nu = ||V~(:,k+1)||^2
// The basis is stored unnormalised: V(:,j) = sigma_j V~(:,j) with sigma_j = 1/H(j+1,j)
// kept in FP64, so normalising costs no extra pass.  Each pass reduces per-CTA partial
// sums in a fixed order in the last CTA to finish (deterministic, no waiting).  The last
// CTA of pass 3 also runs the FP64 Givens step, the finish test and, when the cycle ends,
// the triangular solve for Q.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "psp_kernels.cuh"

namespace psp {

constexpr double kBreakdownRel = 1e-14;

template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int W = 4;
  // A load the compiler may not merge with an earlier load of the same address (the
  // second sweep of pass 2 re-reads V from L1/L2 instead of holding k vectors in registers).
  __device__ static __forceinline__ float4 reload(const float4 *p) {
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
  }
  __device__ static __forceinline__ float dot(float4 a, float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
  }
  __device__ static __forceinline__ float4 axpy(float c, float4 x, float4 y) {  // y - c x
    return make_float4(y.x - c * x.x, y.y - c * x.y, y.z - c * x.z, y.w - c * x.w);
  }
};
template <> struct Vec<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static __forceinline__ double2 reload(const double2 *p) {
    double2 r;
    asm volatile("ld.global.nc.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
  }
  __device__ static __forceinline__ double dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
  __device__ static __forceinline__ double2 axpy(double c, double2 x, double2 y) {
    return make_double2(y.x - c * x.x, y.y - c * x.y);
  }
};

// ---------------------------------------------------------------------------------------
// Tile pipeline.  A pass streams the basis in row tiles of 1 KB per column (64 vectors of
// 16 bytes: 256 floats or 128 doubles).  One CTA per SM walks its tiles; warp 0 issues one
// bulk copy (cp.async.bulk, global -> shared) per column segment into a ring of kStages
// buffers, each completed through an mbarrier transaction count, so the copies of the next
// tiles are in flight while the current one is consumed.  Every wait on an mbarrier is
// bounded; on timeout the CTA records DevState::error and skips the tile.
// ---------------------------------------------------------------------------------------
constexpr int kArnThreads = 512;
constexpr int kArnWarps = kArnThreads / 32;
constexpr int kMaxArnCta = 256;
constexpr int kMaxStages = 8;
constexpr int kStageBudget = 200 * 1024;         // shared memory for the stage ring
constexpr int kSegBytes = 1024;                  // one column segment of a tile
constexpr int kSegVec = kSegBytes / 16;          // 64 vectors of 16 B
constexpr uint32_t kWaitLimit = 1u << 20;        // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase completed, false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Stage s holds ncols column segments: seg c at buf + (s*ncols + c)*kSegBytes.  Columns
// 0..k-1 are V(:,0..k-1), column ucol = k is U (the P_y ring column).  Tensor maps of V
// with boxes of 16, 4 and 1 columns x 1 KB cover exactly k columns in at most
// k/16 + 3 + 3 copies; a map of the P_y ring (box of 1 column) brings U.
constexpr int kBoxCols = 16;
__host__ __device__ inline int ucol_for(int k) { return k; }

struct TilePipe {
  char *buf;
  uint64_t *bar;
  int ncols;      // ucol + 1
  int ucol;       // segment index of U
  int ntiles;     // tiles of the vectors
  int first, step;
  int nst;        // stages in the ring (<= kMaxStages)
  int uring;      // ring column of U
};

__host__ __device__ inline int stages_for(int k) {
  const int s = kStageBudget / ((ucol_for(k) + 1) * kSegBytes);
  return s > kMaxStages ? kMaxStages : (s < 2 ? 2 : s);
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Issue the copies of one tile into `stage` (thread 0 of the CTA).
// The three V maps (boxes of 16, 4 and 1 columns), passed together as one kernel parameter.
struct VMaps {
  CUtensorMap m[3];
};

template <typename T>
__device__ __forceinline__ void issue_tile(const TilePipe &p, int stage, int tile, const CUtensorMap *mapV,
                                           const CUtensorMap *mapU) {
  constexpr int TR = kSegBytes / sizeof(T);   // rows per tile
  char *base = p.buf + (int64_t)stage * p.ncols * kSegBytes;
  mbar_expect_tx(&p.bar[stage], (uint32_t)(p.ncols * kSegBytes));
  int cb = 0;
  for (; cb + 16 <= p.ucol; cb += 16) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[0], tile * TR, cb, &p.bar[stage]);
  for (; cb + 4 <= p.ucol; cb += 4) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[1], tile * TR, cb, &p.bar[stage]);
  for (; cb < p.ucol; ++cb) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[2], tile * TR, cb, &p.bar[stage]);
  tma_load_2d(base + (int64_t)p.ucol * kSegBytes, mapU, tile * TR, p.uring, &p.bar[stage]);
}

// Drives the pipeline: calls body(stage_ptr, tile) for each of this CTA's tiles.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

template <typename T, typename Body, typename Pro>
__device__ __forceinline__ void run_tiles(TilePipe &p, const CUtensorMap *mapV, const CUtensorMap *mapU, DevState *st,
                                          Pro prologue, Body body) {
  const int kStages = p.nst;
  // the stage ring must fit the dynamic shared memory of this launch; otherwise no copy
  // is issued and the error flag is set
  if ((uint64_t)kStages * p.ncols * kSegBytes > dynamic_smem_bytes()) {
    if (threadIdx.x == 0) atomicExch(&st->error, 2);
    return;
  }
  if (threadIdx.x == 0)
    for (int s = 0; s < kStages; ++s) mbar_init(&p.bar[s], 1);
  fence_mbar_init();
  __syncthreads();
  const int my = (p.ntiles - p.first + p.step - 1) / p.step;   // tiles of this CTA
  if (threadIdx.x == 0)
    for (int i = 0; i < kStages && i < my; ++i) issue_tile<T>(p, i, p.first + i * p.step, mapV, mapU);
  prologue();          // runs while the first tiles are in flight
  __syncthreads();
  bool ok = true;
  for (int i = 0; i < my; ++i) {
    const int s = i % kStages;
    const uint32_t parity = (uint32_t)((i / kStages) & 1);
    // warp 0 polls the stage's mbarrier (bounded; acquire), the other warps sleep in the CTA
    // barrier that publishes its result, so the tile is consumed by all threads or by none
    const int mine = (threadIdx.x < 32) ? (mbar_wait(&p.bar[s], parity) ? 1 : 0) : 1;
    const bool ready = __syncthreads_and(mine) != 0;
    if (!ready) ok = false;
    if (ready) body(reinterpret_cast<const T *>(p.buf + (int64_t)s * p.ncols * kSegBytes), p.first + i * p.step);
    __syncthreads();                       // every thread is done with stage s
    if (threadIdx.x == 0 && i + kStages < my) {
      fence_proxy_async();
      issue_tile<T>(p, s, p.first + (i + kStages) * p.step, mapV, mapU);
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(&st->error, 1);
    // drain: wait (bounded) for copies still in flight before the CTA exits
    if (threadIdx.x < 32)
      for (int i = (my > kStages ? my - kStages : 0); i < my; ++i) mbar_wait(&p.bar[i % kStages], (uint32_t)((i / kStages) & 1));
    __syncthreads();
  }
}

// Per-warp column ownership: warp w owns columns j = w + kArnWarps * s, s < KS.  Lane l
// works on vectors l and l + 32 of the tile.
template <typename T, int KS>
__device__ __forceinline__ void tile_dots(const T *tile, int k, const typename Vec<T>::type (&u)[2], T (&acc)[KS]) {
  using VT = typename Vec<T>::type;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const int j = wid + kArnWarps * s;
    if (j < k) {
      const VT *seg = reinterpret_cast<const VT *>(tile) + (int64_t)j * kSegVec;
      acc[s] += Vec<T>::dot(seg[lane], u[0]) + Vec<T>::dot(seg[lane + 32], u[1]);
    }
  }
}

// out[r] = U[r] - sum_j c_j V_j[r] for the 64 vectors of a tile: 4 column groups of 64
// threads form partial sums, combined through shared memory.
template <typename T>
__device__ __forceinline__ void tile_axpy(const T *tile, int k, int ucol, const T *c, typename Vec<T>::type *part,
                                          typename Vec<T>::type *out) {
  using VT = typename Vec<T>::type;
  constexpr int NG = kArnThreads / kSegVec;   // column groups
  const int r = threadIdx.x & (kSegVec - 1), g = threadIdx.x / kSegVec;
  const VT *segs = reinterpret_cast<const VT *>(tile);
  VT p0 = VT{}, p1 = VT{};   // two independent chains
  int j = g;
  for (; j + NG < k; j += 2 * NG) {
    p0 = Vec<T>::axpy(-c[j], segs[(int64_t)j * kSegVec + r], p0);            // p += c_j V_j
    p1 = Vec<T>::axpy(-c[j + NG], segs[(int64_t)(j + NG) * kSegVec + r], p1);
  }
  if (j < k) p0 = Vec<T>::axpy(-c[j], segs[(int64_t)j * kSegVec + r], p0);
  part[g * kSegVec + r] = Vec<T>::axpy((T)-1, p1, p0);                         // p0 + p1
  __syncthreads();
  if (threadIdx.x < kSegVec) {
    VT u = segs[(int64_t)ucol * kSegVec + r];
#pragma unroll
    for (int q = 0; q < NG; ++q) u = Vec<T>::axpy((T)1, part[q * kSegVec + r], u);  // u -= part
    out[r] = u;
  }
  __syncthreads();
}

// Column sums of the CTA -> partial[j * kMaxCta + cta] (each column has one owning warp).
template <typename T, int KS>
__device__ __forceinline__ void write_col_partials(const T (&acc)[KS], int k, double *partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const int j = wid + kArnWarps * s;
    const T v = warp_sum(acc[s]);
    if (lane == 0 && j < k) partial[(int64_t)j * kMaxCta + blockIdx.x] = (double)v;
  }
}

// out[j] = sum over CTAs of partial[j][cta] in a fixed order, j < nvals (partial rows of
// length kMaxCta).  Warp w takes j = w, w + 8, ...; lane l takes CTAs l, l + 32, ...;
// every load is issued before any add.  Ends with a CTA barrier.
__device__ __forceinline__ void grid_sums(const double *partial, int nvals, int nb, double *out) {
  constexpr int MJ = (kMaxM + 2 + kArnWarps - 1) / kArnWarps;   // j values per warp
  constexpr int MB = kMaxArnCta / 32;                            // CTAs per lane
  constexpr int BATCH = 3;                                       // j values loaded together
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t0 = 0; t0 < MJ; t0 += BATCH) {
    if (wid + t0 * kArnWarps >= nvals) break;
    double v[BATCH][MB];
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      const int j = wid + (t0 + t) * kArnWarps;
#pragma unroll
      for (int q = 0; q < MB; ++q) {
        const int b = lane + 32 * q;
        v[t][q] = (j < nvals && b < nb) ? __ldcg(partial + (int64_t)j * kMaxCta + b) : 0.0;
      }
    }
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < MB; ++q) s += v[t][q];
      s = warp_sum(s);
      const int j = wid + (t0 + t) * kArnWarps;
      if (lane == 0 && j < nvals) out[j] = s;
    }
  }
  __syncthreads();
}

// pass 1: partial sums of V^T U (columns 0..k-1) and ||U||^2 (slot k); reduced by pass 2
template <typename T, int KS>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass1(const __grid_constant__ VMaps mapV,
                                                           const __grid_constant__ CUtensorMap mapU, int k,
                                                           DevState *st, double *partial, int ntiles) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kMaxStages];
  const int ucol = ucol_for(k);
  TilePipe p{smem, bars, ucol + 1, ucol, ntiles, (int)blockIdx.x, (int)gridDim.x, stages_for(k), st->hist_count % st->mmax};
  T acc[KS];
#pragma unroll
  for (int s = 0; s < KS; ++s) acc[s] = (T)0;
  T uu = (T)0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  run_tiles<T>(p, mapV.m, &mapU, st, [] {}, [&](const T *tile, int) {
    const VT *useg = reinterpret_cast<const VT *>(tile) + (int64_t)ucol * kSegVec;
    const VT u[2] = {useg[lane], useg[lane + 32]};
    if (wid == kArnWarps - 1) uu += Vec<T>::dot(u[0], u[0]) + Vec<T>::dot(u[1], u[1]);
    tile_dots<T, KS>(tile, k, u, acc);
  });
  write_col_partials<T, KS>(acc, k, partial);
  if (wid == kArnWarps - 1) {
    const T v = warp_sum(uu);
    if (lane == 0) partial[(int64_t)k * kMaxCta + blockIdx.x] = (double)v;
  }
}

// pass 2: reduces pass 1 (h1, ||U||^2) in its prologue; U' = U - V h1 formed per tile in
// shared memory, partial sums of h2 = V^T U' from the same tile
template <typename T, int KS>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass2(const __grid_constant__ VMaps mapV,
                                                           const __grid_constant__ CUtensorMap mapU, int k,
                                                           DevState *st, const double *partial1, double *partial,
                                                           int ntiles, int nb1) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ T s_c[kMaxM];
  __shared__ double s_sum[kMaxM + 2];
  __shared__ VT s_part[kArnThreads];
  __shared__ VT s_u[kSegVec];
  const int ucol = ucol_for(k);
  TilePipe p{smem, bars, ucol + 1, ucol, ntiles, (int)blockIdx.x, (int)gridDim.x, stages_for(k), st->hist_count % st->mmax};
  T acc[KS];
#pragma unroll
  for (int s = 0; s < KS; ++s) acc[s] = (T)0;
  const int lane = threadIdx.x & 31;
  run_tiles<T>(p, mapV.m, &mapU, st, [&] {
    grid_sums(partial1, k + 1, nb1, s_sum);
    for (int j = threadIdx.x; j <= k; j += blockDim.x) {
      if (j < k) {
        const double h = st->sigma[j] * s_sum[j];
        s_c[j] = (T)(h * st->sigma[j]);
        if (blockIdx.x == 0) st->h1[j] = h;
      } else if (blockIdx.x == 0) {
        st->unorm2 = s_sum[k];
      }
    }
  }, [&](const T *tile, int) {
    tile_axpy<T>(tile, k, ucol, s_c, s_part, s_u);
    const VT u[2] = {s_u[lane], s_u[lane + 32]};
    tile_dots<T, KS>(tile, k, u, acc);
  });
  write_col_partials<T, KS>(acc, k, partial);
}

// FP64 Givens step of Algorithm 1 for column k (1-based), then the finish test.
__device__ void arnoldi_finish(DevState *st, int k, double nu, int mixed) {
  const int kk = k - 1;
  const int ld = kMaxM + 1;
  double *Hc = st->H + (int64_t)kk * ld;
  for (int j = 0; j < k; ++j) Hc[j] = st->h1[j] + st->h2[j];
  const double hk1 = sqrt(nu);
  Hc[k] = hk1;
  const bool brk = !(hk1 > kBreakdownRel * sqrt(st->unorm2));
  st->sigma[k] = hk1 > 0.0 ? 1.0 / hk1 : 0.0;
  for (int j = 0; j < kk; ++j) {  // old rotations
    const double d = Hc[j];
    Hc[j] = d * st->C[j] + st->S[j] * Hc[j + 1];
    Hc[j + 1] = -d * st->S[j] + st->C[j] * Hc[j + 1];
  }
  const double gamma = hypot(Hc[kk], Hc[k]);
  if (gamma > 0.0) {
    st->C[kk] = Hc[kk] / gamma;
    st->S[kk] = Hc[k] / gamma;
  } else {
    st->C[kk] = 1.0;
    st->S[kk] = 0.0;
  }
  Hc[kk] = gamma;
  Hc[k] = 0.0;
  st->G[k] = 0.0;
  const double d = st->G[kk];
  st->G[kk] = st->C[kk] * d + st->S[kk] * st->G[k];
  st->G[k] = -st->S[kk] * d + st->C[kk] * st->G[k];
  const double R = fabs(st->G[k]);
  st->R[kk] = R;
  int status = st->status;
  if (!isfinite(R) || !isfinite(hk1)) status |= kStNumeric;
  if (brk) status |= kStBreakdown;
  if (!mixed && R <= st->eps_abs) status |= kStConverged;
  const bool end = (R <= st->eps_cycle) || brk || (k >= st->m) || (status & kStNumeric);
  st->status = status;
  st->k_end = k;
  st->hist_count += 1;
  if (end) {
    st->active = 0;
    for (int j = k - 1; j >= 0; --j) {  // Q = H^{-1} G, back substitution
      double s = st->G[j];
      for (int l = j + 1; l < k; ++l) s -= st->H[(int64_t)l * ld + j] * st->Q[l];
      const double hjj = st->H[(int64_t)j * ld + j];
      st->Q[j] = hjj != 0.0 ? s / hjj : 0.0;
    }
  }
  st->sum.k_end = k;
  st->sum.error = st->error;
  st->sum.status = status;
  st->sum.hist_count = st->hist_count;
  st->sum.R_end = R;
}

// pass 3: reduces pass 2 (h2) in its prologue; V~(:,k+1) = U - V (h1 + h2),
// nu = ||V~(:,k+1)||^2; the last CTA to finish runs the Givens step
template <typename T, int KS>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass3(const __grid_constant__ VMaps mapV,
                                                           const __grid_constant__ CUtensorMap mapU, T *__restrict__ V,
                                                           int64_t ldv, int k, DevState *st, const double *partial2,
                                                           double *partial, int ntiles, int nb2, int mixed) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ T s_c[kMaxM];
  __shared__ double s_sum[kMaxM + 2];
  __shared__ VT s_part[kArnThreads];
  __shared__ VT s_u[kSegVec];
  VT *Vout = reinterpret_cast<VT *>(V + (int64_t)k * ldv);
  const int ucol = ucol_for(k);
  TilePipe p{smem, bars, ucol + 1, ucol, ntiles, (int)blockIdx.x, (int)gridDim.x, stages_for(k), st->hist_count % st->mmax};
  T nu = (T)0;
  run_tiles<T>(p, mapV.m, &mapU, st, [&] {
    grid_sums(partial2, k, nb2, s_sum);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const double h2 = st->sigma[j] * s_sum[j];
      s_c[j] = (T)((st->h1[j] + h2) * st->sigma[j]);
      if (blockIdx.x == 0) st->h2[j] = h2;
    }
  }, [&](const T *tile, int t) {
    tile_axpy<T>(tile, k, ucol, s_c, s_part, s_u);
    if (threadIdx.x < kSegVec) {
      const VT u = s_u[threadIdx.x];
      Vout[(int64_t)t * kSegVec + threadIdx.x] = u;
      nu += Vec<T>::dot(u, u);
    }
  });
  __shared__ double s_nu[kArnWarps];
  {
    const T v = warp_sum(nu);
    if ((threadIdx.x & 31) == 0) s_nu[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0;
      for (int w = 0; w < kArnWarps; ++w) a += s_nu[w];
      partial[blockIdx.x] = a;
    }
  }
  if (!last_block_arrive(&st->counter[3])) return;
  grid_sums(partial, 1, gridDim.x, s_sum);
  if (threadIdx.x == 0) arnoldi_finish(st, k, s_sum[0], mixed);
  __syncthreads();
  last_block_reset(&st->counter[3]);
}

// P_x(:,i) = Y_k = V(:,k) when N = I (unpreconditioned cycle).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_scale_copy(int k, int64_t n, const T *__restrict__ V,
                                                         int64_t ldv, OutRef<T> yref, const DevState *st) {
  if (st->active == 0) return;
  const T c = (T)st->sigma[k - 1];
  const T *v = V + (int64_t)(k - 1) * ldv;
  T *y = yref.get();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = c * v[i];
}

// Z = sum_{j < k_end} Q(j) V(:,j); with add_to_x, X += Z instead (N = I).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_update_z(int64_t n, const T *__restrict__ V, int64_t ldv,
                                                       T *Z, double *X, int add_to_x, const DevState *st) {
  const int k = st->k_end;
  if (k == 0) return;
  __shared__ T s_q[kMaxM];
  for (int j = threadIdx.x; j < k; j += blockDim.x) s_q[j] = (T)(st->Q[j] * st->sigma[j]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T z = (T)0;
    for (int j = 0; j < k; ++j) z += s_q[j] * V[(int64_t)j * ldv + i];
    if (add_to_x) X[i] += (double)z;
    else Z[i] = z;
  }
}

// ---------------------------------------------------------------------------------------

int arnoldi_grid() {
  static int g = 0;
  if (g == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    g = sms > 0 ? std::min(sms, kMaxArnCta) : 152;
  }
  return g;
}

static size_t pass_smem(int k) { return (size_t)stages_for(k) * (ucol_for(k) + 1) * kSegBytes; }

// Opt the pipelined passes in to their dynamic shared memory (once, outside capture).
template <typename T>
static void set_attrs_t() {
#define PSP_ATTR(KS_)                                                                                    \
  cudaFuncSetAttribute(k_cgs_pass1<T, KS_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBudget); \
  cudaFuncSetAttribute(k_cgs_pass2<T, KS_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBudget); \
  cudaFuncSetAttribute(k_cgs_pass3<T, KS_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBudget);
  PSP_ATTR(1) PSP_ATTR(2) PSP_ATTR(3) PSP_ATTR(4) PSP_ATTR(5) PSP_ATTR(6) PSP_ATTR(7) PSP_ATTR(8)
#undef PSP_ATTR
}

void arnoldi_setup() {
  arnoldi_grid();
  set_attrs_t<float>();
  set_attrs_t<double>();
}

template <typename T>
void launch_arnoldi(int k, int64_t n, const ArnoldiMaps &maps, T *V, int64_t ldv, DevState *st, double *partial,
                    int mixed, cudaStream_t s, cudaEvent_t *ev) {
  // tiles cover the padded column length ldv (a multiple of the tile)
  const int ntiles = (int)((ldv * (int64_t)sizeof(T)) / kSegBytes);
  int grid = std::min(ntiles, arnoldi_grid());
  if (grid < 1) grid = 1;
  const size_t sm = pass_smem(k);
  const VMaps &mV = *reinterpret_cast<const VMaps *>(maps.V);
  const CUtensorMap &mU = *reinterpret_cast<const CUtensorMap *>(maps.Py);
  double *p1 = partial, *p2 = partial + (int64_t)(kMaxM + 2) * kMaxCta, *p3 = partial + 2 * (int64_t)(kMaxM + 2) * kMaxCta;
#define PSP_CGS(KS_)                                                                                       \
  case KS_:                                                                                                \
    k_cgs_pass1<T, KS_><<<grid, kArnThreads, sm, s>>>(mV, mU, k, st, p1, ntiles);                          \
    if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);                                   \
    k_cgs_pass2<T, KS_><<<grid, kArnThreads, sm, s>>>(mV, mU, k, st, p1, p2, ntiles, grid);                \
    if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);                                   \
    k_cgs_pass3<T, KS_><<<grid, kArnThreads, sm, s>>>(mV, mU, V, ldv, k, st, p2, p3, ntiles, grid, mixed); \
    if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);                                   \
    break;
  switch ((k + kArnWarps - 1) / kArnWarps) {
    PSP_CGS(1) PSP_CGS(2) PSP_CGS(3) PSP_CGS(4) PSP_CGS(5) PSP_CGS(6) PSP_CGS(7) PSP_CGS(8)
    default: break;
  }
#undef PSP_CGS
}

// Tensor maps of the Krylov basis (ncols x ld) and of the P_y ring (mmax x ld), element
// type T, boxes of 1 KB along the vector and kBoxCols (V) or 1 (ring) columns.
template <typename T>
bool encode_arnoldi_maps(ArnoldiMaps &maps, const T *V, int ncols, const T *Py, int mmax, int64_t ld) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  const cuuint32_t tr = (cuuint32_t)(kSegBytes / sizeof(T));
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t stride[1] = {(cuuint64_t)(ld * sizeof(T))};
  const cuuint32_t cols[3] = {16, 4, 1};
  for (int b = 0; b < 3; ++b) {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)ncols};
    const cuuint32_t box[2] = {tr, cols[b]};
    if (encode(reinterpret_cast<CUtensorMap *>(maps.V) + b, dt, 2, const_cast<T *>(V), dims, stride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)mmax};
    const cuuint32_t box[2] = {tr, 1};
    if (encode(reinterpret_cast<CUtensorMap *>(maps.Py), dt, 2, const_cast<T *>(Py), dims, stride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

template bool encode_arnoldi_maps<float>(ArnoldiMaps &, const float *, int, const float *, int, int64_t);
template bool encode_arnoldi_maps<double>(ArnoldiMaps &, const double *, int, const double *, int, int64_t);

template <typename T>
void launch_scale_copy(int k, int64_t n, const T *V, int64_t ldv, OutRef<T> y, const DevState *st,
                       cudaStream_t s) {
  int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_scale_copy<T><<<grid < 1 ? 1 : grid, kThreads, 0, s>>>(k, n, V, ldv, y, st);
}

template <typename T>
void launch_update_z(int64_t n, const T *V, int64_t ldv, T *Z, double *X, int add_to_x, const DevState *st,
                     cudaStream_t s) {
  int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_update_z<T><<<grid < 1 ? 1 : grid, kThreads, 0, s>>>(n, V, ldv, Z, X, add_to_x, st);
}

template void launch_arnoldi<float>(int, int64_t, const ArnoldiMaps &, float *, int64_t, DevState *, double *, int,
                                    cudaStream_t, cudaEvent_t *);
template void launch_arnoldi<double>(int, int64_t, const ArnoldiMaps &, double *, int64_t, DevState *, double *, int,
                                     cudaStream_t, cudaEvent_t *);
template void launch_scale_copy<float>(int, int64_t, const float *, int64_t, OutRef<float>, const DevState *,
                                       cudaStream_t);
template void launch_scale_copy<double>(int, int64_t, const double *, int64_t, OutRef<double>,
                                        const DevState *, cudaStream_t);
template void launch_update_z<float>(int64_t, const float *, int64_t, float *, double *, int, const DevState *,
                                     cudaStream_t);
template void launch_update_z<double>(int64_t, const double *, int64_t, double *, double *, int,
                                      const DevState *, cudaStream_t);

}  // namespace psp
