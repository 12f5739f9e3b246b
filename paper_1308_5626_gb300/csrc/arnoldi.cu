// Arnoldi step of Algorithm 1 (orthogonalisation, H(:,k), V(:,k+1)), the Givens update of the
// Hessenberg least-squares problem with the residual R(k) = |G(k+1)| and the finish test,
// and the cycle update Z = sum_j Q(j) V(:,j) with Q = H^{-1} G.
//
// The paper orthogonalises with modified Gram-Schmidt, one global reduction per basis
// vector.  Here the orthogonalisation is classical Gram-Schmidt with re-orthogonalisation
// delayed by one iteration (DCGS2; Bielich, Langou, Thomas, Swirydowicz, Yamazaki, Boman,
// "Low-synch Gram-Schmidt with delayed reorthogonalization for Krylov solvers", Parallel
// Computing 2022): the same Arnoldi relation in exact arithmetic, the stability of CGS2,
// and only two streaming passes over the basis per iteration j:
//
//   pass A (k_dcgs_dots):   a = Q^T v_j, alpha = v_j^T v_j, b = Q^T w_j, beta = v_j^T w_j,
//                           w_j = A N^{-1} v_j, Q = [q_0 .. q_{j-1}] (per-CTA partial sums);
//   pass B (k_dcgs_update): every CTA reduces the partials and forms, in FP64,
//                           nu_j = sqrt(alpha - a^T a)             (q_j = (v_j - Q a) / nu_j),
//                           column j-1 of H completed: H(:, j-1) = h_{j-1} + a, H(j, j-1) = nu_j,
//                           t = Hbar a, h_j = ([b; (beta - a^T b)/nu_j] - t) / nu_j,
//                           then streams q_j and v_{j+1} = w_j/nu_j - (c_j/nu_j) v_j - Q d,
//                           c = t/nu_j + h_j, d = c_{0..j-1} - (c_j/nu_j) a.
//
// CTA 0 of pass B alone owns the persistent state (Hessenberg columns, Givens rotations,
// R(j), the finish test, the triangular solve at the end of the cycle).  The Krylov
// vector v_j handed to the preconditioner and the matvec is the once-orthogonalised,
// unnormalised one; (N^{-1} v_j, A N^{-1} v_j) is still an exact matvec pair for the
// history of Algorithm 2.  Column j-1 is completed one iteration late, so a cycle runs one
// matvec past the iteration that meets the tolerance, and a cycle that reaches m columns
// ends with a reduction-only step.
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
  __device__ static __forceinline__ float4 scale(float c, float4 x) { return make_float4(c * x.x, c * x.y, c * x.z, c * x.w); }
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
  __device__ static __forceinline__ double2 scale(double c, double2 x) { return make_double2(c * x.x, c * x.y); }
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

// V segments of one tile into `stage` (thread 0); the mbarrier expects the whole stage,
// U included.
template <typename T>
__device__ __forceinline__ void issue_tile_v(const TilePipe &p, int stage, int tile, const CUtensorMap *mapV) {
  constexpr int TR = kSegBytes / sizeof(T);   // rows per tile
  char *base = p.buf + (int64_t)stage * p.ncols * kSegBytes;
  mbar_expect_tx(&p.bar[stage], (uint32_t)(p.ncols * kSegBytes));
  int cb = 0;
  for (; cb + 16 <= p.ucol; cb += 16) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[0], tile * TR, cb, &p.bar[stage]);
  for (; cb + 4 <= p.ucol; cb += 4) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[1], tile * TR, cb, &p.bar[stage]);
  for (; cb < p.ucol; ++cb) tma_load_2d(base + (int64_t)cb * kSegBytes, &mapV[2], tile * TR, cb, &p.bar[stage]);
}
// U segment of one tile (thread 0).
template <typename T>
__device__ __forceinline__ void issue_tile_u(const TilePipe &p, int stage, int tile, const CUtensorMap *mapU) {
  constexpr int TR = kSegBytes / sizeof(T);
  char *base = p.buf + (int64_t)stage * p.ncols * kSegBytes;
  tma_load_2d(base + (int64_t)p.ucol * kSegBytes, mapU, tile * TR, p.uring, &p.bar[stage]);
}
template <typename T>
__device__ __forceinline__ void issue_tile(const TilePipe &p, int stage, int tile, const CUtensorMap *mapV,
                                           const CUtensorMap *mapU) {
  issue_tile_v<T>(p, stage, tile, mapV);
  issue_tile_u<T>(p, stage, tile, mapU);
}

// Drives the pipeline: calls body(stage_ptr, tile) for each of this CTA's tiles.
__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// With defer_u the prologue writes U itself (the matvec folded into the pass): the V
// segments of the first stages are issued before it and their U segments after it, once
// its global writes are ordered before the bulk copies that read them.
template <typename T, typename Body, typename Pro>
__device__ __forceinline__ void run_tiles(TilePipe &p, const CUtensorMap *mapV, const CUtensorMap *mapU, DevState *st,
                                          bool defer_u, Pro prologue, Body body) {
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
    for (int i = 0; i < kStages && i < my; ++i) {
      if (defer_u) issue_tile_v<T>(p, i, p.first + i * p.step, mapV);
      else issue_tile<T>(p, i, p.first + i * p.step, mapV, mapU);
    }
  prologue(my);        // runs while the first tiles are in flight
  if (defer_u) asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (defer_u && threadIdx.x == 0)
    for (int i = 0; i < kStages && i < my; ++i) issue_tile_u<T>(p, i, p.first + i * p.step, mapU);
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

// The matvec of the iteration, w = A x (Eq. 4: A = I - dt L with the finite-difference
// stencil of L), on the rows of this CTA's tiles: thread e of the CTA takes vector e % 64
// of tile e / 64 (16-byte vectors of W points along x), one or two vectors per round with
// every load of the round issued before the arithmetic.  The x terms come from a register
// window of the row, the y and z terms from one vector per neighbour row (periodic).  With
// xc set, x is also copied there (P_x column of an unpreconditioned cycle).  Needs
// nx % W == 0 and more vectors per row than halo vectors.
template <typename T, int NDIM, int R>
__device__ __forceinline__ void tile_matvec_t(const T *__restrict__ x, T *__restrict__ w, T *__restrict__ xc,
                                           const T (*c)[2 * kMaxR + 1], int nx, int ny, int nz, int first,
                                           int step, int my) {
  using VT = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  constexpr int NH = (R + W - 1) / W;          // halo vectors on each side along x
  constexpr int NY = NDIM >= 2 ? R : 0, NZ = NDIM >= 3 ? R : 0;
  // vectors per thread and round: two while their loads fit in about 80 registers
  constexpr int kLoads = 2 * NH + 1 + 2 * NY + 2 * NZ;
  constexpr int U = kLoads <= 10 ? 2 : 1;
  const int nxv = nx / W, plane = nx * ny;
  const int nvec = nxv * ny * nz;
  const int total = my * kSegVec;
  for (int e0 = threadIdx.x; e0 < total; e0 += U * blockDim.x) {
    int iv[U];
    bool ok[U];
    VT win[U][2 * NH + 1], ym[U][NY > 0 ? NY : 1], yp[U][NY > 0 ? NY : 1], zm[U][NZ > 0 ? NZ : 1],
        zp[U][NZ > 0 ? NZ : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * blockDim.x;
      iv[u] = (first + (e / kSegVec) * step) * kSegVec + (e % kSegVec);
      ok[u] = e < total && iv[u] < nvec;
      if (!ok[u]) iv[u] = 0;   // loads of a padding lane stay in bounds; nothing is stored
      const int row = iv[u] / nxv;
      const int xv = iv[u] - row * nxv;
      const int iz = row / ny;
      const int iy = row - iz * ny;
      const int base = row * nx;
#pragma unroll
      for (int h = -NH; h <= NH; ++h) {
        int v = xv + h;
        v += (v < 0) ? nxv : 0;
        v -= (v >= nxv) ? nxv : 0;
        win[u][h + NH] = *reinterpret_cast<const VT *>(x + base + v * W);
      }
#pragma unroll
      for (int jj = 1; jj <= NY; ++jj) {
        int m = iy - jj; m += (m < 0) ? ny : 0;
        int p = iy + jj; p -= (p >= ny) ? ny : 0;
        ym[u][jj - 1] = *reinterpret_cast<const VT *>(x + iz * plane + m * nx + xv * W);
        yp[u][jj - 1] = *reinterpret_cast<const VT *>(x + iz * plane + p * nx + xv * W);
      }
#pragma unroll
      for (int jj = 1; jj <= NZ; ++jj) {
        int m = iz - jj; m += (m < 0) ? nz : 0;
        int p = iz + jj; p -= (p >= nz) ? nz : 0;
        zm[u][jj - 1] = *reinterpret_cast<const VT *>(x + m * plane + iy * nx + xv * W);
        zp[u][jj - 1] = *reinterpret_cast<const VT *>(x + p * plane + iy * nx + xv * W);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const T *wn = reinterpret_cast<const T *>(&win[u][0]);   // (2 NH + 1) W points
      T acc[W];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        T s = c[0][kMaxR] * wn[NH * W + i];
#pragma unroll
        for (int jj = 1; jj <= R; ++jj)
          s += c[0][kMaxR - jj] * wn[NH * W + i - jj] + c[0][kMaxR + jj] * wn[NH * W + i + jj];
        acc[i] = s;
      }
#pragma unroll
      for (int jj = 1; jj <= NY; ++jj) {
        const T *me = reinterpret_cast<const T *>(&ym[u][jj - 1]), *pe = reinterpret_cast<const T *>(&yp[u][jj - 1]);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] += c[1][kMaxR - jj] * me[i] + c[1][kMaxR + jj] * pe[i];
      }
#pragma unroll
      for (int jj = 1; jj <= NZ; ++jj) {
        const T *me = reinterpret_cast<const T *>(&zm[u][jj - 1]), *pe = reinterpret_cast<const T *>(&zp[u][jj - 1]);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] += c[2][kMaxR - jj] * me[i] + c[2][kMaxR + jj] * pe[i];
      }
      if (ok[u]) {
        VT out;
        T *oe = reinterpret_cast<T *>(&out);
#pragma unroll
        for (int i = 0; i < W; ++i) oe[i] = acc[i];
        reinterpret_cast<VT *>(w)[iv[u]] = out;
        if (xc) reinterpret_cast<VT *>(xc)[iv[u]] = win[u][NH];
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void tile_matvec(const TileMatvec<T> &mv, const T (*c)[2 * kMaxR + 1], int first, int step,
                                            int my) {
  const T *x = mv.x.get();
  T *w = mv.w.get();
  T *xc = mv.xcopy.base ? mv.xcopy.get() : nullptr;
#define PSP_TMV(D_, R_) \
  tile_matvec_t<T, D_, R_>(x, w, xc, c, mv.nx, mv.ny, mv.nz, first, step, my)
#define PSP_TMV_R(D_)                  \
  switch (mv.R) {                      \
    case 1: PSP_TMV(D_, 1); break;     \
    case 2: PSP_TMV(D_, 2); break;     \
    case 3: PSP_TMV(D_, 3); break;     \
    case 4: PSP_TMV(D_, 4); break;     \
    case 5: PSP_TMV(D_, 5); break;     \
    default: break;                    \
  }
  switch (mv.ndim) {
    case 1: PSP_TMV_R(1); break;
    case 2: PSP_TMV_R(2); break;
    case 3: PSP_TMV_R(3); break;
    default: break;
  }
#undef PSP_TMV_R
#undef PSP_TMV
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
// out[j] = sum over CTAs of partial[j][cta] in a fixed order, j < nvals (rows of length
// kMaxCta, element type TP: float in the mixed form, whose dot products are FP32
// accumulations, double otherwise).  The sums are formed in TP: on GB300 every FP64 warp
// instruction (conversions included) occupies the narrow FP64 pipe for tens of cycles.
template <typename TP>
__device__ __forceinline__ void grid_sums(const TP *partial, int nvals, int nb, TP *out) {
  constexpr int kMinWarps = 8;                                      // blocks of >= 256 threads
  constexpr int MJ = (2 * kMaxM + 2 + kMinWarps - 1) / kMinWarps;   // j values per warp (at most)
  constexpr int MB = kMaxArnCta / 32;                               // CTAs per lane
  constexpr int BATCH = 3;                                          // j values loaded together
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nq = (nb + 31) / 32;
#pragma unroll
  for (int t0 = 0; t0 < MJ; t0 += BATCH) {
    if (wid + t0 * nw >= nvals) break;
    TP v[BATCH][MB];
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      const int j = wid + (t0 + t) * nw;
#pragma unroll
      for (int q = 0; q < MB; ++q) {
        const int b = lane + 32 * q;
        v[t][q] = (q < nq && j < nvals && b < nb) ? __ldcg(partial + (int64_t)j * kMaxCta + b) : (TP)0;
      }
    }
#pragma unroll
    for (int t = 0; t < BATCH; ++t) {
      TP sl = (TP)0;
#pragma unroll
      for (int q = 0; q < MB; ++q)
        if (q < nq) sl += v[t][q];
      sl = warp_sum(sl);
      const int j = wid + (t0 + t) * nw;
      if (lane == 0 && j < nvals) out[j] = sl;
    }
  }
  __syncthreads();
}

// FP64 Givens step for the completed column kk of H (rows 0..kk+1 in hcol, shared memory),
// R(kk+1) and the finish test; run by one thread with the rotations staged in shared
// memory (sC, sS, sG hold C, S, G).  Returns true when the cycle ends.
__device__ bool givens_column(DevState *st, int kk, double *hcol, double *sC, double *sS, double *sG, bool brk,
                              bool force_end, int mixed) {
  const int k = kk + 1;
  for (int i = 0; i < kk; ++i) {   // old rotations
    const double d = hcol[i];
    hcol[i] = d * sC[i] + sS[i] * hcol[i + 1];
    hcol[i + 1] = -d * sS[i] + sC[i] * hcol[i + 1];
  }
  const double gamma = hypot(hcol[kk], hcol[k]);
  double c = 1.0, s = 0.0;
  if (gamma > 0.0) {
    c = hcol[kk] / gamma;
    s = hcol[k] / gamma;
  }
  hcol[kk] = gamma;
  hcol[k] = 0.0;
  const double d = sG[kk];
  const double gk = -s * d;
  sG[kk] = c * d;
  sG[k] = gk;
  sC[kk] = c;
  sS[kk] = s;
  // write back: rotated column, rotation, G
  const int ld = kMaxM + 1;
  for (int r = 0; r <= k; ++r) st->H[(int64_t)kk * ld + r] = hcol[r];
  st->C[kk] = c;
  st->S[kk] = s;
  st->G[kk] = sG[kk];
  st->G[k] = gk;
  const double R = fabs(gk);
  st->R[kk] = R;
  int status = st->status;
  if (!isfinite(R) || !isfinite(gamma)) status |= kStNumeric;
  if (brk) status |= kStBreakdown;
  if (!mixed && R <= st->eps_abs) status |= kStConverged;
  st->status = status;
  st->k_end = k;
  const bool end = (R <= st->eps_cycle) || brk || force_end || (status & kStNumeric);
  st->sum.k_end = k;
  st->sum.error = st->error;
  st->sum.status = status;
  st->sum.R_end = R;
  return end;
}

// ---------------------------------------------------------------------------------------
// DCGS2 scalar engine, run once per iteration by all threads of the last CTA of pass A:
// reduce the partial sums, form nu_j, complete column j-1, t = Hbar a, h_j, the pass-B
// coefficients, the Givens step, the finish test and, when the cycle ends, Q = H^{-1} G.
// Small dense work in FP64 out of shared memory (`scratch`, the freed stage ring).
// ---------------------------------------------------------------------------------------
// Arrays of the scalar engine in the precision of the Krylov vectors (FP32 copies in the
// mixed form; the FP64 Hessenberg used by the Givens step is kept alongside).
template <typename T> __device__ __forceinline__ T *hc_copy(DevState *st);
template <> __device__ __forceinline__ float *hc_copy<float>(DevState *st) { return st->HcF; }
template <> __device__ __forceinline__ double *hc_copy<double>(DevState *st) { return st->Hc; }
template <typename T> __device__ __forceinline__ T *coef_copy(DevState *st, int which);
template <> __device__ __forceinline__ float *coef_copy<float>(DevState *st, int which) {
  return which == 0 ? st->cAF : (which == 1 ? st->cDF : st->c3F);
}
template <> __device__ __forceinline__ double *coef_copy<double>(DevState *st, int which) {
  return which == 0 ? st->cA : (which == 1 ? st->cD : st->c3);
}

template <typename T>
__device__ void dcgs_scalar(DevState *st, int j, int final_step, const T *partial, int nb, T *scratch) {
  constexpr int ld = kMaxM + 1;
  T *s_sum = scratch;                                             // 2 kMaxM + 2
  T *sH = s_sum + 2 * kMaxM + 2;                                  // kMaxM * ld
  T *s_a = sH + kMaxM * ld;                                       // kMaxM
  T *s_t = s_a + kMaxM;                                           // kMaxM + 1
  T *s_hcol = s_t + kMaxM + 1;                                    // kMaxM + 2
  T *s_sc = s_hcol + kMaxM + 2;                                   // 4
  const T *HcT = hc_copy<T>(st);
  T *HcTw = hc_copy<T>(st);
  const int k = j + 1;
  for (int e = threadIdx.x; e < (j > 1 ? (j - 1) * ld : 0); e += blockDim.x) sH[e] = HcT[e];
  if (j >= 1)
    for (int r = threadIdx.x; r < j; r += blockDim.x) s_hcol[r] = (T)st->Hf[(int64_t)(j - 1) * ld + r];
  grid_sums<T>(partial, 2 * k, nb, s_sum);   // ends with a barrier
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid == 0) {
    T aa = (T)0, ab = (T)0;
    for (int i = lane; i < j; i += 32) {
      const T ai = s_sum[i];
      s_a[i] = ai;
      aa += ai * ai;
      ab += ai * s_sum[k + i];
    }
    aa = warp_sum(aa);
    ab = warp_sum(ab);
    if (lane == 0) {
      const T alpha = s_sum[j];
      const T nu2 = alpha - aa;
      const bool brk = !(nu2 > (T)(kBreakdownRel * kBreakdownRel) * alpha) || !isfinite(nu2);
      s_sc[0] = brk ? (T)0 : sqrt(nu2);
      s_sc[2] = ab;
      st->dc_brk = brk ? 1 : 0;
    }
  }
  __syncthreads();
  const T nu = s_sc[0];
  // completed column j-1 (first projection + a, nu in row j): kept for the Givens step
  if (j >= 1)
    for (int r = threadIdx.x; r <= j; r += blockDim.x) {
      const T v = (r < j) ? s_hcol[r] + s_a[r] : nu;
      s_hcol[r] = v;
      st->Hc[(int64_t)(j - 1) * ld + r] = (double)v;
      HcTw[(int64_t)(j - 1) * ld + r] = v;
    }
  __syncthreads();
  for (int r = threadIdx.x; r <= j; r += blockDim.x) {   // t = Hbar a
    T t = (T)0;
    for (int i = (r > 0 ? r - 1 : 0); i < j; ++i) t += ((i == j - 1) ? s_hcol[r] : sH[i * ld + r]) * s_a[i];
    s_t[r] = t;
  }
  __syncthreads();
  const T inv = (nu > (T)0) ? (T)1 / nu : (T)0;
  const T beta = s_sum[k + j];
  for (int r = threadIdx.x; r <= j; r += blockDim.x) {
    const T proj = (r < j) ? s_sum[k + r] : (beta - s_sc[2]) * inv;
    const T h = (proj - s_t[r]) * inv;
    if (!final_step) st->Hf[(int64_t)j * ld + r] = (double)h;
    s_t[r] = s_t[r] * inv + h;                    // c_r
  }
  __syncthreads();
  const T cj = s_t[j];
  T *cA = coef_copy<T>(st, 0), *cD = coef_copy<T>(st, 1), *c3 = coef_copy<T>(st, 2);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cA[i] = s_a[i] * inv;
    cD[i] = s_t[i] - cj * inv * s_a[i];
  }
  if (threadIdx.x == 0) {
    c3[0] = inv;
    c3[1] = cj * inv;
    c3[2] = inv;
  }
}

// Givens step for column j-1 (completed by the scalar engine of this iteration), the
// finish test and, when the cycle ends, Q = H^{-1} G; one CTA of pass B, concurrently with
// the stream of the other CTAs.
__device__ void dcgs_givens(DevState *st, int j, int final_step, int mixed, double *scratch) {
  constexpr int ld = kMaxM + 1;
  double *s_hcol = scratch;                   // kMaxM + 2
  double *sC = s_hcol + kMaxM + 2;            // kMaxM
  double *sS = sC + kMaxM;                    // kMaxM
  double *sG = sS + kMaxM;                    // kMaxM + 1
  double *s_t = sG + kMaxM + 1;               // kMaxM + 1
  double *sH = s_t + kMaxM + 1;               // kMaxM * ld
  __shared__ int s_end;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    if (i < j) { sC[i] = st->C[i]; sS[i] = st->S[i]; }
    sG[i] = st->G[i];
    if (j >= 1) s_hcol[i] = st->Hc[(int64_t)(j - 1) * ld + i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool brk = st->dc_brk != 0;
    bool end = false;
    if (j >= 1) {
      end = givens_column(st, j - 1, s_hcol, sC, sS, sG, brk, final_step != 0, mixed);
    } else if (brk || final_step) {
      end = true;   // v_0 = 0: nothing to do
      st->k_end = 0;
      st->sum.k_end = 0;
    }
    if (end) {
      st->active = 0;
      // matvecs of this cycle: iterations 0..j had one each, the final step none
      st->hist_count = st->hist_base + 1 + (final_step ? j : j + 1);
      st->sum.hist_count = st->hist_count;
    }
    s_end = end ? 1 : 0;
  }
  __syncthreads();
  if (s_end) {
    // Q = H^{-1} G on the leading kend x kend triangle of the rotated H (column-oriented
    // back substitution); the basis scales of the update become 1
    const int kend = st->k_end;
    for (int e = threadIdx.x; e < kend * ld; e += blockDim.x) sH[e] = st->H[e];
    for (int i = threadIdx.x; i <= kend; i += blockDim.x) s_t[i] = st->G[i];
    __syncthreads();
    for (int c = kend - 1; c >= 0; --c) {
      const double hcc = sH[c * ld + c];
      const double q = hcc != 0.0 ? s_t[c] / hcc : 0.0;
      __syncthreads();
      for (int i = threadIdx.x; i < c; i += blockDim.x) s_t[i] -= sH[c * ld + i] * q;
      if (threadIdx.x == 0) { st->Q[c] = q; st->sigma[c] = 1.0; }
      __syncthreads();
    }
  }
}

// Shared memory (doubles) the scalar engine needs.
constexpr int kScalarDoubles = (2 * kMaxM + 2) + kMaxM * (kMaxM + 1) + kMaxM + (kMaxM + 1) + (kMaxM + 2) + 4;
// ... and the Givens CTA of pass B
constexpr int kGivensDoubles = (kMaxM + 2) + 2 * kMaxM + 2 * (kMaxM + 1) + kMaxM * (kMaxM + 1);

// ---------------------------------------------------------------------------------------
// pass A: partial sums of V_i^T v_j (rows 0..j) and V_i^T w_j (rows j+1..2j+1), i <= j
// ---------------------------------------------------------------------------------------
template <typename T, int KS>
__global__ void __launch_bounds__(kArnThreads) k_dcgs_dots(const __grid_constant__ VMaps mapV,
                                                           const __grid_constant__ CUtensorMap mapU, int j, int woff,
                                                           DevState *st, T *partial, int ntiles, int final_step,
                                                           const TileMatvec<T> mv) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  extern __shared__ __align__(128) char smem[];
  __shared__ uint64_t bars[kMaxStages];
  __shared__ T s_c[3][2 * kMaxR + 1];
  const bool fused = mv.x.base != nullptr;
  if (fused && threadIdx.x < 3 * (2 * kMaxR + 1))
    s_c[threadIdx.x / (2 * kMaxR + 1)][threadIdx.x % (2 * kMaxR + 1)] =
        (T)st->coef[threadIdx.x / (2 * kMaxR + 1)][threadIdx.x % (2 * kMaxR + 1)];
  // (the pipeline's first CTA barrier orders these writes before the prologue)
  const int k = j + 1;                      // V columns 0..j
  const int ucol = ucol_for(k);
  TilePipe p{smem, bars, ucol + 1, ucol, ntiles, (int)blockIdx.x, (int)gridDim.x, stages_for(k),
             (st->hist_base + woff) % st->mmax};
  T av[KS], aw[KS];
#pragma unroll
  for (int s = 0; s < KS; ++s) { av[s] = (T)0; aw[s] = (T)0; }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  run_tiles<T>(p, mapV.m, &mapU, st, fused, [&](int my) {
    if (fused) tile_matvec<T>(mv, s_c, p.first, p.step, my);
  }, [&](const T *tile, int) {
    const VT *vseg = reinterpret_cast<const VT *>(tile) + (int64_t)j * kSegVec;
    const VT *wseg = reinterpret_cast<const VT *>(tile) + (int64_t)ucol * kSegVec;
    const VT v0 = vseg[lane], v1 = vseg[lane + 32], w0 = wseg[lane], w1 = wseg[lane + 32];
#pragma unroll
    for (int s = 0; s < KS; ++s) {
      const int i = wid + kArnWarps * s;
      if (i < k) {
        const VT *seg = reinterpret_cast<const VT *>(tile) + (int64_t)i * kSegVec;
        const VT x0 = seg[lane], x1 = seg[lane + 32];
        av[s] += Vec<T>::dot(x0, v0) + Vec<T>::dot(x1, v1);
        aw[s] += Vec<T>::dot(x0, w0) + Vec<T>::dot(x1, w1);
      }
    }
  });
#pragma unroll
  for (int s = 0; s < KS; ++s) {
    const int i = wid + kArnWarps * s;
    const T x = warp_sum(av[s]);
    const T y = warp_sum(aw[s]);
    if (lane == 0 && i < k) {
      partial[(int64_t)i * kMaxCta + blockIdx.x] = x;
      partial[(int64_t)(k + i) * kMaxCta + blockIdx.x] = y;
    }
  }
  if (!last_block_arrive(&st->counter[1])) return;
  // pass B (a programmatic dependent) may start its CTAs now; it waits for this grid
  // before it reads anything the scalar engine writes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  dcgs_scalar<T>(st, j, final_step, partial, gridDim.x, reinterpret_cast<T *>(smem));
  last_block_reset(&st->counter[1]);
}


// ---------------------------------------------------------------------------------------
// pass B: q_j over v_j in V(:,j) and v_{j+1} in V(:,j+1), with the coefficients formed by
// the scalar engine.  Columns are taken in chunks of 8 with the column index clamped to
// j-1 and a zero coefficient past j, so the 8 loads of a chunk (for two vectors per
// thread) are issued together.
// ---------------------------------------------------------------------------------------
constexpr int kUpdThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kUpdThreads) k_dcgs_update(T *__restrict__ V, int64_t ldv, const T *__restrict__ Pyb,
                                                             int64_t ldh, int j, int woff, DevState *st, int64_t nv,
                                                             int final_step, int mixed) {
  // Launched as a programmatic dependent of pass A: the CTAs may be scheduled while pass
  // A's last CTA still forms the coefficients, and wait here for that grid to finish.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (st->active == 0) return;   // the cycle ended: nothing to do
  extern __shared__ __align__(16) double dsm[];
  if (blockIdx.x == gridDim.x - 1) {   // the Givens CTA
    dcgs_givens(st, j, final_step, mixed, dsm);
    return;
  }
  using VT = typename Vec<T>::type;
  __shared__ T s_sa[kMaxM], s_sd[kMaxM];
  const T *cA = coef_copy<T>(st, 0), *cD = coef_copy<T>(st, 1), *c3 = coef_copy<T>(st, 2);
  for (int i = threadIdx.x; i < kMaxM; i += blockDim.x) {
    s_sa[i] = (i < j) ? cA[i] : (T)0;
    s_sd[i] = (i < j) ? cD[i] : (T)0;
  }
  const T sv = c3[0], cv = c3[1], sw = c3[2];
  __syncthreads();
  VT *vj = reinterpret_cast<VT *>(V + (int64_t)j * ldv);
  VT *vn = reinterpret_cast<VT *>(V + (int64_t)(j + 1) * ldv);
  const VT *w = reinterpret_cast<const VT *>(Pyb + (int64_t)((st->hist_base + woff) % st->mmax) * ldh);
  const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;   // streaming CTAs
  for (int64_t iv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; iv < nv; iv += 2 * stride) {
    const int64_t iv2 = iv + stride;
    const bool two = iv2 < nv;
    const int64_t jv2 = two ? iv2 : iv;
    const VT v0 = vj[iv], v1 = vj[jv2];
    const VT x0 = w[iv], x1 = w[jv2];
    VT q0 = Vec<T>::scale(sv, v0), q1 = Vec<T>::scale(sv, v1);
    VT y0 = Vec<T>::axpy(cv, v0, Vec<T>::scale(sw, x0)), y1 = Vec<T>::axpy(cv, v1, Vec<T>::scale(sw, x1));
    for (int c0 = 0; c0 < j; c0 += 8) {
      VT a0[8], a1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = min(c0 + u, j - 1);
        const VT *qc = reinterpret_cast<const VT *>(V + (int64_t)col * ldv);
        a0[u] = qc[iv];
        a1[u] = qc[jv2];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T ca = s_sa[c0 + u], cd = s_sd[c0 + u];
        q0 = Vec<T>::axpy(ca, a0[u], q0);
        y0 = Vec<T>::axpy(cd, a0[u], y0);
        q1 = Vec<T>::axpy(ca, a1[u], q1);
        y1 = Vec<T>::axpy(cd, a1[u], y1);
      }
    }
    vj[iv] = q0;
    vn[iv] = y0;
    if (two) {
      vj[iv2] = q1;
      vn[iv2] = y1;
    }
  }
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

// Opt the pipelined pass in to its dynamic shared memory (once, outside capture).
template <typename T>
static void set_attrs_t() {
#define PSP_ATTR(KS_) \
  cudaFuncSetAttribute(k_dcgs_dots<T, KS_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBudget);
  PSP_ATTR(1) PSP_ATTR(2) PSP_ATTR(3) PSP_ATTR(4) PSP_ATTR(5)
#undef PSP_ATTR
}

void arnoldi_setup() {
  arnoldi_grid();
  set_attrs_t<float>();
  set_attrs_t<double>();
  cudaFuncSetAttribute(k_dcgs_update<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kGivensDoubles * sizeof(double)));
  cudaFuncSetAttribute(k_dcgs_update<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kGivensDoubles * sizeof(double)));
}

template <typename T>
void launch_arnoldi(int j, int final_step, int64_t n, const ArnoldiMaps &maps, T *V, int64_t ldv, const T *Py,
                    int64_t ldh, DevState *st, double *partial, int mixed, cudaStream_t s, cudaEvent_t *ev,
                    const TileMatvec<T> *mv) {
  const TileMatvec<T> m = mv ? *mv : TileMatvec<T>{};
  const int ntiles = (int)((ldv * (int64_t)sizeof(T)) / kSegBytes);
  int grid = std::min(ntiles, arnoldi_grid());
  if (grid < 1) grid = 1;
  const int k = j + 1;
  // the stage ring, later reused by the last CTA as the scalar engine's scratch
  const size_t sm = std::max(pass_smem(k), (size_t)kScalarDoubles * sizeof(double));
  const int woff = 1 + j;   // ring column of w_j relative to the cycle's restart column
  const VMaps &mV = *reinterpret_cast<const VMaps *>(maps.V);
  const CUtensorMap &mU = *reinterpret_cast<const CUtensorMap *>(maps.Py);
  switch ((k + kArnWarps - 1) / kArnWarps) {
#define PSP_DOTS(KS_) \
  case KS_: k_dcgs_dots<T, KS_><<<grid, kArnThreads, sm, s>>>(mV, mU, j, woff, st, reinterpret_cast<T *>(partial), ntiles, final_step, m); break;
    PSP_DOTS(1) PSP_DOTS(2) PSP_DOTS(3) PSP_DOTS(4) PSP_DOTS(5)
#undef PSP_DOTS
    default: break;
  }
  if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
  if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
  {
    // streaming CTAs (none for the final step) plus one CTA for the Givens step
    const int64_t nv = (ldv + Vec<T>::W - 1) / Vec<T>::W;
    int ugrid = final_step ? 0 : (int)std::min<int64_t>((nv + kUpdThreads - 1) / kUpdThreads, (int64_t)arnoldi_grid() * 4);
    if (!final_step && ugrid < 1) ugrid = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ugrid + 1));
    cfg.blockDim = dim3(kUpdThreads);
    cfg.dynamicSmemBytes = kGivensDoubles * sizeof(double);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_dcgs_update<T>, V, ldv, Py, ldh, j, woff, st, nv, final_step, mixed);
  }
  if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
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

template void launch_arnoldi<float>(int, int, int64_t, const ArnoldiMaps &, float *, int64_t, const float *, int64_t,
                                    DevState *, double *, int, cudaStream_t, cudaEvent_t *, const TileMatvec<float> *);
template void launch_arnoldi<double>(int, int, int64_t, const ArnoldiMaps &, double *, int64_t, const double *,
                                     int64_t, DevState *, double *, int, cudaStream_t, cudaEvent_t *,
                                     const TileMatvec<double> *);

bool fused_matvec_ok(const Geometry &g, int elem_bytes) {
  const int W = 16 / elem_bytes;
  const int nh = (g.R + W - 1) / W;
  return g.R >= 1 && g.R <= kMaxR && g.ndim >= 1 && g.ndim <= 3 && g.nx % W == 0 && g.nx / W > nh;
}
template void launch_scale_copy<float>(int, int64_t, const float *, int64_t, OutRef<float>, const DevState *,
                                       cudaStream_t);
template void launch_scale_copy<double>(int, int64_t, const double *, int64_t, OutRef<double>,
                                        const DevState *, cudaStream_t);
template void launch_update_z<float>(int64_t, const float *, int64_t, float *, double *, int, const DevState *,
                                     cudaStream_t);
template void launch_update_z<double>(int64_t, const double *, int64_t, double *, double *, int,
                                      const DevState *, cudaStream_t);

}  // namespace psp
