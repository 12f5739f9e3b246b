// The on-chip step: one CTA runs every restart cycle of Algorithm 1 for one system, with the
// cycle loop on the device, and one launch runs many systems.
//
// For a system of up to kOnChipMaxN unknowns the restart, the preconditioner solve, the
// stencil matvec, the Gram-Schmidt loop, the Givens step, the finish test and the update
// X = X_0 + N^{-1} Z all run inside one CTA, cycle after cycle, until the step converges,
// max_cycles is reached or a cycle breaks down; the host waits once per launch instead of
// once per cycle, and no kernel is launched per iteration.  A launch takes any number of
// systems: every CTA takes the next system from a shared counter, so a batch of independent
// systems of uneven sizes runs in one persistent launch (the batched form of the step).
//
// The arithmetic is that of the grid-wide path, organised for one CTA:
//  * restart (FP64): r = B - A X_0, the pair (X_0, A X_0) into the history ring, V(:,0) =
//    r / ||r||, G(0) = ||r||; ||B|| and the step bound on the first restart of the step;
//  * iteration k: P_x = N^{-1} V(:,k) (the level sweeps of the partitioned banded solve, one
//    thread per group, a CTA barrier between levels; cyclic bands add the
//    Sherman-Morrison-Woodbury correction), P_y = A P_x, then classical Gram-Schmidt applied
//    twice (CGS2: project, subtract, project again, subtract), ||.|| and V(:,k+1); the block
//    reductions sum each warp's values with shuffles and the warps in a fixed order
//    (deterministic);
//  * the FP64 Givens step of column k, R(k) = |G(k+1)|, the finish test;
//  * end of cycle: Q = H^{-1} G, Z = V Q, X += N^{-1} Z in FP64.
// Vectors are read and written through L1/L2: at these sizes the whole Krylov basis of a
// system stays in the 126 MB L2 while its CTA works on it.
#include <algorithm>

#include "band_sweeps.cuh"
#include "onchip.cuh"

namespace psp {

namespace {

constexpr double kOcBreakdownRel = 1e-14;
constexpr int kOcChunk = 16;   // projections reduced together
constexpr int kOcMaxWarps = 32;
constexpr int kOcLdH = kMaxM + 1;
constexpr int kOcMaxLevels = 16;   // levels of a cached slot (small systems have a handful)

struct OcShared {
  double H[kOcLdH * kMaxM];   // rotated Hessenberg, column-major
  double G[kMaxM + 1], C[kMaxM], S[kMaxM], t[kMaxM + 1], R[kMaxM];
  double h[kMaxM + 1], h2[kMaxM + 1];
  double coef[3][2 * kMaxR + 1];
  float coefF[3][2 * kMaxR + 1];
  double red[kOcMaxWarps][kOcChunk];
  double scal[4];
  double sv[8];   // cyclic correction: K^{-1} y(C)
  int flag[4];
  double levbuf[kOcMaxLevels * 16];   // level descriptors of the cached factors (LevelApply)
};

static_assert(sizeof(LevelApply<double>) <= 16 * sizeof(double) && sizeof(LevelApply<float>) <= 16 * sizeof(double),
              "a level descriptor fits its slot of OcShared::levbuf");

template <typename T> __device__ __forceinline__ T coef_of(const OcShared &sh, int d, int j);
template <> __device__ __forceinline__ double coef_of<double>(const OcShared &sh, int d, int j) { return sh.coef[d][j]; }
template <> __device__ __forceinline__ float coef_of<float>(const OcShared &sh, int d, int j) { return sh.coefF[d][j]; }

// Block sums of v[0..cnt) into out[0..cnt) (every thread contributes, fixed order over warps).
template <typename TV, int K>
__device__ __forceinline__ void oc_reduce(TV (&v)[K], OcShared &sh, double *out, int cnt) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const TV s = warp_sum(v[k]);
    if (lane == 0 && k < cnt) sh.red[wid][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh.red[w][threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// (A x)(r) in the arithmetic of TC: the periodic stencil of the handle (coefficients of A =
// I - dt L in DevState::coef, centres folded into direction 0), or the explicit band.
template <typename TC, typename TX>
__device__ __forceinline__ TC oc_apply_A(const OnChipDesc &d, const OcShared &sh, const TX *__restrict__ x, int r) {
  if (d.band_w > 0) {
    const int w = d.band_w, W = 2 * w + 1;
    TC acc = (TC)0;
    for (int p = 0; p < W; ++p) {
      const int j = r + p - w;
      if (j >= 0 && j < d.n) {
        const TC a = (sizeof(TC) == 4) ? (TC)d.Ab32[(int64_t)r * W + p] : (TC)d.Ab[(int64_t)r * W + p];
        acc += a * (TC)x[j];
      }
    }
    return acc;
  }
  const int plane = d.nx * d.ny;
  const int iz = r / plane, rem = r - iz * plane, iy = rem / d.nx, ix = rem - iy * d.nx;
  TC acc = coef_of<TC>(sh, 0, kMaxR) * (TC)x[r];
  for (int dd = 0; dd < d.ndim; ++dd) {
    const int c = dd == 0 ? ix : (dd == 1 ? iy : iz);
    const int len = dd == 0 ? d.nx : (dd == 1 ? d.ny : d.nz);
    const int stride = dd == 0 ? 1 : (dd == 1 ? d.nx : plane);
    const int base = r - c * stride;
    for (int j = 1; j <= d.R; ++j) {
      int qm = c - j;
      qm += (qm < 0) ? len : 0;
      int qp = c + j;
      qp -= (qp >= len) ? len : 0;
      acc = fma(coef_of<TC>(sh, dd, kMaxR - j), (TC)x[base + qm * stride], acc);
      acc = fma(coef_of<TC>(sh, dd, kMaxR + j), (TC)x[base + qp * stride], acc);
    }
  }
  return acc;
}

// Banded solve N_b^{-1} v of the partitioned factorisation (all levels in this CTA):
// y = solution (y != nullptr) or X += solution.
template <typename T, int B, bool RO>
__device__ void oc_band_solve(const OnChipDesc &d, const LevelApply<T> *lev, const T *v, T *y, double *X) {
  const int L = d.nlev;
  constexpr int SPAN = (kQ0 + 1) * B;
  const int G0 = lev[0].G;
  for (int g = threadIdx.x; g < G0; g += blockDim.x) {
    T f[kQ0][B], sep[B];
    const int row0 = g * SPAN;
#pragma unroll
    for (int i = 0; i < kQ0; ++i)
#pragma unroll
      for (int r = 0; r < B; ++r) {
        const int row = row0 + i * B + r;
        f[i][r] = row < d.n ? v[row] : (T)0;
      }
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int row = row0 + kQ0 * B + r;
      sep[r] = row < d.n ? v[row] : (T)0;
    }
    down_group<T, B, kQ0, RO>(lev[0], g, f, sep, G0, g);
  }
  __syncthreads();
  for (int l = 1; l < L; ++l) {
    const int G = lev[l].G;
    for (int g = threadIdx.x; g < G; g += blockDim.x) down_level_group<T, B, RO>(lev[l], lev[l - 1], g, G, g);
    __syncthreads();
  }
  for (int l = L - 1; l >= 1; --l) {
    const int G = lev[l].G;
    const T *solnext = (l + 1 < L) ? lev[l + 1].sol : nullptr;
    for (int g = threadIdx.x; g < G; g += blockDim.x) up_level_group<T, B, RO>(lev[l], solnext, g, G, g);
    __syncthreads();
  }
  const T *sol1 = L > 1 ? lev[1].sol : nullptr;
  for (int g = threadIdx.x; g < G0; g += blockDim.x) {
    const int row0 = g * SPAN;
    auto out = [&](int i, int r, T val) {
      const int row = row0 + i * B + r;
      if (row < d.n) {
        if (y) y[row] = val;
        else X[row] += (double)val;
      }
    };
    up_group<T, B, kQ0, RO>(lev[0], g, sol1, out, G0, g);
  }
  __syncthreads();
}

__device__ __forceinline__ int oc_corner(int n, int b, int c) { return c < b ? n - b + c : c - b; }

// y = N^{-1} v (y != nullptr) or X += N^{-1} v; N = I without a preconditioner.  Ends with a
// CTA barrier.
template <typename T>
__device__ void oc_precond(const OnChipDesc &d, OcShared &sh, const LevelApply<T> *lev, bool cached, const T *v, T *y,
                           double *X) {
  if (!d.lev) {
    for (int r = threadIdx.x; r < d.n; r += blockDim.x) {
      if (y) y[r] = v[r];
      else X[r] += (double)v[r];
    }
    __syncthreads();
    return;
  }
  T *yb = d.cyclic ? reinterpret_cast<T *>(d.tmp) : y;
  double *Xb = d.cyclic ? nullptr : X;
  // factors read through the read-only path from global memory, or plainly from the
  // shared-memory cache
  switch (d.b * 2 + (cached ? 1 : 0)) {
    case 2: oc_band_solve<T, 1, true>(d, lev, v, yb, Xb); break;
    case 3: oc_band_solve<T, 1, false>(d, lev, v, yb, Xb); break;
    case 4: oc_band_solve<T, 2, true>(d, lev, v, yb, Xb); break;
    case 5: oc_band_solve<T, 2, false>(d, lev, v, yb, Xb); break;
    case 6: oc_band_solve<T, 3, true>(d, lev, v, yb, Xb); break;
    case 7: oc_band_solve<T, 3, false>(d, lev, v, yb, Xb); break;
    case 8: oc_band_solve<T, 4, true>(d, lev, v, yb, Xb); break;
    case 9: oc_band_solve<T, 4, false>(d, lev, v, yb, Xb); break;
    default: break;
  }
  if (!d.cyclic) return;
  // cyclic band: N^{-1} v = yb - Z K^{-1} yb(C)
  const T *Zc = reinterpret_cast<const T *>(d.smwZ);
  const T *Kc = reinterpret_cast<const T *>(d.smwK);
  const int w2 = 2 * d.b;
  if (threadIdx.x < w2) {
    double acc = 0.0;
    for (int c = 0; c < w2; ++c) acc += (double)Kc[threadIdx.x * w2 + c] * (double)yb[oc_corner(d.n, d.b, c)];
    sh.sv[threadIdx.x] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < d.n; r += blockDim.x) {
    T val = yb[r];
    for (int c = 0; c < w2; ++c) val -= Zc[(int64_t)r * w2 + c] * (T)sh.sv[c];
    if (y) y[r] = val;
    else X[r] += (double)val;
  }
  __syncthreads();
}

// out[i] = V(:,i) . w for i < kk (block sums).
template <typename T>
__device__ void oc_project(const T *V, int64_t ld, int kk, const T *w, int n, OcShared &sh, double *out) {
  for (int c0 = 0; c0 < kk; c0 += kOcChunk) {
    const int cnt = min(kOcChunk, kk - c0);
    T acc[kOcChunk];
#pragma unroll
    for (int i = 0; i < kOcChunk; ++i) acc[i] = (T)0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const T wr = w[r];
#pragma unroll
      for (int i = 0; i < kOcChunk; ++i)
        if (i < cnt) acc[i] += V[(int64_t)(c0 + i) * ld + r] * wr;
    }
    oc_reduce<T, kOcChunk>(acc, sh, out + c0, cnt);
  }
}

// w -= sum_{i < kk} c[i] V(:,i) on this thread's rows; returns this thread's part of ||w||^2.
template <typename T>
__device__ __forceinline__ T oc_subtract(const T *V, int64_t ld, int kk, const double *c, T *w, int n) {
  T ss = (T)0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    T acc = w[r];
    for (int i = 0; i < kk; ++i) acc -= (T)c[i] * V[(int64_t)i * ld + r];
    w[r] = acc;
    ss += acc * acc;
  }
  return ss;
}

// The FP64 Givens step of column k (one thread): the old rotations, the new one, G, R(k).
__device__ double oc_givens(OcShared &sh, int k) {
  double *hc = sh.H + (int64_t)k * kOcLdH;
  for (int i = 0; i < k; ++i) {
    const double dv = hc[i];
    hc[i] = dv * sh.C[i] + sh.S[i] * hc[i + 1];
    hc[i + 1] = -dv * sh.S[i] + sh.C[i] * hc[i + 1];
  }
  const double gamma = hypot(hc[k], hc[k + 1]);
  double c = 1.0, s = 0.0;
  if (gamma > 0.0) {
    c = hc[k] / gamma;
    s = hc[k + 1] / gamma;
  }
  hc[k] = gamma;
  hc[k + 1] = 0.0;
  const double dg = sh.G[k];
  sh.G[k] = c * dg;
  sh.G[k + 1] = -s * dg;
  sh.C[k] = c;
  sh.S[k] = s;
  const double R = fabs(sh.G[k + 1]);
  sh.R[k] = R;
  return isfinite(gamma) ? R : NAN;
}

template <typename T>
__device__ void oc_run(const OnChipDesc &d, OcShared &sh) {
  const int tid = threadIdx.x, NT = blockDim.x;
  const int n = d.n;
  T *V = reinterpret_cast<T *>(d.V);
  T *Px = reinterpret_cast<T *>(d.Px);
  T *Py = reinterpret_cast<T *>(d.Py);
  T *Z = reinterpret_cast<T *>(d.Z);
  const int64_t ld = d.ld;
  const int m = d.m, mmax = d.mmax;
  constexpr bool mixed = sizeof(T) == 4;
  DevState *st = d.st;
  unsigned long long t_begin = 0;
  if (tid == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_begin));
  for (int e = tid; e < 3 * (2 * kMaxR + 1); e += NT) {
    const double cv = st->coef[e / (2 * kMaxR + 1)][e % (2 * kMaxR + 1)];
    sh.coef[e / (2 * kMaxR + 1)][e % (2 * kMaxR + 1)] = cv;
    sh.coefF[e / (2 * kMaxR + 1)][e % (2 * kMaxR + 1)] = (float)cv;
  }
  // the slot's factor arrays, optionally copied into dynamic shared memory (one 16-byte
  // chunk per thread and round); the level descriptors then point there
  const LevelApply<T> *lev = reinterpret_cast<const LevelApply<T> *>(d.lev);
  const bool cached = d.lev && d.cache_bytes > 0 && d.nlev <= kOcMaxLevels;
  if (cached) {
    extern __shared__ __align__(16) unsigned char oc_dyn[];
    LevelApply<T> *sl = reinterpret_cast<LevelApply<T> *>(sh.levbuf);
    unsigned char *cur = oc_dyn;
    const int BB = d.b * d.b;
    for (int l = 0; l < d.nlev; ++l) {
      LevelApply<T> L = lev[l];
      const size_t gq = (size_t)L.G * L.q * BB, gs = (size_t)L.G * BB;
      const T **arr[7] = {&L.Mul, &L.Minv, &L.Up, &L.W, &L.Vs, &L.LoSep, &L.UpSepPrev};
      const size_t cnt[7] = {gq, gq, gq, gq, gq, gs, gs};
      for (int a = 0; a < 7; ++a) {
        const size_t n16 = (cnt[a] * sizeof(T) + 15) / 16;
        const uint4 *src = reinterpret_cast<const uint4 *>(*arr[a]);
        uint4 *dst = reinterpret_cast<uint4 *>(cur);
        for (size_t e = tid; e < n16; e += NT) dst[e] = __ldg(src + e);
        *arr[a] = reinterpret_cast<const T *>(cur);
        cur += n16 * 16;
      }
      if (tid == 0) sl[l] = L;
    }
    lev = sl;
  }
  const double tol = st->tol, inner = st->inner_tol;
  int first = st->first;
  double bnorm = st->bnorm, eps_abs = st->eps_abs;
  int hist_count = st->hist_count;
  int cycles = 0, iters = 0, status = 0, k_last = 0, first_k = -1, hb = st->hist_base, any_brk = 0;
  double first_beta = -1.0, last_beta = 0.0, last_R = 0.0;
  __syncthreads();
  for (int cyc = 0; cyc < d.max_cycles; ++cyc) {
    // ---- restart (FP64)
    hb = hist_count;
    {
      T *px = Px + (int64_t)(hb % mmax) * ld, *py = Py + (int64_t)(hb % mmax) * ld;
      double rb[2] = {0.0, 0.0};
      for (int r = tid; r < n; r += NT) {
        const double ax = oc_apply_A<double, double>(d, sh, d.X, r);
        const double b = d.Bv[r];
        const double rv = b - ax;
        px[r] = (T)d.X[r];
        py[r] = (T)ax;
        V[r] = (T)rv;
        rb[0] += rv * rv;
        rb[1] += b * b;
      }
      oc_reduce<double, 2>(rb, sh, sh.scal, 2);
    }
    const double beta = sqrt(sh.scal[0]);
    if (first) {
      bnorm = sqrt(sh.scal[1]);
      eps_abs = tol * bnorm;
      first = 0;
    }
    const double eps_cycle = mixed ? fmax(eps_abs, inner * beta) : eps_abs;
    hist_count = hb + 1;
    cycles += 1;
    if (first_beta < 0.0) first_beta = beta;
    last_beta = beta;
    if (!isfinite(beta)) {
      status = kStNumeric;
      k_last = 0;
      last_R = beta;
      if (first_k < 0) first_k = 0;
      break;
    }
    if (beta == 0.0 || (mixed && beta <= eps_abs)) {
      status = kStConverged;
      k_last = 0;
      last_R = beta;
      if (first_k < 0) first_k = 0;
      break;
    }
    {
      const T inv = (T)(1.0 / beta);
      for (int r = tid; r < n; r += NT) V[r] *= inv;
    }
    if (tid == 0) sh.G[0] = beta;
    __syncthreads();
    // ---- Arnoldi iterations
    int k_end = 0;
    status = 0;
    double R = beta;
    for (int k = 0; k < m; ++k) {
      T *vk = V + (int64_t)k * ld, *vn = V + (int64_t)(k + 1) * ld;
      const int col = (hb + 1 + k) % mmax;
      T *pcol = Px + (int64_t)col * ld, *ycol = Py + (int64_t)col * ld;
      oc_precond<T>(d, sh, lev, cached, vk, pcol, nullptr);
      T w0[1] = {(T)0};
      for (int r = tid; r < n; r += NT) {
        const T w = oc_apply_A<T, T>(d, sh, pcol, r);
        ycol[r] = w;
        vn[r] = w;
        w0[0] += w * w;
      }
      oc_reduce<T, 1>(w0, sh, sh.scal + 2, 1);
      oc_project<T>(V, ld, k + 1, vn, n, sh, sh.h);
      T ss[1];
      ss[0] = oc_subtract<T>(V, ld, k + 1, sh.h, vn, n);
      oc_project<T>(V, ld, k + 1, vn, n, sh, sh.h2);
      ss[0] = oc_subtract<T>(V, ld, k + 1, sh.h2, vn, n);
      oc_reduce<T, 1>(ss, sh, sh.scal + 1, 1);
      if (tid == 0) {
        const double nu2 = sh.scal[1], a2 = sh.scal[2];
        // an overflowed ||U_k|| (a preconditioner whose solve blew up in the Krylov precision)
        // is a numeric failure, not a breakdown: it must not end the cycle as if it converged
        const bool bad = !isfinite(nu2) || !isfinite(a2);
        const bool brk = !bad && !(nu2 > kOcBreakdownRel * kOcBreakdownRel * a2);
        const double nu = (brk || bad) ? 0.0 : sqrt(nu2);
        double *hc = sh.H + (int64_t)k * kOcLdH;
        for (int i = 0; i <= k; ++i) hc[i] = sh.h[i] + sh.h2[i];
        hc[k + 1] = nu;
        const double Rk = oc_givens(sh, k);
        int fl = 0;
        if (!isfinite(Rk) || bad) fl |= kStNumeric;
        if (brk) fl |= kStBreakdown;
        if (!mixed && Rk <= eps_abs) fl |= kStConverged;
        sh.flag[0] = fl;
        sh.flag[1] = (Rk <= eps_cycle) || brk || (fl & kStNumeric) || (k + 1 == m);
        sh.scal[3] = Rk;
        sh.scal[0] = nu > 0.0 ? 1.0 / nu : 0.0;
      }
      __syncthreads();
      R = sh.scal[3];
      status = sh.flag[0];
      k_end = k + 1;
      const bool end = sh.flag[1] != 0;
      if (!end) {
        const T inv = (T)sh.scal[0];
        for (int r = tid; r < n; r += NT) vn[r] *= inv;
      }
      __syncthreads();
      if (end) break;
    }
    iters += k_end;
    // ---- Q = H^{-1} G on the leading k_end x k_end triangle (column-oriented back
    // substitution), Z = V Q, X += N^{-1} Z
    for (int i = tid; i <= k_end; i += NT) sh.t[i] = sh.G[i];
    __syncthreads();
    for (int c = k_end - 1; c >= 0; --c) {
      const double hcc = sh.H[(int64_t)c * kOcLdH + c];
      const double q = hcc != 0.0 ? sh.t[c] / hcc : 0.0;
      __syncthreads();
      for (int i = tid; i < c; i += NT) sh.t[i] -= sh.H[(int64_t)c * kOcLdH + i] * q;
      if (tid == 0) sh.h[c] = q;
      __syncthreads();
    }
    if (!d.lev) {
      for (int r = tid; r < n; r += NT) {
        T z = (T)0;
        for (int j = 0; j < k_end; ++j) z += (T)sh.h[j] * V[(int64_t)j * ld + r];
        d.X[r] += (double)z;
      }
      __syncthreads();
    } else {
      for (int r = tid; r < n; r += NT) {
        T z = (T)0;
        for (int j = 0; j < k_end; ++j) z += (T)sh.h[j] * V[(int64_t)j * ld + r];
        Z[r] = z;
      }
      __syncthreads();
      oc_precond<T>(d, sh, lev, cached, Z, nullptr, d.X);
    }
    hist_count = hb + 1 + k_end;
    if (status & kStBreakdown) any_brk = kStBreakdown;
    last_R = R;
    k_last = k_end;
    if (first_k < 0) first_k = k_end;
    if (status & (kStNumeric | kStConverged)) break;
  }
  // ---- state of the handle and the launch summary
  for (int i = tid; i < k_last; i += NT) st->R[i] = sh.R[i];
  if (tid == 0) {
    st->hist_count = hist_count;
    st->hist_base = hb;
    st->first = first;
    st->bnorm = bnorm;
    st->eps_abs = eps_abs;
    st->k_end = k_last;
    st->status = status;
    st->beta = last_beta;
    st->active = 0;
    st->sum.k_end = k_last;
    st->sum.status = status;
    st->sum.hist_count = hist_count;
    st->sum.error = st->error;
    st->sum.beta = last_beta;
    st->sum.R_end = last_R;
    st->sum.bnorm = bnorm;
    OnChipResult res;
    res.cycles = cycles;
    res.iters = iters;
    res.status = status | any_brk;
    res.k_last = k_last;
    res.first_k = first_k < 0 ? 0 : first_k;
    res.error = st->error;
    res.hist_count = hist_count;
    res.first_beta = first_beta;
    res.last_beta = last_beta;
    res.last_R = last_R;
    res.bnorm = bnorm;
    unsigned long long t_end;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
    res.t_begin = t_begin;
    res.t_end = t_end;
    *d.res = res;
  }
}

template <typename T>
__global__ void __launch_bounds__(kOnChipMaxThreads) k_onchip(const OnChipDesc *__restrict__ descs, int count,
                                                              int *counter) {
  __shared__ OcShared sh;
  __shared__ int s_inst;
  if ((blockDim.x & 31) != 0 || blockDim.x > kOnChipMaxThreads || blockDim.x < 64) {
    // launch self-check: the reductions need whole warps and at most kOcMaxWarps of them
    if (threadIdx.x == 0)
      for (int i = 0; i < count; ++i) atomicExch(&descs[i].st->error, 4);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_inst = atomicAdd(counter, 1);
    __syncthreads();
    const int i = s_inst;
    if (i >= count) return;
    oc_run<T>(descs[i], sh);
    __syncthreads();
  }
}

}  // namespace

bool onchip_threads_ok(int threads) { return threads >= 64 && threads <= kOnChipMaxThreads && threads % 32 == 0; }

template <typename T>
void launch_onchip(const OnChipDesc *descs, int count, int *counter, int threads, int grid, cudaStream_t s,
                   int cache_bytes) {
  if (count <= 0) return;
  static const bool attr = [] {   // opt in to the factor cache's dynamic shared memory (once)
    return cudaFuncSetAttribute(k_onchip<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnChipCacheMax) ==
           cudaSuccess;
  }();
  cudaMemsetAsync(counter, 0, sizeof(int), s);
  k_onchip<T><<<std::max(1, grid), threads, attr ? cache_bytes : 0, s>>>(descs, count, counter);
}

template void launch_onchip<float>(const OnChipDesc *, int, int *, int, int, cudaStream_t, int);
template void launch_onchip<double>(const OnChipDesc *, int, int *, int, int, cudaStream_t, int);

}  // namespace psp
