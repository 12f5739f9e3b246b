// The matrix-free product A x = x - dt L x (Eqs. 1, 2, 4) on a periodic grid, and the
// restart residual of Algorithm 1 (P_x(:,i) = X_0, P_y(:,i) = A X_0, R_bar = B - A X_0,
// V(:,1) = R_bar / ||R_bar||, G(1) = ||R_bar||).
//
// L is a sum over directions d of a 1D stencil of radius R (central differences of the
// configured order, all terms of one direction pre-summed); the coefficients of A for the
// current dt live in DevState::coef, the centre weight of all directions folded into
// coef[0][R].  One thread computes one grid point; neighbour loads go through the
// read-only cache, and the y/z neighbours of a warp's 32 consecutive x points are reused
// from L1/L2 by the warps of the neighbouring rows.
#include <algorithm>
#include <type_traits>

#include "dfloat.cuh"
#include "psp_kernels.cuh"

namespace psp {

template <typename TI, int NDIM, int R, typename TC>
__device__ __forceinline__ TC stencil_point(const TI *__restrict__ x, const TC (*c)[2 * R + 1], int ix,
                                            int iy, int iz, int nx, int ny, int nz) {
  const int64_t plane = (int64_t)nx * ny;
  const int64_t base = (int64_t)iz * plane + (int64_t)iy * nx;
  TC acc = c[0][R] * (TC)__ldg(x + base + ix);
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    int xm = ix - j; xm += (xm < 0) ? nx : 0;
    int xp = ix + j; xp -= (xp >= nx) ? nx : 0;
    acc = fma(c[0][R - j], (TC)__ldg(x + base + xm), acc);
    acc = fma(c[0][R + j], (TC)__ldg(x + base + xp), acc);
  }
  if (NDIM >= 2) {
    const int64_t rowx = (int64_t)iz * plane + ix;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      int ym = iy - j; ym += (ym < 0) ? ny : 0;
      int yp = iy + j; yp -= (yp >= ny) ? ny : 0;
      acc = fma(c[1][R - j], (TC)__ldg(x + rowx + (int64_t)ym * nx), acc);
      acc = fma(c[1][R + j], (TC)__ldg(x + rowx + (int64_t)yp * nx), acc);
    }
  }
  if (NDIM >= 3) {
    const int64_t colx = (int64_t)iy * nx + ix;
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      int zm = iz - j; zm += (zm < 0) ? nz : 0;
      int zp = iz + j; zp -= (zp >= nz) ? nz : 0;
      acc = fma(c[2][R - j], (TC)__ldg(x + colx + (int64_t)zm * plane), acc);
      acc = fma(c[2][R + j], (TC)__ldg(x + colx + (int64_t)zp * plane), acc);
    }
  }
  return acc;
}

template <typename TC, int R>
__device__ __forceinline__ void load_coef(const DevState *st, TC (*c)[2 * R + 1]) {
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int j = -R; j <= R; ++j) c[d][R + j] = (TC)st->coef[d][kMaxR + j];
}

// y = A (s x) with s = *scale (1 if scale is null).  If xcopy is set, it receives s x (the
// N = I preconditioner output Y_k = V(:,k), written together with U_k = A Y_k).  TC is
// the arithmetic type (float in the mixed form, double otherwise).  Grids have fewer than
// 2^31 points, so the index arithmetic is 32-bit.
template <typename TI, typename TO, typename TC, int NDIM, int R>
__global__ void __launch_bounds__(kThreads) k_stencil(InRef<TI> xref, OutRef<TO> yref, OutRef<TO> xcopy,
                                                      const double *scale, const DevState *__restrict__ st,
                                                      int nx, int ny, int nz, const int *active) {
  if (active && *active == 0) return;
  TC c[3][2 * R + 1];
  load_coef<TC, R>(st, c);
  const TI *__restrict__ x = xref.get();
  TO *y = yref.get();
  TO *xc = xcopy.base ? xcopy.get() : nullptr;
  const TC sc = scale ? (TC)(*scale) : (TC)1;
  const int n = nx * ny * nz;
  const int plane = nx * ny;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int iz = i / plane;
    const int rem = i - iz * plane;
    const int iy = rem / nx;
    const int ix = rem - iy * nx;
    const TC v = stencil_point<TI, NDIM, R, TC>(x, c, ix, iy, iz, nx, ny, nz);
    y[i] = (TO)(sc * v);
    if (xc) xc[i] = (TO)(sc * (TC)x[i]);
  }
}

// Vectorised y = A (s x): each thread computes VW consecutive x points from aligned
// vector loads (a register window of the row for the x terms, one vector per y/z
// neighbour row), coefficients staged once per CTA in shared memory.  Needs nx % VW == 0.
template <typename T> struct SVec;
template <> struct SVec<float> { using type = float4; static constexpr int W = 4; };
template <> struct SVec<double> { using type = double2; static constexpr int W = 2; };

template <typename T, int W>
__device__ __forceinline__ void vload(const T *p, T (&o)[W]) {
  using VT = typename SVec<T>::type;
  const VT v = __ldg(reinterpret_cast<const VT *>(p));
  const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
  for (int i = 0; i < W; ++i) o[i] = e[i];
}

template <typename T, int NDIM, int R>
__global__ void __launch_bounds__(kThreads) k_stencil_vec(InRef<T> xref, OutRef<T> yref, OutRef<T> xcopy,
                                                          const double *scale, const DevState *__restrict__ st,
                                                          int nx, int ny, int nz, const int *active) {
  constexpr int W = SVec<T>::W;
  constexpr int NH = (R + W - 1) / W;          // halo vectors on each side along x
  if (active && *active == 0) return;
  __shared__ T s_c[3][2 * R + 1];
  if (threadIdx.x < 3 * (2 * R + 1)) {
    const int d = threadIdx.x / (2 * R + 1), j = threadIdx.x % (2 * R + 1);
    s_c[d][j] = (T)st->coef[d][kMaxR - R + j];
  }
  __syncthreads();
  T c[3][2 * R + 1];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int j = 0; j < 2 * R + 1; ++j) c[d][j] = s_c[d][j];
  const T *__restrict__ x = xref.get();
  T *y = yref.get();
  T *xc = xcopy.base ? xcopy.get() : nullptr;
  const T sc = scale ? (T)(*scale) : (T)1;
  const int nxv = nx / W;
  const int nvec = nxv * ny * nz;
  const int plane = nx * ny;
  for (int iv = blockIdx.x * blockDim.x + threadIdx.x; iv < nvec; iv += gridDim.x * blockDim.x) {
    const int row = iv / nxv;               // row index iy + ny*iz
    const int xv = iv - row * nxv;
    const int iz = row / ny;
    const int iy = row - iz * ny;
    const int base = row * nx;
    // x window: vectors xv-NH .. xv+NH (periodic)
    T win[(2 * NH + 1) * W];
#pragma unroll
    for (int h = -NH; h <= NH; ++h) {
      int v = xv + h;
      v += (v < 0) ? nxv : 0;
      v -= (v >= nxv) ? nxv : 0;
      T t[W];
      vload<T, W>(x + base + v * W, t);
#pragma unroll
      for (int i = 0; i < W; ++i) win[(h + NH) * W + i] = t[i];
    }
    T acc[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      T a = c[0][R] * win[NH * W + i];
#pragma unroll
      for (int j = 1; j <= R; ++j) a = fma(c[0][R + j], win[NH * W + i + j], fma(c[0][R - j], win[NH * W + i - j], a));
      acc[i] = a;
    }
    if (NDIM >= 2) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        int ym = iy - j; ym += (ym < 0) ? ny : 0;
        int yp = iy + j; yp -= (yp >= ny) ? ny : 0;
        T tm[W], tp[W];
        vload<T, W>(x + iz * plane + ym * nx + xv * W, tm);
        vload<T, W>(x + iz * plane + yp * nx + xv * W, tp);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = fma(c[1][R + j], tp[i], fma(c[1][R - j], tm[i], acc[i]));
      }
    }
    if (NDIM >= 3) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        int zm = iz - j; zm += (zm < 0) ? nz : 0;
        int zp = iz + j; zp -= (zp >= nz) ? nz : 0;
        T tm[W], tp[W];
        vload<T, W>(x + zm * plane + iy * nx + xv * W, tm);
        vload<T, W>(x + zp * plane + iy * nx + xv * W, tp);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = fma(c[2][R + j], tp[i], fma(c[2][R - j], tm[i], acc[i]));
      }
    }
    using VT = typename SVec<T>::type;
    VT out;
    T *oe = reinterpret_cast<T *>(&out);
#pragma unroll
    for (int i = 0; i < W; ++i) oe[i] = sc * acc[i];
    reinterpret_cast<VT *>(y + base)[xv] = out;
    if (xc) {
#pragma unroll
      for (int i = 0; i < W; ++i) oe[i] = sc * win[NH * W + i];
      reinterpret_cast<VT *>(xc + base)[xv] = out;
    }
  }
}

// The end of a restart: per-CTA sums of ||r||^2 and ||B||^2 (rr, bb of each thread) to
// partial, and the last CTA to arrive adds them in a fixed order and sets the cycle's state
// (beta = ||r||, G(1), the lazy normalisation of V~(:,1), the step bound on the first cycle,
// the active flag, the history columns) and the cycle summary.
__device__ __forceinline__ void restart_finish(double rr, double bb, DevState *st, double *partial, int col,
                                               int mixed) {
  __shared__ double s_rr[kThreads / 32], s_bb[kThreads / 32];
  rr = warp_sum(rr);
  bb = warp_sum(bb);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s_rr[wid] = rr; s_bb[wid] = bb; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += s_rr[w]; b2 += s_bb[w]; }
    partial[blockIdx.x] = a;
    partial[kMaxCta + blockIdx.x] = b2;
  }
  if (!last_block_arrive(&st->counter[0])) return;
  __shared__ double s_tot[2];
  if (wid < 2) {  // warp 0: ||r||^2, warp 1: ||B||^2, fixed order over CTAs
    double a = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) a += partial[wid * kMaxCta + b];
    a = warp_sum(a);
    if (lane == 0) s_tot[wid] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double a = s_tot[0], b2 = s_tot[1];
    const double beta = sqrt(a);
    if (st->first) {
      st->bnorm = sqrt(b2);
      st->eps_abs = st->tol * st->bnorm;
      st->first = 0;
    }
    st->beta = beta;
    st->G[0] = beta;
    st->sigma[0] = beta > 0.0 ? 1.0 / beta : 0.0;
    st->eps_cycle = mixed ? fmax(st->eps_abs, st->inner_tol * beta) : st->eps_abs;
    st->k_end = 0;
    st->status = 0;
    st->hist_base = col;
    st->hist_count = col + 1;
    if (!isfinite(beta)) {
      st->status = kStNumeric;
      st->active = 0;
    } else if (beta == 0.0 || (mixed && beta <= st->eps_abs)) {
      st->status = kStConverged;
      st->active = 0;
    } else {
      st->active = 1;
    }
    st->sum.beta = beta;
    st->sum.error = st->error;
    st->sum.bnorm = st->bnorm;
    st->sum.k_end = 0;
    st->sum.status = st->status;
    st->sum.hist_count = st->hist_count;
    st->sum.R_end = beta;
    last_block_reset(&st->counter[0]);
  }
}

// Restart of Algorithm 1 in FP64: AX = A X_0, r = B - AX; store the history pair
// (X_0, AX) in the ring column hist_count, V~(:,1) = r (normalised lazily through
// sigma[0] = 1/||r||), G(1) = ||r||; ||B|| sets the step bound eps_abs = tol ||B||.
// NDIM == 0: the explicit banded operator (Ab, half-width bw) instead of the stencil.
template <typename TH, typename TV, int NDIM, int R>
__global__ void __launch_bounds__(kThreads) k_restart(const double *__restrict__ X,
                                                      const double *__restrict__ B, TH *Px, TH *Py,
                                                      int64_t ldh, TV *V1, DevState *st, double *partial,
                                                      int nx, int ny, int nz, int mixed,
                                                      const double *__restrict__ Ab, int bw, const int *skip) {
  if (skip && *skip) return;   // the double-float restart of the same cycle runs instead
  double c[3][2 * R + 1];
  if (NDIM > 0) load_coef<double, R>(st, c);
  const int col = st->hist_count;
  TH *px = ring_col(Px, ldh, col, st->mmax);
  TH *py = ring_col(Py, ldh, col, st->mmax);
  const int n = nx * ny * nz;
  const int plane = nx * ny;
  double rr = 0.0, bb = 0.0;
  auto point = [&](int i) {
    const int iz = i / plane;
    const int rem = i - iz * plane;
    const int iy = rem / nx;
    const int ix = rem - iy * nx;
    double ax;
    if constexpr (NDIM == 0) {
      ax = 0.0;
      for (int p = 0; p <= 2 * bw; ++p) {
        const int j = i + p - bw;
        if (j >= 0 && j < n) ax += Ab[(int64_t)i * (2 * bw + 1) + p] * X[j];
      }
    } else {
      ax = stencil_point<double, NDIM, R, double>(X, c, ix, iy, iz, nx, ny, nz);
    }
    const double b = B[i];
    const double r = b - ax;
    px[i] = (TH)X[i];
    py[i] = (TH)ax;
    V1[i] = (TV)r;
    rr += r * r;
    bb += b * b;
  };
  // two points per round, independent: their loads and FP64 chains overlap
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += 2 * stride) {
    point(i);
    if (i + stride < n) point(i + stride);
  }
  restart_finish(rr, bb, st, partial, col, mixed);
}

// The mixed form's restart with its FP64-grade arithmetic on the FP32 pipe.  k_split_x
// writes X_0 as the double-float pair (X_hi, X_lo) (split_double, one pass, integer
// operations); k_restart_df then computes A X_0 and r = B - A X_0 in double-float: every
// term c x of the stencil is an error-free product of the pairs (c_hi + c_lo)(x_hi + x_lo)
// (the c_lo x_lo term, 2^-48 relative, dropped) added by two-sum, the low parts summed in
// FP32 and folded back into the high part after each direction.  The roundings leave r
// with an error of a few 2^-48 sum_t |c_t x_t| per point, about 2^-45 sum_t |c_t| |x|
// (against 2^-53 for FP64): the host sets DevState::restart_df only for tol >= 2^-42
// sum_t |c_t|, else the FP64 restart runs.  Each thread computes four consecutive x points
// (16-byte loads of X_hi and X_lo, a register window along x), two at a time in packed
// FP32x2 registers.  The squares of r and B are summed in FP32 per four points and in FP64
// across them.  Needs nx % 4 == 0, more than (R + 3) / 4 vectors per row and 16-byte
// aligned columns.
__global__ void __launch_bounds__(kThreads) k_split_x(const double *__restrict__ X, float *__restrict__ Xh,
                                                     float *__restrict__ Xl, int nvec, const DevState *st) {
  if (!st->restart_df) return;
  for (int iv = blockIdx.x * blockDim.x + threadIdx.x; iv < nvec; iv += gridDim.x * blockDim.x) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(X) + 2 * iv);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(X) + 2 * iv + 1);
    float4 h, l;
    split_double(a.x, h.x, l.x);
    split_double(a.y, h.y, l.y);
    split_double(b.x, h.z, l.z);
    split_double(b.y, h.w, l.w);
    reinterpret_cast<float4 *>(Xh)[iv] = h;
    reinterpret_cast<float4 *>(Xl)[iv] = l;
  }
}

// (sh, sl) += (ch + cl)(xh + xl) for two lanes; nch = -ch, ncl = -cl (both lanes).
// -e = fma(-ch, xh, p) is exact (p = fl(ch xh)); the cross terms join it, and the two-sum of
// sh and p sends its rounding error to sl.
__device__ __forceinline__ void df2_fma(uint64_t &sh, uint64_t &sl, uint64_t ch, uint64_t nch, uint64_t ncl,
                                        uint64_t xh, uint64_t xl) {
  const uint64_t p = f2mul(ch, xh);
  uint64_t ne = f2fma(nch, xh, p);
  ne = f2fma(nch, xl, ne);
  ne = f2fma(ncl, xh, ne);
  const uint64_t s = f2add(sh, p);
  const uint64_t bb = f2sub(s, sh);
  const uint64_t err = f2add(f2sub(sh, f2sub(s, bb)), f2sub(p, bb));
  sh = s;
  sl = f2add(sl, f2sub(err, ne));
}

// (sh, sl) <- fast two-sum of sh and sl (|sl| < |sh| but for cancellation): bounds sl again
// by half an FP32 ulp of sh, so that its own rounding stays at that scale.
__device__ __forceinline__ void df2_renorm(uint64_t &sh, uint64_t &sl) {
  const uint64_t s = f2add(sh, sl);
  sl = f2sub(sl, f2sub(s, sh));
  sh = s;
}

// Lanes f, f+1 of a window held as packed pairs (pair q = lanes 2q, 2q+1).
__device__ __forceinline__ uint64_t df2_lanes(const uint64_t *w, int f) {
  if ((f & 1) == 0) return w[f >> 1];
  float a, b, c, d;
  f2unpack(w[f >> 1], a, b);
  f2unpack(w[(f >> 1) + 1], c, d);
  return f2pack(b, c);
}

template <int NDIM, int R>
__global__ void __launch_bounds__(kThreads) k_restart_df(const float *__restrict__ Xh, const float *__restrict__ Xl,
                                                         const double *__restrict__ B, float *Px, float *Py,
                                                         int64_t ldh, float *V1, DevState *st, double *partial,
                                                         int nx, int ny, int nz) {
  if (!st->restart_df) return;                // the FP64 restart of the same cycle runs instead
  constexpr int NH = (R + 3) / 4;             // halo vectors on each side along x
  constexpr int NW = 2 * (2 * NH + 1);        // packed pairs of the x window
  constexpr int NC = 3 * (2 * R + 1);
  __shared__ uint64_t s_c[3][NC];             // (c_hi, c_hi), (-c_hi, -c_hi), (-c_lo, -c_lo)
  if (threadIdx.x < NC) {
    const int d = threadIdx.x / (2 * R + 1), j = threadIdx.x % (2 * R + 1);
    float ch, cl;
    split_double(st->coef[d][kMaxR - R + j], ch, cl);
    s_c[0][threadIdx.x] = f2pack(ch, ch);
    s_c[1][threadIdx.x] = f2pack(-ch, -ch);
    s_c[2][threadIdx.x] = f2pack(-cl, -cl);
  }
  const int col = st->hist_count;
  float *px = ring_col(Px, ldh, col, st->mmax);
  float *py = ring_col(Py, ldh, col, st->mmax);
  __syncthreads();
  const int nxv = nx / 4;
  const int nvec = nxv * ny * nz;
  const int plane = nx * ny;
  double rr = 0.0, bb = 0.0;
  auto term = [&](uint64_t (&sh)[2], uint64_t (&sl)[2], int d, int j, const ulonglong2 &h, const ulonglong2 &l) {
    const int k = d * (2 * R + 1) + R + j;
    const uint64_t ch = s_c[0][k], nch = s_c[1][k], ncl = s_c[2][k];
    df2_fma(sh[0], sl[0], ch, nch, ncl, h.x, l.x);
    df2_fma(sh[1], sl[1], ch, nch, ncl, h.y, l.y);
  };
  for (int iv = blockIdx.x * blockDim.x + threadIdx.x; iv < nvec; iv += gridDim.x * blockDim.x) {
    const int row = iv / nxv;                 // iy + ny iz
    const int xv = iv - row * nxv;
    const int iz = row / ny;
    const int iy = row - iz * ny;
    const int base = row * nx;
    uint64_t wh[NW], wl[NW];
#pragma unroll
    for (int q = -NH; q <= NH; ++q) {
      int v = xv + q;
      v += (v < 0) ? nxv : 0;
      v -= (v >= nxv) ? nxv : 0;
      const ulonglong2 h = __ldg(reinterpret_cast<const ulonglong2 *>(Xh + base) + v);
      const ulonglong2 l = __ldg(reinterpret_cast<const ulonglong2 *>(Xl + base) + v);
      wh[2 * (q + NH)] = h.x;
      wh[2 * (q + NH) + 1] = h.y;
      wl[2 * (q + NH)] = l.x;
      wl[2 * (q + NH) + 1] = l.y;
    }
    uint64_t sh[2], sl[2];
    {  // the centre term starts the sums: sh = fl(c x_hi), sl = its exact error and cross terms
      const int k = R;
      const uint64_t ch = s_c[0][k], nch = s_c[1][k], ncl = s_c[2][k];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint64_t xh = wh[2 * NH + q], xl = wl[2 * NH + q];
        const uint64_t p = f2mul(ch, xh);
        uint64_t ne = f2fma(nch, xh, p);
        ne = f2fma(nch, xl, ne);
        ne = f2fma(ncl, xh, ne);
        sh[q] = p;
        sl[q] = f2sub(0ull, ne);
      }
    }
#pragma unroll
    for (int j = 1; j <= R; ++j) {
#pragma unroll
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const int k = R + sgn * j;
        const uint64_t ch = s_c[0][k], nch = s_c[1][k], ncl = s_c[2][k];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int f = 4 * NH + 2 * q + sgn * j;   // window lane of point 2q shifted by sgn j
          df2_fma(sh[q], sl[q], ch, nch, ncl, df2_lanes(wh, f), df2_lanes(wl, f));
        }
      }
    }
    df2_renorm(sh[0], sl[0]);
    df2_renorm(sh[1], sl[1]);
    if (NDIM >= 2) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        int ym = iy - j; ym += (ym < 0) ? ny : 0;
        int yp = iy + j; yp -= (yp >= ny) ? ny : 0;
        const int om = iz * plane + ym * nx + 4 * xv, op = iz * plane + yp * nx + 4 * xv;
        term(sh, sl, 1, -j, __ldg(reinterpret_cast<const ulonglong2 *>(Xh + om)),
             __ldg(reinterpret_cast<const ulonglong2 *>(Xl + om)));
        term(sh, sl, 1, j, __ldg(reinterpret_cast<const ulonglong2 *>(Xh + op)),
             __ldg(reinterpret_cast<const ulonglong2 *>(Xl + op)));
      }
      df2_renorm(sh[0], sl[0]);
      df2_renorm(sh[1], sl[1]);
    }
    if (NDIM >= 3) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        int zm = iz - j; zm += (zm < 0) ? nz : 0;
        int zp = iz + j; zp -= (zp >= nz) ? nz : 0;
        const int om = zm * plane + iy * nx + 4 * xv, op = zp * plane + iy * nx + 4 * xv;
        term(sh, sl, 2, -j, __ldg(reinterpret_cast<const ulonglong2 *>(Xh + om)),
             __ldg(reinterpret_cast<const ulonglong2 *>(Xl + om)));
        term(sh, sl, 2, j, __ldg(reinterpret_cast<const ulonglong2 *>(Xh + op)),
             __ldg(reinterpret_cast<const ulonglong2 *>(Xl + op)));
      }
      df2_renorm(sh[0], sl[0]);
      df2_renorm(sh[1], sl[1]);
    }
    // r = B - A X_0 by the two-sum of B_hi and -(A X_0)_hi, the low parts added after it
    const int i0 = base + 4 * xv;
    const double2 b01 = __ldg(reinterpret_cast<const double2 *>(B + i0));
    const double2 b23 = __ldg(reinterpret_cast<const double2 *>(B + i0 + 2));
    float bh[4], bl[4];
    split_double(b01.x, bh[0], bl[0]);
    split_double(b01.y, bh[1], bl[1]);
    split_double(b23.x, bh[2], bl[2]);
    split_double(b23.y, bh[3], bl[3]);
    ulonglong2 rv, ax, xc;
    uint64_t *rp = reinterpret_cast<uint64_t *>(&rv);
    uint64_t *ap = reinterpret_cast<uint64_t *>(&ax);
    uint64_t *xp = reinterpret_cast<uint64_t *>(&xc);
    float r2 = 0.0f, b2 = 0.0f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint64_t Bh = f2pack(bh[2 * q], bh[2 * q + 1]), Bl = f2pack(bl[2 * q], bl[2 * q + 1]);
      const uint64_t t = f2sub(Bh, sh[q]);
      const uint64_t v = f2sub(t, Bh);
      const uint64_t err = f2sub(f2sub(Bh, f2sub(t, v)), f2add(sh[q], v));
      const uint64_t r = f2add(t, f2add(err, f2sub(Bl, sl[q])));
      rp[q] = r;
      ap[q] = f2add(sh[q], sl[q]);
      xp[q] = wh[2 * NH + q];
      float r0, r1;
      f2unpack(r, r0, r1);
      r2 = fmaf(r0, r0, fmaf(r1, r1, r2));
      b2 = fmaf(bh[2 * q], bh[2 * q], fmaf(bh[2 * q + 1], bh[2 * q + 1], b2));
    }
    reinterpret_cast<ulonglong2 *>(V1 + i0)[0] = rv;
    reinterpret_cast<ulonglong2 *>(py + i0)[0] = ax;
    reinterpret_cast<ulonglong2 *>(px + i0)[0] = xc;
    rr += (double)r2;
    bb += (double)b2;
  }
  restart_finish(rr, bb, st, partial, col, 1);
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

// z = a x + b y (FP64, elementwise; z may alias x or y): the right-hand sides of the
// integrators built on the step.
__global__ void __launch_bounds__(kThreads) k_axpby(int64_t n, double a, const double *x, double b, const double *y,
                                                   double *z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = a * x[i] + b * y[i];
}

void launch_axpby(int64_t n, double a, const double *x, double b, const double *y, double *z, cudaStream_t s) {
  const int64_t g = std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_axpby<<<(unsigned)std::max<int64_t>(g, 1), kThreads, 0, s>>>(n, a, x, b, y, z);
}

// d_t = lambda . (D_t u) for every term t of the operator (unit coefficient, h^-k folded in):
// each term is a 1D stencil along its direction, applied at every point of the periodic grid
// and weighted by lambda there.  Per-CTA sums go to partial[t][cta]; the last CTA to arrive
// adds them in a fixed order (deterministic), so the gradients of an adjoint step need one
// launch and no vector of their own.
__global__ void __launch_bounds__(kThreads) k_term_dots(const double *__restrict__ lam, const double *__restrict__ u,
                                                       int nx, int ny, int nz, TermStencils ts, double *partial,
                                                       unsigned int *counter, double *out) {
  const int n = nx * ny * nz, plane = nx * ny;
  const int R = ts.R;
  double acc[kMaxTerms];
#pragma unroll
  for (int t = 0; t < kMaxTerms; ++t) acc[t] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int iz = i / plane;
    const int rem = i - iz * plane;
    const int iy = rem / nx;
    const int ix = rem - iy * nx;
    const double li = lam[i];
#pragma unroll
    for (int t = 0; t < kMaxTerms; ++t) {
      if (t >= ts.nt) break;
      const int d = ts.dir[t];
      const int c = d == 0 ? ix : (d == 1 ? iy : iz);
      const int len = d == 0 ? nx : (d == 1 ? ny : nz);
      const int stride = d == 0 ? 1 : (d == 1 ? nx : plane);
      const int base = i - c * stride;
      double sum = 0.0;
      for (int j = -R; j <= R; ++j) {
        const double wj = ts.w[t][kMaxR + j];
        if (wj == 0.0) continue;
        int q = c + j;
        q += (q < 0) ? len : 0;
        q -= (q >= len) ? len : 0;
        sum += wj * u[base + q * stride];
      }
      acc[t] += li * sum;
    }
  }
  __shared__ double s_w[kThreads / 32][kMaxTerms];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kMaxTerms; ++t) {
    const double v = warp_sum(acc[t]);
    if (lane == 0) s_w[wid][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < ts.nt) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_w[w][threadIdx.x];
    partial[(int64_t)threadIdx.x * kMaxCta + blockIdx.x] = v;
  }
  if (!last_block_arrive(counter)) return;
  if (threadIdx.x < ts.nt) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += partial[(int64_t)threadIdx.x * kMaxCta + b];
    out[threadIdx.x] = v;
  }
  last_block_reset(counter);
}

void launch_term_dots(const Geometry &g, const double *lam, const double *u, const TermStencils &ts, double *partial,
                      unsigned int *counter, double *out, cudaStream_t s) {
  k_term_dots<<<reduce_grid(g.n), kThreads, 0, s>>>(lam, u, g.nx, g.ny, g.nz, ts, partial, counter, out);
}

int reduce_grid(int64_t n) {
  int64_t g = (n + kThreads * 4 - 1) / (kThreads * 4);
  if (g < 1) g = 1;
  if (g > kMaxCta) g = kMaxCta;
  return (int)g;
}

static int stencil_grid(int64_t n) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

#define PSP_DISPATCH_R(R_, ...)                   \
  switch (R_) {                                   \
    case 1: { constexpr int RR = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int RR = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int RR = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int RR = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int RR = 5; __VA_ARGS__; } break; \
    default: break;                               \
  }

#define PSP_DISPATCH_NDIM(D_, ...)                \
  switch (D_) {                                   \
    case 1: { constexpr int DD = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int DD = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int DD = 3; __VA_ARGS__; } break; \
    default: break;                               \
  }

// 3D vectorised stencil with z-marching (2.5D blocking): a CTA owns a tile of kTileXV
// x-vectors by kTileY rows and walks a range of planes.  Each thread keeps the planes
// z-R .. z+R of its own vector in a register queue (the z terms); the plane loop is unrolled
// by the queue length, so the queue index of every plane is a compile-time constant and
// nothing is moved between planes.  The loads run kAhead3 planes ahead through shared memory,
// not registers: per plane one group of 16-byte asynchronous copies (cp.async) brings the
// thread's own vector of plane z+R+kAhead3 into its slot of an own-vector ring, and the
// tile's halo of plane z+kAhead3 (an x halo of whole vectors and a y halo of R rows on each
// side; no corners, the stencil is a cross; every thread takes the same one or two halo
// positions on every plane) into a ring of plane slots.  At plane z the thread waits for its
// group of plane z, moves its vector of plane z+R into the queue, writes its vector of plane
// z into the plane slot, and one barrier makes the slot whole.  A point is read from HBM
// about once; the halos come from L2.  Needs nx / W and ny to be multiples of the tile (the
// periodic wrap is then tile-exact).
constexpr int kTileXV = 32;
constexpr int kTileY = 8;
constexpr int kAhead3 = 4;   // planes of look-ahead of the asynchronous copies

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T, int R>
__host__ __device__ constexpr int tile3d_slot_vecs() {
  return (kTileY + 2 * R) * (kTileXV + 2 * ((R + SVec<T>::W - 1) / SVec<T>::W));
}
// Dynamic shared memory of k_stencil_3d: kAhead3 + 1 plane slots and as many own-vector slots.
template <typename T, int R>
__host__ __device__ constexpr int tile3d_smem_bytes() {
  return (kAhead3 + 1) * (tile3d_slot_vecs<T, R>() + kTileXV * kTileY) * 16;
}

// Coefficients of the three directions: in registers for FP32 (the kernel is then bound by
// memory and instruction issue), read from shared memory for FP64 (bound by the FP64 pipe).
template <typename T, int R, bool REG>
struct Coef3;
template <typename T, int R>
struct Coef3<T, R, true> {
  T c[3][2 * R + 1];
  __device__ __forceinline__ void load(const T (*s)[2 * R + 1]) {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int j = 0; j < 2 * R + 1; ++j) c[d][j] = s[d][j];
  }
  __device__ __forceinline__ T operator()(int d, int j) const { return c[d][j]; }
};
template <typename T, int R>
struct Coef3<T, R, false> {
  const T (*c)[2 * R + 1];
  __device__ __forceinline__ void load(const T (*s)[2 * R + 1]) { c = s; }
  __device__ __forceinline__ T operator()(int d, int j) const { return c[d][j]; }
};

template <typename T, int R>
__global__ void __launch_bounds__(kTileXV * kTileY, 2) k_stencil_3d(InRef<T> xref, OutRef<T> yref, OutRef<T> xcopy,
                                                                   const double *scale, const DevState *__restrict__ st,
                                                                   int nx, int ny, int nz, int tz, const int *active) {
  using VT = typename SVec<T>::type;
  constexpr int W = SVec<T>::W;
  constexpr int NH = (R + W - 1) / W;
  constexpr int SX = kTileXV + 2 * NH;
  constexpr int SLOT = tile3d_slot_vecs<T, R>();
  constexpr int NS = kAhead3 + 1;                     // ring slots (planes z .. z+kAhead3)
  constexpr int QL = 2 * R + 1;                       // queue length: planes z-R .. z+R
  constexpr int NHALO = 2 * R * kTileXV + 2 * NH * kTileY;
  constexpr int NT = kTileXV * kTileY;
  if (active && *active == 0) return;
  extern __shared__ __align__(16) unsigned char smem3[];
  VT *ring = reinterpret_cast<VT *>(smem3);           // [NS][SLOT] plane slots
  VT *own_ring = ring + NS * SLOT;                    // [NS][NT] own vectors
  __shared__ T s_c[3][2 * R + 1];
  if (threadIdx.x < 3 * (2 * R + 1)) {
    const int d = threadIdx.x / (2 * R + 1), j = threadIdx.x % (2 * R + 1);
    s_c[d][j] = (T)st->coef[d][kMaxR - R + j];
  }
  const T *__restrict__ x = xref.get();
  T *y = yref.get();
  T *xc = xcopy.base ? xcopy.get() : nullptr;
  const T sc = scale ? (T)(*scale) : (T)1;
  const int nxv = nx / W;
  const int64_t plane = (int64_t)nx * ny;
  const int tx = threadIdx.x % kTileXV, ty = threadIdx.x / kTileXV;
  const int xv0 = blockIdx.x * kTileXV, y0 = blockIdx.y * kTileY;
  const int64_t own = (int64_t)(y0 + ty) * nx + (int64_t)(xv0 + tx) * W;   // offset inside a plane
  const int z0 = blockIdx.z * tz;
  const int z1 = min(z0 + tz, nz);
  auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
  auto ldv = [&](int z) { return __ldg(reinterpret_cast<const VT *>(x + (int64_t)wrapz(z) * plane + own)); };
  // this thread's halo positions (the same on every plane): e = threadIdx.x and e + NT of
  // the list [y halo rows (2R x kTileXV), x halo vectors of the tile rows (kTileY x 2NH)]
  int h_s[2];
  int64_t h_g[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int e = threadIdx.x + k * NT;
    h_s[k] = -1;
    h_g[k] = 0;
    if (e < 2 * R * kTileXV) {
      const int hr = e / kTileXV, hx = e % kTileXV;
      int row = (hr < R) ? y0 - R + hr : y0 + kTileY + (hr - R);
      row += (row < 0) ? ny : 0;
      row -= (row >= ny) ? ny : 0;
      h_s[k] = ((hr < R) ? hr : kTileY + hr) * SX + hx + NH;
      h_g[k] = (int64_t)row * nx + (int64_t)(xv0 + hx) * W;
    } else if (e < NHALO) {
      const int f = e - 2 * R * kTileXV;
      const int r = f / (2 * NH), c = f % (2 * NH);
      int v = (c < NH) ? xv0 - NH + c : xv0 + kTileXV + (c - NH);
      v += (v < 0) ? nxv : 0;
      v -= (v >= nxv) ? nxv : 0;
      h_s[k] = (r + R) * SX + ((c < NH) ? c : kTileXV + c);
      h_g[k] = (int64_t)(y0 + r) * nx + (int64_t)v * W;
    }
  }
  // the copy group of plane z (z0 <= z < z1): the halo of plane z into plane slot z % NS and
  // this thread's vector of plane z + R into own slot (z + R) % NS
  auto issue = [&](int z) {
    if (z < z1) {
      const T *pz = x + (int64_t)wrapz(z) * plane;
      VT *slot = ring + ((z - z0) % NS) * SLOT;
#pragma unroll
      for (int k = 0; k < 2; ++k)
        if (h_s[k] >= 0) cp_async16(slot + h_s[k], pz + h_g[k]);
      cp_async16(own_ring + ((z - z0) % NS) * NT + threadIdx.x, x + (int64_t)wrapz(z + R) * plane + own);
    }
    cp_async_commit();   // one group per plane, empty past the end (the wait counts stay exact)
  };
  // queue: plane z0 - R + i in q[i] for i < 2R; groups of planes z0 .. z0 + kAhead3 - 1
  VT q[QL];
#pragma unroll
  for (int i = 0; i < 2 * R; ++i) q[i] = ldv(z0 - R + i);
#pragma unroll
  for (int k = 0; k < kAhead3; ++k) issue(z0 + k);
  __syncthreads();   // s_c
  Coef3<T, R, sizeof(T) == 4> c;
  c.load(s_c);
  for (int zb = z0; zb < z1; zb += QL) {
#pragma unroll
    for (int u = 0; u < QL; ++u) {
      const int z = zb + u;
      if (z >= z1) break;
      // plane z + k sits in q[(u + k + R) % QL]; plane z + R arrives through the own ring
      // into the entry of plane z - R - 1, which the previous plane used last
      cp_async_wait<kAhead3 - 1>();   // this thread's group of plane z has landed
      q[(u + 2 * R) % QL] = own_ring[((z - z0) % NS) * NT + threadIdx.x];
      VT *slot = ring + ((z - z0) % NS) * SLOT;
      slot[(ty + R) * SX + tx + NH] = q[(u + R) % QL];
      __syncthreads();      // every thread's halo copies and centre vectors of plane z
      issue(z + kAhead3);   // into the slots of plane z - 1, which every thread has finished
      T win[(2 * NH + 1) * W];
#pragma unroll
      for (int hh = 0; hh <= 2 * NH; ++hh) {
        const VT v = slot[(ty + R) * SX + tx + hh];
        const T *ve = reinterpret_cast<const T *>(&v);
#pragma unroll
        for (int i = 0; i < W; ++i) win[hh * W + i] = ve[i];
      }
      T acc[W];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        T a = c(0, R) * win[NH * W + i];
#pragma unroll
        for (int j = 1; j <= R; ++j) a = fma(c(0, R + j), win[NH * W + i + j], fma(c(0, R - j), win[NH * W + i - j], a));
        acc[i] = a;
      }
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const VT tm = slot[(ty + R - j) * SX + tx + NH], tp = slot[(ty + R + j) * SX + tx + NH];
        const T *me = reinterpret_cast<const T *>(&tm), *pe = reinterpret_cast<const T *>(&tp);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = fma(c(1, R + j), pe[i], fma(c(1, R - j), me[i], acc[i]));
      }
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const T *me = reinterpret_cast<const T *>(&q[(u + R - j + QL) % QL]);
        const T *pe = reinterpret_cast<const T *>(&q[(u + R + j) % QL]);
#pragma unroll
        for (int i = 0; i < W; ++i) acc[i] = fma(c(2, R + j), pe[i], fma(c(2, R - j), me[i], acc[i]));
      }
      VT out;
      T *oe = reinterpret_cast<T *>(&out);
#pragma unroll
      for (int i = 0; i < W; ++i) oe[i] = sc * acc[i];
      const int64_t o = (int64_t)z * plane + own;
      *reinterpret_cast<VT *>(y + o) = out;
      if (xc) {
        const T *ce = reinterpret_cast<const T *>(&q[(u + R) % QL]);
#pragma unroll
        for (int i = 0; i < W; ++i) oe[i] = sc * ce[i];
        *reinterpret_cast<VT *>(xc + o) = out;
      }
    }
  }
  cp_async_wait<0>();
}

// Planes per CTA of k_stencil_3d: the fewest chunks of z that fill the resident slots.
template <typename T, int R>
static int tile3d_tz(int gx, int gy, int nz) {
  static const int resident = [] {   // thread-safe one-time initialisation
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int bytes = tile3d_smem_bytes<T, R>();
    cudaFuncSetAttribute(k_stencil_3d<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stencil_3d<T, R>, kTileXV * kTileY, bytes);
    return std::max(1, sms) * std::max(1, per);
  }();
  const int chunks = std::max(1, std::min(nz, resident / std::max(1, gx * gy)));
  return (nz + chunks - 1) / chunks;
}

bool stencil_3d_tiled(const Geometry &g, int elem_bytes) {
  const int W = 16 / elem_bytes;
  return g.ndim == 3 && g.nx % W == 0 && (g.nx / W) % kTileXV == 0 && g.ny % kTileY == 0 && g.nz >= g.R;
}

// Grid of the vectorised stencil: one vector per thread when that many CTAs are resident
// at once, else every resident slot (a grid-stride loop covers the rest).
template <typename T, int NDIM, int R>
static int vec_grid(int64_t nvec) {
  static const int resident = [] {   // thread-safe one-time initialisation
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stencil_vec<T, NDIM, R>, kThreads, 0);
    return std::max(1, sms) * std::max(1, per);
  }();
  return (int)std::max<int64_t>(1, std::min<int64_t>((nvec + kThreads - 1) / kThreads, resident));
}

// y = A (s x) for the explicit banded operator, one row per thread (xcopy as for the stencil).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_band_matvec(const T *__restrict__ Ab, int bw, InRef<T> xref, OutRef<T> yref,
                                                         OutRef<T> xcopy, const double *scale, int64_t n,
                                                         const int *active) {
  if (active && *active == 0) return;
  const T *__restrict__ x = xref.get();
  T *y = yref.get();
  T *xc = xcopy.base ? xcopy.get() : nullptr;
  const T sc = scale ? (T)(*scale) : (T)1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T acc = (T)0;
    for (int p = 0; p <= 2 * bw; ++p) {
      const int64_t j = i + p - bw;
      if (j >= 0 && j < n) acc += Ab[i * (2 * bw + 1) + p] * x[j];
    }
    y[i] = sc * acc;
    if (xc) xc[i] = sc * x[i];
  }
}

template <typename TI, typename TO, typename TC>
void launch_stencil(const Geometry &g, InRef<TI> x, OutRef<TO> y, const DevState *st, const int *active,
                    cudaStream_t s, OutRef<TO> xcopy, const double *scale) {
  constexpr bool same = std::is_same<TI, TO>::value && std::is_same<TI, TC>::value;
  if constexpr (same) {
    if (g.band_w > 0) {
      const TI *Ab = nullptr;
      if constexpr (std::is_same<TI, float>::value) Ab = g.Ab32;
      else Ab = g.Ab;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + kThreads - 1) / kThreads, 4096));
      k_band_matvec<TI><<<grid, kThreads, 0, s>>>(Ab, g.band_w, x, y, xcopy, scale, g.n, active);
      return;
    }
    constexpr int W = SVec<TI>::W;
    // vector path: rows split into whole aligned vectors, and more vectors per row than
    // halo vectors (so one periodic wrap suffices)
    const int nh = (g.R + W - 1) / W;
    auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const bool aligned = (x.counter ? (al(x.base) && (x.ld * sizeof(TI)) % 16 == 0) : al(x.base)) &&
                         (y.counter ? (al(y.base) && (y.ld * sizeof(TO)) % 16 == 0) : al(y.base)) &&
                         (!xcopy.base || (xcopy.counter ? (al(xcopy.base) && (xcopy.ld * sizeof(TO)) % 16 == 0)
                                                        : al(xcopy.base)));
    if (stencil_3d_tiled(g, sizeof(TI)) && aligned) {
      const int gx = g.nx / W / kTileXV, gy = g.ny / kTileY;
      PSP_DISPATCH_R(g.R, {
        const int tz = tile3d_tz<TI, RR>(gx, gy, g.nz);
        const dim3 grid3(gx, gy, (g.nz + tz - 1) / tz);
        const int bytes = tile3d_smem_bytes<TI, RR>();
        k_stencil_3d<TI, RR><<<grid3, kTileXV * kTileY, bytes, s>>>(x, y, xcopy, scale, st, g.nx, g.ny, g.nz, tz, active);
      });
      return;
    }
    if (g.nx % W == 0 && g.nx / W > nh && aligned) {
      const int64_t nvec = g.n / W;
      PSP_DISPATCH_NDIM(g.ndim, PSP_DISPATCH_R(g.R, (k_stencil_vec<TI, DD, RR><<<vec_grid<TI, DD, RR>(nvec), kThreads, 0, s>>>(
                                                        x, y, xcopy, scale, st, g.nx, g.ny, g.nz, active))));
      return;
    }
  }
  const int grid = stencil_grid(g.n);
  PSP_DISPATCH_NDIM(g.ndim, PSP_DISPATCH_R(g.R, (k_stencil<TI, TO, TC, DD, RR><<<grid, kThreads, 0, s>>>(
                                                    x, y, xcopy, scale, st, g.nx, g.ny, g.nz, active))));
}

template <typename TH, typename TV>
void launch_restart(const Geometry &g, const double *X, const double *B, TH *Px, TH *Py, int64_t ldh,
                    TV *V1, DevState *st, double *partial, int mixed, cudaStream_t s, const int *skip) {
  const int grid = reduce_grid(g.n);
  if (g.band_w > 0) {
    k_restart<TH, TV, 0, 1><<<grid, kThreads, 0, s>>>(X, B, Px, Py, ldh, V1, st, partial, g.nx, g.ny, g.nz, mixed,
                                                     g.Ab, g.band_w, skip);
    return;
  }
  PSP_DISPATCH_NDIM(g.ndim, PSP_DISPATCH_R(g.R, (k_restart<TH, TV, DD, RR><<<grid, kThreads, 0, s>>>(
                                                    X, B, Px, Py, ldh, V1, st, partial, g.nx, g.ny,
                                                    g.nz, mixed, nullptr, 0, skip))));
}

// Grid of k_restart_df: one wave of resident CTAs.  The grid-stride loop then walks the grid
// in lockstep, a few planes at a time, so every neighbour plane is in L2 when it is read; with
// more CTAs than fit, the waves scatter over the grid and the neighbours come from DRAM again.
template <int NDIM, int R>
static int restart_df_grid(int64_t n) {
  static const int resident = [] {   // thread-safe one-time initialisation
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_restart_df<NDIM, R>, kThreads, 0);
    return std::max(1, sms) * std::max(1, per);
  }();
  return std::max(1, std::min(reduce_grid(n), resident));
}

// The mixed form's restart.  On stencil grids the double-float kernels take (k_split_x into
// the scratch columns Xh and Xl, then k_restart_df) all three kernels are enqueued and
// DevState::restart_df, set per step, picks the double-float pair or the FP64 kernel (the
// others return at once); returns whether the pair was enqueued.  Elsewhere: the FP64
// kernel alone.
bool launch_restart_mixed(const Geometry &g, const double *X, const double *B, float *Px, float *Py, int64_t ldh,
                          float *V1, float *Xh, float *Xl, DevState *st, double *partial, cudaStream_t s) {
  auto al = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int nh = (g.R + 3) / 4;
  const bool df = g.band_w == 0 && Xh && Xl && g.R >= 1 && g.R <= 5 && g.nx % 4 == 0 && g.nx / 4 > nh &&
                  ldh % 4 == 0 && al(X) && al(B) && al(Px) && al(Py) && al(V1) && al(Xh) && al(Xl);
  if (!df) {
    launch_restart<float, float>(g, X, B, Px, Py, ldh, V1, st, partial, 1, s);
    return false;
  }
  const int nvec = (int)(g.n / 4);
  const int gs = std::max(1, std::min((nvec + kThreads - 1) / kThreads, 152 * 8));
  k_split_x<<<gs, kThreads, 0, s>>>(X, Xh, Xl, nvec, st);
  PSP_DISPATCH_NDIM(g.ndim, PSP_DISPATCH_R(g.R, (k_restart_df<DD, RR><<<restart_df_grid<DD, RR>(g.n), kThreads, 0, s>>>(
                                                    Xh, Xl, B, Px, Py, ldh, V1, st, partial, g.nx, g.ny, g.nz))));
  launch_restart<float, float>(g, X, B, Px, Py, ldh, V1, st, partial, 1, s, &st->restart_df);
  return true;
}

template void launch_stencil<double, double, double>(const Geometry &, InRef<double>, OutRef<double>,
                                                     const DevState *, const int *, cudaStream_t,
                                                     OutRef<double>, const double *);
template void launch_stencil<float, float, float>(const Geometry &, InRef<float>, OutRef<float>,
                                                  const DevState *, const int *, cudaStream_t, OutRef<float>,
                                                  const double *);
template void launch_restart<double, double>(const Geometry &, const double *, const double *, double *,
                                             double *, int64_t, double *, DevState *, double *, int,
                                             cudaStream_t, const int *);
template void launch_restart<float, float>(const Geometry &, const double *, const double *, float *,
                                           float *, int64_t, float *, DevState *, double *, int,
                                           cudaStream_t, const int *);

}  // namespace psp
