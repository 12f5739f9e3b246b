// Restarted right-preconditioned BiCGSTAB (van der Vorst 1992) as an alternative Krylov
// solver for the implicit step, with the progressive history of Algorithm 1: every
// iteration stores two matvec pairs, (p^, A p^) and (s^, A s^), in the P_x / P_y rings, so
// Algorithm 2 fits N from them exactly as from GMRES's pairs.  FP64 only.
//
// One restart cycle (captured as a graph like a GMRES cycle): the restart kernel forms the
// true residual r = B - A X_0 (V column 0) and the restart pair; k_bi_start sets the
// shadow residual rh = r (column 1) and the scalars; iteration j then runs
//   k_bi_p      p = r (j = 0) or r + beta (p - omega v)         (column 2; P_x ring if N = I)
//   [band solve p^ = N^{-1} (sigma p) into the P_x ring]        (N != I)
//   stencil     sigma v = A (sigma p^)                          (P_y ring)
//   k_bi_alpha  alpha = rho / (rh . v)
//   k_bi_s      s = r - alpha v                                 (column 3; P_x ring if N = I)
//   [band solve, stencil: sigma s^, sigma t = A sigma s^]
//   k_bi_omega  omega = (t . s) / (t . t)  (0 when t = 0)
//   k_bi_xr     X += alpha p^ + omega s^, r = s - omega t, rho' = rh . r, ||r||: the finish
//               test, beta = (rho' / rho)(alpha / omega), sigma' = 1 / ||r||, the summary.
// The stored pairs are scaled by sigma = 1 / ||r|| of the iteration's start (BiCGSTAB's
// directions shrink with the residual; unscaled they make the fit's designs
// ill-conditioned), and the kernels that read them back divide by sigma.  The scalars
// live in DevState::bi; each reduction is the counting last-block pattern in a fixed
// order over CTAs, so a run is deterministic.
#include "psp_kernels.cuh"

namespace psp {

namespace {

enum { kRho = 0, kAlpha = 1, kOmega = 2, kBeta = 3, kSig = 4, kRr = 5 };

// Block sum of two values into partial[t * kMaxCta + blockIdx.x] (t = 0, 1); true in the
// last CTA to arrive, whose tot[] then holds the fixed-order grid sums.
__device__ __forceinline__ bool grid_sum2(double a, double b, double *partial, unsigned int *counter,
                                          double (&tot)[2]) {
  __shared__ double s_w[2][kThreads / 32];
  __shared__ double s_tot[2];
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s_w[0][wid] = a; s_w[1][wid] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { x += s_w[0][w]; y += s_w[1][w]; }
    partial[blockIdx.x] = x;
    partial[kMaxCta + blockIdx.x] = y;
  }
  if (!last_block_arrive(counter)) return false;
  if (wid < 2) {
    double x = 0.0;
    for (int c = lane; c < (int)gridDim.x; c += 32) x += __ldcg(partial + wid * kMaxCta + c);
    x = warp_sum(x);
    if (lane == 0) s_tot[wid] = x;
  }
  __syncthreads();
  tot[0] = s_tot[0];
  tot[1] = s_tot[1];
  return true;
}

__global__ void __launch_bounds__(kThreads) k_bi_start(int64_t n, double *__restrict__ V, int64_t ldv, DevState *st) {
  if (st->active == 0) return;
  const double *r = V;
  double *rh = V + ldv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    rh[i] = r[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const double beta = st->beta;   // ||r|| of the restart (> 0 while active)
    st->bi[kRho] = beta * beta;
    st->bi[kRr] = beta * beta;
    st->bi[kAlpha] = 1.0;
    st->bi[kOmega] = 1.0;
    st->bi[kBeta] = 0.0;
    st->bi[kSig] = 1.0 / beta;
    st->bi_flag = 0;
  }
}

// p = r (first) or r + beta (p - omega v), v = vs / sigma_prev; px (if set) = sigma p.
__global__ void __launch_bounds__(kThreads) k_bi_p(int64_t n, int first, double *__restrict__ V, int64_t ldv,
                                                   InRef<double> vref, OutRef<double> pxref, DevState *st) {
  if (st->active == 0) return;
  const double *r = V;
  double *p = V + 2 * ldv;
  const double beta = st->bi[kBeta], omega = st->bi[kOmega], sig = st->bi[kSig];
  const double ivs = st->bi_isig_prev;   // 1 / sigma of the previous iteration
  const double *vs = first ? nullptr : vref.get();
  double *px = pxref.base ? pxref.get() : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = first ? r[i] : r[i] + beta * (p[i] - omega * ivs * vs[i]);
    p[i] = pi;
    if (px) px[i] = sig * pi;
  }
}

// alpha = rho / (rh . v), with v = vs / sigma.
__global__ void __launch_bounds__(kThreads) k_bi_alpha(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                       InRef<double> vref, DevState *st, double *partial) {
  if (st->active == 0) return;
  const double *rh = V + ldv;
  const double *vs = vref.get();
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += rh[i] * vs[i];
  double tot[2];
  if (!grid_sum2(a, 0.0, partial, &st->counter[2], tot)) return;
  if (threadIdx.x == 0) {
    const double rv = tot[0] / st->bi[kSig];
    st->bi[kAlpha] = (rv != 0.0) ? st->bi[kRho] / rv : 0.0;
    if (rv == 0.0) st->bi_flag = 1;
    last_block_reset(&st->counter[2]);
  }
}

// s = r - alpha v (v = vs / sigma); sx (if set) = sigma s.
__global__ void __launch_bounds__(kThreads) k_bi_s(int64_t n, double *__restrict__ V, int64_t ldv,
                                                   InRef<double> vref, OutRef<double> sxref, DevState *st) {
  if (st->active == 0) return;
  const double *r = V;
  double *s = V + 3 * ldv;
  const double sig = st->bi[kSig];
  const double c = st->bi[kAlpha] / sig;
  const double *vs = vref.get();
  double *sx = sxref.base ? sxref.get() : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = r[i] - c * vs[i];
    s[i] = si;
    if (sx) sx[i] = sig * si;
  }
}

// omega = (t . s) / (t . t) with t = ts / sigma, i.e. sigma (ts . s) / (ts . ts); 0 if t = 0.
__global__ void __launch_bounds__(kThreads) k_bi_omega(int64_t n, const double *__restrict__ V, int64_t ldv,
                                                       InRef<double> tref, DevState *st, double *partial) {
  if (st->active == 0) return;
  const double *s = V + 3 * ldv;
  const double *ts = tref.get();
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    a += ts[i] * s[i];
    b += ts[i] * ts[i];
  }
  double tot[2];
  if (!grid_sum2(a, b, partial, &st->counter[2], tot)) return;
  if (threadIdx.x == 0) {
    st->bi[kOmega] = (tot[1] != 0.0) ? st->bi[kSig] * tot[0] / tot[1] : 0.0;
    last_block_reset(&st->counter[2]);
  }
}

// X += (alpha ps + omega ss) / sigma, r = s - (omega / sigma) ts; rho' = rh . r, ||r||^2;
// the last CTA: finish test, next beta and sigma, the cycle summary.
__global__ void __launch_bounds__(kThreads) k_bi_xr(int64_t n, int j, int m, double *__restrict__ X,
                                                    double *__restrict__ V, int64_t ldv, InRef<double> pref,
                                                    InRef<double> sref, InRef<double> tref, DevState *st,
                                                    double *partial) {
  if (st->active == 0) return;
  double *r = V;
  const double *rh = V + ldv;
  const double *s = V + 3 * ldv;
  const double sig = st->bi[kSig];
  const double ca = st->bi[kAlpha] / sig, co = st->bi[kOmega] / sig;
  const double *ps = pref.get(), *ss = sref.get(), *ts = tref.get();
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    X[i] += ca * ps[i] + co * ss[i];
    const double ri = s[i] - co * ts[i];
    r[i] = ri;
    a += rh[i] * ri;
    b += ri * ri;
  }
  double tot[2];
  if (!grid_sum2(a, b, partial, &st->counter[2], tot)) return;
  if (threadIdx.x == 0) {
    const double rho_new = tot[0], rr = tot[1];
    const double R = sqrt(rr);
    const double alpha = st->bi[kAlpha], omega = st->bi[kOmega], rho = st->bi[kRho];
    int status = st->status;
    bool end = false;
    if (!isfinite(R) || !isfinite(rho_new)) { status |= kStNumeric; end = true; }
    else if (R <= st->eps_abs) { status |= kStConverged; end = true; }
    else if (st->bi_flag || omega == 0.0 || rho_new == 0.0 || rho == 0.0) { status |= kStBreakdown; end = true; }
    st->bi[kBeta] = (omega != 0.0 && rho != 0.0) ? (rho_new / rho) * (alpha / omega) : 0.0;
    st->bi[kRho] = rho_new;
    st->bi[kRr] = rr;
    st->bi_isig_prev = 1.0 / sig;
    st->bi[kSig] = R > 0.0 ? 1.0 / R : 1.0;
    const int k = j + 1;
    st->R[j] = R;
    st->k_end = k;
    st->status = status;
    st->hist_count = st->hist_base + 1 + 2 * k;
    if (end || k == m) st->active = 0;
    st->sum.k_end = k;
    st->sum.status = status;
    st->sum.R_end = R;
    st->sum.hist_count = st->hist_count;
    st->sum.error = st->error;
    last_block_reset(&st->counter[2]);
  }
}

int bi_grid(int64_t n) { return reduce_grid(n); }

}  // namespace

void launch_bi_start(int64_t n, double *V, int64_t ldv, DevState *st, cudaStream_t s) {
  k_bi_start<<<bi_grid(n), kThreads, 0, s>>>(n, V, ldv, st);
}
void launch_bi_p(int first, int64_t n, double *V, int64_t ldv, InRef<double> v, OutRef<double> px, DevState *st,
                 cudaStream_t s) {
  k_bi_p<<<bi_grid(n), kThreads, 0, s>>>(n, first, V, ldv, v, px, st);
}
void launch_bi_alpha(int64_t n, const double *V, int64_t ldv, InRef<double> v, DevState *st, double *partial,
                     cudaStream_t s) {
  k_bi_alpha<<<bi_grid(n), kThreads, 0, s>>>(n, V, ldv, v, st, partial);
}
void launch_bi_s(int64_t n, double *V, int64_t ldv, InRef<double> v, OutRef<double> sx, DevState *st, cudaStream_t s) {
  k_bi_s<<<bi_grid(n), kThreads, 0, s>>>(n, V, ldv, v, sx, st);
}
void launch_bi_omega(int64_t n, const double *V, int64_t ldv, InRef<double> t, DevState *st, double *partial,
                     cudaStream_t s) {
  k_bi_omega<<<bi_grid(n), kThreads, 0, s>>>(n, V, ldv, t, st, partial);
}
void launch_bi_xr(int j, int m, int64_t n, double *X, double *V, int64_t ldv, InRef<double> p, InRef<double> sx,
                  InRef<double> t, DevState *st, double *partial, cudaStream_t s) {
  k_bi_xr<<<bi_grid(n), kThreads, 0, s>>>(n, j, m, X, V, ldv, p, sx, t, st, partial);
}

}  // namespace psp
