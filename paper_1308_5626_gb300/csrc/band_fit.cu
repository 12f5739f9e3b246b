// Algorithm 2 (MREP): the banded preconditioner N fitted row by row to the matvec history
// P_x, P_y (n x M, column c = one pair (x, A x)).
//
// Row i of the interior regresses P_y(i,:) on [1; P_x(i-b..i+b, :)] by the normal
// equations.  Its Gram matrix only needs lagged products of P_x rows,
//     S_l(j) = sum_c P_x(j,c) P_x(j+l,c),  l = 0..2b,
// because G(p,q) = S_|q-p|(i - b + min(p,q)); the right-hand side needs
//     r_p(i) = sum_c P_x(i-b+p,c) P_y(i,c),  p = 0..2b,
// and the intercept row the sums s(j) = sum_c P_x(j,c), t(i) = sum_c P_y(i,c).  So one
// streaming pass (k_fit_moments) reads every history element once and accumulates
// 2(2b+1)+2 FP64 moments per row; a second kernel (k_fit_solve) assembles each row's
// Gram from the moments of rows i-b..i+b and solves it by Cholesky in registers.  The
// first and last b rows take the slope of the simple linear fit on P_x(i,:) (diagonal
// of N only), as the paper prescribes; with a cyclic band (periodic 1D grid) every row is an
// interior row and the neighbour indices wrap modulo n.  A row whose relative Cholesky pivot is <= 1e-12
// (regressors collinear in the sample) gets the identity row and is counted.
//
// Moments of an FP32 history are accumulated in double-float (an FP32 pair): every product
// of two FP32 values is split exactly into p + e with one FMA and added by an error-free
// two-sum, so a moment carries about 48 significant bits -- FP64-grade for sums of a few
// hundred terms -- at FP32 instruction rates (GB300 runs FP64 at 1/64 of the FP32 rate).
// An FP64 history is accumulated in FP64.
#include <algorithm>

#include "psp_kernels.cuh"

namespace psp {

constexpr double kRelPivot = 1e-12;
constexpr int kFitRows = 256;   // rows per CTA
constexpr int kFitCols = 8;     // history columns staged per round

// Accumulators of the moments: FP64, or double-float for FP32 data (see above).
struct AccD {
  double v = 0.0;
  __device__ __forceinline__ void fma(double a, double b) { v = ::fma(a, b, v); }
  __device__ __forceinline__ void add(double a) { v += a; }
  __device__ __forceinline__ double get() const { return v; }
};
struct AccF2 {
  float hi = 0.0f, lo = 0.0f;
  // hi + lo += a b: two-product a b = p + e (FMA), two-sum hi + p = s + err (Knuth); the
  // _rn intrinsics keep the compiler from contracting or reassociating these steps
  __device__ __forceinline__ void fma(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    add2(p, e);
  }
  __device__ __forceinline__ void add(float a) { add2(a, 0.0f); }
  __device__ __forceinline__ void add2(float p, float e) {
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
template <typename TH> struct FitAcc;
template <> struct FitAcc<double> { using type = AccD; };
template <> struct FitAcc<float> { using type = AccF2; };

template <typename TH, int B>
__global__ void __launch_bounds__(kFitRows) k_fit_moments(int64_t n, int M, const TH *__restrict__ Px,
                                                          const TH *__restrict__ Py, int64_t ld,
                                                          double *__restrict__ mom, int cyclic) {
  constexpr int TW = kFitRows + 3 * B;   // P_x rows r0-B .. r0+kFitRows+2B-1
  constexpr int NM = 4 * B + 4;
  using Acc = typename FitAcc<TH>::type;
  __shared__ TH sx[kFitCols][TW];
  __shared__ TH sy[kFitCols][kFitRows];
  const int64_t r0 = (int64_t)blockIdx.x * kFitRows;
  const int tid = threadIdx.x;
  Acc S[2 * B + 1], Rp[2 * B + 1], sx_sum, sy_sum;
  for (int c0 = 0; c0 < M; c0 += kFitCols) {
    const int nc = min(kFitCols, M - c0);
    __syncthreads();
    for (int cc = 0; cc < kFitCols; ++cc) {
      const TH *px = Px + (int64_t)(c0 + cc) * ld;
      const TH *py = Py + (int64_t)(c0 + cc) * ld;
      for (int t = tid; t < TW; t += kFitRows) {
        int64_t row = r0 - B + t;
        if (cyclic) row = ((row % n) + n) % n;   // periodic neighbours
        sx[cc][t] = (cc < nc && row >= 0 && row < n) ? px[row] : (TH)0;
      }
      const int64_t row = r0 + tid;
      sy[cc][tid] = (cc < nc && row < n) ? py[row] : (TH)0;
    }
    __syncthreads();
#pragma unroll 2
    for (int cc = 0; cc < kFitCols; ++cc) {
      const TH *x = &sx[cc][tid + B];   // x[0] = P_x(row, c)
      const TH y = sy[cc][tid];
#pragma unroll
      for (int l = 0; l <= 2 * B; ++l) S[l].fma(x[0], x[l]);
#pragma unroll
      for (int p = 0; p <= 2 * B; ++p) Rp[p].fma(x[p - B], y);
      sx_sum.add(x[0]);
      sy_sum.add(y);
    }
  }
  const int64_t row = r0 + tid;
  if (row < n) {
    double *o = mom + row * NM;
#pragma unroll
    for (int l = 0; l <= 2 * B; ++l) { o[l] = S[l].get(); o[2 * B + 1 + l] = Rp[l].get(); }
    o[4 * B + 2] = sx_sum.get();
    o[4 * B + 3] = sy_sum.get();
  }
}

// Cholesky solve of a Q x Q SPD system in registers (one square root and one division per
// pivot; the substitutions multiply by the pivot's reciprocal).  Returns false if degenerate.
template <int Q>
__device__ __forceinline__ bool chol_solve(double (&G)[Q][Q], double (&rhs)[Q], int q) {
  double L[Q][Q], rd[Q];
#pragma unroll
  for (int j = 0; j < Q; ++j) {
    if (j >= q) break;
    double d = G[j][j];
#pragma unroll
    for (int l = 0; l < Q; ++l) if (l < j) d -= L[j][l] * L[j][l];
    if (!(G[j][j] > 0.0) || !(d > kRelPivot * G[j][j])) return false;
    const double ljj = sqrt(d);
    const double r = 1.0 / ljj;
    L[j][j] = ljj;
    rd[j] = r;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i > j && i < q) {
        double s = G[i][j];
#pragma unroll
        for (int l = 0; l < Q; ++l) if (l < j) s -= L[i][l] * L[j][l];
        L[i][j] = s * r;
      }
    }
  }
  double z[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i < q) {
      double s = rhs[i];
#pragma unroll
      for (int l = 0; l < Q; ++l) if (l < i) s -= L[i][l] * z[l];
      z[i] = s * rd[i];
    }
  }
#pragma unroll
  for (int i = Q - 1; i >= 0; --i) {
    if (i < q) {
      double s = z[i];
#pragma unroll
      for (int l = 0; l < Q; ++l) if (l > i && l < q) s -= L[l][i] * rhs[l];
      rhs[i] = s * rd[i];
    }
  }
  return true;
}

template <int B>
__global__ void __launch_bounds__(128) k_fit_solve(int64_t n, int M, int intercept,
                                                   const double *__restrict__ mom, double *__restrict__ band,
                                                   int *singular_count, int cyclic) {
  constexpr int NM = 4 * B + 4;
  constexpr int W = 2 * B + 1;
  constexpr int Q = 2 * B + 2;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double *out = band + i * W;
  const double *mi = mom + i * NM;
  bool ok;
  double beta[Q];
  const bool interior = cyclic || ((i >= B) && (i < n - B));
  // moments of row i - B + p (taken modulo n for a cyclic band)
  auto mrow = [&](int p) -> const double * {
    int64_t r = i - B + p;
    r += (r < 0) ? n : ((r >= n) ? -n : 0);
    return mom + r * NM;
  };
  if (interior) {
    double G[Q][Q], rhs[Q];
    const int o = intercept ? 1 : 0;
    const int q = W + o;
    if (intercept) {
      G[0][0] = (double)M;
#pragma unroll
      for (int p = 0; p < W; ++p) {
        const double s = mrow(p)[4 * B + 2];
        G[0][1 + p] = s;
        G[1 + p][0] = s;
      }
      rhs[0] = mi[4 * B + 3];
    }
#pragma unroll
    for (int p = 0; p < W; ++p) {
#pragma unroll
      for (int qq = 0; qq < W; ++qq) {
        const int lo = p < qq ? p : qq;
        const int lag = p < qq ? qq - p : p - qq;
        const double v = mrow(lo)[lag];
        if (intercept) G[1 + p][1 + qq] = v; else G[p][qq] = v;
      }
      rhs[o + p] = mi[W + p];
    }
    if (!intercept) { G[Q - 1][Q - 1] = 1.0; rhs[Q - 1] = 0.0; }
    ok = chol_solve<Q>(G, rhs, q);
#pragma unroll
    for (int p = 0; p < W; ++p) out[p] = ok ? rhs[o + p] : (p == B ? 1.0 : 0.0);
  } else {
    double G[2][2], rhs[2];
    if (intercept) {
      G[0][0] = (double)M; G[0][1] = G[1][0] = mi[4 * B + 2]; G[1][1] = mi[0];
      rhs[0] = mi[4 * B + 3]; rhs[1] = mi[W + B];
      ok = chol_solve<2>(G, rhs, 2);
      beta[1] = rhs[1];
    } else {
      double g1[1][1] = {{mi[0]}}, r1[1] = {mi[W + B]};
      ok = chol_solve<1>(g1, r1, 1);
      beta[1] = r1[0];
    }
#pragma unroll
    for (int p = 0; p < W; ++p) out[p] = (p == B) ? (ok ? beta[1] : 1.0) : 0.0;
  }
  if (!ok) atomicAdd(singular_count, 1);
}

template <typename TH>
void launch_fit(int b, int intercept, int64_t n, int M, const TH *Px, const TH *Py, int64_t ld, double *moments,
                double *band, int *singular_count, cudaStream_t s, int cyclic) {
  const int g1 = (int)((n + kFitRows - 1) / kFitRows);
  const int g2 = (int)((n + 127) / 128);
  switch (b) {
#define PSP_FIT(B_)                                                                              \
  case B_:                                                                                       \
    k_fit_moments<TH, B_><<<g1, kFitRows, 0, s>>>(n, M, Px, Py, ld, moments, cyclic);            \
    k_fit_solve<B_><<<g2, 128, 0, s>>>(n, M, intercept, moments, band, singular_count, cyclic);  \
    break;
    PSP_FIT(1) PSP_FIT(2) PSP_FIT(3) PSP_FIT(4)
#undef PSP_FIT
    default: break;
  }
}

// The history ring in chronological order: output column c (of `cols`) is ring column
// (first + c) mod mmax, widened to FP64 (exact for FP32 values).
template <typename TH>
__global__ void __launch_bounds__(kThreads) k_history_copy(int64_t n, int cols, int first, int mmax,
                                                           const TH *__restrict__ Px, const TH *__restrict__ Py,
                                                           int64_t ld, double *__restrict__ ox,
                                                           double *__restrict__ oy, int64_t ldo) {
  const int c = blockIdx.y;
  const int64_t src = (int64_t)((first + c) % mmax) * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    ox[(int64_t)c * ldo + i] = (double)Px[src + i];
    oy[(int64_t)c * ldo + i] = (double)Py[src + i];
  }
}

template <typename TH>
void launch_history_copy(int64_t n, int cols, int first, int mmax, const TH *Px, const TH *Py, int64_t ld,
                         double *ox, double *oy, int64_t ldo, cudaStream_t s) {
  if (cols <= 0) return;
  const int gx = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 1024);
  k_history_copy<TH><<<dim3((unsigned)std::max(gx, 1), (unsigned)cols), kThreads, 0, s>>>(n, cols, first, mmax, Px, Py,
                                                                                            ld, ox, oy, ldo);
}
template void launch_history_copy<float>(int64_t, int, int, int, const float *, const float *, int64_t, double *,
                                         double *, int64_t, cudaStream_t);
template void launch_history_copy<double>(int64_t, int, int, int, const double *, const double *, int64_t,
                                          double *, double *, int64_t, cudaStream_t);

template void launch_fit<float>(int, int, int64_t, int, const float *, const float *, int64_t, double *, double *,
                                int *, cudaStream_t, int);
template void launch_fit<double>(int, int, int64_t, int, const double *, const double *, int64_t, double *,
                                 double *, int *, cudaStream_t, int);

}  // namespace psp
