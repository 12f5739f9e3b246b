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
#include <type_traits>

#include "dfloat.cuh"
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

// FP32 history, the fast form of the moments: every thread owns two consecutive rows (i,
// i+1), and each of its moments is a pair (row i, row i+1) of double-float accumulators held
// in packed FP32x2 registers, so one packed instruction advances both rows (the error-free
// product a b = p + e by a multiply and an FMA, the error-free sum by Knuth's two-sum, as in
// AccF2).  The history is staged in shared memory column chunk by column chunk with 16-byte
// asynchronous copies, two chunks in flight, so the copies of the next chunk overlap the
// arithmetic of this one.  Row windows: P_x rows i-B .. i+1+2B, P_y rows i, i+1.
constexpr int kFm2Threads = 256;
constexpr int kFm2Rows = 2 * kFm2Threads;        // rows per CTA
constexpr int kFm2Cols = 8;                      // history columns per staged chunk
constexpr int kFm2Lead = 4;                      // staged rows before the CTA's first row (>= B, 16-byte aligned)
constexpr int kFm2Span = kFm2Rows + 12;          // staged P_x rows: r0-4 .. r0+kFm2Rows+7 (covers i+1+2B for B <= 4)

// A pair of double-float accumulators (hi, lo packed per row).
struct Acc2 {
  uint64_t hi = 0, lo = 0;
  // += a b, with na = -a: p = fl(a b), p - a b = fma(na, b, p) = -e exactly
  __device__ __forceinline__ void fma(uint64_t a, uint64_t na, uint64_t b) {
    const uint64_t p = f2mul(a, b);
    const uint64_t ne = f2fma(na, b, p);
    sum2(p, ne);
  }
  __device__ __forceinline__ void add(uint64_t v) { sum2(v, 0ull); }
  // hi + lo += p - ne (two-sum of hi and p; the rounding error and -ne go to lo)
  __device__ __forceinline__ void sum2(uint64_t p, uint64_t ne) {
    const uint64_t s = f2add(hi, p);
    const uint64_t bb = f2sub(s, hi);
    const uint64_t err = f2add(f2sub(hi, f2sub(s, bb)), f2sub(p, bb));
    hi = s;
    lo = f2add(lo, f2sub(err, ne));
  }
  __device__ __forceinline__ void get(double &r0, double &r1) const {
    float h0, h1, l0, l1;
    f2unpack(hi, h0, h1);
    f2unpack(lo, l0, l1);
    r0 = (double)h0 + (double)l0;
    r1 = (double)h1 + (double)l1;
  }
};

template <int B>
__global__ void __launch_bounds__(kFm2Threads) k_fit_moments_f32(int64_t n, int M, const float *__restrict__ Px,
                                                                 const float *__restrict__ Py, int64_t ld,
                                                                 double *__restrict__ mom, int cyclic, int vec) {
  constexpr int NM = 4 * B + 4;
  extern __shared__ __align__(16) float fm2[];
  float *sx = fm2;                                   // [2][kFm2Cols][kFm2Span]
  float *sy = fm2 + 2 * kFm2Cols * kFm2Span;         // [2][kFm2Cols][kFm2Rows]
  const int64_t r0 = (int64_t)blockIdx.x * kFm2Rows;
  const int tid = threadIdx.x;
  // the 16-byte path: every staged row inside [0, n) and every column 16-byte aligned
  const bool fast = vec && r0 - kFm2Lead >= 0 && r0 - kFm2Lead + kFm2Span <= n;
  auto stage = [&](int c0, int buf) {
    const int nc = min(kFm2Cols, M - c0);
    float *bx = sx + buf * kFm2Cols * kFm2Span;
    float *by = sy + buf * kFm2Cols * kFm2Rows;
    if (fast) {
      constexpr int CX = kFm2Span / 4, CY = kFm2Rows / 4;
      for (int e = tid; e < kFm2Cols * (CX + CY); e += kFm2Threads) {
        const int cc = e / (CX + CY), k = e % (CX + CY);
        if (cc >= nc) continue;
        if (k < CX) {
          const float *src = Px + (int64_t)(c0 + cc) * ld + r0 - kFm2Lead + 4 * k;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                           static_cast<uint32_t>(__cvta_generic_to_shared(bx + cc * kFm2Span + 4 * k))),
                       "l"(src)
                       : "memory");
        } else {
          const int kk = k - CX;
          const float *src = Py + (int64_t)(c0 + cc) * ld + r0 + 4 * kk;
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                           static_cast<uint32_t>(__cvta_generic_to_shared(by + cc * kFm2Rows + 4 * kk))),
                       "l"(src)
                       : "memory");
        }
      }
    } else {
      for (int e = tid; e < kFm2Cols * kFm2Span; e += kFm2Threads) {
        const int cc = e / kFm2Span, k = e % kFm2Span;
        int64_t row = r0 - kFm2Lead + k;
        if (cyclic) row = (row < 0) ? row + n : (row >= n ? row - n : row);   // B <= 4 < n: one wrap
        bx[cc * kFm2Span + k] = (cc < nc && row >= 0 && row < n) ? Px[(int64_t)(c0 + cc) * ld + row] : 0.0f;
      }
      for (int e = tid; e < kFm2Cols * kFm2Rows; e += kFm2Threads) {
        const int cc = e / kFm2Rows, k = e % kFm2Rows;
        const int64_t row = r0 + k;
        by[cc * kFm2Rows + k] = (cc < nc && row < n) ? Py[(int64_t)(c0 + cc) * ld + row] : 0.0f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  Acc2 S[2 * B + 1], Rp[2 * B + 1], ssx, ssy;
  const int nch = (M + kFm2Cols - 1) / kFm2Cols;
  stage(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      stage((ch + 1) * kFm2Cols, (ch + 1) & 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const int buf = ch & 1;
    const int nc = min(kFm2Cols, M - ch * kFm2Cols);
    const float *bx = sx + buf * kFm2Cols * kFm2Span;
    const float *by = sy + buf * kFm2Cols * kFm2Rows;
    for (int cc = 0; cc < nc; ++cc) {
      // x[k] = P_x(i - kFm2Lead + k) with i = r0 + 2 tid, k = 0 .. kFm2Lead + 2B + 1
      const float *xw = bx + cc * kFm2Span + 2 * tid;
      constexpr int NW = (kFm2Lead + 2 * B + 2 + 1) / 2;   // aligned pairs of the window
      uint64_t pr[NW];
#pragma unroll
      for (int q = 0; q < NW; ++q) pr[q] = *reinterpret_cast<const uint64_t *>(xw + 2 * q);
      // the pair (P_x(i + o), P_x(i + 1 + o)) for offset o (from the aligned pairs)
      auto pair_at = [&](int o) -> uint64_t {
        const int k = kFm2Lead + o;
        if ((k & 1) == 0) return pr[k / 2];
        float a0, a1, b0, b1;
        f2unpack(pr[k / 2], a0, a1);
        f2unpack(pr[k / 2 + 1], b0, b1);
        return f2pack(a1, b0);
      };
      const uint64_t x0 = pr[kFm2Lead / 2];
      const uint64_t nx0 = f2neg(x0);
      const uint64_t y = *reinterpret_cast<const uint64_t *>(by + cc * kFm2Rows + 2 * tid);
      const uint64_t ny = f2neg(y);
#pragma unroll
      for (int l = 0; l <= 2 * B; ++l) S[l].fma(x0, nx0, pair_at(l));
#pragma unroll
      for (int p = 0; p <= 2 * B; ++p) Rp[p].fma(y, ny, pair_at(p - B));
      ssx.add(x0);
      ssy.add(y);
    }
    __syncthreads();   // the buffer is refilled by the stage issued in the next round
  }
  const int64_t row = r0 + 2 * tid;
  double v0, v1;
#pragma unroll
  for (int l = 0; l <= 2 * B; ++l) {
    S[l].get(v0, v1);
    if (row < n) mom[row * NM + l] = v0;
    if (row + 1 < n) mom[(row + 1) * NM + l] = v1;
    Rp[l].get(v0, v1);
    if (row < n) mom[row * NM + 2 * B + 1 + l] = v0;
    if (row + 1 < n) mom[(row + 1) * NM + 2 * B + 1 + l] = v1;
  }
  ssx.get(v0, v1);
  if (row < n) mom[row * NM + 4 * B + 2] = v0;
  if (row + 1 < n) mom[(row + 1) * NM + 4 * B + 2] = v1;
  ssy.get(v0, v1);
  if (row < n) mom[row * NM + 4 * B + 3] = v0;
  if (row + 1 < n) mom[(row + 1) * NM + 4 * B + 3] = v1;
}

constexpr size_t kFm2Smem = (size_t)2 * kFm2Cols * (kFm2Span + kFm2Rows) * sizeof(float);

// Cholesky solve of a Q x Q SPD system in registers (one reciprocal square root per pivot,
// L_jj = d rsqrt(d); the substitutions multiply by rsqrt(d)).  Returns false if degenerate.
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
    const double r = rsqrt(d);
    const double ljj = d * r;
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

template <int B, int INTERCEPT>
__global__ void __launch_bounds__(128) k_fit_solve(int64_t n, int M, const double *__restrict__ mom,
                                                   double *__restrict__ band, int *singular_count, int cyclic) {
  constexpr int intercept = INTERCEPT;
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
  const int g1f = (int)((n + kFm2Rows - 1) / kFm2Rows);
  const int g2 = (int)((n + 127) / 128);
  // 16-byte staging needs 16-byte aligned columns
  const int vec = ((reinterpret_cast<uintptr_t>(Px) | reinterpret_cast<uintptr_t>(Py)) % 16 == 0) && (ld % 4 == 0);
  switch (b) {
#define PSP_FIT(B_)                                                                              \
  case B_:                                                                                       \
    if constexpr (std::is_same<TH, float>::value) {                                              \
      static const bool attr_ = [] {                                                             \
        return cudaFuncSetAttribute(k_fit_moments_f32<B_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)kFm2Smem) == cudaSuccess;                               \
      }();                                                                                       \
      (void)attr_;                                                                               \
      k_fit_moments_f32<B_><<<g1f, kFm2Threads, kFm2Smem, s>>>(n, M, Px, Py, ld, moments, cyclic, vec); \
    } else {                                                                                     \
      k_fit_moments<TH, B_><<<g1, kFitRows, 0, s>>>(n, M, Px, Py, ld, moments, cyclic);          \
    }                                                                                            \
    if (intercept) k_fit_solve<B_, 1><<<g2, 128, 0, s>>>(n, M, moments, band, singular_count, cyclic); \
    else k_fit_solve<B_, 0><<<g2, 128, 0, s>>>(n, M, moments, band, singular_count, cyclic);           \
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
