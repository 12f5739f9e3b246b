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
//   pass A (k_dcgs_dots):   w_j = A N^{-1} v_j (the matvec, when it is folded into the pass),
//                           a = Q^T v_j, alpha = v_j^T v_j, b = Q^T w_j, beta = v_j^T w_j,
//                           Q = [q_0 .. q_{j-1}], as per-CTA partial sums; the last CTA to
//                           finish reduces them and forms (the scalar engine)
//                           nu_j = sqrt(alpha - a^T a)             (q_j = (v_j - Q a) / nu_j),
//                           column j-1 of H completed: H(:, j-1) = h_{j-1} + a, H(j, j-1) = nu_j,
//                           t = Hbar a, h_j = ([b; (beta - a^T b)/nu_j] - t) / nu_j,
//                           c = t/nu_j + h_j, d = c_{0..j-1} - (c_j/nu_j) a;
//   pass B (k_dcgs_update): streams q_j and v_{j+1} = w_j/nu_j - (c_j/nu_j) v_j - Q d; its
//                           extra first CTA (block 0) runs the FP64 Givens step of column j-1.
//
// That Givens CTA alone owns the persistent state (Givens rotations, R(j), the finish test,
// the triangular solve at the end of the cycle).  The Krylov vector v_j handed to the
// preconditioner and the matvec is the once-orthogonalised, unnormalised one;
// (N^{-1} v_j, A N^{-1} v_j) is still an exact matvec pair for the history of Algorithm 2.
// Column j-1 is completed one iteration late, so a cycle runs one matvec past the
// iteration that meets the tolerance, and a cycle that reaches m columns ends with a
// reduction-only step.
//
// Both passes stream the basis with plain 16-byte loads, many in flight per thread: on
// GB300 that moved these column sweeps faster than a TMA tile pipeline with one CTA per SM.
#include "psp_kernels.cuh"

namespace psp {

constexpr double kBreakdownRel = 1e-14;

// L2 eviction-priority policies (PTX createpolicy): the first basis columns of a cycle are
// read by both passes of every iteration, so they are loaded and stored with evict_last and
// stay resident in L2; the other columns stream through with evict_first.
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <typename T> struct Vec;
template <> struct Vec<float> {
  using type = float4;
  static constexpr int W = 4;
  // 16-byte loads and stores with an L2 cache policy (ldnc: read-only for the kernel)
  __device__ static __forceinline__ float4 ldnc(const float4 *p, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
    return v;
  }
  __device__ static __forceinline__ float4 ld(const float4 *p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol) : "memory");
    return v;
  }
  __device__ static __forceinline__ void st(float4 *p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
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
  __device__ static __forceinline__ double2 ldnc(const double2 *p, uint64_t pol) {
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
  }
  __device__ static __forceinline__ double2 ld(const double2 *p, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol) : "memory");
    return v;
  }
  __device__ static __forceinline__ void st(double2 *p, double2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" :: "l"(p), "d"(v.x), "d"(v.y), "l"(pol)
                 : "memory");
  }
  __device__ static __forceinline__ double dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
  __device__ static __forceinline__ double2 axpy(double c, double2 x, double2 y) {
    return make_double2(y.x - c * x.x, y.y - c * x.y);
  }
  __device__ static __forceinline__ double2 scale(double c, double2 x) { return make_double2(c * x.x, c * x.y); }
};

constexpr int kMaxArnCta = 256;   // CTAs of pass A (one per SM)

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
                              bool force_end, int mixed, bool bad = false) {
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
  if (!isfinite(R) || !isfinite(gamma) || bad) status |= kStNumeric;
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

// The inputs from earlier iterations (columns 0..j-2 of the Hessenberg copy into sH, h_{j-1}
// into hf_pre) were staged into shared memory by engine_stage at the start of the kernel.
template <typename T>
__device__ void dcgs_scalar(DevState *st, int j, int final_step, const T *partial, int nb, T *scratch,
                            const double *hf_pre) {
  constexpr int ld = kMaxM + 1;
  T *s_sum = scratch;                                             // 2 kMaxM + 2
  T *sH = s_sum + 2 * kMaxM + 2;                                  // kMaxM * ld
  T *s_a = sH + kMaxM * ld;                                       // kMaxM
  T *s_t = s_a + kMaxM;                                           // kMaxM + 1
  T *s_hcol = s_t + kMaxM + 1;                                    // kMaxM + 2
  T *s_sc = s_hcol + kMaxM + 2;                                   // 4
  T *HcTw = hc_copy<T>(st);
  const int k = j + 1;
  cp_async_wait_all();
  __syncthreads();
  if (j >= 1)
    for (int r = threadIdx.x; r < j; r += blockDim.x) s_hcol[r] = (T)hf_pre[r];
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
      // an overflowed ||w_j|| (a preconditioner whose solve blew up in the Krylov precision)
      // is a numeric failure (dc_brk = 2), not a breakdown that would end the cycle as converged
      const bool bad = !isfinite(nu2) || !isfinite(alpha);
      const bool brk = !bad && !(nu2 > (T)(kBreakdownRel * kBreakdownRel) * alpha);
      s_sc[0] = (brk || bad) ? (T)0 : sqrt(nu2);
      s_sc[2] = ab;
      st->dc_brk = bad ? 2 : (brk ? 1 : 0);
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
  {  // t = Hbar a: 8 lanes per row, each a strided share of the row's terms, then a shuffle sum
    constexpr int LPR = 8;
    const int sub = threadIdx.x % LPR, rows = blockDim.x / LPR;
    for (int rb = 0; rb <= j; rb += rows) {   // the same trip count for every lane of a warp
      const int r = rb + threadIdx.x / LPR;
      T t = (T)0;
      if (r <= j)
        for (int i = (r > 0 ? r - 1 : 0) + sub; i < j; i += LPR)
          t += ((i == j - 1) ? s_hcol[r] : sH[i * ld + r]) * s_a[i];
#pragma unroll
      for (int off = LPR / 2; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (r <= j && sub == 0) s_t[r] = t;
    }
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

// Stage the scalar engine's inputs from earlier iterations (written by earlier launches)
// into shared memory with asynchronous copies: issued by every CTA of pass A right after its
// grid-dependency wait, so that they are in place, at no latency, when the last CTA to
// arrive runs the engine.  Layout as in dcgs_scalar.
template <typename T>
__device__ __forceinline__ void engine_stage(DevState *st, int j, T *scratch, double *hf_pre) {
  constexpr int ld = kMaxM + 1;
  T *sH = scratch + 2 * kMaxM + 2;
  const T *HcT = hc_copy<T>(st);
  for (int e = threadIdx.x; e < (j > 1 ? (j - 1) * ld : 0); e += blockDim.x) cp_async_elem(sH + e, HcT + e);
  if (j >= 1)
    for (int r = threadIdx.x; r < j; r += blockDim.x) cp_async_elem(hf_pre + r, st->Hf + (int64_t)(j - 1) * ld + r);
  asm volatile("cp.async.commit_group;" ::: "memory");
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
    const bool bad = st->dc_brk == 2;
    const bool brk = st->dc_brk == 1;
    bool end = false;
    if (j >= 1) {
      end = givens_column(st, j - 1, s_hcol, sC, sS, sG, brk, final_step != 0, mixed, bad);
    } else if (bad) {
      end = true;   // ||v_0|| overflowed
      st->status |= kStNumeric;
      st->sum.status = st->status;
      st->k_end = 0;
      st->sum.k_end = 0;
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
// pass A: one CTA per SM, two 16-byte vectors per thread and row round (the folded matvec
// makes w_j for them first), basis columns in chunks of 8 with the index clamped to j; a
// chunk's 16 sums (a_i and b_i of 8 columns) are reduced across the warp by a butterfly
// and added to the warp's row of s_acc; the CTA's totals go to partial[row][cta].
// ---------------------------------------------------------------------------------------
constexpr int kDotThreads = 512;
constexpr int kDotWarps = kDotThreads / 32;
constexpr int kAccLd = 2 * kMaxM + 2;

// v[16] lane-local -> lane l returns the warp total of value (l >> 1) & 15
template <typename T>
__device__ __forceinline__ T warp_reduce16(T (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int h = 8 >> s, off = 16 >> s;
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (i < h) {
        const T send = up ? v[i] : v[i + h];
        const T keep = up ? v[i + h] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// w = A x at vector iv (W points along x) with the centre vector of x.
template <typename T, int NDIM, int R>
__device__ __forceinline__ void matvec_vec(const T *__restrict__ x, const T (*c)[2 * kMaxR + 1], int iv, int nx,
                                           int ny, int nz, typename Vec<T>::type &wout,
                                           typename Vec<T>::type &centre) {
  using VT = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  constexpr int NH = (R + W - 1) / W;
  constexpr int NY = NDIM >= 2 ? R : 0, NZ = NDIM >= 3 ? R : 0;
  const int nxv = nx / W, plane = nx * ny;
  const int row = iv / nxv;
  const int xv = iv - row * nxv;
  const int iz = row / ny;
  const int iy = row - iz * ny;
  const int base = row * nx;
  VT win[2 * NH + 1], ym[NY > 0 ? NY : 1], yp[NY > 0 ? NY : 1], zm[NZ > 0 ? NZ : 1], zp[NZ > 0 ? NZ : 1];
#pragma unroll
  for (int h = -NH; h <= NH; ++h) {
    int v = xv + h;
    v += (v < 0) ? nxv : 0;
    v -= (v >= nxv) ? nxv : 0;
    win[h + NH] = *reinterpret_cast<const VT *>(x + base + v * W);
  }
#pragma unroll
  for (int jj = 1; jj <= NY; ++jj) {
    int m = iy - jj; m += (m < 0) ? ny : 0;
    int p = iy + jj; p -= (p >= ny) ? ny : 0;
    ym[jj - 1] = *reinterpret_cast<const VT *>(x + iz * plane + m * nx + xv * W);
    yp[jj - 1] = *reinterpret_cast<const VT *>(x + iz * plane + p * nx + xv * W);
  }
#pragma unroll
  for (int jj = 1; jj <= NZ; ++jj) {
    int m = iz - jj; m += (m < 0) ? nz : 0;
    int p = iz + jj; p -= (p >= nz) ? nz : 0;
    zm[jj - 1] = *reinterpret_cast<const VT *>(x + m * plane + iy * nx + xv * W);
    zp[jj - 1] = *reinterpret_cast<const VT *>(x + p * plane + iy * nx + xv * W);
  }
  const T *wn = reinterpret_cast<const T *>(&win[0]);
  T acc[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    T s = c[0][kMaxR] * wn[NH * W + i];
#pragma unroll
    for (int jj = 1; jj <= R; ++jj) {
      s = fma(c[0][kMaxR - jj], wn[NH * W + i - jj], s);
      s = fma(c[0][kMaxR + jj], wn[NH * W + i + jj], s);
    }
    acc[i] = s;
  }
#pragma unroll
  for (int jj = 1; jj <= NY; ++jj) {
    const T *me = reinterpret_cast<const T *>(&ym[jj - 1]), *pe = reinterpret_cast<const T *>(&yp[jj - 1]);
#pragma unroll
    for (int i = 0; i < W; ++i) acc[i] = fma(c[1][kMaxR + jj], pe[i], fma(c[1][kMaxR - jj], me[i], acc[i]));
  }
#pragma unroll
  for (int jj = 1; jj <= NZ; ++jj) {
    const T *me = reinterpret_cast<const T *>(&zm[jj - 1]), *pe = reinterpret_cast<const T *>(&zp[jj - 1]);
#pragma unroll
    for (int i = 0; i < W; ++i) acc[i] = fma(c[2][kMaxR + jj], pe[i], fma(c[2][kMaxR - jj], me[i], acc[i]));
  }
  T *oe = reinterpret_cast<T *>(&wout);
#pragma unroll
  for (int i = 0; i < W; ++i) oe[i] = acc[i];
  centre = win[NH];
}

template <typename T, int MV>
__global__ void __launch_bounds__(kDotThreads, 1) k_dcgs_dots(const T *__restrict__ V, int64_t ldv,
                                                                const T *__restrict__ Pyb, int64_t ldh, int j,
                                                                int woff, DevState *st, T *partial, int64_t nv,
                                                                int final_step, const TileMatvec<T> mv, int hot) {
  // launch self-check: the engine's cross-CTA sums cover at most kMaxArnCta CTAs and the
  // partial rows kMaxCta; a larger grid records a device error instead of reading past them
  if (gridDim.x > kMaxArnCta || gridDim.x > kMaxCta || blockDim.x != kDotThreads) {
    if (threadIdx.x == 0) atomicExch(&st->error, 3);
    return;
  }
  using VT = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  extern __shared__ __align__(16) double dsm[];
  __shared__ T s_acc[kDotWarps][kAccLd];
  __shared__ T s_c[3][2 * kMaxR + 1];
  __shared__ double s_hfpre[kMaxM + 1];
  for (int e = threadIdx.x; e < kDotWarps * kAccLd; e += blockDim.x) (&s_acc[0][0])[e] = (T)0;
  // launched as a programmatic dependent of the previous kernel (pass B of the last
  // iteration): nothing it writes is read before this wait
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the state this pass needs is read in one batch of independent loads (the active flag,
  // the ring positions, the stencil coefficients) before anything waits on one of them
  const int active = st->active;
  int64_t nvg = nv;   // vectors inside the grid (the rest of the column is zero padding)
  const T *xin = nullptr;
  VT *wout = nullptr, *xcp = nullptr;
  const VT *wp = nullptr;
  if constexpr (MV != 0) {
    nvg = (int64_t)mv.nx * mv.ny * mv.nz / W;
    xin = mv.x.get();
    wout = reinterpret_cast<VT *>(mv.w.get());
    xcp = mv.xcopy.base ? reinterpret_cast<VT *>(mv.xcopy.get()) : nullptr;
    if (threadIdx.x < 3 * (2 * kMaxR + 1))
      s_c[threadIdx.x / (2 * kMaxR + 1)][threadIdx.x % (2 * kMaxR + 1)] =
          (T)st->coef[threadIdx.x / (2 * kMaxR + 1)][threadIdx.x % (2 * kMaxR + 1)];
  } else {
    wp = reinterpret_cast<const VT *>(Pyb + (int64_t)((st->hist_base + woff) % st->mmax) * ldh);
  }
  if (active) engine_stage<T>(st, j, reinterpret_cast<T *>(dsm), s_hfpre);
  __syncthreads();
  if (active == 0) return;
  const int k = j + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const VT *vjp = reinterpret_cast<const VT *>(V + (int64_t)j * ldv);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t iters = (nv + 2 * stride - 1) / (2 * stride);
  // columns below `hot` stay resident in L2 between the passes and iterations
  const uint64_t pol_last = l2_evict_last(), pol_first = l2_evict_first();
  const uint64_t pol_j = j < hot ? pol_last : pol_first;
  for (int64_t it = 0; it < iters; ++it) {
    const int64_t i0 = it * 2 * stride + blockIdx.x * (int64_t)blockDim.x + threadIdx.x, i1 = i0 + stride;
    const bool ok0 = i0 < nv, ok1 = i1 < nv;
    VT v0{}, v1{}, w0{}, w1{};
    if constexpr (MV != 0) {
      VT c0{}, c1{};
      if (i0 < nvg) matvec_vec<T, MV / 8, MV % 8>(xin, s_c, (int)i0, mv.nx, mv.ny, mv.nz, w0, c0);
      if (i1 < nvg) matvec_vec<T, MV / 8, MV % 8>(xin, s_c, (int)i1, mv.nx, mv.ny, mv.nz, w1, c1);
      // w_j is read again by pass B; the P_x copy only by the next fit: it streams out with
      // evict_first instead of displacing basis lines pass B re-reads
      if (i0 < nvg) { wout[i0] = w0; if (xcp) Vec<T>::st(xcp + i0, c0, pol_first); }
      if (i1 < nvg) { wout[i1] = w1; if (xcp) Vec<T>::st(xcp + i1, c1, pol_first); }
      if (xcp) { v0 = c0; v1 = c1; }
      else {
        if (ok0) v0 = Vec<T>::ldnc(vjp + i0, pol_j);
        if (ok1) v1 = Vec<T>::ldnc(vjp + i1, pol_j);
      }
    } else {
      if (ok0) { v0 = Vec<T>::ldnc(vjp + i0, pol_j); if (!final_step) w0 = wp[i0]; }
      if (ok1) { v1 = Vec<T>::ldnc(vjp + i1, pol_j); if (!final_step) w1 = wp[i1]; }
    }
    for (int c0 = 0; c0 < k; c0 += 8) {
      VT a0[8], a1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = min(c0 + u, j);
        const VT *qc = reinterpret_cast<const VT *>(V + (int64_t)col * ldv);
        const uint64_t pol = col < hot ? pol_last : pol_first;
        a0[u] = ok0 ? Vec<T>::ldnc(qc + i0, pol) : VT{};
        a1[u] = ok1 ? Vec<T>::ldnc(qc + i1, pol) : VT{};
      }
      T val[16];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        val[u] = Vec<T>::dot(a0[u], v0) + Vec<T>::dot(a1[u], v1);
        val[8 + u] = Vec<T>::dot(a0[u], w0) + Vec<T>::dot(a1[u], w1);
      }
      const T tot = warp_reduce16(val);
      if ((lane & 1) == 0) {
        const int idx = (lane >> 1) & 15;
        const int col = c0 + (idx & 7);
        if (col <= j) s_acc[wid][(idx >> 3) * (kMaxM + 1) + col] += tot;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * k; t += blockDim.x) {
    const int half = t < k ? 0 : 1, i = t - half * k;
    T s = (T)0;
#pragma unroll 4
    for (int g = 0; g < kDotWarps; ++g) s += s_acc[g][half * (kMaxM + 1) + i];
    partial[(int64_t)t * kMaxCta + blockIdx.x] = s;
  }
  if (!last_block_arrive(&st->counter[1])) {
    cp_async_wait_all();   // no copies left in flight when the CTA exits
    return;
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  dcgs_scalar<T>(st, j, final_step, partial, gridDim.x, reinterpret_cast<T *>(dsm), s_hfpre);
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
__global__ void __launch_bounds__(kUpdThreads, 4) k_dcgs_update(T *__restrict__ V, int64_t ldv, const T *__restrict__ Pyb,
                                                             int64_t ldh, int j, int woff, DevState *st, int64_t nv,
                                                             int final_step, int mixed, int hot) {
  // Launched as a programmatic dependent of pass A: the CTAs may be scheduled while pass
  // A's last CTA still forms the coefficients, and wait here for that grid to finish.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the next pass A (a programmatic dependent of this grid) may be scheduled onto SMs as
  // this grid's CTAs retire; it waits for this grid's completion before reading its data
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(16) double dsm[];
  // block 0 is the Givens CTA: the first block is scheduled first, so it runs alongside the
  // streaming CTAs instead of waiting for a free slot after them
  if (blockIdx.x == 0) {
    if (st->active == 0) return;   // the cycle ended: nothing to do
    dcgs_givens(st, j, final_step, mixed, dsm);
    return;
  }
  using VT = typename Vec<T>::type;
  __shared__ T s_sa[kMaxM], s_sd[kMaxM];
  // the active flag, the coefficients and the ring position in one batch of independent loads
  const int active = st->active;
  const T *cA = coef_copy<T>(st, 0), *cD = coef_copy<T>(st, 1), *c3 = coef_copy<T>(st, 2);
  for (int i = threadIdx.x; i < kMaxM; i += blockDim.x) {
    s_sa[i] = (i < j) ? cA[i] : (T)0;
    s_sd[i] = (i < j) ? cD[i] : (T)0;
  }
  const T sv = c3[0], cv = c3[1], sw = c3[2];
  const VT *w = reinterpret_cast<const VT *>(Pyb + (int64_t)((st->hist_base + woff) % st->mmax) * ldh);
  __syncthreads();
  if (active == 0) return;   // the cycle ended: nothing to do
  VT *vj = reinterpret_cast<VT *>(V + (int64_t)j * ldv);
  VT *vn = reinterpret_cast<VT *>(V + (int64_t)(j + 1) * ldv);
  const int64_t stride = (int64_t)(gridDim.x - 1) * blockDim.x;   // streaming CTAs
  // columns below `hot` stay resident in L2 (as in pass A); v_j and v_{j+1} are stored with
  // the policy of their column, the others are read with evict_first
  const uint64_t pol_last = l2_evict_last(), pol_first = l2_evict_first();
  const uint64_t pol_j = j < hot ? pol_last : pol_first;
  const uint64_t pol_n = j + 1 < hot ? pol_last : pol_first;
  for (int64_t iv = (blockIdx.x - 1) * (int64_t)blockDim.x + threadIdx.x; iv < nv; iv += 2 * stride) {
    const int64_t iv2 = iv + stride;
    const bool two = iv2 < nv;
    const int64_t jv2 = two ? iv2 : iv;
    const VT v0 = Vec<T>::ld(vj + iv, pol_j), v1 = Vec<T>::ld(vj + jv2, pol_j);
    const VT x0 = w[iv], x1 = w[jv2];
    VT q0 = Vec<T>::scale(sv, v0), q1 = Vec<T>::scale(sv, v1);
    VT y0 = Vec<T>::axpy(cv, v0, Vec<T>::scale(sw, x0)), y1 = Vec<T>::axpy(cv, v1, Vec<T>::scale(sw, x1));
    for (int c0 = 0; c0 < j; c0 += 8) {
      VT a0[8], a1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int col = min(c0 + u, j - 1);
        const VT *qc = reinterpret_cast<const VT *>(V + (int64_t)col * ldv);
        // columns below j are not written by this grid: read-only loads
        const uint64_t pol = col < hot ? pol_last : pol_first;
        a0[u] = Vec<T>::ldnc(qc + iv, pol);
        a1[u] = Vec<T>::ldnc(qc + jv2, pol);
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
    Vec<T>::st(vj + iv, q0, pol_j);
    Vec<T>::st(vn + iv, y0, pol_n);
    if (two) {
      Vec<T>::st(vj + iv2, q1, pol_j);
      Vec<T>::st(vn + iv2, y1, pol_n);
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

// Basis columns kept resident in L2 across the two passes and the iterations of a cycle:
// as many as fit in PSP_L2_HOT_FRACTION of the L2 (the rest of it serves the streamed
// columns, the matvec and the other kernels of the step).
#ifndef PSP_L2_HOT_FRACTION
#define PSP_L2_HOT_FRACTION 0.4
#endif
int l2_hot_columns(int64_t col_bytes) {
  static const int64_t l2 = [] {
    int dev = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, dev);
    return (int64_t)b;
  }();
  if (col_bytes <= 0) return 0;
  return (int)std::min<int64_t>(kMaxM + 1, (int64_t)(PSP_L2_HOT_FRACTION * (double)l2) / col_bytes);
}

int arnoldi_grid() {
  static const int g = [] {   // thread-safe one-time initialisation
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? std::min(sms, kMaxArnCta) : 152;
  }();
  return g;
}

// Opt the passes in to their shared memory (once, outside capture): pass A keeps its
// per-warp sums statically and the scalar engine's scratch dynamically, pass B's Givens CTA
// its scratch dynamically.
template <typename T>
static void set_attrs_t() {
#define PSP_ATTR(MV_) \
  cudaFuncSetAttribute(k_dcgs_dots<T, MV_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kScalarDoubles * sizeof(double)));
  PSP_ATTR(0) PSP_ATTR(9) PSP_ATTR(10) PSP_ATTR(11) PSP_ATTR(12) PSP_ATTR(13) PSP_ATTR(17) PSP_ATTR(18) PSP_ATTR(19)
  PSP_ATTR(20) PSP_ATTR(21) PSP_ATTR(25) PSP_ATTR(26) PSP_ATTR(27) PSP_ATTR(28) PSP_ATTR(29)
#undef PSP_ATTR
  cudaFuncSetAttribute(k_dcgs_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kGivensDoubles * sizeof(double)));
}

void arnoldi_setup() {
  arnoldi_grid();
  l2_hot_columns(1);
  set_attrs_t<float>();
  set_attrs_t<double>();
}

template <typename T>
void launch_arnoldi(int j, int final_step, int64_t n, T *V, int64_t ldv, const T *Py, int64_t ldh, DevState *st,
                    double *partial, int mixed, cudaStream_t s, cudaEvent_t *ev, const TileMatvec<T> *mv) {
  const TileMatvec<T> m = mv ? *mv : TileMatvec<T>{};
  const int hot = l2_hot_columns(ldv * (int64_t)sizeof(T));
  const int woff = 1 + j;   // ring column of w_j relative to the cycle's restart column
  const int64_t nv = (ldv + Vec<T>::W - 1) / Vec<T>::W;
  {
    // one CTA per SM at most, and no more CTAs than two vectors per thread need: a small
    // system leaves the other SMs to the work on other streams (and the engine sums fewer
    // partials)
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(arnoldi_grid(), (nv + 2 * kDotThreads - 1) / (2 * kDotThreads)));
    const size_t sm = (size_t)kScalarDoubles * sizeof(double);
    // the folded matvec is instantiated per dimension and stencil radius: 8 ndim + R
    const int sel = (mv && !final_step) ? 8 * m.ndim + m.R : 0;
    T *pt = reinterpret_cast<T *>(partial);
    // a programmatic dependent of the previous kernel (see k_dcgs_dots and k_dcgs_update)
    cudaLaunchConfig_t cfa = {};
    cfa.gridDim = dim3((unsigned)grid);
    cfa.blockDim = dim3(kDotThreads);
    cfa.dynamicSmemBytes = sm;
    cfa.stream = s;
    cudaLaunchAttribute ata[1];
    ata[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    ata[0].val.programmaticStreamSerializationAllowed = 1;
    cfa.attrs = ata;
    cfa.numAttrs = 1;
    switch (sel) {
#define PSP_DOTS(MV_) \
  case MV_: cudaLaunchKernelEx(&cfa, k_dcgs_dots<T, MV_>, (const T *)V, ldv, Py, ldh, j, woff, st, pt, nv, final_step, m, hot); break;
      PSP_DOTS(0) PSP_DOTS(9) PSP_DOTS(10) PSP_DOTS(11) PSP_DOTS(12) PSP_DOTS(13) PSP_DOTS(17) PSP_DOTS(18)
      PSP_DOTS(19) PSP_DOTS(20) PSP_DOTS(21) PSP_DOTS(25) PSP_DOTS(26) PSP_DOTS(27) PSP_DOTS(28) PSP_DOTS(29)
#undef PSP_DOTS
      default: break;
    }
  }
  if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);
  if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);
  {
    // one CTA for the Givens step plus the streaming CTAs (none for the final step), all in
    // one wave of four CTAs per SM, launched as a programmatic dependent of pass A
    int ugrid = final_step ? 0 : (int)std::min<int64_t>((nv + kUpdThreads - 1) / kUpdThreads, (int64_t)arnoldi_grid() * 4 - 1);
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
    cudaLaunchKernelEx(&cfg, k_dcgs_update<T>, V, ldv, Py, ldh, j, woff, st, nv, final_step, mixed, hot);
  }
  if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);
}

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

template void launch_arnoldi<float>(int, int, int64_t, float *, int64_t, const float *, int64_t, DevState *, double *,
                                    int, cudaStream_t, cudaEvent_t *, const TileMatvec<float> *);
template void launch_arnoldi<double>(int, int, int64_t, double *, int64_t, const double *, int64_t, DevState *,
                                     double *, int, cudaStream_t, cudaEvent_t *, const TileMatvec<double> *);

bool fused_matvec_ok(const Geometry &g, int elem_bytes) {
  const int W = 16 / elem_bytes;
  const int nh = (g.R + W - 1) / W;
  // FP32 3D grids fold the matvec too (each vector gathers its 4R+2NH+1 neighbour vectors
  // from L2, under pass A's stream: measured faster on the 256^3 workload than the z-marching
  // stencil kernel, which needs its own pass over v and w); the FP64 form, bound by the FP64
  // pipe, keeps the z-marching kernel on the grids it takes
  if (g.ndim == 3 && elem_bytes == 8 && stencil_3d_tiled(g, elem_bytes)) return false;
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
