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

constexpr int kArnThreads = 512;                 // one CTA of 16 warps per SM
constexpr int kArnWarps = kArnThreads / 32;
constexpr int kMaxArnCta = 256;

// Sum NV per-thread values over the CTA; thread j < nvals writes partial[j*kMaxCta + cta].
template <typename T, int NV>
__device__ __forceinline__ void cta_partials(const T (&acc)[NV], int nvals, double *partial) {
  __shared__ double s_red[kArnWarps][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    if (j < nvals) {
      T v = warp_sum(acc[j]);
      if (lane == 0) s_red[wid][j] = (double)v;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nvals; j += blockDim.x) {
    double a = 0.0;
#pragma unroll
    for (int w = 0; w < kArnWarps; ++w) a += s_red[w][j];
    partial[(int64_t)j * kMaxCta + blockIdx.x] = a;
  }
}

// In the last CTA: out[j] = sum over CTAs of partial[j][cta] in a fixed order, j < nvals.
// Every load is issued before any add (warp w takes j = w, w + 16, ...; lane l takes CTAs
// l, l + 32, ...).
__device__ __forceinline__ void grid_sums(const double *partial, int nvals, double *out) {
  constexpr int MJ = (kMaxM + 2 + kArnWarps - 1) / kArnWarps;
  constexpr int MB = kMaxArnCta / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = gridDim.x;
  double a[MJ];
#pragma unroll
  for (int t = 0; t < MJ; ++t) {
    const int j = wid + t * kArnWarps;
    double s = 0.0;
    if (j < nvals) {
      const double *p = partial + (int64_t)j * kMaxCta;
#pragma unroll
      for (int q = 0; q < MB; ++q) {
        const int b = lane + 32 * q;
        if (b < nb) s += p[b];
      }
    }
    a[t] = s;
  }
#pragma unroll
  for (int t = 0; t < MJ; ++t) {
    const double s = warp_sum(a[t]);
    const int j = wid + t * kArnWarps;
    if (lane == 0 && j < nvals) out[j] = s;
  }
  __syncthreads();
}

template <typename T, int KC>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass1(const T *__restrict__ V, int64_t ldv, int k,
                                                           const T *__restrict__ Pyb, int64_t ldh, DevState *st,
                                                           double *partial, int64_t nv) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  const VT *U = reinterpret_cast<const VT *>(ring_col(Pyb, ldh, st->hist_count, st->mmax));
  T acc[KC + 1];
#pragma unroll
  for (int j = 0; j <= KC; ++j) acc[j] = (T)0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t iv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; iv < nv; iv += 2 * stride) {
    const int64_t iv2 = iv + stride;
    const bool two = iv2 < nv;
    const VT u0 = U[iv];
    const VT u1 = two ? U[iv2] : VT{};
    acc[KC] += Vec<T>::dot(u0, u0) + Vec<T>::dot(u1, u1);
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j < k) {
        const VT *vj = reinterpret_cast<const VT *>(V + j * ldv);
        const VT v0 = vj[iv];
        const VT v1 = two ? vj[iv2] : VT{};
        acc[j] += Vec<T>::dot(v0, u0) + Vec<T>::dot(v1, u1);
      }
    }
  }
  // slot k carries ||U||^2
  T acc2[KC + 1];
#pragma unroll
  for (int j = 0; j <= KC; ++j) acc2[j] = (j < k) ? acc[j] : ((j == k) ? acc[KC] : (T)0);
  cta_partials<T, KC + 1>(acc2, k + 1, partial);
  if (!last_block_arrive(&st->counter[1])) return;
  __shared__ double s_sum[kMaxM + 2];
  grid_sums(partial, k + 1, s_sum);
  for (int j = threadIdx.x; j <= k; j += blockDim.x) {
    if (j < k) st->h1[j] = st->sigma[j] * s_sum[j];
    else st->unorm2 = s_sum[k];
  }
  last_block_reset(&st->counter[1]);
}

template <typename T, int KC>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass2(const T *__restrict__ V, int64_t ldv, int k,
                                                           const T *__restrict__ Pyb, int64_t ldh, DevState *st,
                                                           double *partial, int64_t nv) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  __shared__ T s_c[KC];
  for (int j = threadIdx.x; j < KC; j += blockDim.x) s_c[j] = (j < k) ? (T)(st->h1[j] * st->sigma[j]) : (T)0;
  __syncthreads();
  const VT *U = reinterpret_cast<const VT *>(ring_col(Pyb, ldh, st->hist_count, st->mmax));
  T acc[KC];
#pragma unroll
  for (int j = 0; j < KC; ++j) acc[j] = (T)0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t iv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; iv < nv; iv += 2 * stride) {
    const int64_t iv2 = iv + stride;
    const bool two = iv2 < nv;
    VT u0 = U[iv];
    VT u1 = two ? U[iv2] : VT{};
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j < k) {
        const VT *vj = reinterpret_cast<const VT *>(V + j * ldv);
        u0 = Vec<T>::axpy(s_c[j], vj[iv], u0);
        if (two) u1 = Vec<T>::axpy(s_c[j], vj[iv2], u1);
      }
    }
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j < k) {
        const VT *vj = reinterpret_cast<const VT *>(V + j * ldv);
        acc[j] += Vec<T>::dot(Vec<T>::reload(vj + iv), u0) + (two ? Vec<T>::dot(Vec<T>::reload(vj + iv2), u1) : (T)0);
      }
    }
  }
  cta_partials<T, KC>(acc, k, partial);
  if (!last_block_arrive(&st->counter[2])) return;
  __shared__ double s_sum[kMaxM + 2];
  grid_sums(partial, k, s_sum);
  for (int j = threadIdx.x; j < k; j += blockDim.x) st->h2[j] = st->sigma[j] * s_sum[j];
  last_block_reset(&st->counter[2]);
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
  st->sum.status = status;
  st->sum.hist_count = st->hist_count;
  st->sum.R_end = R;
}

template <typename T, int KC>
__global__ void __launch_bounds__(kArnThreads) k_cgs_pass3(T *__restrict__ V, int64_t ldv, int k,
                                                           const T *__restrict__ Pyb, int64_t ldh, DevState *st,
                                                           double *partial, int64_t nv, int mixed) {
  if (st->active == 0) return;
  using VT = typename Vec<T>::type;
  __shared__ T s_c[KC];
  for (int j = threadIdx.x; j < KC; j += blockDim.x)
    s_c[j] = (j < k) ? (T)((st->h1[j] + st->h2[j]) * st->sigma[j]) : (T)0;
  __syncthreads();
  const VT *U = reinterpret_cast<const VT *>(ring_col(Pyb, ldh, st->hist_count, st->mmax));
  VT *Vout = reinterpret_cast<VT *>(V + (int64_t)k * ldv);
  T acc[1] = {(T)0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t iv = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; iv < nv; iv += 2 * stride) {
    const int64_t iv2 = iv + stride;
    const bool two = iv2 < nv;
    VT u0 = U[iv];
    VT u1 = two ? U[iv2] : VT{};
#pragma unroll
    for (int j = 0; j < KC; ++j) {
      if (j < k) {
        const VT *vj = reinterpret_cast<const VT *>(V + j * ldv);
        u0 = Vec<T>::axpy(s_c[j], vj[iv], u0);
        if (two) u1 = Vec<T>::axpy(s_c[j], vj[iv2], u1);
      }
    }
    Vout[iv] = u0;
    acc[0] += Vec<T>::dot(u0, u0);
    if (two) {
      Vout[iv2] = u1;
      acc[0] += Vec<T>::dot(u1, u1);
    }
  }
  cta_partials<T, 1>(acc, 1, partial);
  if (!last_block_arrive(&st->counter[3])) return;
  __shared__ double s_sum[kMaxM + 2];
  grid_sums(partial, 1, s_sum);
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

template <typename T>
void launch_arnoldi(int k, int64_t n, const T *V, int64_t ldv, const T *Py, int64_t ldh, DevState *st,
                    double *partial, int mixed, cudaStream_t s, cudaEvent_t *ev) {
  const int64_t nv = (n + Vec<T>::W - 1) / Vec<T>::W;
  int grid = (int)std::min<int64_t>((nv + kArnThreads - 1) / kArnThreads, arnoldi_grid());
  if (grid < 1) grid = 1;
#define PSP_CGS(KC_)                                                                                   \
  case KC_ / 4:                                                                                        \
    k_cgs_pass1<T, KC_><<<grid, kArnThreads, 0, s>>>(V, ldv, k, Py, ldh, st, partial, nv);             \
    if (ev) cudaEventRecordWithFlags(ev[0], s, cudaEventRecordExternal);                               \
    k_cgs_pass2<T, KC_><<<grid, kArnThreads, 0, s>>>(V, ldv, k, Py, ldh, st, partial, nv);             \
    if (ev) cudaEventRecordWithFlags(ev[1], s, cudaEventRecordExternal);                               \
    k_cgs_pass3<T, KC_><<<grid, kArnThreads, 0, s>>>(const_cast<T *>(V), ldv, k, Py, ldh, st, partial, \
                                                     nv, mixed);                                       \
    if (ev) cudaEventRecordWithFlags(ev[2], s, cudaEventRecordExternal);                               \
    break;
  switch ((k + 3) / 4) {
    PSP_CGS(4) PSP_CGS(8) PSP_CGS(12) PSP_CGS(16) PSP_CGS(20) PSP_CGS(24) PSP_CGS(28) PSP_CGS(32)
    PSP_CGS(36) PSP_CGS(40) PSP_CGS(44) PSP_CGS(48) PSP_CGS(52) PSP_CGS(56) PSP_CGS(60) PSP_CGS(64)
    default: break;
  }
#undef PSP_CGS
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

template void launch_arnoldi<float>(int, int64_t, const float *, int64_t, const float *, int64_t, DevState *,
                                    double *, int, cudaStream_t, cudaEvent_t *);
template void launch_arnoldi<double>(int, int64_t, const double *, int64_t, const double *, int64_t,
                                     DevState *, double *, int, cudaStream_t, cudaEvent_t *);
template void launch_scale_copy<float>(int, int64_t, const float *, int64_t, OutRef<float>, const DevState *,
                                       cudaStream_t);
template void launch_scale_copy<double>(int, int64_t, const double *, int64_t, OutRef<double>,
                                        const DevState *, cudaStream_t);
template void launch_update_z<float>(int64_t, const float *, int64_t, float *, double *, int, const DevState *,
                                     cudaStream_t);
template void launch_update_z<double>(int64_t, const double *, int64_t, double *, double *, int,
                                      const DevState *, cudaStream_t);

}  // namespace psp
