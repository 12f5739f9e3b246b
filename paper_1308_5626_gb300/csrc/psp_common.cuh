// Internal definitions shared by the libpsp translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/psp.h"

namespace psp {

constexpr int kMaxM = 64;         // largest restart length
constexpr int kMaxR = 5;          // largest stencil radius (k <= 4, order <= 8)
constexpr int kMaxB = 4;          // largest band half-width
constexpr int kThreads = 256;     // block size of the vector kernels
constexpr int kMaxCta = 1216;     // cap on CTAs of the reduction kernels (8 per SM)

// Bits of DevState::status
constexpr int kStConverged = 1;
constexpr int kStBreakdown = 2;
constexpr int kStNumeric = 4;

// What the host reads after every restart cycle (one small device-to-host copy).
struct CycleSummary {
  int k_end;         // Arnoldi iterations completed in the cycle
  int status;        // kSt* bits
  int hist_count;    // history columns written since the history was cleared
  int error;         // internal error flag
  double beta;       // ||B - A X_0|| at the start of the cycle (FP64 true residual)
  double R_end;      // R(k_end) (beta if k_end == 0)
  double bnorm;      // ||B||
  double pad;
};

// Device-resident solver state.  Everything a captured cycle needs that changes from
// launch to launch lives here, so the CUDA graphs keep fixed kernel parameters.
struct DevState {
  CycleSummary sum;  // first member: copied to the host after every cycle
  // cycle control
  int active;        // 1 while the current restart cycle runs
  int k_end;         // Arnoldi iterations completed in the current cycle
  int status;        // kSt* bits of the current cycle
  int hist_count;    // history columns written since the history was cleared
  int hist_base;     // ring column of the current cycle's restart pair (X_0, A X_0)
  int mmax;          // history ring length
  int m;             // restart length
  int restart_df;    // 1: the mixed form's restart runs in double-float (k_restart_df), else FP64
  int pad1;
  double beta;       // ||B - A X_0|| at the start of the cycle
  double eps_abs;    // step bound on R(k): tol * ||B||
  double eps_cycle;  // cycle bound on R(k): eps_abs (FP64) or max(eps_abs, inner*beta)
  double inner_tol;
  double tol;        // relative tolerance of the step
  double bnorm;      // ||B||
  double unorm2;     // ||U_k||^2 before orthogonalisation (breakdown test)
  // Arnoldi / Givens (FP64, Algorithm 1)
  double sigma[kMaxM + 2];            // V(:,j) = sigma[j] * Vt(:,j) (lazy normalisation)
  double H[(kMaxM + 1) * kMaxM];      // rotated Hessenberg, column-major (ld = kMaxM+1)
  double Hf[(kMaxM + 1) * kMaxM];     // first projection of each column (DCGS2)
  double Hc[(kMaxM + 1) * kMaxM];     // completed, unrotated columns (DCGS2)
  double G[kMaxM + 1];
  double C[kMaxM];
  double S[kMaxM];
  double Q[kMaxM];
  double h1[kMaxM + 1];               // first Gram-Schmidt projection coefficients
  double h2[kMaxM + 1];               // second (re-orthogonalisation) coefficients
  double R[kMaxM];                    // R(k) of the current cycle
  double cA[kMaxM];                   // DCGS2 update coefficients of the current iteration
  double cD[kMaxM];
  double c3[4];
  float HcF[(kMaxM + 1) * kMaxM];     // FP32 copies for the mixed form's scalar engine
  float cAF[kMaxM];
  float cDF[kMaxM];
  float c3F[4];
  int dc_brk;                         // this iteration's scalar engine saw 1: a breakdown, 2: an overflowed norm
  int pad2;
  // stencil coefficients of A = I - dt L for the current dt: coef[d][j + kMaxR]
  double coef[3][2 * kMaxR + 1];
  // last-block counters of the grid reductions
  unsigned int counter[8];
  int error;         // internal error flag (0 = none)
  int first;         // 1 before the first restart of a step (sets ||B|| and eps_abs)
  // BiCGSTAB scalars (rho, alpha, omega, beta, sigma = 1/||r||, ||r||^2), 1/sigma of the
  // previous iteration, and the rh . v = 0 breakdown flag
  double bi[6];
  double bi_isig_prev;
  int bi_flag;
  int bi_pad;
};

// Column `col` of a ring of `mmax` columns of length ld.
template <typename T>
__device__ __forceinline__ T *ring_col(T *base, int64_t ld, int col, int mmax) {
  return base + (int64_t)(col % mmax) * ld;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Signal that this CTA finished writing its partials; returns true in the last CTA.
// Standard "last block" pattern: fence, count, the last arriving CTA reduces.  No
// thread waits for another CTA.
// The barrier makes every thread's writes visible to thread 0, whose GPU-scope fence then
// releases them (fences are cumulative) before its arrival is counted.
__device__ __forceinline__ bool last_block_arrive(unsigned int *counter) {
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
    if (s_last) __threadfence();
  }
  __syncthreads();
  return s_last;
}

__device__ __forceinline__ void last_block_reset(unsigned int *counter) {
  if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace psp
