// The on-chip step (internal): one CTA runs every restart cycle of one implicit step of a
// system small enough for it, and one launch runs many such systems (see onchip.cu).
#pragma once

#include "psp_kernels.cuh"

namespace psp {

// What one launch did for one system: its cycles and the summary of the last one.
struct OnChipResult {
  int cycles;         // restart cycles run (a restart that finds the step converged counts)
  int iters;          // Arnoldi iterations of those cycles
  int status;         // kSt* bits of the last cycle
  int k_last;         // iterations of the last cycle
  int first_k;        // iterations of the first cycle
  int error;          // device error flag (a misconfigured launch)
  int hist_count;     // history columns written since the history was cleared, after the launch
  double first_beta;  // ||B - A X_0|| at the start of the first cycle
  double last_beta;   // ... of the last cycle
  double last_R;      // R(k_last) of the last cycle (its beta if k_last == 0)
  double bnorm;       // ||B||
  unsigned long long t_begin, t_end;   // device clock (%globaltimer, ns) around the system's cycles
};

// One system of an on-chip launch (device memory).  The vectors, history ring and state are
// the handle's own workspace; the preconditioner is the LevelApply array of one factor slot
// (nullptr: N = I).
struct OnChipDesc {
  int ndim, nx, ny, nz, R, n;
  int band_w, b;              // explicit banded operator (band_w > 0); band half-width of N
  const double *Ab;
  const float *Ab32;
  double *X;
  const double *Bv;
  void *V, *Px, *Py, *Z;      // Krylov precision
  int64_t ld;
  int m, mmax;
  DevState *st;               // coefficients, history position, ||B|| / eps, last cycle's R(k)
  const void *lev;            // LevelApply<T>[nlev] of the slot, or nullptr
  int nlev, cyclic;
  const void *smwZ, *smwK;    // cyclic band: Z (n x 2b) and K^{-1} (2b x 2b) in the Krylov precision
  void *tmp;                  // n values: the banded part of a cyclic solve
  int max_cycles;             // cycles this launch may run (1 for a candidate's trial cycle)
  int cache_bytes;            // > 0: the slot's factor blocks are staged in this much dynamic
                              // shared memory once per launch (a single small system)
  OnChipResult *res;
};

// Dynamic shared memory the factor cache of a slot needs (0 if the slot does not fit
// kOnChipCacheMax): every factor array of every level, each rounded up to 16 bytes.
constexpr int kOnChipCacheMax = 160 * 1024;

// Largest system of the on-chip path, and the largest that takes it by default (opts.onchip
// = -1) when stepped on its own: below it a step's cycle graphs are bound by launch latency.
constexpr int kOnChipMaxN = 1 << 18;
constexpr int kOnChipAutoN = 1 << 15;
constexpr int kOnChipMaxThreads = 512;   // CTA size limit (the kernel's register budget)
bool onchip_threads_ok(int threads);
// CTA size for one system of n unknowns stepped on its own (about four rows per thread,
// 128 to kOnChipMaxThreads threads).
inline int onchip_threads_for(int64_t n) {
  const int64_t t = ((n / 4 + 31) / 32) * 32;
  return (int)(t < 128 ? 128 : (t > kOnChipMaxThreads ? kOnChipMaxThreads : t));
}
// Run the cycles of descs[0..count) (T = float: the mixed form, double: FP64), `grid` CTAs of
// `threads` threads taking systems from *counter (reset by the launcher).
template <typename T>
void launch_onchip(const OnChipDesc *descs, int count, int *counter, int threads, int grid, cudaStream_t s,
                   int cache_bytes = 0);

}  // namespace psp
