// Per-group sweeps of the partitioned banded solve (internal): the block-Thomas down sweep
// and the spike up sweep of one group of a level, shared by the level kernels of
// band_solve.cu and the single-CTA solve of the on-chip step.
#pragma once

#include "band_solve.cuh"

namespace psp {

// element e of block i of group g (group-interleaved)
__device__ __forceinline__ int64_t gi(int i, int e, int G, int g, int BB) {
  return ((int64_t)i * BB + e) * G + g;
}

// Factor blocks are read-only during an apply: in global memory (RO) they are read
// through the read-only path, so the loads may be issued ahead of the recurrence that
// consumes them; in the shared-memory tail they are plain loads.
template <bool RO, typename T>
__device__ __forceinline__ T ldf(const T *p) {
  if constexpr (RO) return __ldg(p);
  else return *p;
}

template <typename T, int B, bool RO>
__device__ __forceinline__ void mv_sub(T (&y)[B], const T *M, int i, int G, int g, const T (&x)[B]) {
  T m[B][B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) m[r][c] = ldf<RO>(M + gi(i, r * B + c, G, g, B * B));
#pragma unroll
  for (int r = 0; r < B; ++r) {
    T s = y[r];
#pragma unroll
    for (int c = 0; c < B; ++c) s -= m[r][c] * x[c];
    y[r] = s;
  }
}

template <typename T, int B, bool RO>
__device__ __forceinline__ void mv(T (&y)[B], const T *M, int i, int G, int g, const T (&x)[B]) {
  T m[B][B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) m[r][c] = ldf<RO>(M + gi(i, r * B + c, G, g, B * B));
#pragma unroll
  for (int r = 0; r < B; ++r) {
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < B; ++c) s += m[r][c] * x[c];
    y[r] = s;
  }
}

// Down sweep of group g (Q interior blocks, the level's q), all in registers: f holds the
// right-hand sides of the interior blocks and sep that of the separator block.  Forward
// elimination y_i = f_i - Mul_i y_{i-1}, back substitution x_i = Minv_i (y_i - Up_i x_{i+1})
// (both in place in f); p = x goes to L.p (group-interleaved), and the separator terms of
// the next level to cR, cL and seprhs.
// The factor blocks are read at stride fG and index fg (the level's G and g in global memory,
// or the CTA's group count and the thread's slot when staged in shared memory); the outputs
// always use G and g.
template <typename T, int B, int Q, bool RO>
__device__ __forceinline__ void down_group(const LevelApply<T> &L, int g, T (&f)[Q][B], const T (&sep)[B], int fG,
                                           int fg) {
  const int G = L.G;
#pragma unroll
  for (int i = 1; i < Q; ++i) mv_sub<T, B, RO>(f[i], L.Mul, i, fG, fg, f[i - 1]);
#pragma unroll
  for (int i = Q - 1; i >= 0; --i) {
    if (i < Q - 1) mv_sub<T, B, RO>(f[i], L.Up, i, fG, fg, f[i + 1]);
    T x[B];
    mv<T, B, RO>(x, L.Minv, i, fG, fg, f[i]);
#pragma unroll
    for (int r = 0; r < B; ++r) f[i][r] = x[r];
  }
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int r = 0; r < B; ++r) L.p[gi(i, r, G, g, B)] = f[i][r];
  if (G > 1) {
    if (g < G - 1) {
      T c[B];
      mv<T, B, RO>(c, L.LoSep, 0, fG, fg, f[Q - 1]);
#pragma unroll
      for (int r = 0; r < B; ++r) { L.cR[g * B + r] = -c[r]; L.seprhs[g * B + r] = sep[r]; }
    }
    if (g > 0) {
      T c[B];
      mv<T, B, RO>(c, L.UpSepPrev, 0, fG, fg, f[0]);
#pragma unroll
      for (int r = 0; r < B; ++r) L.cL[g * B + r] = -c[r];
    }
  }
}

// Up sweep of group g: x_i = p_i - W_i sl - V_i sr (independent blocks); out(i, r)
// receives interior block i (i < Q) and the separator block (i == Q, only for g < G-1).
template <typename T, int B, int Q, bool RO, typename Out>
__device__ __forceinline__ void up_group(const LevelApply<T> &L, int g, const T *solnext, Out out, int fG, int fg) {
  const int G = L.G;
  T sl[B], sr[B];
#pragma unroll
  for (int r = 0; r < B; ++r) {
    sl[r] = (g > 0) ? solnext[(g - 1) * B + r] : (T)0;
    sr[r] = (g < G - 1) ? solnext[g * B + r] : (T)0;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    T x[B];
#pragma unroll
    for (int r = 0; r < B; ++r) x[r] = L.p[gi(i, r, G, g, B)];
    if (G > 1) {
      mv_sub<T, B, RO>(x, L.W, i, fG, fg, sl);
      mv_sub<T, B, RO>(x, L.Vs, i, fG, fg, sr);
    }
#pragma unroll
    for (int r = 0; r < B; ++r) out(i, r, x[r]);
  }
  if (g < G - 1) {
#pragma unroll
    for (int r = 0; r < B; ++r) out(Q, r, sr[r]);
  }
}

constexpr int kQ0 = 8;           // interior blocks per group on level 0
constexpr int kQ = 4;            // ... on the levels above

// Level >= 1 down: right-hand side of block j = prev.seprhs[j] + prev.cR[j] + prev.cL[j+1].
template <typename T, int B, bool RO>
__device__ __forceinline__ void down_level_group(const LevelApply<T> &L, const LevelApply<T> &P, int g, int fG,
                                                 int fg) {
  const int G = L.G;
  T f[kQ][B], sep[B];
#pragma unroll
  for (int i = 0; i <= kQ; ++i) {
    const int j = g * (kQ + 1) + i;
    const bool real = (i < kQ) ? (j < L.nb) : (g < G - 1);
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const T v = real ? P.seprhs[j * B + r] + P.cR[j * B + r] + P.cL[(j + 1) * B + r] : (T)0;
      if (i < kQ) f[i][r] = v;
      else sep[r] = v;
    }
  }
  down_group<T, B, kQ, RO>(L, g, f, sep, fG, fg);
}

template <typename T, int B, bool RO>
__device__ __forceinline__ void up_level_group(const LevelApply<T> &L, const T *solnext, int g, int fG, int fg) {
  T *sol = L.sol;
  const int nb = L.nb;
  auto out = [&](int i, int r, T v) {
    const int j = g * (kQ + 1) + i;
    if (j < nb) sol[j * B + r] = v;
  };
  up_group<T, B, kQ, RO>(L, g, solnext, out, fG, fg);
}

}  // namespace psp
