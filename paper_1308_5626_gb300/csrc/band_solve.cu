// The preconditioner solve y = N^{-1} v of Algorithm 1 for the banded N of Algorithm 2.
//
// The paper solves the tridiagonal case (d = 1) with the sequential Thomas algorithm.  On
// a GPU the solve is partitioned instead (nested dissection in one dimension, a
// multi-level form of the SPIKE / cyclic-reduction family):
//
//  * Rows are grouped in blocks of b rows; a matrix of half-bandwidth b is block
//    tridiagonal with b x b blocks (Lo_i, Di_i, Up_i).
//  * A level splits its blocks into groups of q interior blocks followed by one
//    separator block.  Given the separator values, the interiors of different groups
//    are independent: one thread per group runs block Thomas (forward elimination,
//    back substitution) over its q blocks.
//  * Eliminating the interiors leaves a block-tridiagonal Schur system on the separators
//    (b x b blocks again), which is the next level.  Levels recurse until one group is
//    left; the top levels with few blocks run inside one CTA.
//
// Factorisation (once per fitted N, FP64): per group the block-Thomas pivots
// Minv_i = S_i^{-1} and multipliers Mul_i = Lo_i S_{i-1}^{-1}, and the two spikes
// W = T^{-1} [Lo_0; 0..] and V = T^{-1} [0..; Up_{q-1}] (response of the interior to the
// left and right separators); then the separator system Lo', Di', Up' of the next level.
// No pivoting across blocks (within a b x b inverse, partial pivoting); a zero or
// non-finite pivot marks the factorisation as failed.
//
// Apply (per preconditioner solve, FP32 in the mixed form or FP64):
//   down: per group p = T^{-1} f_I, separator right-hand sides f_s - Lo_s p_last - Up_s p_first;
//   up:   x_I = p - W x_{s-1} - V x_s.
// Arrays of a level are stored group-interleaved (element e of block i of group g at
// (i*b*b + e)*G + g) so that the one-thread-per-group sweeps read coalesced.
#include <algorithm>
#include <cmath>
#include <vector>

#include "band_solve.cuh"
#include "band_sweeps.cuh"

namespace psp {

// ---------------------------------------------------------------------------------------
// small dense helpers (b x b, row-major)
// ---------------------------------------------------------------------------------------

template <int B>
__device__ __forceinline__ bool inv_block(const double (&A)[B][B], double (&X)[B][B]) {
  double M[B][2 * B];
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < 2 * B; ++c) M[r][c] = c < B ? A[r][c] : (c - B == r ? 1.0 : 0.0);
  double scale = 0.0;
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) scale = fmax(scale, fabs(A[r][c]));
  bool ok = isfinite(scale) && scale > 0.0;
#pragma unroll
  for (int col = 0; col < B; ++col) {
    int piv = col;
    double best = fabs(M[col][col]);
#pragma unroll
    for (int r = 0; r < B; ++r)
      if (r > col && fabs(M[r][col]) > best) { best = fabs(M[r][col]); piv = r; }
    if (!(best > 1e-13 * scale)) ok = false;
#pragma unroll
    for (int c = 0; c < 2 * B; ++c) {
      double t = M[col][c];
      // swap rows col and piv (piv >= col), written without dynamic indexing
#pragma unroll
      for (int r = 0; r < B; ++r)
        if (r == piv && r != col) { M[col][c] = M[r][c]; M[r][c] = t; }
    }
    const double p = M[col][col];
    const double ip = (p != 0.0) ? 1.0 / p : 0.0;
#pragma unroll
    for (int c = 0; c < 2 * B; ++c) M[col][c] *= ip;
#pragma unroll
    for (int r = 0; r < B; ++r) {
      if (r != col) {
        const double f = M[r][col];
#pragma unroll
        for (int c = 0; c < 2 * B; ++c) M[r][c] -= f * M[col][c];
      }
    }
  }
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      X[r][c] = M[r][B + c];
      if (!isfinite(X[r][c])) ok = false;
    }
  return ok;
}

template <int B>
__device__ __forceinline__ void mm(const double (&A)[B][B], const double (&C)[B][B], double (&X)[B][B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < B; ++l) s += A[r][l] * C[l][c];
      X[r][c] = s;
    }
}

template <int B>
__device__ __forceinline__ void store_blk(double *dst, float *dstf, int i, int G, int g,
                                          const double (&M)[B][B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const int64_t o = gi(i, r * B + c, G, g, B * B);
      dst[o] = M[r][c];
      if (dstf) dstf[o] = (float)M[r][c];
    }
}

template <int B>
__device__ __forceinline__ void load_blk(const double *src, int i, int G, int g, double (&M)[B][B]) {
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) M[r][c] = src[gi(i, r * B + c, G, g, B * B)];
}

// Blocks of the level input.  Level 0 reads the band (rows >= n are identity rows,
// columns outside [0, n) are zero); higher levels read natural-order block arrays.
struct LevelInput {
  const double *band;     // level 0: n x (2b+1) band, else nullptr
  int64_t n;
  const double *bLo, *bDi, *bUp;   // levels >= 1: [blk * b*b + e]
  int nb;
};

template <int B>
__device__ __forceinline__ void input_blocks(const LevelInput &in, int blk, double (&Lo)[B][B],
                                             double (&Di)[B][B], double (&Up)[B][B]) {
  if (in.band) {
    constexpr int W = 2 * B + 1;
#pragma unroll
    for (int r = 0; r < B; ++r) {
      const int64_t row = (int64_t)blk * B + r;
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const int64_t cl = (int64_t)(blk - 1) * B + c, cd = (int64_t)blk * B + c, cu = (int64_t)(blk + 1) * B + c;
        double lo = 0.0, di = 0.0, up = 0.0;
        if (row < in.n) {
          const double *br = in.band + row * W;
          if (cl >= 0 && cl - row >= -B) lo = br[cl - row + B];
          if (cd < in.n && cd - row >= -B && cd - row <= B) di = br[cd - row + B];
          if (cu < in.n && cu - row <= B) up = br[cu - row + B];
        } else {
          di = (r == c) ? 1.0 : 0.0;
        }
        Lo[r][c] = lo; Di[r][c] = di; Up[r][c] = up;
      }
    }
  } else {
    const bool real = blk < in.nb;
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int c = 0; c < B; ++c) {
        const int64_t o = (int64_t)blk * B * B + r * B + c;
        Lo[r][c] = real ? in.bLo[o] : 0.0;
        Up[r][c] = real ? in.bUp[o] : 0.0;
        Di[r][c] = real ? in.bDi[o] : (r == c ? 1.0 : 0.0);
      }
  }
}

// ---------------------------------------------------------------------------------------
// factorisation
// ---------------------------------------------------------------------------------------

template <int B>
__global__ void k_factor_level(LevelInput in, int q, int G, LevelF64 f, LevelF32 h, int *fail) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  double Lo[B][B], Di[B][B], Up[B][B], Minv[B][B], UpPrev[B][B], Mul[B][B], T1[B][B], S[B][B];
  double E[B][B], F[B][B];
  bool ok = true;
  for (int i = 0; i < q; ++i) {
    const int blk = g * (q + 1) + i;
    input_blocks<B>(in, blk, Lo, Di, Up);
    if (i == 0) {
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) { S[r][c] = Di[r][c]; Mul[r][c] = 0.0; E[r][c] = Lo[r][c]; }
    } else {
      mm<B>(Lo, Minv, Mul);
      mm<B>(Mul, UpPrev, T1);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) S[r][c] = Di[r][c] - T1[r][c];
    }
    ok = inv_block<B>(S, Minv) && ok;
    store_blk<B>(f.Mul, h.Mul, i, G, g, Mul);
    store_blk<B>(f.Minv, h.Minv, i, G, g, Minv);
    store_blk<B>(f.Up, h.Up, i, G, g, Up);
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int c = 0; c < B; ++c) { UpPrev[r][c] = Up[r][c]; F[r][c] = Up[r][c]; }
  }
  // separator couplings of this group
  {
    double L2[B][B], D2[B][B], U2[B][B];
    if (g < G - 1) {
      input_blocks<B>(in, g * (q + 1) + q, L2, D2, U2);
      store_blk<B>(f.LoSep, h.LoSep, 0, G, g, L2);
    }
    if (g > 0) {
      input_blocks<B>(in, g * (q + 1) - 1, L2, D2, U2);
      store_blk<B>(f.UpSepPrev, h.UpSepPrev, 0, G, g, U2);
    }
  }
  // spike W = T^{-1} [E; 0; ...]: forward Y_0 = E, Y_i = -Mul_i Y_{i-1} (kept in W),
  // backward W_{q-1} = Minv Y_{q-1}, W_i = Minv_i (Y_i - Up_i W_{i+1})
  double Y[B][B], Xn[B][B];
  if (g > 0) {
#pragma unroll
    for (int r = 0; r < B; ++r)
#pragma unroll
      for (int c = 0; c < B; ++c) Y[r][c] = E[r][c];
    store_blk<B>(f.W, nullptr, 0, G, g, Y);
    for (int i = 1; i < q; ++i) {
      load_blk<B>(f.Mul, i, G, g, Mul);
      mm<B>(Mul, Y, T1);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) Y[r][c] = -T1[r][c];
      store_blk<B>(f.W, nullptr, i, G, g, Y);
    }
    for (int i = q - 1; i >= 0; --i) {
      load_blk<B>(f.W, i, G, g, Y);
      if (i < q - 1) {
        load_blk<B>(f.Up, i, G, g, Up);
        mm<B>(Up, Xn, T1);
#pragma unroll
        for (int r = 0; r < B; ++r)
#pragma unroll
          for (int c = 0; c < B; ++c) Y[r][c] -= T1[r][c];
      }
      load_blk<B>(f.Minv, i, G, g, Minv);
      mm<B>(Minv, Y, Xn);
      store_blk<B>(f.W, h.W, i, G, g, Xn);
    }
  } else {
    double Z0[B][B] = {};
    for (int i = 0; i < q; ++i) store_blk<B>(f.W, h.W, i, G, g, Z0);
  }
  // spike V = T^{-1} [0; ...; F]: V_{q-1} = Minv F, V_i = -Minv_i Up_i V_{i+1}
  if (g < G - 1) {
    load_blk<B>(f.Minv, q - 1, G, g, Minv);
    mm<B>(Minv, F, Xn);
    store_blk<B>(f.Vs, h.Vs, q - 1, G, g, Xn);
    for (int i = q - 2; i >= 0; --i) {
      load_blk<B>(f.Up, i, G, g, Up);
      mm<B>(Up, Xn, T1);
      load_blk<B>(f.Minv, i, G, g, Minv);
      mm<B>(Minv, T1, Y);
#pragma unroll
      for (int r = 0; r < B; ++r)
#pragma unroll
        for (int c = 0; c < B; ++c) Xn[r][c] = -Y[r][c];
      store_blk<B>(f.Vs, h.Vs, i, G, g, Xn);
    }
  } else {
    double Z0[B][B] = {};
    for (int i = 0; i < q; ++i) store_blk<B>(f.Vs, h.Vs, i, G, g, Z0);
  }
  if (!ok) atomicOr(fail, 1);
}

// Separator system of the next level: for separator t (block s = t(q+1)+q)
//   Lo' = -LoSep_t W_t[q-1],  Di' = Di_s - LoSep_t V_t[q-1] - UpSep_t W_{t+1}[0],
//   Up' = -UpSep_t V_{t+1}[0],  UpSep_t = UpSepPrev_{t+1}.
template <int B>
__global__ void k_assemble(LevelInput in, int q, int G, LevelF64 f, double *nLo, double *nDi, double *nUp,
                           int *fail) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= G - 1) return;
  double Lo[B][B], Di[B][B], Up[B][B], Ls[B][B], Us[B][B], Wl[B][B], Vl[B][B], Wn[B][B], Vn[B][B];
  double T1[B][B], T2[B][B], T3[B][B];
  input_blocks<B>(in, t * (q + 1) + q, Lo, Di, Up);
  load_blk<B>(f.LoSep, 0, G, t, Ls);
  load_blk<B>(f.UpSepPrev, 0, G, t + 1, Us);
  load_blk<B>(f.W, q - 1, G, t, Wl);
  load_blk<B>(f.Vs, q - 1, G, t, Vl);
  load_blk<B>(f.W, 0, G, t + 1, Wn);
  load_blk<B>(f.Vs, 0, G, t + 1, Vn);
  mm<B>(Ls, Wl, T1);
  mm<B>(Ls, Vl, T2);
  mm<B>(Us, Wn, T3);
  bool ok = true;
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) {
      const int64_t o = (int64_t)t * B * B + r * B + c;
      nLo[o] = -T1[r][c];
      nDi[o] = Di[r][c] - T2[r][c] - T3[r][c];
      if (!isfinite(nDi[o]) || !isfinite(nLo[o])) ok = false;
    }
  mm<B>(Us, Vn, T1);
#pragma unroll
  for (int r = 0; r < B; ++r)
#pragma unroll
    for (int c = 0; c < B; ++c) nUp[(int64_t)t * B * B + r * B + c] = -T1[r][c];
  if (!ok) atomicOr(fail, 1);
}

// ---------------------------------------------------------------------------------------
// apply
// ---------------------------------------------------------------------------------------

constexpr int kMaxLevels = 24;
constexpr int kTailSmem = 200 * 1024;   // shared memory of the single-CTA top levels

// The factor blocks a CTA's groups read are staged in shared memory before the sweeps:
// every thread issues asynchronous copies (cp.async, 4 or 8 bytes) of its own group's
// elements, all in flight at once, instead of the sweep's dependent loads one step at a
// time.  Shared layout: element e of the array for CTA slot t at e * nt + t (nt = groups per
// CTA), the global layout with stride nt.
template <typename T>
__device__ __forceinline__ void stage_group(T *dst, const T *src, int cnt, int G, int g, int nt, int t) {
  for (int e = 0; e < cnt; ++e) cp_async_elem(dst + e * nt + t, src + (int64_t)e * G + g);
}

// Shared memory of the staged factors (elements of T) for nt groups of q blocks: the down
// sweep reads Mul, Minv, Up (q blocks each) and LoSep, UpSepPrev (one block each); the up
// sweep W and Vs (q blocks each).
__host__ __device__ constexpr int down_stage_elems(int q, int B, int nt) { return (3 * q + 2) * B * B * nt; }
__host__ __device__ constexpr int up_stage_elems(int q, int B, int nt) { return 2 * q * B * B * nt; }

// A copy of L whose down-sweep factors point at the staged arrays (outputs unchanged).
template <typename T, int B>
__device__ __forceinline__ LevelApply<T> stage_down(const LevelApply<T> &L, T *sm, int q, int g, int nt) {
  constexpr int BB = B * B;
  const int t = threadIdx.x;
  LevelApply<T> S = L;
  T *mul = sm, *minv = mul + q * BB * nt, *up = minv + q * BB * nt, *lo = up + q * BB * nt, *usp = lo + BB * nt;
  if (g < L.G) {
    stage_group(mul, L.Mul, q * BB, L.G, g, nt, t);
    stage_group(minv, L.Minv, q * BB, L.G, g, nt, t);
    stage_group(up, L.Up, q * BB, L.G, g, nt, t);
    stage_group(lo, L.LoSep, BB, L.G, g, nt, t);
    stage_group(usp, L.UpSepPrev, BB, L.G, g, nt, t);
  }
  S.Mul = mul; S.Minv = minv; S.Up = up; S.LoSep = lo; S.UpSepPrev = usp;
  return S;
}
template <typename T, int B>
__device__ __forceinline__ LevelApply<T> stage_up(const LevelApply<T> &L, T *sm, int q, int g, int nt) {
  constexpr int BB = B * B;
  const int t = threadIdx.x;
  LevelApply<T> S = L;
  T *w = sm, *vs = w + q * BB * nt;
  if (g < L.G) {
    stage_group(w, L.W, q * BB, L.G, g, nt, t);
    stage_group(vs, L.Vs, q * BB, L.G, g, nt, t);
  }
  S.W = w; S.Vs = vs;
  return S;
}

// Level 0 down: the CTA's rows of v (times *scale) through a shared-memory tile (coalesced),
// one group per thread.  The factor blocks are streamed: every thread keeps a private ring of kRing block
// slots in shared memory (interleaved by thread, element e of slot r at (r B^2 + e) NT + t) and
// fills it with 4- or 8-byte asynchronous copies of its own group's blocks, in the order
// the sweep uses them, kRing-1 blocks ahead of the one it consumes.  No thread reads another's
// slots, so the stream needs no barrier; the ring is small, so many more groups (threads) are
// resident per SM than when a group's whole factor set is staged first.
constexpr int kRing = 4;

template <typename T, int B, int NT>
__device__ __forceinline__ void ring_stage(T *ring, int r, const T *arr, int i, int G, int g) {
  constexpr int BB = B * B;
#pragma unroll
  for (int e = 0; e < BB; ++e) cp_async_elem(ring + ((r % kRing) * BB + e) * NT + threadIdx.x, arr + gi(i, e, G, g, BB));
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void ring_commit_empty() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <typename T, int B, int NT>
__device__ __forceinline__ void ring_take(const T *ring, int r, T (&m)[B][B]) {
  constexpr int BB = B * B;
  // kRing-1 blocks were staged ahead of this one: the copies of the kRing-2 newest may still
  // be in flight, this block's (the oldest outstanding group) must have landed
  asm volatile("cp.async.wait_group %0;" ::"n"(kRing - 2) : "memory");
#pragma unroll
  for (int rr = 0; rr < B; ++rr)
#pragma unroll
    for (int c = 0; c < B; ++c) m[rr][c] = ring[((r % kRing) * BB + rr * B + c) * NT + threadIdx.x];
}

template <typename T, int B>
__device__ __forceinline__ void mat_sub(T (&y)[B], const T (&m)[B][B], const T (&x)[B]) {
#pragma unroll
  for (int r = 0; r < B; ++r) {
    T s = y[r];
#pragma unroll
    for (int c = 0; c < B; ++c) s -= m[r][c] * x[c];
    y[r] = s;
  }
}
template <typename T, int B>
__device__ __forceinline__ void mat_vec(T (&y)[B], const T (&m)[B][B], const T (&x)[B]) {
#pragma unroll
  for (int r = 0; r < B; ++r) {
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < B; ++c) s += m[r][c] * x[c];
    y[r] = s;
  }
}

// The down sweep's blocks in order of use: Mul[1..Q-1], then Minv[Q-1], Up[Q-2], Minv[Q-2],
// ..., Up[0], Minv[0], then LoSep, UpSepPrev (3Q blocks).
template <typename T, int B, int Q>
__device__ __forceinline__ void down_seq(const LevelApply<T> &L, int k, const T *&arr, int &i) {
  if (k < Q - 1) { arr = L.Mul; i = k + 1; return; }
  const int k1 = k - (Q - 1);
  if (k1 < 2 * Q - 1) {
    const int j = (k1 + 1) / 2;
    if (k1 & 1) { arr = L.Up; i = Q - 1 - j; }
    else { arr = L.Minv; i = Q - 1 - j; }
    return;
  }
  if (k1 == 2 * Q - 1) { arr = L.LoSep; i = 0; return; }
  arr = L.UpSepPrev;
  i = 0;
}

template <typename T, int B, int NT>
__global__ void __launch_bounds__(NT) k_down0s(const T *__restrict__ v, const double *scale, const int *active,
                                               LevelApply<T> L, int64_t n) {
  asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent: inputs complete
  if (active && *active == 0) return;
  constexpr int Q = kQ0;
  constexpr int SPAN = (Q + 1) * B;
  constexpr int PITCH = SPAN + 1;
  constexpr int NSEQ = 3 * Q;
  __shared__ T tile[NT * PITCH];
  __shared__ T ring[kRing * B * B * NT];
  const int g0 = blockIdx.x * NT;
  const int g = g0 + threadIdx.x;
  const int G = L.G;
  const bool mine = g < G;
  if (mine)
#pragma unroll
    for (int k = 0; k < kRing - 1; ++k) {
      const T *arr;
      int i;
      down_seq<T, B, Q>(L, k, arr, i);
      ring_stage<T, B, NT>(ring, k, arr, i, G, g);
    }
  const T sc = scale ? (T)(*scale) : (T)1;
  const int64_t row0 = (int64_t)g0 * SPAN;
  for (int e = threadIdx.x; e < NT * SPAN; e += NT) {
    const int64_t row = row0 + e;
    tile[(e / SPAN) * PITCH + (e % SPAN)] = (row < n) ? sc * v[row] : (T)0;
  }
  __syncthreads();
  if (!mine) return;
  T f[Q][B], sep[B];
  const T *my = tile + threadIdx.x * PITCH;
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int r = 0; r < B; ++r) f[i][r] = my[i * B + r];
#pragma unroll
  for (int r = 0; r < B; ++r) sep[r] = my[Q * B + r];
  T m[B][B];
  int k = 0;
  auto next = [&]() {
    ring_take<T, B, NT>(ring, k, m);
    if (k + kRing - 1 < NSEQ) {
      const T *arr;
      int i;
      down_seq<T, B, Q>(L, k + kRing - 1, arr, i);
      ring_stage<T, B, NT>(ring, k + kRing - 1, arr, i, G, g);
    } else {
      ring_commit_empty();
    }
    ++k;
  };
  // forward elimination y_i = f_i - Mul_i y_{i-1}
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    next();
    mat_sub<T, B>(f[i], m, f[i - 1]);
  }
  // back substitution x_i = Minv_i (y_i - Up_i x_{i+1})
#pragma unroll
  for (int i = Q - 1; i >= 0; --i) {
    if (i < Q - 1) {
      next();
      mat_sub<T, B>(f[i], m, f[i + 1]);
    }
    next();
    T x[B];
    mat_vec<T, B>(x, m, f[i]);
#pragma unroll
    for (int r = 0; r < B; ++r) f[i][r] = x[r];
  }
#pragma unroll
  for (int i = 0; i < Q; ++i)
#pragma unroll
    for (int r = 0; r < B; ++r) L.p[gi(i, r, G, g, B)] = f[i][r];
  next();   // LoSep
  if (G > 1 && g < G - 1) {
    T c[B];
    mat_vec<T, B>(c, m, f[Q - 1]);
#pragma unroll
    for (int r = 0; r < B; ++r) { L.cR[g * B + r] = -c[r]; L.seprhs[g * B + r] = sep[r]; }
  }
  next();   // UpSepPrev
  if (G > 1 && g > 0) {
    T c[B];
    mat_vec<T, B>(c, m, f[0]);
#pragma unroll
    for (int r = 0; r < B; ++r) L.cL[g * B + r] = -c[r];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Level 0 up with W and V streamed in order (W_0, V_0, W_1, V_1, ...): x for the CTA's groups
// goes to the shared-memory tile and is written in row order through the epilogue: mode 0 y = x
// (fixed or ring-column output), mode 1 X += x (FP64).
template <typename T, int B, int NT>
__global__ void __launch_bounds__(NT) k_up0s(const int *active, LevelApply<T> L, const T *solnext, OutRef<T> yref,
                                             double *X, int mode, int64_t n) {
  asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent: inputs complete
  if (active && *active == 0) return;
  constexpr int Q = kQ0;
  constexpr int SPAN = (Q + 1) * B;
  constexpr int PITCH = SPAN + 1;
  constexpr int NSEQ = 2 * Q;
  __shared__ T tile[NT * PITCH];
  __shared__ T ring[kRing * B * B * NT];
  const int g0 = blockIdx.x * NT;
  const int g = g0 + threadIdx.x;
  const int G = L.G;
  const bool mine = g < G;
  const bool spikes = G > 1;
  if (mine && spikes)
#pragma unroll
    for (int k = 0; k < kRing - 1; ++k) ring_stage<T, B, NT>(ring, k, (k & 1) ? L.Vs : L.W, k >> 1, G, g);
  if (mine) {
    T sl[B], sr[B];
#pragma unroll
    for (int r = 0; r < B; ++r) {
      sl[r] = (g > 0) ? solnext[(g - 1) * B + r] : (T)0;
      sr[r] = (g < G - 1) ? solnext[g * B + r] : (T)0;
    }
    T *my = tile + threadIdx.x * PITCH;
    T m[B][B];
    int k = 0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      T x[B];
#pragma unroll
      for (int r = 0; r < B; ++r) x[r] = L.p[gi(i, r, G, g, B)];
      if (spikes) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          ring_take<T, B, NT>(ring, k, m);
          if (k + kRing - 1 < NSEQ) {
            const int kk = k + kRing - 1;
            ring_stage<T, B, NT>(ring, kk, (kk & 1) ? L.Vs : L.W, kk >> 1, G, g);
          } else {
            ring_commit_empty();
          }
          ++k;
          mat_sub<T, B>(x, m, h == 0 ? sl : sr);
        }
      }
#pragma unroll
      for (int r = 0; r < B; ++r) my[i * B + r] = x[r];
    }
    if (g < G - 1)
#pragma unroll
      for (int r = 0; r < B; ++r) my[Q * B + r] = sr[r];
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  }
  __syncthreads();
  const int64_t row0 = (int64_t)g0 * SPAN;
  T *y = (mode == 0) ? yref.get() : nullptr;
  for (int e = threadIdx.x; e < NT * SPAN; e += NT) {
    const int64_t row = row0 + e;
    if (row < n && (g0 + e / SPAN) < G) {
      const T val = tile[(e / SPAN) * PITCH + (e % SPAN)];
      if (mode == 0) y[row] = val;
      else X[row] += (double)val;
    }
  }
}

constexpr int kLevelCta = 64;   // groups per CTA of the level kernels

template <typename T, int B>
__global__ void __launch_bounds__(kLevelCta) k_down_level(const int *active, LevelApply<T> L, LevelApply<T> P) {
  // the next level's CTAs may be placed now; the factor blocks (constant during the solve)
  // are staged before the wait for the previous level's outputs, so the copies overlap it
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(16) unsigned char bsm[];
  const int g = blockIdx.x * kLevelCta + threadIdx.x;
  const LevelApply<T> S = stage_down<T, B>(L, reinterpret_cast<T *>(bsm), kQ, g, kLevelCta);
  asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent: inputs complete
  if (active && *active == 0) {
    cp_async_wait_all();   // no copies left in flight when the CTA exits
    return;
  }
  cp_async_wait_all();
  __syncthreads();
  if (g < L.G) down_level_group<T, B, false>(S, P, g, kLevelCta, threadIdx.x);
}

template <typename T, int B>
__global__ void __launch_bounds__(kLevelCta) k_up_level(const int *active, LevelApply<T> L, const T *solnext) {
  // as k_down_level: dependents placed now, the spikes staged before the wait
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(16) unsigned char bsm[];
  const int g = blockIdx.x * kLevelCta + threadIdx.x;
  const LevelApply<T> S = stage_up<T, B>(L, reinterpret_cast<T *>(bsm), kQ, g, kLevelCta);
  asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent: inputs complete
  if (active && *active == 0) {
    cp_async_wait_all();   // no copies left in flight when the CTA exits
    return;
  }
  cp_async_wait_all();
  __syncthreads();
  if (g < L.G) up_level_group<T, B, false>(S, solnext, g, kLevelCta, threadIdx.x);
}

// Levels first..last (last = top, one group) in one CTA: their factors and vectors are
// copied to shared memory, then the down sweeps and the up sweeps run there.  Level
// first reads the separator vectors of level first-1 and writes its solution to global
// memory (the up sweep of level first-1 reads it).
// Shared-memory arrays of the tail start on 16-byte boundaries; a staged array is copied
// in 16-byte chunks, four per thread in flight (global arrays are 256-byte aligned and
// padded, so the last chunk stays inside the array's allocation).
__device__ __forceinline__ size_t tail_bytes(size_t count, size_t es) { return (count * es + 15) & ~size_t(15); }

template <typename T>
__device__ __forceinline__ void stage(unsigned char *&cur, const T *&ptr, size_t count) {
  const size_t n16 = tail_bytes(count, sizeof(T)) / 16;
  const uint4 *__restrict__ src = reinterpret_cast<const uint4 *>(ptr);
  uint4 *dst = reinterpret_cast<uint4 *>(cur);
  for (size_t e = threadIdx.x; e < n16; e += 4 * (size_t)blockDim.x) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t k = e + (size_t)u * blockDim.x;
      if (k < n16) v[u] = __ldg(src + k);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const size_t k = e + (size_t)u * blockDim.x;
      if (k < n16) dst[k] = v[u];
    }
  }
  ptr = reinterpret_cast<const T *>(cur);
  cur += n16 * 16;
}
template <typename T>
__device__ __forceinline__ T *carve_s(unsigned char *&cur, size_t count) {
  T *d = reinterpret_cast<T *>(cur);
  cur += tail_bytes(count, sizeof(T));
  return d;
}

template <typename T, int B>
__global__ void __launch_bounds__(512) k_tail(const int *active, const LevelApply<T> *lv, int first, int last) {
  // dependents placed now; the levels' factors (constant during the solve) are staged before
  // the wait for the level below, which is the only input written by the previous kernel
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  extern __shared__ __align__(16) unsigned char tail_smem[];
  __shared__ LevelApply<T> S[kMaxLevels];
  if (last - first + 1 > kMaxLevels) return;
  constexpr int BB = B * B;
  unsigned char *cur = tail_smem;
  for (int l = first; l <= last; ++l) {
    LevelApply<T> L = lv[l];
    const size_t gq = (size_t)L.G * L.q * BB, gs = (size_t)L.G * BB;
    stage(cur, L.Mul, gq);
    stage(cur, L.Minv, gq);
    stage(cur, L.Up, gq);
    stage(cur, L.W, gq);
    stage(cur, L.Vs, gq);
    stage(cur, L.LoSep, gs);
    stage(cur, L.UpSepPrev, gs);
    L.p = carve_s<T>(cur, (size_t)L.G * L.q * B);
    L.cR = carve_s<T>(cur, (size_t)L.G * B + 64);
    L.cL = carve_s<T>(cur, (size_t)L.G * B + 64);
    L.seprhs = carve_s<T>(cur, (size_t)L.G * B + 64);
    if (l > first) L.sol = carve_s<T>(cur, (size_t)(L.nb + 1) * B);
    if (threadIdx.x == 0) S[l - first] = L;
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");   // programmatic dependent: inputs complete
  if (active && *active == 0) return;
  for (int l = first; l <= last; ++l) {
    const LevelApply<T> L = S[l - first];
    const LevelApply<T> P = (l == first) ? lv[l - 1] : S[l - 1 - first];
    for (int g = threadIdx.x; g < L.G; g += blockDim.x) down_level_group<T, B, false>(L, P, g, L.G, g);
    __syncthreads();
  }
  for (int l = last; l >= first; --l) {
    const LevelApply<T> L = S[l - first];
    const T *solnext = (l < last) ? S[l + 1 - first].sol : nullptr;
    for (int g = threadIdx.x; g < L.G; g += blockDim.x) up_level_group<T, B, false>(L, solnext, g, L.G, g);
    __syncthreads();
  }
}

// N^T in band storage: bandT[i][p] = N^T(i, i+p-b) = N(i+p-b, i) = band[i+p-b][2b-p]
// (zero where row i+p-b is outside [0, n); taken modulo n for a cyclic band).
__global__ void k_transpose_band(const double *__restrict__ band, double *__restrict__ bandT, int64_t n, int b,
                                 int cyclic) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int w = 2 * b + 1;
  for (int p = 0; p < w; ++p) {
    int64_t r = i + p - b;
    if (cyclic) r += (r < 0) ? n : ((r >= n) ? -n : 0);
    bandT[i * w + p] = (r >= 0 && r < n) ? band[r * w + (2 * b - p)] : 0.0;
  }
}

void launch_transpose_band(const double *band, double *bandT, int64_t n, int b, cudaStream_t s, bool cyclic) {
  k_transpose_band<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(band, bandT, n, b, cyclic ? 1 : 0);
}

// ---------------------------------------------------------------------------------------
// cyclic band (Sherman-Morrison-Woodbury on the in-range band; see BandSolver::cyclic)
// ---------------------------------------------------------------------------------------

// Corner column c of the 2b: C_c = n-b+c for c < b, c-b otherwise.
__device__ __forceinline__ int64_t corner_col(int64_t n, int b, int c) { return c < b ? n - b + c : c - b; }

// u = U(:, c): the wrapped entries of N in column C_c (rows 0..b-1 and n-b..n-1).
__global__ void k_corner_rhs(const double *__restrict__ band, int64_t n, int b, int c, double *__restrict__ u) {
  const int w = 2 * b + 1;
  const int64_t cc = corner_col(n, b, c);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (i < b || i >= n - b)
      for (int p = 0; p < w; ++p) {
        const int64_t col = i + p - b;
        if (col < 0 && col + n == cc) v = band[i * w + p];
        if (col >= n && col - n == cc) v = band[i * w + p];
      }
    u[i] = v;
  }
}

// Z(:, c) = z (Z row-major n x 2b).
__global__ void k_put_z(const double *__restrict__ z, double *__restrict__ Z, int64_t n, int w2, int c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    Z[i * w2 + c] = z[i];
}

// Kc = Z(C, :) (2b x 2b), one thread.
__global__ void k_gather_corner_rows(const double *__restrict__ Z, int64_t n, int b, double *__restrict__ Kc) {
  const int w2 = 2 * b;
  for (int r = 0; r < w2; ++r)
    for (int c = 0; c < w2; ++c) Kc[r * w2 + c] = Z[corner_col(n, b, r) * w2 + c];
}

// y = yb - Z K^{-1} yb(C) (mode 0, into the fixed or ring column of yref), or X += that
// (mode 1).  Every CTA forms s = K^{-1} yb(C) itself from the 2b gathered values.
template <typename T>
__global__ void __launch_bounds__(256) k_smw(const T *__restrict__ yb, const T *__restrict__ Z,
                                             const T *__restrict__ Kinv, int64_t n, int b, const int *active,
                                             OutRef<T> yref, double *X, int mode) {
  if (active && *active == 0) return;
  __shared__ T g[8], sv[8];
  const int w2 = 2 * b;
  if (threadIdx.x < w2) g[threadIdx.x] = yb[corner_col(n, b, threadIdx.x)];
  __syncthreads();
  if (threadIdx.x < w2) {
    T acc = (T)0;
    for (int c = 0; c < w2; ++c) acc += Kinv[threadIdx.x * w2 + c] * g[c];
    sv[threadIdx.x] = acc;
  }
  __syncthreads();
  T *y = (mode == 0) ? yref.get() : nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T v = yb[i];
    for (int c = 0; c < w2; ++c) v -= Z[i * w2 + c] * sv[c];
    if (mode == 0) y[i] = v;
    else X[i] += (double)v;
  }
}

__global__ void k_to_f32(const double *__restrict__ in, float *__restrict__ out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

void launch_to_f32(const double *in, float *out, int64_t count, cudaStream_t s) {
  const int64_t g = std::min<int64_t>((count + 255) / 256, 4096);
  k_to_f32<<<(unsigned)std::max<int64_t>(g, 1), 256, 0, s>>>(in, out, count);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------

void BandSolver::plan(int64_t n_, int b_) {
  n = n_;
  b = b_;
  levels.clear();
  int nb = (int)((n + b - 1) / b);
  int q = kQ0;
  while (true) {
    LevelShape s;
    s.nb = nb;
    s.q = q;
    s.G = (nb <= q) ? 1 : (nb + 1 + q) / (q + 1);
    levels.push_back(s);
    if (s.G == 1) break;
    nb = s.G - 1;
    q = kQ;
  }
  // the top levels run in one CTA with their factors and vectors in shared memory: as
  // many levels (at least the top one, never level 0) as fit in kTailSmem in FP64
  tail_first = (int)levels.size() - 1;
  while (tail_first > 1 && tail_smem_bytes(tail_first - 1, (int)levels.size() - 1, 8) <= kTailSmem) --tail_first;
  if (levels.size() == 1) tail_first = 1;  // no tail: level 0 is the top
}

// Shared memory of the tail kernel for levels first..last in elements of `es` bytes: the
// factor blocks, p, the separator vectors and (above `first`) the solution of each level,
// every array rounded up to 16 bytes exactly as k_tail carves them.
size_t BandSolver::tail_smem_bytes(int first, int last, int es) const {
  auto ev = [es](size_t c) { return ((c * es + 15) & ~size_t(15)) / es; };
  size_t e = 0;
  const int BB = b * b;
  for (int l = first; l <= last; ++l) {
    const LevelShape &s = levels[l];
    const size_t gq = (size_t)s.G * s.q * BB, gs = (size_t)s.G * BB;
    e += 5 * ev(gq) + 2 * ev(gs);                           // Mul Minv Up W Vs, LoSep UpSepPrev
    e += ev((size_t)s.G * s.q * b) + 3 * ev((size_t)s.G * b + 64);   // p, cR cL seprhs
    if (l > first) e += ev((size_t)(s.nb + 1) * b);         // sol
  }
  return e * es;
}

template <typename T>
static T *carve(char *&p, size_t count) {
  T *r = reinterpret_cast<T *>(p);
  p += ((count * sizeof(T) + 255) / 256) * 256;
  return r;
}

size_t BandSolver::slot_bytes() const {
  size_t total = 0;
  const int BB = b * b;
  for (size_t l = 0; l < levels.size(); ++l) {
    const LevelShape &s = levels[l];
    const size_t gq = (size_t)s.G * s.q * BB;
    const size_t gs = (size_t)s.G * BB;
    total += 5 * (((gq * 8 + 255) / 256) * 256) + 2 * (((gs * 8 + 255) / 256) * 256);  // FP64
    total += 5 * (((gq * 4 + 255) / 256) * 256) + 2 * (((gs * 4 + 255) / 256) * 256);  // FP32
    if (l + 1 < levels.size()) total += 3 * ((((size_t)(s.G - 1) * BB * 8 + 255) / 256) * 256);
  }
  if (cyclic) {
    const size_t nz = (size_t)n * 2 * b, nk = (size_t)4 * b * b;
    total += ((nz * 8 + 255) / 256) * 256 + ((nz * 4 + 255) / 256) * 256;
    total += ((nk * 8 + 255) / 256) * 256 + ((nk * 4 + 255) / 256) * 256;
  }
  return total + 4096;
}

template <typename T>
static size_t apply_bytes_t(const std::vector<LevelShape> &lv, int b) {
  size_t total = 0;
  for (const LevelShape &s : lv) {
    total += ((((size_t)s.G * s.q * b * sizeof(T)) + 255) / 256) * 256;
    total += 3 * (((((size_t)s.G * b + 64) * sizeof(T)) + 255) / 256) * 256;
    total += ((((size_t)(s.nb + 1) * b * sizeof(T)) + 255) / 256) * 256;
  }
  return total + 2 * ((((size_t)lv.size() * sizeof(LevelApply<T>)) + 255) / 256) * 256 + 4096;
}

size_t BandSolver::apply_bytes() const {
  const size_t cyc = cyclic ? 2 * ((((size_t)n * 8) + 255) / 256) * 256 : 0;
  return apply_bytes_t<double>(levels, b) + apply_bytes_t<float>(levels, b) + cyc;
}

void BandSolver::bind(void *slot_mem, int slot) {
  char *p = reinterpret_cast<char *>(slot_mem);
  const int BB = b * b;
  Slot &S = slots[slot];
  S.f.assign(levels.size(), LevelF64{});
  S.h.assign(levels.size(), LevelF32{});
  S.nLo.assign(levels.size(), nullptr);
  S.nDi.assign(levels.size(), nullptr);
  S.nUp.assign(levels.size(), nullptr);
  for (size_t l = 0; l < levels.size(); ++l) {
    const LevelShape &s = levels[l];
    const size_t gq = (size_t)s.G * s.q * BB, gs = (size_t)s.G * BB;
    LevelF64 &f = S.f[l];
    f.Mul = carve<double>(p, gq); f.Minv = carve<double>(p, gq); f.Up = carve<double>(p, gq);
    f.W = carve<double>(p, gq); f.Vs = carve<double>(p, gq);
    f.LoSep = carve<double>(p, gs); f.UpSepPrev = carve<double>(p, gs);
    LevelF32 &h = S.h[l];
    h.Mul = carve<float>(p, gq); h.Minv = carve<float>(p, gq); h.Up = carve<float>(p, gq);
    h.W = carve<float>(p, gq); h.Vs = carve<float>(p, gq);
    h.LoSep = carve<float>(p, gs); h.UpSepPrev = carve<float>(p, gs);
    if (l + 1 < levels.size()) {
      const size_t nn = (size_t)(s.G - 1) * BB;
      S.nLo[l] = carve<double>(p, nn); S.nDi[l] = carve<double>(p, nn); S.nUp[l] = carve<double>(p, nn);
    }
  }
  if (cyclic) {
    const size_t nz = (size_t)n * 2 * b, nk = (size_t)4 * b * b;
    S.Z64 = carve<double>(p, nz); S.Z32 = carve<float>(p, nz);
    S.K64 = carve<double>(p, nk); S.K32 = carve<float>(p, nk);
  }
}

template <typename T, typename FS>
static void bind_apply_t(const std::vector<LevelShape> &lv, int b, char *&p, const FS (&fac)[BandSolver::kSlots],
                         std::vector<LevelApply<T>> (&out)[BandSolver::kSlots],
                         LevelApply<T> *(&dev)[BandSolver::kSlots]) {
  std::vector<LevelApply<T>> scratch(lv.size(), LevelApply<T>{});
  for (size_t l = 0; l < lv.size(); ++l) {
    LevelApply<T> &a = scratch[l];
    a.nb = lv[l].nb; a.q = lv[l].q; a.G = lv[l].G;
    a.p = carve<T>(p, (size_t)lv[l].G * lv[l].q * b);
    a.cR = carve<T>(p, (size_t)lv[l].G * b + 64);
    a.cL = carve<T>(p, (size_t)lv[l].G * b + 64);
    a.seprhs = carve<T>(p, (size_t)lv[l].G * b + 64);
    a.sol = carve<T>(p, (size_t)(lv[l].nb + 1) * b);
  }
  for (int s = 0; s < BandSolver::kSlots; ++s) {
    out[s] = scratch;
    for (size_t l = 0; l < lv.size(); ++l) {
      const auto &f = fac[s][l];
      LevelApply<T> &a = out[s][l];
      a.Mul = f.Mul; a.Minv = f.Minv; a.Up = f.Up; a.W = f.W; a.Vs = f.Vs;
      a.LoSep = f.LoSep; a.UpSepPrev = f.UpSepPrev;
    }
    dev[s] = carve<LevelApply<T>>(p, lv.size());
    cudaMemcpy(dev[s], out[s].data(), lv.size() * sizeof(LevelApply<T>), cudaMemcpyHostToDevice);
  }
}

// Groups (threads) per CTA of the level-0 kernels: 64 in FP32, 32 in FP64 (a CTA's block ring
// and input tile then take the same ~26 KB of static shared memory).
template <typename T>
constexpr int level0_cta() { return sizeof(T) == 4 ? 64 : 32; }

template <typename T, int B>
static void set_apply_attrs() {
  cudaFuncSetAttribute(k_down_level<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(down_stage_elems(kQ, B, kLevelCta) * sizeof(T)));
  cudaFuncSetAttribute(k_up_level<T, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(up_stage_elems(kQ, B, kLevelCta) * sizeof(T)));
}

void BandSolver::bind_apply(void *mem) {
  char *p = reinterpret_cast<char *>(mem);
  const std::vector<LevelF64> f64[kSlots] = {slots[0].f, slots[1].f, slots[2].f};
  const std::vector<LevelF32> f32[kSlots] = {slots[0].h, slots[1].h, slots[2].h};
  bind_apply_t<double>(levels, b, p, f64, app64, dev_app64);
  bind_apply_t<float>(levels, b, p, f32, app32, dev_app32);
  if (cyclic) {
    cyc_y = carve<double>(p, (size_t)n);
    cyc_u = carve<double>(p, (size_t)n);
  }
  static bool attrs = false;
  if (!attrs) {
    attrs = true;
#define PSP_TAIL_ATTR(T_, B_) \
  cudaFuncSetAttribute(k_tail<T_, B_>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmem + 1024); \
  set_apply_attrs<T_, B_>();
    PSP_TAIL_ATTR(float, 1) PSP_TAIL_ATTR(float, 2) PSP_TAIL_ATTR(float, 3) PSP_TAIL_ATTR(float, 4)
    PSP_TAIL_ATTR(double, 1) PSP_TAIL_ATTR(double, 2) PSP_TAIL_ATTR(double, 3) PSP_TAIL_ATTR(double, 4)
#undef PSP_TAIL_ATTR
  }
}

template <int B>
static void factor_b(BandSolver &bs, int slot, const double *band, int *fail, cudaStream_t s) {
  BandSolver::Slot &S = bs.slots[slot];
  for (size_t l = 0; l < bs.levels.size(); ++l) {
    const LevelShape &sh = bs.levels[l];
    LevelInput in;
    if (l == 0) {
      in.band = band; in.n = bs.n; in.bLo = in.bDi = in.bUp = nullptr; in.nb = sh.nb;
    } else {
      in.band = nullptr; in.n = 0; in.bLo = S.nLo[l - 1]; in.bDi = S.nDi[l - 1]; in.bUp = S.nUp[l - 1];
      in.nb = sh.nb;
    }
    const int th = 64;
    k_factor_level<B><<<(sh.G + th - 1) / th, th, 0, s>>>(in, sh.q, sh.G, S.f[l], S.h[l], fail);
    if (l + 1 < bs.levels.size())
      k_assemble<B><<<(sh.G - 1 + th - 1) / th, th, 0, s>>>(in, sh.q, sh.G, S.f[l], S.nLo[l], S.nDi[l],
                                                            S.nUp[l], fail);
  }
}

void BandSolver::factor(int slot, const double *band, int *fail, cudaStream_t s) {
  switch (b) {
    case 1: factor_b<1>(*this, slot, band, fail, s); break;
    case 2: factor_b<2>(*this, slot, band, fail, s); break;
    case 3: factor_b<3>(*this, slot, band, fail, s); break;
    case 4: factor_b<4>(*this, slot, band, fail, s); break;
    default: break;
  }
}

template <typename T, int B>
static void apply_b(const BandSolver &bs, const std::vector<LevelApply<T>> &a, const LevelApply<T> *dev,
                    const T *v, const double *scale, const int *active, OutRef<T> y, double *X, int mode,
                    cudaStream_t s) {
  constexpr int NT = level0_cta<T>();
  const int L = (int)a.size();
  const int g0 = (a[0].G + NT - 1) / NT;
  // every kernel of the solve is a programmatic dependent of the one before it (each waits
  // for its inputs before touching memory), so its CTAs are scheduled while that one drains
  launch_pdl(k_down0s<T, B, NT>, dim3(g0), dim3(NT), 0, s, v, scale, active, a[0], bs.n);
  const int tf = bs.tail_first;
  for (int l = 1; l < tf && l < L; ++l)
    launch_pdl(k_down_level<T, B>, dim3((a[l].G + kLevelCta - 1) / kLevelCta), dim3(kLevelCta),
               (int)(down_stage_elems(kQ, B, kLevelCta) * sizeof(T)), s, active, a[l], a[l - 1]);
  if (L > 1)
    launch_pdl(k_tail<T, B>, dim3(1), dim3(512), (int)bs.tail_smem_bytes(tf, L - 1, sizeof(T)), s, active, dev, tf,
               L - 1);
  for (int l = std::min(tf, L) - 1; l >= 1; --l)
    launch_pdl(k_up_level<T, B>, dim3((a[l].G + kLevelCta - 1) / kLevelCta), dim3(kLevelCta),
               (int)(up_stage_elems(kQ, B, kLevelCta) * sizeof(T)), s, active, a[l], (const T *)a[l + 1].sol);
  launch_pdl(k_up0s<T, B, NT>, dim3(g0), dim3(NT), 0, s, active, a[0], (const T *)(L > 1 ? a[1].sol : nullptr), y, X,
             mode, bs.n);
}

template <typename T>
static const std::vector<LevelApply<T>> &apps_of(const BandSolver &bs, int slot);
template <>
const std::vector<LevelApply<double>> &apps_of<double>(const BandSolver &bs, int slot) { return bs.app64[slot]; }
template <>
const std::vector<LevelApply<float>> &apps_of<float>(const BandSolver &bs, int slot) { return bs.app32[slot]; }
static const LevelApply<double> *dev_of(const BandSolver &bs, int slot, double *) { return bs.dev_app64[slot]; }
static const LevelApply<float> *dev_of(const BandSolver &bs, int slot, float *) { return bs.dev_app32[slot]; }

template <typename T>
void BandSolver::apply(int slot, const T *v, const double *scale, const int *active, OutRef<T> y, double *X,
                       int mode, cudaStream_t s) const {
  if (!cyclic) {
    apply_banded<T>(slot, v, scale, active, y, X, mode, s);
    return;
  }
  T *yb = reinterpret_cast<T *>(cyc_y);
  apply_banded<T>(slot, v, scale, active, fixed_out<T>(yb), nullptr, 0, s);
  const Slot &S = slots[slot];
  const T *Z = sizeof(T) == 8 ? reinterpret_cast<const T *>(S.Z64) : reinterpret_cast<const T *>(S.Z32);
  const T *K = sizeof(T) == 8 ? reinterpret_cast<const T *>(S.K64) : reinterpret_cast<const T *>(S.K32);
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
  k_smw<T><<<g, 256, 0, s>>>(yb, Z, K, n, b, active, y, X, mode);
}

bool BandSolver::prepare_cyclic(int slot, const double *band, cudaStream_t s) {
  Slot &S = slots[slot];
  const int w2 = 2 * b;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
  for (int c = 0; c < w2; ++c) {
    k_corner_rhs<<<g, 256, 0, s>>>(band, n, b, c, cyc_u);
    apply_banded<double>(slot, cyc_u, nullptr, nullptr, fixed_out<double>(cyc_y), nullptr, 0, s);
    k_put_z<<<g, 256, 0, s>>>(cyc_y, S.Z64, n, w2, c);
  }
  k_gather_corner_rows<<<1, 1, 0, s>>>(S.Z64, n, b, S.K64);
  std::vector<double> Kc((size_t)w2 * w2);
  if (cudaMemcpyAsync(Kc.data(), S.K64, Kc.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return false;
  // K = I + Z(C, :), inverted by Gauss-Jordan elimination with partial pivoting in long double
  std::vector<long double> M((size_t)w2 * 2 * w2, 0.0L);
  long double scale = 0.0L;
  for (int r = 0; r < w2; ++r)
    for (int c = 0; c < w2; ++c) {
      const long double v = (long double)Kc[(size_t)r * w2 + c] + (r == c ? 1.0L : 0.0L);
      M[(size_t)r * 2 * w2 + c] = v;
      scale = std::max(scale, std::fabs(v));
    }
  for (int r = 0; r < w2; ++r) M[(size_t)r * 2 * w2 + w2 + r] = 1.0L;
  if (!(scale > 0.0L) || !std::isfinite((double)scale)) return false;
  for (int col = 0; col < w2; ++col) {
    int piv = col;
    for (int r = col + 1; r < w2; ++r)
      if (std::fabs(M[(size_t)r * 2 * w2 + col]) > std::fabs(M[(size_t)piv * 2 * w2 + col])) piv = r;
    if (!(std::fabs(M[(size_t)piv * 2 * w2 + col]) > 1e-13L * scale)) return false;
    if (piv != col)
      for (int c = 0; c < 2 * w2; ++c) std::swap(M[(size_t)piv * 2 * w2 + c], M[(size_t)col * 2 * w2 + c]);
    const long double d = M[(size_t)col * 2 * w2 + col];
    for (int c = 0; c < 2 * w2; ++c) M[(size_t)col * 2 * w2 + c] /= d;
    for (int r = 0; r < w2; ++r) {
      if (r == col) continue;
      const long double f = M[(size_t)r * 2 * w2 + col];
      if (f != 0.0L)
        for (int c = 0; c < 2 * w2; ++c) M[(size_t)r * 2 * w2 + c] -= f * M[(size_t)col * 2 * w2 + c];
    }
  }
  std::vector<double> K64((size_t)w2 * w2);
  std::vector<float> K32((size_t)w2 * w2);
  for (int r = 0; r < w2; ++r)
    for (int c = 0; c < w2; ++c) {
      const double v = (double)M[(size_t)r * 2 * w2 + w2 + c];
      if (!std::isfinite(v)) return false;
      K64[(size_t)r * w2 + c] = v;
      K32[(size_t)r * w2 + c] = (float)v;
    }
  launch_to_f32(S.Z64, S.Z32, n * w2, s);
  return cudaMemcpyAsync(S.K64, K64.data(), K64.size() * 8, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaMemcpyAsync(S.K32, K32.data(), K32.size() * 4, cudaMemcpyHostToDevice, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
}

template <typename T>
void BandSolver::apply_banded(int slot, const T *v, const double *scale, const int *active, OutRef<T> y, double *X,
                              int mode, cudaStream_t s) const {
  const std::vector<LevelApply<T>> &a = apps_of<T>(*this, slot);
  const LevelApply<T> *dev = dev_of(*this, slot, (T *)nullptr);
  switch (b) {
    case 1: apply_b<T, 1>(*this, a, dev, v, scale, active, y, X, mode, s); break;
    case 2: apply_b<T, 2>(*this, a, dev, v, scale, active, y, X, mode, s); break;
    case 3: apply_b<T, 3>(*this, a, dev, v, scale, active, y, X, mode, s); break;
    case 4: apply_b<T, 4>(*this, a, dev, v, scale, active, y, X, mode, s); break;
    default: break;
  }
}

template void BandSolver::apply_banded<float>(int, const float *, const double *, const int *, OutRef<float>,
                                              double *, int, cudaStream_t) const;
template void BandSolver::apply_banded<double>(int, const double *, const double *, const int *, OutRef<double>,
                                               double *, int, cudaStream_t) const;
template void BandSolver::apply<float>(int, const float *, const double *, const int *, OutRef<float>, double *,
                                       int, cudaStream_t) const;
template void BandSolver::apply<double>(int, const double *, const double *, const int *, OutRef<double>,
                                        double *, int, cudaStream_t) const;

}  // namespace psp
