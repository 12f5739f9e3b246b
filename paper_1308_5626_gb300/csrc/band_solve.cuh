// Partitioned banded solver for the preconditioner N (internal).
#pragma once

#include <vector>

#include "psp_kernels.cuh"

namespace psp {

struct LevelShape {
  int nb;  // real blocks of the level
  int q;   // interior blocks per group
  int G;   // groups (1 = top level)
};

// FP64 factors of one level (group-interleaved)
struct LevelF64 {
  double *Mul, *Minv, *Up, *W, *Vs, *LoSep, *UpSepPrev;
};
struct LevelF32 {
  float *Mul, *Minv, *Up, *W, *Vs, *LoSep, *UpSepPrev;
};

// What an apply kernel needs of one level.
template <typename T>
struct LevelApply {
  int nb, q, G, pad;
  const T *Mul, *Minv, *Up, *W, *Vs, *LoSep, *UpSepPrev;
  T *p, *cR, *cL, *seprhs, *sol;
};

struct BandSolver {
  int64_t n = 0;
  int b = 0;
  std::vector<LevelShape> levels;
  int tail_first = 1;

  struct Slot {
    std::vector<LevelF64> f;
    std::vector<LevelF32> h;
    std::vector<double *> nLo, nDi, nUp;   // separator systems (input of the next level)
  };
  // slots 0 and 1: the adopted and the candidate N; slot 2: N^T for the transposed solve
  static constexpr int kSlots = 3;
  Slot slots[kSlots];
  std::vector<LevelApply<double>> app64[kSlots];
  std::vector<LevelApply<float>> app32[kSlots];
  LevelApply<double> *dev_app64[kSlots] = {nullptr, nullptr, nullptr};
  LevelApply<float> *dev_app32[kSlots] = {nullptr, nullptr, nullptr};

  void plan(int64_t n, int b);
  // shared memory of the single-CTA kernel for levels first..last, elements of es bytes
  size_t tail_smem_bytes(int first, int last, int es) const;
  size_t slot_bytes() const;     // factor storage of one slot
  size_t apply_bytes() const;    // shared apply scratch + per-slot descriptors
  void bind(void *slot_mem, int slot);
  // Bind the apply scratch and upload the per-slot descriptors (synchronous).
  void bind_apply(void *mem);
  void factor(int slot, const double *band, int *fail, cudaStream_t s);
  // y = N^{-1} (scale * v) with the factors of `slot`; mode 0: y (fixed or ring column),
  // mode 1: X += N^{-1} (scale * v) in FP64.
  template <typename T>
  void apply(int slot, const T *v, const double *scale, const int *active, OutRef<T> y, double *X, int mode,
             cudaStream_t s) const;
};

// bandT = N^T in the same band storage (n x (2b+1) FP64).
void launch_transpose_band(const double *band, double *bandT, int64_t n, int b, cudaStream_t s);
// out = (float) in, count elements.
void launch_to_f32(const double *in, float *out, int64_t count, cudaStream_t s);

}  // namespace psp
