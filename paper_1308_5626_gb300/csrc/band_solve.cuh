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
  // Cyclic band: N(i, (i+p-b) mod n) = band[i][p].  N = N_b + U V^T with N_b the band's
  // in-range part (what the partitioned factorisation takes) and U V^T the 2b corner
  // columns C = (n-b .. n-1, 0 .. b-1) of the wrapped entries; the solve is
  // N^{-1} v = y - Z K^{-1} y(C), y = N_b^{-1} v, Z = N_b^{-1} U, K = I + Z(C, :)
  // (Sherman-Morrison-Woodbury).  Set before slot_bytes / apply_bytes / bind.
  bool cyclic = false;

  struct Slot {
    std::vector<LevelF64> f;
    std::vector<LevelF32> h;
    std::vector<double *> nLo, nDi, nUp;   // separator systems (input of the next level)
    // cyclic band: Z (n x 2b row-major) and K^{-1} (2b x 2b), FP64 and FP32 copies
    double *Z64 = nullptr, *K64 = nullptr;
    float *Z32 = nullptr, *K32 = nullptr;
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
  // Cyclic band, after factor() succeeded: Z and K^{-1} of the slot (2b solves with N_b,
  // K inverted on the host with partial pivoting; synchronous on s).  Returns false if K
  // is singular (relative pivot below 1e-13) or not finite.
  bool prepare_cyclic(int slot, const double *band, cudaStream_t s);
  // y = N^{-1} (scale * v) with the factors of `slot`; mode 0: y (fixed or ring column),
  // mode 1: X += N^{-1} (scale * v) in FP64.
  template <typename T>
  void apply(int slot, const T *v, const double *scale, const int *active, OutRef<T> y, double *X, int mode,
             cudaStream_t s) const;
  // the same with N_b alone (the band's in-range part)
  template <typename T>
  void apply_banded(int slot, const T *v, const double *scale, const int *active, OutRef<T> y, double *X, int mode,
                    cudaStream_t s) const;

  // cyclic scratch (apply memory): the banded solve's output and a factor-time column
  double *cyc_y = nullptr, *cyc_u = nullptr;
};

// bandT = N^T in the same band storage (n x (2b+1) FP64); cyclic: row index modulo n.
void launch_transpose_band(const double *band, double *bandT, int64_t n, int b, cudaStream_t s, bool cyclic = false);
// out = (float) in, count elements.
void launch_to_f32(const double *in, float *out, int64_t count, cudaStream_t s);

}  // namespace psp
