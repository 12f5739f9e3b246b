// Launchers of the libpsp kernels (internal).
#pragma once

#include "psp_common.cuh"

namespace psp {

// Grid geometry and stencil radius as the kernels see them.
struct Geometry {
  int ndim;
  int nx, ny, nz;
  int64_t n;
  int R;   // stencil radius (max over directions)
  // explicit banded operator (psp_create_banded): A in row-major band storage with half-width
  // band_w, A(i, i+p-band_w) = Ab[i (2 band_w + 1) + p]; band_w == 0: the stencil operator
  int band_w = 0;
  const double *Ab = nullptr;
  const float *Ab32 = nullptr;
};

// Output array that is either a fixed pointer or the ring column selected at run time by
// a device counter (the history column of the current matvec).
template <typename T>
struct OutRef {
  T *base;
  int64_t ld;
  const int *counter;  // nullptr: fixed output `base`
  int mmax;
  int off;             // column = (*counter + off) % mmax
  __device__ __forceinline__ T *get() const {
    return counter ? base + (int64_t)((*counter + off) % mmax) * ld : base;
  }
};

template <typename T>
inline OutRef<T> fixed_out(T *p) { return OutRef<T>{p, 0, nullptr, 1, 0}; }

// Read-only counterpart of OutRef.
template <typename T>
struct InRef {
  const T *base;
  int64_t ld;
  const int *counter;
  int mmax;
  int off;
  __device__ __forceinline__ const T *get() const {
    return counter ? base + (int64_t)((*counter + off) % mmax) * ld : base;
  }
};
template <typename T>
inline InRef<T> fixed_in(const T *p) { return InRef<T>{p, 0, nullptr, 1, 0}; }
template <typename T>
inline InRef<T> ring_in(const T *base, int64_t ld, const int *counter, int mmax, int off = 0) {
  return InRef<T>{base, ld, counter, mmax, off};
}
template <typename T>
inline OutRef<T> ring_out(T *base, int64_t ld, const int *counter, int mmax, int off = 0) {
  return OutRef<T>{base, ld, counter, mmax, off};
}

// One 4- or 8-byte asynchronous copy global -> shared (cp.async), and the wait for all of
// the calling thread's copies.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element of 4 or 8 bytes");
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

int reduce_grid(int64_t n);
// z = a x + b y (FP64; z may alias x or y)
void launch_axpby(int64_t n, double a, const double *x, double b, const double *y, double *z, cudaStream_t s);
// The 3D geometry is taken by the z-marching tiled stencil (x a whole number of tiles of
// 32 16-byte vectors, y of 8 rows).
bool stencil_3d_tiled(const Geometry &g, int elem_bytes);

// Matvec folded into the first Gram-Schmidt pass (see launch_arnoldi).
template <typename T>
struct TileMatvec {
  InRef<T> x;          // input; x.base == nullptr: no matvec in the pass
  OutRef<T> w;         // w = A x (P_y ring column)
  OutRef<T> xcopy;     // copy of x (P_x ring column of an unpreconditioned cycle) or base nullptr
  int nx, ny, nz, ndim, R;
};

// Unit-coefficient 1D stencils of the operator's terms (for the adjoint gradients).
constexpr int kMaxTerms = 16;
struct TermStencils {
  int nt;                              // terms (<= kMaxTerms)
  int R;                               // widest radius
  int dir[kMaxTerms];
  double w[kMaxTerms][2 * kMaxR + 1];  // w[t][kMaxR + j]: weight of u(x + j h e_dir)
};
// out[t] = lambda . (D_t u), t < ts.nt; per-CTA sums in partial (rows of kMaxCta), one
// last-block counter
void launch_term_dots(const Geometry &g, const double *lam, const double *u, const TermStencils &ts, double *partial,
                      unsigned int *counter, double *out, cudaStream_t s);

// stencil.cu
template <typename TI, typename TO, typename TC>
void launch_stencil(const Geometry &g, InRef<TI> x, OutRef<TO> y, const DevState *st, const int *active,
                    cudaStream_t s, OutRef<TO> xcopy = OutRef<TO>{nullptr, 0, nullptr, 1, 0},
                    const double *scale = nullptr);
template <typename TH, typename TV>
void launch_restart(const Geometry &g, const double *X, const double *B, TH *Px, TH *Py, int64_t ldh,
                    TV *V1, DevState *st, double *partial, int mixed, cudaStream_t s,
                    const int *skip = nullptr);   // skip: the kernel returns at once while *skip != 0
// The mixed form's restart (FP32 history and basis) with its FP64-grade arithmetic in
// double-float where the grid allows and DevState::restart_df asks for it (returns whether
// the double-float kernels were enqueued); Xh, Xl: two scratch columns of n floats.
bool launch_restart_mixed(const Geometry &g, const double *X, const double *B, float *Px, float *Py, int64_t ldh,
                          float *V1, float *Xh, float *Xl, DevState *st, double *partial, cudaStream_t s);

// Launch `kernel` as a programmatic dependent of the previous kernel in the stream: its CTAs
// may be scheduled while that kernel drains; the kernel itself must wait
// (griddepcontrol.wait) before it touches memory.
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, int smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// cycle_loop.cu: the summary of one segment (up to max_cycles restart cycles in one graph
// launch, the loop on the device), folded together from the cycles' summaries.
struct SegSummary {
  int cycles;       // cycles run
  int iters;        // Arnoldi iterations of those cycles
  int k_last;       // iterations of the last cycle
  int status;       // kSt* bits of the last cycle, kStBreakdown if any cycle broke down
  int error;        // internal error flag
  int hist_count;   // history columns written since the history was cleared
  int max_cycles;   // the segment's cycle budget (set by the host before the launch)
  int pad;
  double first_beta, last_beta, last_R, bnorm;
};
void launch_seg_control(const DevState *st, SegSummary *seg, cudaGraphConditionalHandle cond, cudaStream_t s);

// arnoldi.cu
int arnoldi_grid();   // CTAs of the Gram-Schmidt passes (one per SM)
void arnoldi_setup(); // grid size and shared-memory attributes; call once outside capture
// DCGS2 step of iteration j (0-based) of a cycle: pass A (dots) and pass B (update).  With
// final_step, pass B only completes column j-1 (no matvec was made at this j).  If
// ev != nullptr, ev[0..2] are recorded after pass A, (nothing), pass B (profiling).  With
// mv, pass A also makes the iteration's matvec w_j = A x into mv->w (and the copy of x
// into mv->xcopy) for the vectors each thread streams, and uses w_j from registers; mv is
// only valid when fused_matvec_ok(geometry) holds.
template <typename T>
void launch_arnoldi(int j, int final_step, int64_t n, T *V, int64_t ldv, const T *Py, int64_t ldh, DevState *st,
                    double *partial, int mixed, cudaStream_t s, cudaEvent_t *ev = nullptr,
                    const TileMatvec<T> *mv = nullptr);
// The folded matvec handles the geometry: x rows of whole 16-byte vectors (elem bytes each)
// with more vectors per row than stencil halo vectors.
bool fused_matvec_ok(const Geometry &g, int elem_bytes);
template <typename T>
void launch_scale_copy(int k, int64_t n, const T *V, int64_t ldv, OutRef<T> y, const DevState *st,
                       cudaStream_t s);
template <typename T>
void launch_update_z(int64_t n, const T *V, int64_t ldv, T *Z, double *X, int add_to_x, const DevState *st,
                     cudaStream_t s);

// bicgstab.cu: the kernels of one BiCGSTAB iteration (FP64; V columns 0..3 = r, rh, p, s)
void launch_bi_start(int64_t n, double *V, int64_t ldv, DevState *st, cudaStream_t s);
void launch_bi_p(int first, int64_t n, double *V, int64_t ldv, InRef<double> v, OutRef<double> px, DevState *st,
                 cudaStream_t s);
void launch_bi_alpha(int64_t n, const double *V, int64_t ldv, InRef<double> v, DevState *st, double *partial,
                     cudaStream_t s);
void launch_bi_s(int64_t n, double *V, int64_t ldv, InRef<double> v, OutRef<double> sx, DevState *st, cudaStream_t s);
void launch_bi_omega(int64_t n, const double *V, int64_t ldv, InRef<double> t, DevState *st, double *partial,
                     cudaStream_t s);
void launch_bi_xr(int j, int m, int64_t n, double *X, double *V, int64_t ldv, InRef<double> p, InRef<double> sx,
                  InRef<double> t, DevState *st, double *partial, cudaStream_t s);

// band_fit.cu: the history ring in chronological order, widened to FP64 (psp_get_history)
template <typename TH>
void launch_history_copy(int64_t n, int cols, int first, int mmax, const TH *Px, const TH *Py, int64_t ld,
                         double *ox, double *oy, int64_t ldo, cudaStream_t s);
// band_fit.cu (cyclic: every row regresses on its neighbours modulo n)
template <typename TH>
void launch_fit(int b, int intercept, int64_t n, int M, const TH *Px, const TH *Py, int64_t ld,
                double *moments, double *band, int *singular_count, cudaStream_t s, int cyclic = 0);

}  // namespace psp
