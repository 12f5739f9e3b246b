// The restart loop of Algorithm 1 on the device for the captured cycle graphs: a segment
// graph wraps one restart cycle in a WHILE conditional node, and k_seg_control, the last
// kernel of the cycle, folds the cycle's summary into the segment's and sets the node's
// condition (another cycle while the step has not converged, no cycle broke, and the
// segment's cycle budget is not spent).  The host then waits once per segment instead of
// once per cycle.
#include "psp_kernels.cuh"

namespace psp {

namespace {

// No segment runs more cycles than this, whatever its budget says, so the loop always ends
// (psp_step starts another segment while its restart budget lasts).
constexpr int kSegHardCap = 4096;

__global__ void k_seg_control(const DevState *__restrict__ st, SegSummary *seg, cudaGraphConditionalHandle cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const CycleSummary c = st->sum;
  SegSummary g = *seg;
  g.cycles += 1;
  g.iters += c.k_end;
  if (g.cycles == 1) g.first_beta = c.beta;
  g.last_beta = c.beta;
  g.last_R = c.R_end;
  g.k_last = c.k_end;
  g.status = c.status | (g.status & kStBreakdown);   // a breakdown of any cycle of the segment
  g.error = c.error;
  g.hist_count = c.hist_count;
  g.bnorm = c.bnorm;
  *seg = g;
  const bool broken = (c.status & kStNumeric) || c.error || !isfinite(c.beta) || !isfinite(c.R_end);
  const bool more = !broken && !(c.status & kStConverged) && g.cycles < g.max_cycles && g.cycles < kSegHardCap;
  cudaGraphSetConditional(cond, more ? 1u : 0u);
}

}  // namespace

void launch_seg_control(const DevState *st, SegSummary *seg, cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_seg_control<<<1, 32, 0, s>>>(st, seg, cond);
}

}  // namespace psp
