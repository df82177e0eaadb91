// dispatch.h -- host-side selection of the fused-kernel instantiation.
#pragma once
#include <cuda_runtime.h>

namespace gna {
// ph: 0 = double-float phase, 1 = double phase (both FP32 + Kahan bulk), 2 = all double.
// nl: instantiated baseline count (1, 2, 4, 8 or 16).  args points to
// SplitArgs / BinArgs (ph 0, 1) or SplitArgs64 / BinArgs64 (ph 2).
cudaError_t dispatch_split(int ph, int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s);
cudaError_t dispatch_bins(int ph, int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s);
// registers per thread of the split kernel (for occupancy-aware grid sizing)
int split_regs(int ph, int nl, bool grad, bool spec);
// second step of the slice mapping (slices.cu): S slices of NV values per
// (point, group) in part [npts][ngroups][S][NV][32]
struct EpiArgs;
cudaError_t launch_slices_reduce(const float2* part, int S, int NV, const EpiArgs& ea, int npts, cudaStream_t s);
// epilogue only, on kept node sums [npts][nbins][ea.NV] (slices.cu)
cudaError_t launch_cached_epilogue(const double* sums, const EpiArgs& ea, cudaStream_t s);
}  // namespace gna
