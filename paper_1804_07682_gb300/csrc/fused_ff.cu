// fused_ff.cu -- explicit instantiations of the fused kernels with the double-float phase, for 1, 2, 4, 8 and 16 baselines.
#include "dispatch.h"
#include "fused.cuh"
namespace gna {
cudaError_t dispatch_split_ph0(int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    const SplitArgs& a = *static_cast<const SplitArgs*>(args);
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: return launch_split<0, 1, false, false>(a, grid, block, s);
        case 5: return launch_split<0, 1, false, true>(a, grid, block, s);
        case 6: return launch_split<0, 1, true, false>(a, grid, block, s);
        case 7: return launch_split<0, 1, true, true>(a, grid, block, s);
        case 8: return launch_split<0, 2, false, false>(a, grid, block, s);
        case 9: return launch_split<0, 2, false, true>(a, grid, block, s);
        case 10: return launch_split<0, 2, true, false>(a, grid, block, s);
        case 11: return launch_split<0, 2, true, true>(a, grid, block, s);
        case 16: return launch_split<0, 4, false, false>(a, grid, block, s);
        case 17: return launch_split<0, 4, false, true>(a, grid, block, s);
        case 18: return launch_split<0, 4, true, false>(a, grid, block, s);
        case 19: return launch_split<0, 4, true, true>(a, grid, block, s);
        case 32: return launch_split<0, 8, false, false>(a, grid, block, s);
        case 33: return launch_split<0, 8, false, true>(a, grid, block, s);
        case 34: return launch_split<0, 8, true, false>(a, grid, block, s);
        case 35: return launch_split<0, 8, true, true>(a, grid, block, s);
        case 64: return launch_split<0, 16, false, false>(a, grid, block, s);
        case 65: return launch_split<0, 16, false, true>(a, grid, block, s);
        case 66: return launch_split<0, 16, true, false>(a, grid, block, s);
        case 67: return launch_split<0, 16, true, true>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t dispatch_bins_ph0(int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    const BinArgs& a = *static_cast<const BinArgs*>(args);
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: return launch_bins<0, 1, false, false>(a, grid, block, s);
        case 5: return launch_bins<0, 1, false, true>(a, grid, block, s);
        case 6: return launch_bins<0, 1, true, false>(a, grid, block, s);
        case 7: return launch_bins<0, 1, true, true>(a, grid, block, s);
        case 8: return launch_bins<0, 2, false, false>(a, grid, block, s);
        case 9: return launch_bins<0, 2, false, true>(a, grid, block, s);
        case 10: return launch_bins<0, 2, true, false>(a, grid, block, s);
        case 11: return launch_bins<0, 2, true, true>(a, grid, block, s);
        case 16: return launch_bins<0, 4, false, false>(a, grid, block, s);
        case 17: return launch_bins<0, 4, false, true>(a, grid, block, s);
        case 18: return launch_bins<0, 4, true, false>(a, grid, block, s);
        case 19: return launch_bins<0, 4, true, true>(a, grid, block, s);
        case 32: return launch_bins<0, 8, false, false>(a, grid, block, s);
        case 33: return launch_bins<0, 8, false, true>(a, grid, block, s);
        case 34: return launch_bins<0, 8, true, false>(a, grid, block, s);
        case 35: return launch_bins<0, 8, true, true>(a, grid, block, s);
        case 64: return launch_bins<0, 16, false, false>(a, grid, block, s);
        case 65: return launch_bins<0, 16, false, true>(a, grid, block, s);
        case 66: return launch_bins<0, 16, true, false>(a, grid, block, s);
        case 67: return launch_bins<0, 16, true, true>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}
int split_regs_ph0(int nl, bool grad, bool spec) {
    cudaFuncAttributes at{};
    cudaError_t e = cudaErrorInvalidValue;
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: e = cudaFuncGetAttributes(&at, k_fused_split<0, 1, false, false>); break;
        case 5: e = cudaFuncGetAttributes(&at, k_fused_split<0, 1, false, true>); break;
        case 6: e = cudaFuncGetAttributes(&at, k_fused_split<0, 1, true, false>); break;
        case 7: e = cudaFuncGetAttributes(&at, k_fused_split<0, 1, true, true>); break;
        case 8: e = cudaFuncGetAttributes(&at, k_fused_split<0, 2, false, false>); break;
        case 9: e = cudaFuncGetAttributes(&at, k_fused_split<0, 2, false, true>); break;
        case 10: e = cudaFuncGetAttributes(&at, k_fused_split<0, 2, true, false>); break;
        case 11: e = cudaFuncGetAttributes(&at, k_fused_split<0, 2, true, true>); break;
        case 16: e = cudaFuncGetAttributes(&at, k_fused_split<0, 4, false, false>); break;
        case 17: e = cudaFuncGetAttributes(&at, k_fused_split<0, 4, false, true>); break;
        case 18: e = cudaFuncGetAttributes(&at, k_fused_split<0, 4, true, false>); break;
        case 19: e = cudaFuncGetAttributes(&at, k_fused_split<0, 4, true, true>); break;
        case 32: e = cudaFuncGetAttributes(&at, k_fused_split<0, 8, false, false>); break;
        case 33: e = cudaFuncGetAttributes(&at, k_fused_split<0, 8, false, true>); break;
        case 34: e = cudaFuncGetAttributes(&at, k_fused_split<0, 8, true, false>); break;
        case 35: e = cudaFuncGetAttributes(&at, k_fused_split<0, 8, true, true>); break;
        case 64: e = cudaFuncGetAttributes(&at, k_fused_split<0, 16, false, false>); break;
        case 65: e = cudaFuncGetAttributes(&at, k_fused_split<0, 16, false, true>); break;
        case 66: e = cudaFuncGetAttributes(&at, k_fused_split<0, 16, true, false>); break;
        case 67: e = cudaFuncGetAttributes(&at, k_fused_split<0, 16, true, true>); break;
        default: break;
    }
    return e == cudaSuccess ? at.numRegs : -1;
}
}  // namespace gna
