// fused_fp64.cu -- explicit instantiations of the all-double fused kernels, for 1, 8 and 16 baselines.
#include "dispatch.h"
#include "fused64.cuh"
namespace gna {
cudaError_t dispatch_split_ph2(int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    const SplitArgs64& a = *static_cast<const SplitArgs64*>(args);
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: return launch_split64<1, false, false>(a, grid, block, s);
        case 5: return launch_split64<1, false, true>(a, grid, block, s);
        case 6: return launch_split64<1, true, false>(a, grid, block, s);
        case 7: return launch_split64<1, true, true>(a, grid, block, s);
        case 32: return launch_split64<8, false, false>(a, grid, block, s);
        case 33: return launch_split64<8, false, true>(a, grid, block, s);
        case 34: return launch_split64<8, true, false>(a, grid, block, s);
        case 35: return launch_split64<8, true, true>(a, grid, block, s);
        case 64: return launch_split64<16, false, false>(a, grid, block, s);
        case 65: return launch_split64<16, false, true>(a, grid, block, s);
        case 66: return launch_split64<16, true, false>(a, grid, block, s);
        case 67: return launch_split64<16, true, true>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t dispatch_bins_ph2(int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    const BinArgs64& a = *static_cast<const BinArgs64*>(args);
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: return launch_bins64<1, false, false>(a, grid, block, s);
        case 5: return launch_bins64<1, false, true>(a, grid, block, s);
        case 6: return launch_bins64<1, true, false>(a, grid, block, s);
        case 7: return launch_bins64<1, true, true>(a, grid, block, s);
        case 32: return launch_bins64<8, false, false>(a, grid, block, s);
        case 33: return launch_bins64<8, false, true>(a, grid, block, s);
        case 34: return launch_bins64<8, true, false>(a, grid, block, s);
        case 35: return launch_bins64<8, true, true>(a, grid, block, s);
        case 64: return launch_bins64<16, false, false>(a, grid, block, s);
        case 65: return launch_bins64<16, false, true>(a, grid, block, s);
        case 66: return launch_bins64<16, true, false>(a, grid, block, s);
        case 67: return launch_bins64<16, true, true>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}
int split_regs_ph2(int nl, bool grad, bool spec) {
    cudaFuncAttributes at{};
    cudaError_t e = cudaErrorInvalidValue;
    const int key = nl * 4 + (grad ? 2 : 0) + (spec ? 1 : 0);
    switch (key) {
        case 4: e = cudaFuncGetAttributes(&at, k_fused64_split<1, false, false>); break;
        case 5: e = cudaFuncGetAttributes(&at, k_fused64_split<1, false, true>); break;
        case 6: e = cudaFuncGetAttributes(&at, k_fused64_split<1, true, false>); break;
        case 7: e = cudaFuncGetAttributes(&at, k_fused64_split<1, true, true>); break;
        case 32: e = cudaFuncGetAttributes(&at, k_fused64_split<8, false, false>); break;
        case 33: e = cudaFuncGetAttributes(&at, k_fused64_split<8, false, true>); break;
        case 34: e = cudaFuncGetAttributes(&at, k_fused64_split<8, true, false>); break;
        case 35: e = cudaFuncGetAttributes(&at, k_fused64_split<8, true, true>); break;
        case 64: e = cudaFuncGetAttributes(&at, k_fused64_split<16, false, false>); break;
        case 65: e = cudaFuncGetAttributes(&at, k_fused64_split<16, false, true>); break;
        case 66: e = cudaFuncGetAttributes(&at, k_fused64_split<16, true, false>); break;
        case 67: e = cudaFuncGetAttributes(&at, k_fused64_split<16, true, true>); break;
        default: break;
    }
    return e == cudaSuccess ? at.numRegs : -1;
}
}  // namespace gna
