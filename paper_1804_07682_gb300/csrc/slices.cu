// slices.cu -- second step of the slice mapping: for each (point, group of
// 32 bins) the slices' values are summed in slice order (double-float, so the
// result does not depend on which warp computed which slice), then the bin
// epilogue runs for the group's bins and the group and point reductions
// follow (steps a7-a9 of the chain).
#include <mutex>

#include "dispatch.h"
#include "epilogue.cuh"

namespace gna {

// One block of kWarps warps per (point, group).  Warp w sums slices
// w, w + kWarps, ... in order for every value (lane l: bin 32 g + l; the
// loads of a slice for all values are in flight together); the warps' sums
// are then added in warp order through shared memory, one value per warp,
// and warp 0 runs the epilogue of the group.  The fixed order makes the
// result independent of timing.
constexpr int kWarps = 16;

__global__ void __launch_bounds__(kWarps * 32) k_slices_reduce(const float2* __restrict__ part, int S, int NV, EpiArgs ea) {
    extern __shared__ float2 red[];  // [kWarps][NV][32], then [NV][32] doubles
    double* fin = reinterpret_cast<double*>(red + kWarps * NV * 32);
    const int pg = blockIdx.x;
    const int p = pg / ea.ngroups;
    const int g = pg - p * ea.ngroups;
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    float2 acc[kMaxNV];
#pragma unroll
    for (int v = 0; v < kMaxNV; v++) acc[v] = make_float2(0.f, 0.f);
    // launched as a programmatic dependent of the node kernel: the blocks may
    // be resident before it ends; wait (in hardware) until it has completed
    // and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float2* base = part + (int64_t)pg * S * NV * 32 + lane;
    const int64_t stride = (int64_t)NV * 32;
    // warp w: slices w, w + kWarps, ... (all values' loads of a slice in flight)
    for (int sl = w; sl < S; sl += kWarps) {
        const float2* src = base + sl * stride;
        float2 t[kMaxNV];
#pragma unroll
        for (int v = 0; v < kMaxNV; v++) t[v] = (v < NV) ? __ldg(src + v * 32) : make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < kMaxNV; v++)
            if (v < NV) acc[v] = ff_add(acc[v], t[v]);
    }
#pragma unroll
    for (int v = 0; v < kMaxNV; v++)
        if (v < NV) red[(w * NV + v) * 32 + lane] = acc[v];
    __syncthreads();
    // value v: warps' sums added in warp order by warp v (all values at once)
    for (int v = w; v < NV; v += kWarps) {
        float2 sum = red[v * 32 + lane];
        for (int k = 1; k < kWarps; k++) sum = ff_add(sum, red[(k * NV + v) * 32 + lane]);
        fin[v * 32 + lane] = (double)sum.x + (double)sum.y;
    }
    __syncthreads();
    if (w == 0) {
        const int i = g * 32 + lane;
        double vals[kMaxNV];
        for (int v = 0; v < NV; v++) vals[v] = fin[v * 32 + lane];
        if (i < ea.nbins) bin_epilogue(ea, p, i, vals);
        group_done(ea, p, g, lane);
    }
}

cudaError_t launch_slices_reduce(const float2* part, int S, int NV, const EpiArgs& ea, int npts, cudaStream_t s) {
    if (NV < 1 || NV > kMaxNV) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * kWarps * NV * 32 + sizeof(double) * NV * 32;
    // more than the default 48 KB of dynamic shared memory: opt in once per device
    static std::once_flag once[64];
    static cudaError_t attr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        attr[dev] = cudaFuncSetAttribute(k_slices_reduce, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) * kWarps * kMaxNV * 32 + sizeof(double) * kMaxNV * 32));
    });
    if (attr[dev] != cudaSuccess) return attr[dev];
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((int64_t)npts * ea.ngroups));
    cfg.blockDim = dim3(kWarps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slices_reduce, part, S, NV, ea);
}

}  // namespace gna
