// slices.cu -- second step of the slice mapping: for each (point, group of
// 32 bins) the slices' values are summed in slice order (double-float, so the
// result does not depend on which warp computed which slice), then the bin
// epilogue runs for the group's bins and the group and point reductions
// follow (steps a7-a9 of the chain).
#include <mutex>

#include "dispatch.h"
#include "epilogue.cuh"

namespace gna {

// One block of W warps per (point, group).  Warp w sums slices w, w + W, ...
// in order for every value (lane l: bin 32 g + l; the loads of a slice for
// all values are in flight together); the warps' sums are then added in warp
// order through shared memory, one value per warp, and warp 0 runs the
// epilogue of the group.  The fixed order makes the result independent of
// timing.  NVM bounds the value count so that the per-lane arrays stay in
// registers: 32 warps for up to 5 values, 24 for up to 13, 16 beyond.
template <int NVM, int W>
__global__ void __launch_bounds__(W * 32) k_slices_reduce(const float2* __restrict__ part, int S, int NV, EpiArgs ea) {
    extern __shared__ float2 red[];  // [W][NV][32], then [NV][32] doubles
    double* fin = reinterpret_cast<double*>(red + W * NV * 32);
    const int pg = blockIdx.x;
    const int p = pg / ea.ngroups;
    const int g = pg - p * ea.ngroups;
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // the next evaluation's first kernel may be placed now; it waits for this
    // kernel to complete before it touches anything
    asm volatile("griddepcontrol.launch_dependents;");
    float2 acc[NVM];
#pragma unroll
    for (int v = 0; v < NVM; v++) acc[v] = make_float2(0.f, 0.f);
    // the epilogue's inputs do not depend on the node kernel: load them first
    const int i = g * 32 + lane;
    BinIn in{0.0, 0.0, 0.0};
    if (w == 0 && i < ea.nbins) in = bin_inputs(ea, p, i);
    // launched as a programmatic dependent of the node kernel: the blocks may
    // be resident before it ends; wait (in hardware) until it has completed
    // and its writes are visible
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const float2* base = part + (int64_t)pg * S * NV * 32 + lane;
    const int64_t stride = (int64_t)NV * 32;
    for (int sl = w; sl < S; sl += W) {
        const float2* src = base + sl * stride;
        float2 t[NVM];
#pragma unroll
        for (int v = 0; v < NVM; v++) t[v] = (v < NV) ? __ldg(src + v * 32) : make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < NVM; v++)
            if (v < NV) acc[v] = ff_add(acc[v], t[v]);
    }
#pragma unroll
    for (int v = 0; v < NVM; v++)
        if (v < NV) red[(w * NV + v) * 32 + lane] = acc[v];
    __syncthreads();
    for (int v = w; v < NV; v += W) {
        float2 sum = red[v * 32 + lane];
        for (int k = 1; k < W; k++) sum = ff_add(sum, red[(k * NV + v) * 32 + lane]);
        fin[v * 32 + lane] = (double)sum.x + (double)sum.y;
    }
    __syncthreads();
    if (w == 0) {
        double vals[kMaxNV];
        for (int v = 0; v < NV; v++) vals[v] = fin[v * 32 + lane];
        float2 regs[15];  // this lane's per-bin values: the warp reduces its own group
        if (i < ea.nbins) bin_epilogue(ea, p, i, vals, in, regs);
        group_done(ea, p, g, lane, regs);
    }
}

template <int NVM, int W>
cudaError_t launch_reduce(const float2* part, int S, int NV, const EpiArgs& ea, int npts, cudaStream_t s) {
    // more than the default 48 KB of dynamic shared memory: opt in once per device
    static std::once_flag once[64];
    static cudaError_t attr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        attr[dev] = cudaFuncSetAttribute(k_slices_reduce<NVM, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) * W * NVM * 32 + sizeof(double) * NVM * 32));
    });
    if (attr[dev] != cudaSuccess) return attr[dev];
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((int64_t)npts * ea.ngroups));
    cfg.blockDim = dim3(W * 32);
    cfg.dynamicSmemBytes = sizeof(float2) * W * NV * 32 + sizeof(double) * NV * 32;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_slices_reduce<NVM, W>, part, S, NV, ea);
}

cudaError_t launch_slices_reduce(const float2* part, int S, int NV, const EpiArgs& ea, int npts, cudaStream_t s) {
    if (NV < 1 || NV > kMaxNV) return cudaErrorInvalidValue;
    if (NV <= 5) return launch_reduce<5, 32>(part, S, NV, ea, npts, s);
    if (NV <= 13) return launch_reduce<13, 24>(part, S, NV, ea, npts, s);
    return launch_reduce<kMaxNV, 16>(part, S, NV, ea, npts, s);
}

// Epilogue-only evaluation (steps a7-a9) on the node sums a previous
// evaluation kept: one warp per (point, group of 32 bins), lane l bin 32 g + l.
__global__ void __launch_bounds__(256) k_cached_epilogue(const double* __restrict__ sums, EpiArgs ea) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (int64_t)ea.npts * ea.ngroups) return;
    const int p = (int)(wid / ea.ngroups);
    const int g = (int)(wid - (int64_t)p * ea.ngroups);
    const int i = g * 32 + lane;
    float2 regs[15];
    if (i < ea.nbins) {
        double v[kMaxNV];
        const double* src = sums + ((int64_t)p * ea.nbins + i) * ea.NV;
        for (int j = 0; j < ea.NV; j++) v[j] = src[j];
        bin_epilogue(ea, p, i, v, bin_inputs(ea, p, i), regs);
    }
    group_done(ea, p, g, lane, regs);
}

cudaError_t launch_cached_epilogue(const double* sums, const EpiArgs& ea, cudaStream_t s) {
    const int64_t threads = (int64_t)ea.npts * ea.ngroups * 32;
    k_cached_epilogue<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(sums, ea);
    return cudaGetLastError();
}

}  // namespace gna
