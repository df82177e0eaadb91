// fused64.cuh -- the fused chain with every step in double precision
// (GNA_FP64).  Same mappings as fused.cuh; the phase is reduced modulo pi in
// double and sin/cos are CUDA's double sincos on the reduced argument.
#pragma once

#include "common.cuh"
#include "fused.cuh"

namespace gna {

template <int NL, bool GRAD, bool SPEC>
struct NodeMath64 {
    static constexpr int NV = 1 + (GRAD ? 4 : 0) + (SPEC ? NL : 0);
    double c21[NL], c32[NL], om[NL], kl2[NL];
    double omsum, A21, A31, A32, d12[3], d13[3];

    __device__ __forceinline__ void load(const PointConst* pc, const BaseConst& bc) {
        omsum = 0.0;
#pragma unroll
        for (int r = 0; r < NL; r++) {
            c21[r] = pc->c21[r];
            c32[r] = pc->c32[r];
            om[r] = bc.omd[r];
            kl2[r] = 2.0 * bc.omd[r] * bc.kld[r];
            omsum += bc.omd[r];
        }
        A21 = pc->A[0];
        A31 = pc->A[1];
        A32 = pc->A[2];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            d12[j] = pc->dA12[j];
            d13[j] = pc->dA13[j];
        }
    }

    // g = {invE, W}
    __device__ __forceinline__ void update(double2 g, double (&acc)[NV]) const {
        const double e = g.x, W = g.y;
        double U21 = 0, U31 = 0, U32 = 0, V21 = 0, V31 = 0, V32 = 0;
#pragma unroll
        for (int r = 0; r < NL; r++) {
            double s1, c1, s2, c2;
            sincos(reduce_pi_d(c21[r] * e), &s1, &c1);
            sincos(reduce_pi_d(c32[r] * e), &s2, &c2);
            double s3 = s1 * c2 + c1 * s2;
            double S21 = s1 * s1, S31 = s3 * s3, S32 = s2 * s2;
            U21 += om[r] * S21;
            U31 += om[r] * S31;
            U32 += om[r] * S32;
            if (GRAD) {
                double c3 = c1 * c2 - s1 * s2;
                V21 += kl2[r] * s1 * c1;
                V31 += kl2[r] * s3 * c3;
                V32 += kl2[r] * s2 * c2;
            }
            if (SPEC) acc[1 + (GRAD ? 4 : 0) + r] += W * (1.0 - A21 * S21 - A31 * S31 - A32 * S32);
        }
        acc[0] += W * (omsum - A21 * U21 - A31 * U31 - A32 * U32);
        if (GRAD) {
            acc[1] += W * (d12[0] * U21 + d12[1] * U31 + d12[2] * U32);
            acc[2] += W * (d13[0] * U21 + d13[1] * U31 + d13[2] * U32);
            acc[3] += W * e * (A21 * V21 + A31 * V31);
            acc[4] += W * e * (A31 * V31 + A32 * V32);
        }
    }
};

struct SplitArgs64 {
    const double2* grid;
    int nbins, n, npts;
    int64_t per;
    int maxseg;
    const PointConst* pcs;
    BaseConst bc;
    double* part;  // [npts][nbins][maxseg][NV]
    EpiArgs ea;
};

// Same equal-range structure as k_fused_split, all in double.
template <int NL, bool GRAD, bool SPEC>
__global__ void __launch_bounds__(256) k_fused64_split(SplitArgs64 a) {
    using M = NodeMath64<NL, GRAD, SPEC>;
    constexpr int NV = M::NV;
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t gn = (int64_t)a.nbins * a.n;
    const int64_t total = gn * a.npts;
    const int64_t f0 = w * a.per;
    const int64_t f1 = min(total, f0 + a.per);
    int last_p = -1;
    M m;
    int64_t f = f0 + lane;
    for (int64_t pos = f0; pos < f1;) {
        const int64_t q = pos / a.n;
        const int p = (int)(q / a.nbins);
        const int i = (int)(q - (int64_t)p * a.nbins);
        const int64_t seg_end = min(f1, (q + 1) * a.n);
        if (p != last_p) {
            m.load(a.pcs + p, a.bc);
            last_p = p;
        }
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) acc[v] = 0.0;
        for (; f < seg_end; f += 32) m.update(a.grid[f % gn], acc);
        const int64_t w_first = (q * a.n) / a.per;
        const int64_t w_last = ((q + 1) * a.n - 1) / a.per;
        const int nseg = (int)(w_last - w_first + 1);
        double* pp = a.part + q * a.maxseg * NV;
#pragma unroll
        for (int v = 0; v < NV; v++) {
            double x = acc[v];
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == v) pp[(w - w_first) * NV + v] = x;
        }
        __threadfence();
        __syncwarp();
        int last = 0;
        if (lane == 0) last = (atomicAdd(a.ea.bin_cnt + q, 1) == nseg - 1);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double val = 0.0;
            if (lane < NV)
                for (int sg = 0; sg < nseg; sg++) val += __ldcg(pp + sg * NV + lane);
            double sv[NV];
#pragma unroll
            for (int j = 0; j < NV; j++) sv[j] = __shfl_sync(0xffffffffu, val, j);
            if (lane == 0) bin_epilogue(a.ea, p, i, sv, bin_inputs(a.ea, p, i));
            bin_done(a.ea, p, i, lane);
        }
        pos = seg_end;
    }
}

struct BinArgs64 {
    const double2* grid;
    const int64_t* goff;
    const int* gn;
    const int* gid;  // [npts] grid of each point, or NULL: every point uses grid 0
    const int* tasks;
    int ntasks, ngroups, nbins;
    const PointConst* pcs;
    BaseConst bc;
    int* counter;
    EpiArgs ea;
};

template <int NL, bool GRAD, bool SPEC>
__global__ void __launch_bounds__(256) k_fused64_bins(BinArgs64 a) {
    using M = NodeMath64<NL, GRAD, SPEC>;
    constexpr int NV = M::NV;
    const int lane = threadIdx.x & 31;
    int last_p = -1;
    M m;
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.ntasks) break;
        const int task = a.tasks[t];
        const int p = task / a.ngroups;
        const int b = task - p * a.ngroups;
        const int gi = a.gid ? a.gid[p] : 0;
        const int n = a.gn[gi];
        if (p != last_p) {
            m.load(a.pcs + p, a.bc);
            last_p = p;
        }
        double acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) acc[v] = 0.0;
        const double2* g = a.grid + a.goff[gi] + (int64_t)b * n * 32 + lane;
        for (int k = 0; k < n; k++) m.update(g[(int64_t)k * 32], acc);
        const int i = b * 32 + lane;
        float2 regs[15];  // this lane's per-bin values: the warp reduces its own group
        if (i < a.nbins) bin_epilogue(a.ea, p, i, acc, bin_inputs(a.ea, p, i), regs);
        group_done(a.ea, p, b, lane, regs);
    }
}

template <int NL, bool GRAD, bool SPEC>
cudaError_t launch_split64(const SplitArgs64& a, int grid, int block, cudaStream_t s) {
    k_fused64_split<NL, GRAD, SPEC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NL, bool GRAD, bool SPEC>
cudaError_t launch_bins64(const BinArgs64& a, int grid, int block, cudaStream_t s) {
    k_fused64_bins<NL, GRAD, SPEC><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gna
