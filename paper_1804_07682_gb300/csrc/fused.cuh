// fused.cuh -- the fused probability -> weight -> bin-integrate kernels.
//
// One pass over the energy nodes computes, per node, the survival
// probability of every baseline (paper Sec. 4.1 formula, alpha = beta = e),
// folds the baselines with their weights omega_r, multiplies by the node's
// spectrum x Gauss-Legendre weight and accumulates the bin sum of the
// prediction and of its four tangents with Kahan compensation.
//
// Per node (invE = 1/E, W = (b-a)/2 w_k S(E), We = W invE) and baseline r:
//   D21 = c21_r invE, D32 = c32_r invE reduced mod pi (c = K dm2 L_r),
//   (sin, cos) of both by FP32 polynomials, D31 = D21 + D32 by angle addition,
//   U_ij += omega_r sin^2 D_ij,   V_ij += 2 omega_r K L_r sin D_ij cos D_ij.
// Then Pc = sum_r omega_r P_r = sum omega - sum_ij A_ij U_ij, and
//   d Pc / d s2_12 = -sum_ij dA12_ij U_ij, d Pc / d s2_13 = -sum_ij dA13_ij U_ij,
//   d Pc / d dm2_21 = -invE (A21 V21 + A31 V31), d Pc / d dm2_32 = -invE (A31 V31 + A32 V32).
// Accumulated values per (point, bin): [0] sum W Pc, [1..4] sum of W (or We)
// times the bracketed tangent terms (sign applied in the epilogue), then
// [5 + r] sum W P_r per baseline when spectra are requested.
#pragma once

#include "common.cuh"
#include "epilogue.cuh"

namespace gna {

// Phase-evaluation policy: 0 = double-float (FF), 1 = double (F64 phase).
template <int PH, int NL>
struct PhaseConsts {
    float ch21[NL], cl21[NL], ch32[NL], cl32[NL];
    double cd21[NL], cd32[NL];

    __device__ __forceinline__ void load(const PointConst* pc) {
#pragma unroll
        for (int r = 0; r < NL; r++) {
            if (PH == 0) {
                ch21[r] = pc->c21h[r];
                cl21[r] = pc->c21l[r];
                ch32[r] = pc->c32h[r];
                cl32[r] = pc->c32l[r];
            } else {
                cd21[r] = pc->c21[r];
                cd32[r] = pc->c32[r];
            }
        }
    }
};

template <int PH, int NL, bool GRAD, bool SPEC>
struct NodeMath {
    static constexpr int NV = 1 + (GRAD ? 4 : 0) + (SPEC ? NL : 0);

    // With more than one baseline and no per-baseline sums, the weights enter
    // as hi + lo so that the FP32 rounding of omega_r leaves no bias; with
    // per-baseline sums the epilogue corrects sum_r (omega_r - om_r) mu_r exactly.
    static constexpr bool OMLO = (NL > 1) && !SPEC;

    PhaseConsts<PH, NL> ph;
    float om[NL], omlo[NL], wkl[NL];
    float wsum;
    float A21, A31, A32, A21l, A31l, A32l;
    float d12[3], d13[3];

    __device__ __forceinline__ void load(const PointConst* pc, const BaseConst& bc) {
        ph.load(pc);
#pragma unroll
        for (int r = 0; r < NL; r++) {
            om[r] = bc.om[r];
            omlo[r] = bc.omlo[r];
            wkl[r] = bc.wkl[r];
        }
        wsum = bc.wsum;
        A21 = pc->Af[0];
        A31 = pc->Af[1];
        A32 = pc->Af[2];
        A21l = pc->Alo[0];
        A31l = pc->Alo[1];
        A32l = pc->Alo[2];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            d12[j] = pc->dA12f[j];
            d13[j] = pc->dA13f[j];
        }
    }

    // One energy node: g = {invE_hi, invE_lo, W, We}.
    __device__ __forceinline__ void update(float4 g, KahanF (&acc)[NV]) const {
        const float eh = g.x, el = g.y, W = g.z, We = g.w;
        double ed = 0.0;
        if (PH == 1) ed = (double)eh + (double)el;
        float U21 = 0.f, U31 = 0.f, U32 = 0.f;
        float L21 = 0.f, L31 = 0.f, L32 = 0.f;  // lo-weight sums (OMLO)
        float V21 = 0.f, V31 = 0.f, V32 = 0.f;
#pragma unroll
        for (int r = 0; r < NL; r++) {
            float s1, c1, s2, c2;
            float r21, r32;
            if (PH == 0) {
                r21 = reduce_pi_ff(ph.ch21[r], ph.cl21[r], eh, el);
                r32 = reduce_pi_ff(ph.ch32[r], ph.cl32[r], eh, el);
            } else {
                r21 = reduce_pi_f64(ph.cd21[r], ed);
                r32 = reduce_pi_f64(ph.cd32[r], ed);
            }
            sincos_poly(r21, s1, c1);
            sincos_poly(r32, s2, c2);
            // D31 = D21 + D32 (up to a multiple of pi, which flips a common sign
            // of sin and cos and leaves sin^2 and sin cos unchanged)
            float s3 = fmaf(s1, c2, c1 * s2);
            float S21 = s1 * s1, S31 = s3 * s3, S32 = s2 * s2;
            if constexpr (NL == 1) {
                // one baseline: omega = w / w = 1 exactly, so the weighting is the identity
                U21 = S21;
                U31 = S31;
                U32 = S32;
            } else {
                U21 = fmaf(om[r], S21, U21);
                U31 = fmaf(om[r], S31, U31);
                U32 = fmaf(om[r], S32, U32);
            }
            if (OMLO) {
                L21 = fmaf(omlo[r], S21, L21);
                L31 = fmaf(omlo[r], S31, L31);
                L32 = fmaf(omlo[r], S32, L32);
            }
            if (GRAD) {
                float c3 = fmaf(c1, c2, -(s1 * s2));
                V21 = fmaf(wkl[r], s1 * c1, V21);
                V31 = fmaf(wkl[r], s3 * c3, V31);
                V32 = fmaf(wkl[r], s2 * c2, V32);
            }
            if (SPEC) {
                float Pr = fmaf(-A32, S32, fmaf(-A31, S31, fmaf(-A21, S21, 1.0f)));
                kadd_prod(acc[1 + (GRAD ? 4 : 0) + r], W, Pr);
            }
        }
        // Pc = wsum - sum_ij (A_ij + A_ij,lo)(U_ij + L_ij): large terms first
        float Pc = fmaf(-A32, U32, fmaf(-A31, U31, fmaf(-A21, U21, wsum)));
        float Plo = fmaf(-A32l, U32, fmaf(-A31l, U31, -A21l * U21));
        if (OMLO) Plo = fmaf(-A32, L32, fmaf(-A31, L31, fmaf(-A21, L21, Plo)));
        Pc = __fadd_rn(Pc, Plo);
        kadd_prod(acc[0], W, Pc);
        if (GRAD) {
            float g12 = fmaf(d12[2], U32, fmaf(d12[1], U31, d12[0] * U21));
            float g13 = fmaf(d13[2], U32, fmaf(d13[1], U31, d13[0] * U21));
            float g21 = fmaf(A31, V31, A21 * V21);
            float g32 = fmaf(A32, V32, A31 * V31);
            kadd_prod(acc[1], W, g12);
            kadd_prod(acc[2], W, g13);
            kadd_prod(acc[3], We, g21);
            kadd_prod(acc[4], We, g32);
        }
    }
};

__host__ __device__ constexpr int pow2ceil(int v) { return v <= 1 ? 1 : v <= 2 ? 2 : v <= 4 ? 4 : v <= 8 ? 8 : v <= 16 ? 16 : 32; }
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// ---------------------------------------------------------------------------
// Split mapping (uniform grids): the flat node space f = (p nbins + i) n + k of
// all points is cut into equal contiguous ranges, one per resident warp
// (range length `per`).  A warp walks its range: lane l takes nodes f + l,
// f + l + 32, ... (bin-major grid, node f at f mod (nbins n): every warp load is
// 512 contiguous bytes, the next two prefetched while the current node is
// computed, across bin boundaries too).  At each bin boundary the warp reduces
// its Kahan sums with a transposed shuffle reduction and stores the segment's
// partial in slot w - w_first(bin); the warp storing a bin's last segment sums
// the segments in order (double-float) and runs the bin epilogue, and the
// last bin of a point to finish reduces the point.  Equal ranges keep every
// warp busy to the end; there is no queue and no CTA barrier.
struct SplitArgs {
    const float4* grid;
    int nbins, n, npts;
    int64_t per;    // nodes per warp range
    int maxseg;     // partial slots per (point, bin)
    int gstep;      // 32 mod (nbins n): a lane's step through the grid
    const PointConst* pcs;
    BaseConst bc;
    float2* part;   // [npts][nbins][maxseg][NV]
    EpiArgs ea;
};

#ifndef GNA_SPLIT_MIN_BLOCKS
#define GNA_SPLIT_MIN_BLOCKS 2
#endif

template <int PH, int NL, bool GRAD, bool SPEC>
__global__ void __launch_bounds__(256, GNA_SPLIT_MIN_BLOCKS) k_fused_split(SplitArgs a) {
    using M = NodeMath<PH, NL, GRAD, SPEC>;
    constexpr int NV = M::NV;
    constexpr int NVP = pow2ceil(NV);
    constexpr int SH = 5 - ilog2(NVP);
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t gn = (int64_t)a.nbins * a.n;  // nodes of the (shared) grid
    const int64_t total = gn * a.npts;
    const int64_t f0 = w * a.per;
    const int64_t f1 = min(total, f0 + a.per);
    int last_p = -1;
    M m;
    int64_t f = f0 + lane;
    // two nodes in flight per lane (f + 32 and f + 64 while f is computed): one
    // was too few to cover the load latency at 4 warps per scheduler.  Grid
    // indices are taken mod gn, so loads past the range end stay in bounds.
    int64_t gi = f % gn;
    float4 cur = __ldg(a.grid + gi);
    gi += a.gstep;  // gi + 32 mod gn, with gi, gstep < gn
    if (gi >= gn) gi -= gn;
    float4 nx1 = __ldg(a.grid + gi);  // gi: grid index of f + 32
    // a programmatic dependent of the kernel that prepares the per-point
    // constants and zeroes the counters: wait (in hardware) for it here
    asm volatile("griddepcontrol.wait;" ::: "memory");
    for (int64_t pos = f0; pos < f1;) {
        const int64_t q = pos / a.n;  // (point, bin) pair
        const int p = (int)(q / a.nbins);
        const int i = (int)(q - (int64_t)p * a.nbins);
        const int64_t seg_end = min(f1, (q + 1) * a.n);
        if (p != last_p) {
            m.load(a.pcs + p, a.bc);
            last_p = p;
        }
        KahanF acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) kzero(acc[v]);
        while (f < seg_end) {
            int64_t gin = gi + a.gstep;
            if (gin >= gn) gin -= gn;
            const float4 nx2 = __ldg(a.grid + gin);  // node f + 64
            m.update(cur, acc);
            cur = nx1;
            nx1 = nx2;
            f += 32;
            gi = gin;
        }
        // lanes whose next node lies past this segment wait here with f >= seg_end
        float2 v[NVP];
#pragma unroll
        for (int j = 0; j < NVP; j++) v[j] = (j < NV) ? kahan_to_ff(acc[j < NV ? j : 0]) : make_float2(0.f, 0.f);
        warp_transpose_reduce<NVP>(v, lane);
        const int64_t w_first = (q * a.n) / a.per;
        const int64_t w_last = ((q + 1) * a.n - 1) / a.per;
        const int nseg = (int)(w_last - w_first + 1);
        float2* pp = a.part + q * a.maxseg * NV;
        const int vi = lane >> SH;
        if ((lane & ((1 << SH) - 1)) == 0 && vi < NV) {
            pp[(w - w_first) * NV + vi] = v[0];
            __threadfence();
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) last = (atomicAdd(a.ea.bin_cnt + q, 1) == nseg - 1);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            // last segment of bin (p, i): lane j < NV sums value j over the segments in order
            __threadfence();
            double val = 0.0;
            if (lane < NV) {
                // slots in order; loads issued eight at a time
                float2 sum = make_float2(0.f, 0.f);
                for (int s0 = 0; s0 < nseg; s0 += 8) {
                    float2 t[8];
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        t[j] = (s0 + j < nseg) ? __ldcg(pp + (s0 + j) * NV + lane) : make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 8; j++)
                        if (s0 + j < nseg) sum = ff_add(sum, t[j]);
                }
                val = (double)sum.x + (double)sum.y;
            }
            double sv[NV];
#pragma unroll
            for (int j = 0; j < NV; j++) sv[j] = __shfl_sync(0xffffffffu, val, j);
            if (lane == 0) bin_epilogue(a.ea, p, i, sv, bin_inputs(a.ea, p, i));
            bin_done(a.ea, p, i, lane);
        }
        pos = seg_end;
    }
}

// ---------------------------------------------------------------------------
// Bin mapping: a warp task is (point p, group b of 32 consecutive bins); lane
// l owns bin 32 b + l and walks its nodes (grid layout [group][k][lane], so
// each warp load is 512 contiguous bytes, the next one prefetched).  Each
// lane finishes its own bin; the warp sums its group and the last group of a
// point sums the groups.  Warps take tasks from a global counter; tasks are
// ordered by decreasing node count so that uneven grids balance.
//
// Slice mapping (S > 1, one grid shared by all points): the same kernel with
// each group's nodes cut into S slices of L nodes; task t = (p, b, s) in
// that order.  A lane keeps its own bin's sums for its slice and stores them
// as float pairs; k_slices_reduce then sums the slices in order and runs the
// epilogue.  Unlike the split mapping no warp reduction or counter is needed
// per node range, and the node loop is the same as for whole bins.
struct BinArgs {
    const float4* grid;
    const int64_t* goff;  // [ngrids] float4 offset of each grid
    const int* gn;        // [ngrids] Gauss-Legendre order of each grid
    const int* gid;       // [npts] grid of each point, or NULL: every point uses grid 0
    const int* tasks;     // [ntasks] p * ngroups + b, in execution order
    int ntasks, ngroups, nbins;
    const PointConst* pcs;
    BaseConst bc;
    int* counter;  // zeroed before the launch
    EpiArgs ea;
    int S, L;      // slices per group and nodes per slice (S = 1: whole bins)
    float2* part;  // slice values [ntasks][NV][32] (S > 1)
};

template <int PH, int NL, bool GRAD, bool SPEC>
__global__ void __launch_bounds__(256) k_fused_bins(BinArgs a) {
    using M = NodeMath<PH, NL, GRAD, SPEC>;
    constexpr int NV = M::NV;
    const int lane = threadIdx.x & 31;
    int last_p = -1;
    M m;
    // a programmatic dependent of the kernel that prepares the per-point
    // constants and zeroes the counters: wait (in hardware) for it here
    asm volatile("griddepcontrol.wait;" ::: "memory");
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.ntasks) break;
        int p, b, k0, n;
        if (a.S > 1) {
            const int per_point = a.ngroups * a.S;
            p = t / per_point;
            const int rem = t - p * per_point;
            b = rem / a.S;
            k0 = (rem - b * a.S) * a.L;
            n = a.gn[0];
        } else {
            const int task = a.tasks[t];
            p = task / a.ngroups;
            b = task - p * a.ngroups;
            k0 = 0;
            n = a.gn[a.gid ? a.gid[p] : 0];
        }
        const int gi = a.gid ? a.gid[p] : 0;
        const int kn = min(n, k0 + (a.S > 1 ? a.L : n)) - k0;  // nodes of this task per lane
        if (p != last_p) {
            m.load(a.pcs + p, a.bc);
            last_p = p;
        }
        KahanF acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) kzero(acc[v]);
        const float4* g = a.grid + a.goff[gi] + ((int64_t)b * n + k0) * 32 + lane;
        // ring of D nodes in flight: with few baselines a node is too little
        // work to cover the load latency of the next one
        constexpr int D = (NL >= 4) ? 1 : 4;
        float4 buf[D];
#pragma unroll
        for (int j = 0; j < D; j++) buf[j] = (j < kn) ? __ldg(g + (int64_t)j * 32) : make_float4(1.f, 0.f, 0.f, 0.f);
        int k = 0;
        for (; k + D <= kn; k += D) {
#pragma unroll
            for (int j = 0; j < D; j++) {
                const float4 cur = buf[j];
                const int kx = k + j + D;
                buf[j] = (kx < kn) ? __ldg(g + (int64_t)kx * 32) : cur;
                m.update(cur, acc);
            }
        }
#pragma unroll
        for (int j = 0; j < D; j++)
            if (k + j < kn) m.update(buf[j], acc);
        if (a.S > 1) {
            float2* pp = a.part + (int64_t)t * NV * 32 + lane;
#pragma unroll
            for (int v = 0; v < NV; v++) pp[v * 32] = kahan_to_ff(acc[v]);
            // the slice reduction (a programmatic dependent launch) may start
            // placing its blocks once this warp's last task is done
            continue;
        }
        const int i = b * 32 + lane;
        float2 regs[15];  // this lane's per-bin values: the warp reduces its own group
        if (i < a.nbins) {
            double v[NV];
            if constexpr (NL == 1) {
                // one baseline (the scans): the tangent sums rounded once to
                // FP32 (the epilogue uses them in FP32), the rest in double
                constexpr int T1 = GRAD ? 5 : 1;
#pragma unroll
                for (int j = 0; j < NV; j++)
                    v[j] = (j >= 1 && j < T1) ? (double)__fsub_rn(acc[j].s, acc[j].c)
                                              : (double)acc[j].s - (double)acc[j].c;
            } else {
#pragma unroll
                for (int j = 0; j < NV; j++) v[j] = (double)acc[j].s - (double)acc[j].c;
            }
            bin_epilogue(a.ea, p, i, v, bin_inputs(a.ea, p, i), regs);
        }
        group_done(a.ea, p, b, lane, regs);
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

// Launch as a programmatic dependent of the previous kernel in the stream
// (the kernel preparing the constants): the node kernel's launch and block
// placement overlap it; the kernel waits with griddepcontrol.wait.
template <typename Kernel, typename Args>
cudaError_t launch_dependent(Kernel k, const Args& a, int grid, int block, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

template <int PH, int NL, bool GRAD, bool SPEC>
cudaError_t launch_split(const SplitArgs& a, int grid, int block, cudaStream_t s) {
    return launch_dependent(k_fused_split<PH, NL, GRAD, SPEC>, a, grid, block, s);
}

template <int PH, int NL, bool GRAD, bool SPEC>
cudaError_t launch_bins(const BinArgs& a, int grid, int block, cudaStream_t s) {
    return launch_dependent(k_fused_bins<PH, NL, GRAD, SPEC>, a, grid, block, s);
}

// Number of values per (point, bin) for the given flags.
__host__ __device__ inline int fused_nv(int nl, bool grad, bool spec) { return 1 + (grad ? 4 : 0) + (spec ? nl : 0); }

}  // namespace gna
