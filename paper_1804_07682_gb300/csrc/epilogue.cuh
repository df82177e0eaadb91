// epilogue.cuh -- steps a7-a9, run by the warps that finish the node sums
// (last-arriver pattern), or by the slice reduction and the cached re-evaluation.
//
// Per (point, bin), once its node sums are complete:
//   M_i = sum_r omega_r mu_r,i,  mu_i = N (1 + eta_i) M_i,
//   Pearson chi2_i = (d - mu)^2 / mu,  g_i = 1 - d^2 / mu^2,
//   Poisson chi2_i = 2 (mu - d + d ln(d/mu)) (2 mu if d = 0), g_i = 2 (1 - d/mu),
// plus eta_i^2 / sigma^2, the gradient terms g_i N (1+eta_i) dM_i/dtheta,
// d chi2 / d eta_i = g_i N M_i + 2 eta_i / sigma^2 and, for the fitter,
// (2 / mu_i) J_i J_i^T with J_i = N (1+eta_i) dM_i/dtheta.
// The per-bin values are then summed per group of 32 bins and per point, each
// in a fixed order (deterministic), and chi2, the gradient and J^T W J written.
//
// In the mixed modes only mu_i and d_i - mu_i are formed in double (FP64
// instructions are 1/64 of the FP32 rate on this part); t_i = (d_i - mu_i) /
// mu_i, the Poisson term 2 mu_i h(t_i), h(t) = (1 + t) log1p(t) - t, the
// adjoint g_i, the gradient and J^T W J terms and the corrections of the FP32
// weights are FP32 (relative error ~1e-7 in each bin's term, far inside the
// mixed-mode tolerance).  Per-bin values are stored as float
// pairs (hi + lo) and summed over bins in double-float arithmetic.
#pragma once

#include "common.cuh"
#include "gnaosc.h"

namespace gna {

// Largest number of values per (point, bin): chi2, four tangents, 16 spectra.
constexpr int kMaxNV = 1 + 4 + GNA_NLMAX;

struct EpiArgs {
    int is64;
    int NV, has_grad, nspec, nL_out;
    int npts, nbins;
    double norm;
    int kind;
    const double* eta;
    double sigma;
    const double* data;
    int data_per_point;
    double* mu_out;        // [npts][nbins] or NULL
    double* spectra_out;   // [npts][nL][nbins] or NULL
    double* grad_eta_out;  // [npts][nbins] or NULL
    float2* binvals;       // [npts][nbins][NBV] scratch (double-float values)
    int NBV;               // 1 (chi2), 5 (+ gradient), 15 (+ J^T W J)
    const double* sumW;    // [ngrids][nbins] summed FP32 node weights (mixed modes)
    const int* gid;        // [npts] grid of each point, or NULL: every point uses grid 0
    float wsum_lo;               // exact sum of the FP32 weights - the kernel's constant term
    float om_delta[GNA_NLMAX];   // omega_r - om_r (corrections ~1e-8 relative: FP32 suffices)
    double* chi2;          // [npts]
    double* grad;          // [npts][4] or NULL
    double* H;             // [npts][10] or NULL
    float2* gvals;         // [npts][ngroups][NBV] sums over groups of 32 bins
    int ngroups;           // ceil(nbins / 32)
    int* pt_cnt;           // [npts] groups finished, zeroed before the launch
    int* grp_cnt;          // [npts][ngroups] bins finished, zeroed before the launch
    int* bin_cnt;          // [npts][nbins] segments finished (split mapping), zeroed before the launch
    double* binsums;       // [npts][nbins][NV] node sums kept for epilogue-only re-evaluations, or NULL
};

__device__ __forceinline__ float2 to_ff(double x) {
    const float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

// h(t) = (1 + t) log1p(t) - t in FP32: series sum_{k>=2} (-1)^k t^k / (k (k-1))
// for |t| < 1/2 (24 terms: truncation below 1e-9 relative), where the closed
// form would cancel; log1pf beyond (cancellation there is at most ~5x).
__device__ __forceinline__ float poisson_h(float t) {
    if (fabsf(t) < 0.5f) {
        float s = 0.f;
#pragma unroll
        for (int k = 25; k >= 2; k--) s = fmaf(s, -t, 1.0f / (float)(k * (k - 1)));
        return t * t * s;
    }
    return fmaf(1.0f + t, log1pf(t), -t);
}

// Inputs of one bin's epilogue that do not depend on the node sums (so that
// a caller may load them before the sums are ready).
struct BinIn {
    double d;     // data count
    double e;     // nuisance eta_i (0 without nuisances)
    double sumw;  // summed FP32 node weights (mixed modes; 0 without)
};

__device__ __forceinline__ BinIn bin_inputs(const EpiArgs& a, int p, int i) {
    const int64_t idx = (int64_t)p * a.nbins + i;
    BinIn in;
    in.d = a.data[a.data_per_point ? idx : i];
    in.e = a.eta ? a.eta[i] : 0.0;
    in.sumw = a.sumW ? a.sumW[(a.gid ? (int64_t)a.gid[p] * a.nbins : 0) + i] : 0.0;
    return in;
}

// v: the NV summed values of (p, i): [0] sum W Pc, [1..4] tangent sums, [off + r]
// per-baseline sums.  The NBV per-bin values go to binvals, or, with regs, to
// the caller's registers (when the caller's warp reduces its own group).
__device__ inline void bin_epilogue(const EpiArgs& a, int p, int i, const double* v, const BinIn& in,
                                    float2* regs = nullptr) {
    const int64_t idx = (int64_t)p * a.nbins + i;
    if (a.binsums)
        for (int j = 0; j < a.NV; j++) a.binsums[idx * a.NV + j] = v[j];
    double M = v[0];
    const int off = 1 + (a.has_grad ? 4 : 0);
    if (!a.is64) {
        // exact corrections of the FP32 weights: the constant term of P carries
        // wsum_lo times the bin's summed node weights, and with per-baseline
        // sums the rounding of omega_r is undone with those sums
        float corr = a.wsum_lo * (float)in.sumw;
        if (a.nspec > 0)
            for (int r = 0; r < a.nL_out; r++) corr = fmaf(a.om_delta[r], (float)v[off + r], corr);
        M += (double)corr;
    }
    const double e = in.e;
    const double f = a.norm * (1.0 + e);
    const double mu = f * M;
    const double d = in.d;
    double term;
    float g;
    if (a.is64) {
        double gd;
        if (a.kind == GNA_PEARSON) {
            term = (d - mu) * (d - mu) / mu;
            gd = 1.0 - (d * d) / (mu * mu);
        } else {
            term = (d > 0.0) ? 2.0 * (mu - d + d * log(d / mu)) : 2.0 * mu;
            gd = 2.0 * (1.0 - d / mu);
        }
        g = (float)gd;
        float2* bv = regs ? regs : a.binvals + idx * a.NBV;
        const bool pen = a.eta && a.sigma > 0.0;
        if (pen) term += e * e / (a.sigma * a.sigma);
        bv[0] = to_ff(term);
        if (a.has_grad && a.NBV >= 5) {
            double J[4];
            for (int q = 0; q < 4; q++) {
                J[q] = -f * v[1 + q];
                bv[1 + q] = to_ff(gd * J[q]);
            }
            if (a.NBV >= 15) {
                const double h = 2.0 / mu;
                int t = 5;
                for (int q = 0; q < 4; q++)
                    for (int r = q; r < 4; r++) bv[t++] = to_ff(h * J[q] * J[r]);
            }
        }
        if (a.mu_out) a.mu_out[idx] = mu;
        if (a.grad_eta_out) a.grad_eta_out[idx] = gd * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
    } else {
        const double dm = d - mu;                   // in double: d and mu are close
        const float tf = (float)dm / (float)mu;     // relative residual, 1e-7 is enough
        if (a.kind == GNA_PEARSON) {
            term = dm * (double)tf;  // (d - mu)^2 / mu
            g = 1.0f - (1.0f + tf) * (1.0f + tf);  // 1 - d^2 / mu^2
        } else {
            term = (d > 0.0) ? 2.0 * mu * (double)poisson_h(tf) : 2.0 * mu;
            g = -2.0f * tf;  // 2 (1 - d / mu)
        }
        float2* bv = regs ? regs : a.binvals + idx * a.NBV;
        const bool pen = a.eta && a.sigma > 0.0;
        if (pen) term += e * e / (a.sigma * a.sigma);
        bv[0] = to_ff(term);
        if (a.has_grad && a.NBV >= 5) {
            const float ff = (float)f;
            float J[4];
            for (int q = 0; q < 4; q++) {
                J[q] = -ff * (float)v[1 + q];
                bv[1 + q] = make_float2(g * J[q], 0.f);
            }
            if (a.NBV >= 15) {
                const float h = 2.0f / (float)mu;
                int tt = 5;
                for (int q = 0; q < 4; q++)
                    for (int r = q; r < 4; r++) bv[tt++] = make_float2(h * J[q] * J[r], 0.f);
            }
        }
        if (a.mu_out) a.mu_out[idx] = mu;
        if (a.grad_eta_out)
            a.grad_eta_out[idx] = (double)g * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
    }
    if (a.spectra_out && a.nspec > 0)
        for (int r = 0; r < a.nL_out; r++) a.spectra_out[((int64_t)p * a.nL_out + r) * a.nbins + i] = v[off + r];
}

// The per-bin values are summed in two levels, each one warp-wide reduction
// in a fixed order (so the result does not depend on which warp finished
// what): the warp that finishes the last bin of a group of 32 bins sums the
// group, and the warp that finishes the last group of a point sums the
// groups and writes the point's outputs.  At the end of a launch this leaves
// two short reductions after the last bin instead of one over all bins.
// Reads go through L2 (__ldcg): other SMs wrote the values.

// Group g of point p: lane l holds (regs) or loads (binvals) the values of
// bin 32 g + l; one transposed reduction; lanes holding value lane / 2 store it.
__device__ inline void group_reduce(const EpiArgs& a, int p, int g, int lane, const float2* regs) {
    const int i = (g << 5) + lane;
    float2 v[16];
    if (regs) {
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = (j < a.NBV && i < a.nbins) ? regs[j] : make_float2(0.f, 0.f);
    } else {
        const float2* bv = a.binvals + ((int64_t)p * a.nbins + i) * a.NBV;
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = (j < a.NBV && i < a.nbins) ? __ldcg(bv + j) : make_float2(0.f, 0.f);
    }
    warp_transpose_reduce<16>(v, lane);
    const int vi = lane >> 1;
    if ((lane & 1) == 0 && vi < a.NBV) a.gvals[((int64_t)p * a.ngroups + g) * a.NBV + vi] = v[0];
}

// Point p: lane l sums groups l, l + 32, ... in order, then one transposed
// reduction over the lanes; the point's outputs are written.
__device__ inline void point_reduce(const EpiArgs& a, int p, int lane) {
    float2 v[16];
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = make_float2(0.f, 0.f);
    for (int g = lane; g < a.ngroups; g += 32) {
        const float2* gv = a.gvals + ((int64_t)p * a.ngroups + g) * a.NBV;
#pragma unroll
        for (int j = 0; j < 15; j++)
            if (j < a.NBV) v[j] = ff_add(v[j], __ldcg(gv + j));
    }
    warp_transpose_reduce<16>(v, lane);
    const int vi = lane >> 1;
    if ((lane & 1) == 0 && vi < a.NBV) {
        const double tot = (double)v[0].x + (double)v[0].y;
        if (vi == 0) a.chi2[p] = tot;
        else if (vi < 5) {
            if (a.grad) a.grad[(int64_t)p * 4 + vi - 1] = tot;
        } else if (a.H) {
            a.H[(int64_t)p * 10 + vi - 5] = tot;
        }
    }
}

// The whole group g of point p has its per-bin values ready (whole warp
// calls): in regs (each lane its bin's values) or in binvals.  Not inlined:
// its registers stay out of the node loops' allocation.
static __device__ __noinline__ void group_done(const EpiArgs& a, int p, int g, int lane, const float2* regs) {
    if (!regs) {
        __threadfence();
        __syncwarp();
    }
    group_reduce(a, p, g, lane, regs);
    // every lane that stored a group value makes it visible before lane 0 counts the group
    __threadfence();
    __syncwarp();
    int lastp = 0;
    if (lane == 0) lastp = (atomicAdd(a.pt_cnt + p, 1) == a.ngroups - 1);
    lastp = __shfl_sync(0xffffffffu, lastp, 0);
    if (lastp) {
        __threadfence();
        point_reduce(a, p, lane);
    }
}

// Bin i of point p has its per-bin values stored by lane 0 (whole warp calls).
__device__ inline void bin_done(const EpiArgs& a, int p, int i, int lane) {
    const int g = i >> 5;
    const int gsize = min(32, a.nbins - (g << 5));
    int lastg = 0;
    if (lane == 0) {
        __threadfence();
        lastg = (atomicAdd(a.grp_cnt + (int64_t)p * a.ngroups + g, 1) == gsize - 1);
    }
    lastg = __shfl_sync(0xffffffffu, lastg, 0);
    if (lastg) group_done(a, p, g, lane, nullptr);
}

}  // namespace gna
