// epilogue.cuh -- steps a7-a9 inside the node kernels (last-arriver pattern).
//
// Per (point, bin), once its node sums are complete:
//   M_i = sum_r omega_r mu_r,i,  mu_i = N (1 + eta_i) M_i,
//   Pearson chi2_i = (d - mu)^2 / mu,  g_i = 1 - d^2 / mu^2,
//   Poisson chi2_i = 2 (mu - d + d ln(d/mu)) (2 mu if d = 0), g_i = 2 (1 - d/mu),
// plus eta_i^2 / sigma^2, the gradient terms g_i N (1+eta_i) dM_i/dtheta,
// d chi2 / d eta_i = g_i N M_i + 2 eta_i / sigma^2 and, for the fitter,
// (2 / mu_i) J_i J_i^T with J_i = N (1+eta_i) dM_i/dtheta.
// The last bin of a point to finish sums the per-bin values over bins in a
// fixed order (deterministic) and writes chi2, the gradient and J^T W J.
#pragma once

#include "common.cuh"
#include "gnaosc.h"

namespace gna {

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
    double* binvals;       // [npts][nbins][NBV] scratch
    int NBV;               // 1 (chi2), 5 (+ gradient), 15 (+ J^T W J)
    const double* sumW;    // [ngrids][nbins] summed FP32 node weights (mixed modes)
    int shared_grid;
    double wsum_lo;
    double om_delta[GNA_NLMAX];  // omega_r - om_r
    double* chi2;          // [npts]
    double* grad;          // [npts][4] or NULL
    double* H;             // [npts][10] or NULL
    int* pt_cnt;           // [npts] bins finished, zeroed before the launch
    int* bin_cnt;          // [npts][nbins] chunks finished (split mapping), zeroed before the launch
};

// v: the NV summed values of (p, i): [0] sum W Pc, [1..4] tangent sums, [off + r] per-baseline sums.
__device__ inline void bin_epilogue(const EpiArgs& a, int p, int i, const double* v) {
    const int64_t idx = (int64_t)p * a.nbins + i;
    double M = v[0];
    const int off = 1 + (a.has_grad ? 4 : 0);
    if (!a.is64) {
        // exact corrections of the FP32 weights: the constant term of P carries
        // wsum_lo times the bin's summed node weights, and with per-baseline
        // sums the rounding of omega_r is undone with those sums
        if (a.sumW) M += a.wsum_lo * a.sumW[(a.shared_grid ? 0 : (int64_t)p * a.nbins) + i];
        if (a.nspec > 0)
            for (int r = 0; r < a.nL_out; r++) M += a.om_delta[r] * v[off + r];
    }
    const double e = a.eta ? a.eta[i] : 0.0;
    const double f = a.norm * (1.0 + e);
    const double mu = f * M;
    const double d = a.data[a.data_per_point ? idx : i];
    double term, g;
    if (a.kind == GNA_PEARSON) {
        term = (d - mu) * (d - mu) / mu;
        g = 1.0 - (d * d) / (mu * mu);
    } else {
        term = (d > 0.0) ? 2.0 * (mu - d + d * log(d / mu)) : 2.0 * mu;
        g = 2.0 * (1.0 - d / mu);
    }
    const bool pen = a.eta && a.sigma > 0.0;
    if (pen) term += e * e / (a.sigma * a.sigma);
    double* bv = a.binvals + idx * a.NBV;
    bv[0] = term;
    if (a.has_grad && a.NBV >= 5) {
        double J[4];
        for (int q = 0; q < 4; q++) {
            J[q] = -f * v[1 + q];
            bv[1 + q] = g * J[q];
        }
        if (a.NBV >= 15) {
            const double h = 2.0 / mu;
            int t = 5;
            for (int q = 0; q < 4; q++)
                for (int r = q; r < 4; r++) bv[t++] = h * J[q] * J[r];
        }
    }
    if (a.mu_out) a.mu_out[idx] = mu;
    if (a.grad_eta_out) a.grad_eta_out[idx] = g * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
    if (a.spectra_out && a.nspec > 0)
        for (int r = 0; r < a.nL_out; r++) a.spectra_out[((int64_t)p * a.nL_out + r) * a.nbins + i] = v[off + r];
}

// Warps w = 0..nw-1 of the caller sum the per-bin values of point p (value v
// by warp v mod nw; lane l takes bins l, l+32, ...; xor butterfly) and write
// the point's outputs.  Reads go through L2 (__ldcg): other SMs wrote them.
__device__ inline void point_reduce(const EpiArgs& a, int p, int w, int nw, int lane) {
    const double* bv = a.binvals + (int64_t)p * a.nbins * a.NBV;
    for (int v = w; v < a.NBV; v += nw) {
        double s = 0.0;
        for (int i = lane; i < a.nbins; i += 32) s += __ldcg(bv + (int64_t)i * a.NBV + v);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (v == 0) a.chi2[p] = s;
            else if (v < 5) {
                if (a.grad) a.grad[(int64_t)p * 4 + v - 1] = s;
            } else if (a.H) {
                a.H[(int64_t)p * 10 + v - 5] = s;
            }
        }
    }
}

}  // namespace gna
