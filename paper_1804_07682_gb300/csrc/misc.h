// misc.h -- argument structs and launchers of kernels_misc.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "epilogue.cuh"
#include "gnaosc.h"

namespace gna {

// Plain FP64 chain over one chunk of points p0 .. p0 + cnt - 1, flattened
// over (point, baseline, node): len = off[p0 + cnt] - off[p0] elements.
struct PlainArgs {
    const double2* nodes;   // bin-major grids {1/E, W}, one per distinct node count
    const int64_t* goff;    // [ngrids] first node of each grid
    const int* gn;          // [ngrids] nodes per bin
    const int* gid;         // [npts] grid of each point, or NULL (one grid)
    const int64_t* off;     // [npts + 1] first element of each point (nL nbins n_p elements per point)
    const PointConst* pcs;  // [npts]
    BaseConst bc;
    int nbins, nL, p0, cnt, grad;
    int64_t len;
    double* P;              // [len]
    double* dP;             // [4][len]
    double* mu_r;           // [cnt][nL][nbins]
    double* dmu;            // [4][cnt][nL][nbins]
};

struct PlainChi2Args {
    const double* mu_r;  // [cnt][nL][nbins]
    const double* dmu;   // [4][cnt][nL][nbins] or NULL
    BaseConst bc;
    int nL, nbins, p0, cnt;
    double norm;
    int kind;
    const double* eta;
    double sigma;
    const double* data;  // [npts][nbins] if dpp else [nbins]
    int dpp;
    double* chi2;        // [npts]
    double* grad;        // [npts][4] or NULL
    double* mu_out;      // [npts][nbins] or NULL
    double* grad_eta_out;
    double* spectra_out;  // [npts][nL][nbins] or NULL
};

struct OscConst {
    double c21[GNA_NLMAX], c32[GNA_NLMAX];
    float c21h[GNA_NLMAX], c21l[GNA_NLMAX], c32h[GNA_NLMAX], c32l[GNA_NLMAX], c31h[GNA_NLMAX], c31l[GNA_NLMAX];
    double A[3];
    float Af[3];
    float one_minus_A21f;
    int nL;
};

// Constants of the general-channel kernel: phases q = (21, 31, 32) per
// baseline (double and hi + lo floats), coefficients -4 Re X and 2 Im X.
struct OscGenConst {
    double c[3][GNA_NLMAX];
    float ch[3][GNA_NLMAX], cl[3][GNA_NLMAX];
    double cr[3], ci[3];
    float crf[3], cif[3];
    double dab;  // delta_ab
    int nL;
};
cudaError_t launch_oscgen(const double* E, int64_t n, const OscGenConst& oc, int prec, void* P, cudaStream_t s);

// Levenberg-Marquardt state of one data set for NP parameters.
template <int NP>
struct LMStateT {
    double best[NP];
    double chi2;
    double g[NP];
    double H[NP * (NP + 1) / 2];
    double lam;
};
using LMState = LMStateT<4>;

// Per-point constants (step a0); also zeroes nz ints at zero (the evaluation's
// counters) and sets *status to GNA_EINVAL for a point outside the physical domain.
cudaError_t launch_prepare(const gna_osc* prm, int npts, const BaseConst& bc, PointConst* out, cudaStream_t s,
                           int* zero = nullptr, int64_t nz = 0, int* status = nullptr);
cudaError_t launch_gl(int n, double* x, double* w, double* tmp_ab, cudaStream_t s);
cudaError_t launch_build_grid(int nbins, int nbins_pad, const double* edges, int n, const double* x, const double* w,
                              double e_scale, int layout, float4* ff, double2* d64, double2* plain64, cudaStream_t s);
cudaError_t launch_sum_weights(const float4* grid, int nbins, int n, int layout, double* out, cudaStream_t s);
// The plain chain's kernels for one chunk of points: OscProb (+ tangents),
// weights, bin integration, chi^2 (4 launches, 6 with the tangents).
cudaError_t launch_plain_chunk(const PlainArgs& a, const PlainChi2Args& ca, cudaStream_t s);
cudaError_t launch_oscprob(const double* E, int64_t n, const OscConst& oc, int prec, void* P, cudaStream_t s);
template <int NP>
cudaError_t launch_lm_init(LMStateT<NP>* st, int npts, double lam0, cudaStream_t s);
template <int NP>
cudaError_t launch_lm_update(int npts, const double* chi2, const double* grad, const double* H, LMStateT<NP>* st,
                             double* prm, double* chi2_best, cudaStream_t s);
cudaError_t launch_fma_probe(int blocks, int iters, float* out, cudaStream_t s);
cudaError_t launch_grad_scale(double* a, int64_t na, double* b, int64_t nb, const double* s, cudaStream_t st);
template <int NP>
cudaError_t launch_lm_finish(int npts, const LMStateT<NP>* st, double* prm, cudaStream_t s);

}  // namespace gna
