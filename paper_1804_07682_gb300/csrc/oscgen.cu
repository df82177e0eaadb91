// oscgen.cu -- element-wise OscProb for any channel (paper Sec. 4.1, the
// general vacuum formula, neutrinos and antineutrinos, with theta23 and the
// CP phase):
//   P(a -> b) = delta_ab + sum_{i>j} [ -4 Re X_ij sin^2 x_ij + 2 Im X_ij sin 2x_ij ],
//   X_ij = V*_ai V_bi V_aj V*_bj,  V = U (neutrinos) or U* (antineutrinos),
//   x_ij = K dm2_ij L / E.
// The host folds U into the six real coefficients (cr = -4 Re X, ci = 2 Im X)
// per channel; the kernel evaluates three phases per (baseline, energy).
#include <algorithm>

#include "common.cuh"
#include "misc.h"

namespace gna {

// FP64: the phases in double, double sincos.
__global__ void k_oscgen64(const double* __restrict__ E, int64_t n, OscGenConst oc, double* __restrict__ P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double inv = 1.0 / E[k];
    for (int r = 0; r < oc.nL; r++) {
        double p = oc.dab;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            double s, c;
            sincos(oc.c[q][r] * inv, &s, &c);
            p = fma(oc.cr[q], s * s, fma(oc.ci[q], 2.0 * s * c, p));
        }
        P[(int64_t)r * n + k] = p;
    }
}

// Mixed: each phase as a double-float product (PH = 0) or in double (PH = 1),
// reduced modulo pi (sin^2 x and sin 2x have period pi), FP32 polynomials.
template <int PH>
__global__ void k_oscgen_mixed(const double* __restrict__ E, int64_t n, OscGenConst oc, float* __restrict__ P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float eh, el;
    ff_recip(E[k], eh, el);
    const double ed = (double)eh + (double)el;
    for (int r = 0; r < oc.nL; r++) {
        float p = 0.f;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float x = (PH == 0) ? reduce_pi_ff(oc.ch[q][r], oc.cl[q][r], eh, el) : reduce_pi_f64(oc.c[q][r], ed);
            float s, c;
            sincos_poly(x, s, c);
            p = fmaf(oc.crf[q], s * s, fmaf(oc.cif[q], 2.0f * s * c, p));
        }
        P[(int64_t)r * n + k] = p + (float)oc.dab;  // exact for delta_ab = 1 when p <= -1/2 (Sterbenz)
    }
}

cudaError_t launch_oscgen(const double* E, int64_t n, const OscGenConst& oc, int prec, void* P, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == GNA_FP64)
        k_oscgen64<<<blocks, 256, 0, s>>>(E, n, oc, (double*)P);
    else if (prec == GNA_MIXED_F64PHASE)
        k_oscgen_mixed<1><<<blocks, 256, 0, s>>>(E, n, oc, (float*)P);
    else
        k_oscgen_mixed<0><<<blocks, 256, 0, s>>>(E, n, oc, (float*)P);
    return cudaGetLastError();
}

}  // namespace gna
