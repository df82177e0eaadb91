// general.cu -- the any-channel chain: per-point coefficients (step a0 for
// P(alpha -> beta)), the node and slice-reduction kernels of general.cuh and
// their launchers.
#include <algorithm>
#include <mutex>

#include "general.cuh"

namespace gna {

// ------------------------------------------------------------ step a0 ----
// A real number with its derivatives in (s2_12, s2_13, s2_23, delta):
// forward-mode differentiation of the written-out mixing matrix.
struct Dn {
    double v, d[4];
};

__device__ inline Dn dn_const(double v) {
    Dn x;
    x.v = v;
    for (int q = 0; q < 4; q++) x.d[q] = 0.0;
    return x;
}
__device__ inline Dn dn_var(double v, int q, double dq) {
    Dn x = dn_const(v);
    x.d[q] = dq;
    return x;
}
__device__ inline Dn operator+(const Dn& a, const Dn& b) {
    Dn x;
    x.v = a.v + b.v;
    for (int q = 0; q < 4; q++) x.d[q] = a.d[q] + b.d[q];
    return x;
}
__device__ inline Dn operator-(const Dn& a, const Dn& b) {
    Dn x;
    x.v = a.v - b.v;
    for (int q = 0; q < 4; q++) x.d[q] = a.d[q] - b.d[q];
    return x;
}
__device__ inline Dn operator-(const Dn& a) { return dn_const(0.0) - a; }
__device__ inline Dn operator*(const Dn& a, const Dn& b) {
    Dn x;
    x.v = a.v * b.v;
    for (int q = 0; q < 4; q++) x.d[q] = a.d[q] * b.v + a.v * b.d[q];
    return x;
}

// Complex number of such reals.
struct Cn {
    Dn re, im;
};
__device__ inline Cn cn(const Dn& re, const Dn& im) { return Cn{re, im}; }
__device__ inline Cn operator+(const Cn& a, const Cn& b) { return Cn{a.re + b.re, a.im + b.im}; }
__device__ inline Cn operator*(const Cn& a, const Cn& b) {
    return Cn{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ inline Cn operator*(const Dn& a, const Cn& b) { return Cn{a * b.re, a * b.im}; }
__device__ inline Cn conjn(const Cn& a) { return Cn{a.re, -a.im}; }

// Coefficients of P(alpha -> beta) at one point: the mixing matrix in the
// standard parameterisation written out element by element (U = R23
// U13(delta) R12), X_ij = U*_ai U_bi U_aj U*_bj for the pairs (21, 31, 32),
// a = -4 Re X, b = 4 Im X, and for antineutrinos (V = U*, so X -> X*) b -> -b.
__device__ void general_coefficients(const gna_osc_full& o, int alpha, int beta, int anti, GenConst& gc) {
    const double s12v = sqrt(o.s2_12), c12v = sqrt(1.0 - o.s2_12);
    const double s13v = sqrt(o.s2_13), c13v = sqrt(1.0 - o.s2_13);
    const double s23v = sqrt(o.s2_23), c23v = sqrt(1.0 - o.s2_23);
    // d sin(theta) / d sin^2(theta) = 1 / (2 sin), d cos / d sin^2 = -1 / (2 cos)
    const Dn s12 = dn_var(s12v, 0, 0.5 / s12v), c12 = dn_var(c12v, 0, -0.5 / c12v);
    const Dn s13 = dn_var(s13v, 1, 0.5 / s13v), c13 = dn_var(c13v, 1, -0.5 / c13v);
    const Dn s23 = dn_var(s23v, 2, 0.5 / s23v), c23 = dn_var(c23v, 2, -0.5 / c23v);
    double sd, cd;
    sincos(o.delta_cp, &sd, &cd);
    const Dn cosd = dn_var(cd, 3, -sd), sind = dn_var(sd, 3, cd);
    const Cn ep = cn(cosd, sind);   // e^{+i delta}
    const Cn em = cn(cosd, -sind);  // e^{-i delta}
    const Dn zero = dn_const(0.0);
    const Cn s13ep = s13 * ep;
    Cn U[3][3];
    U[0][0] = cn(c12 * c13, zero);
    U[0][1] = cn(s12 * c13, zero);
    U[0][2] = s13 * em;
    U[1][0] = cn(-(s12 * c23), zero) + (-(c12 * s23)) * s13ep;
    U[1][1] = cn(c12 * c23, zero) + (-(s12 * s23)) * s13ep;
    U[1][2] = cn(s23 * c13, zero);
    U[2][0] = cn(s12 * s23, zero) + (-(c12 * c23)) * s13ep;
    U[2][1] = cn(-(c12 * s23), zero) + (-(s12 * c23)) * s13ep;
    U[2][2] = cn(c23 * c13, zero);
    const int pi_[3] = {1, 2, 2}, pj_[3] = {0, 0, 1};
    gc.dab = (alpha == beta) ? 1.0 : 0.0;
    for (int k = 0; k < 3; k++) {
        const int i = pi_[k], j = pj_[k];
        const Cn X = conjn(U[alpha][i]) * U[beta][i] * U[alpha][j] * conjn(U[beta][j]);
        const double sb = anti ? -4.0 : 4.0;
        gc.a[k] = -4.0 * X.re.v;
        gc.b[k] = sb * X.im.v;
        gc.af[k] = (float)gc.a[k];
        gc.bf[k] = (float)gc.b[k];
        for (int q = 0; q < 4; q++) {
            gc.da[q][k] = -4.0 * X.re.d[q];
            gc.db[q][k] = sb * X.im.d[q];
            gc.daf[q][k] = (float)gc.da[q][k];
            gc.dbf[q][k] = (float)gc.db[q][k];
        }
    }
}

// One thread per (point, baseline slot): the phase constants as for the
// survival chain; the point's first thread also forms its coefficients and
// checks that the mixing parameters lie inside (0, 1) (the derivatives are
// singular on the boundary).  Zeroes the evaluation's counters.
__global__ void k_prepare_general(const gna_osc_full* __restrict__ prm, int npts, BaseConst bc, int alpha, int beta,
                                  int anti, PointConst* __restrict__ out, GenConst* __restrict__ gout,
                                  int* __restrict__ zero, int64_t nz, int* __restrict__ status) {
    asm volatile("griddepcontrol.launch_dependents;");
    // a programmatic dependent of the kernel before it: wait for it first
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t k = tid; k < nz; k += (int64_t)gridDim.x * blockDim.x) zero[k] = 0;
    const int p = (int)(tid / GNA_NLMAX), r = (int)(tid % GNA_NLMAX);
    if (p >= npts) return;
    const gna_osc_full o = prm[p];
    PointConst& pc = out[p];
    const double kl = (r < bc.nL) ? bc.kld[r] : 0.0;
    const double c21 = o.dm2_21 * kl, c32 = o.dm2_32 * kl;
    pc.c21[r] = c21;
    pc.c32[r] = c32;
    split_ff(c21, pc.c21h[r], pc.c21l[r]);
    split_ff(c32, pc.c32h[r], pc.c32l[r]);
    if (r != 0) return;
    const bool inside = o.s2_12 > 0.0 && o.s2_12 < 1.0 && o.s2_13 > 0.0 && o.s2_13 < 1.0 && o.s2_23 > 0.0 &&
                        o.s2_23 < 1.0 && isfinite(o.delta_cp) && isfinite(o.dm2_21) && isfinite(o.dm2_32);
    if (!inside && status) atomicExch(status, (int)GNA_EINVAL);
    general_coefficients(o, alpha, beta, anti, gout[p]);
    double w = 0.0;
    for (int q = 0; q < bc.nL; q++) w += (double)bc.om[q] + (double)bc.omlo[q];
    gout[p].wsum = w;
}

cudaError_t launch_prepare_general(const gna_osc_full* prm, int npts, const BaseConst& bc, int alpha, int beta,
                                   int anti, PointConst* out, GenConst* gout, int* zero, int64_t nz, int* status,
                                   cudaStream_t s) {
    const int64_t threads = std::max<int64_t>((int64_t)npts * GNA_NLMAX, std::min<int64_t>(nz, 1LL << 20));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)((threads + 255) / 256));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_prepare_general, prm, npts, bc, alpha, beta, anti, out, gout, zero, nz, status);
}

// ------------------------------------------------------------ launchers ----
template <int PH, int NL, bool GRAD, bool SURV>
static cudaError_t launch_gen(const GenArgs& a, int grid, int block, cudaStream_t s) {
    return launch_dependent(k_fused_bins_gen<PH, NL, GRAD, SURV>, a, grid, block, s);
}

template <int PH, int NL>
static cudaError_t launch_gen_nl(bool grad, bool surv, const GenArgs& a, int grid, int block, cudaStream_t s) {
    if (grad) return surv ? launch_gen<PH, NL, true, true>(a, grid, block, s) : launch_gen<PH, NL, true, false>(a, grid, block, s);
    return surv ? launch_gen<PH, NL, false, true>(a, grid, block, s) : launch_gen<PH, NL, false, false>(a, grid, block, s);
}

template <int PH>
static cudaError_t dispatch_gen_ph(int nl, bool grad, bool surv, const GenArgs& a, int grid, int block, cudaStream_t s) {
    switch (nl) {
        case 1: return launch_gen_nl<PH, 1>(grad, surv, a, grid, block, s);
        case 2: return launch_gen_nl<PH, 2>(grad, surv, a, grid, block, s);
        case 4: return launch_gen_nl<PH, 4>(grad, surv, a, grid, block, s);
        case 8: return launch_gen_nl<PH, 8>(grad, surv, a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename Kernel>
static int occupancy(Kernel k, int block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

template <int PH, int NL>
static int resident_gen_nl(bool grad, bool surv, int block) {
    if (grad) return surv ? occupancy(k_fused_bins_gen<PH, NL, true, true>, block) : occupancy(k_fused_bins_gen<PH, NL, true, false>, block);
    return surv ? occupancy(k_fused_bins_gen<PH, NL, false, true>, block) : occupancy(k_fused_bins_gen<PH, NL, false, false>, block);
}

template <int PH>
static int resident_gen_ph(int nl, bool grad, bool surv, int block) {
    switch (nl) {
        case 1: return resident_gen_nl<PH, 1>(grad, surv, block);
        case 2: return resident_gen_nl<PH, 2>(grad, surv, block);
        case 4: return resident_gen_nl<PH, 4>(grad, surv, block);
        case 8: return resident_gen_nl<PH, 8>(grad, surv, block);
        default: return 1;
    }
}

static int resident_gen64(int nl, bool grad, int block) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (nl * 2 + (grad ? 1 : 0)) {
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<1, false>, block, 0); break;
        case 3: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<1, true>, block, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<2, false>, block, 0); break;
        case 5: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<2, true>, block, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<4, false>, block, 0); break;
        case 9: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<4, true>, block, 0); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<8, false>, block, 0); break;
        case 17: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused64_bins_gen<8, true>, block, 0); break;
        default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

int general_resident_ctas(int ph, int nl, bool grad, bool surv, int block) {
    if (ph == 2) return resident_gen64(nl, grad, block);
    return ph == 0 ? resident_gen_ph<0>(nl, grad, surv, block) : resident_gen_ph<1>(nl, grad, surv, block);
}

template <int NL, bool GRAD>
static cudaError_t launch_gen64(const GenArgs64& a, int grid, int block, cudaStream_t s) {
    k_fused64_bins_gen<NL, GRAD><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch_general64(int nl, bool grad, const GenArgs64& a, int grid, int block, cudaStream_t s) {
    switch (nl * 2 + (grad ? 1 : 0)) {
        case 2: return launch_gen64<1, false>(a, grid, block, s);
        case 3: return launch_gen64<1, true>(a, grid, block, s);
        case 4: return launch_gen64<2, false>(a, grid, block, s);
        case 5: return launch_gen64<2, true>(a, grid, block, s);
        case 8: return launch_gen64<4, false>(a, grid, block, s);
        case 9: return launch_gen64<4, true>(a, grid, block, s);
        case 16: return launch_gen64<8, false>(a, grid, block, s);
        case 17: return launch_gen64<8, true>(a, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t dispatch_general(int ph, int nl, bool grad, bool surv, const GenArgs& a, int grid, int block,
                             cudaStream_t s) {
    if (ph == 0) return dispatch_gen_ph<0>(nl, grad, surv, a, grid, block, s);
    if (ph == 1) return dispatch_gen_ph<1>(nl, grad, surv, a, grid, block, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_slices_reduce_general(const float2* part, int S, int NV, const EpiArgs& ea, const GenConst* gc,
                                         int npts, cudaStream_t s) {
    constexpr int W = 24;
    if (NV != gen_nv(false) && NV != gen_nv(true)) return cudaErrorInvalidValue;
    static std::once_flag once[64];
    static cudaError_t attr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::call_once(once[dev], [&] {
        attr[dev] = cudaFuncSetAttribute(k_slices_reduce_gen<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(float2) * W * gen_nv(true) * 32 + sizeof(double) * gen_nv(true) * 32));
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
    return cudaLaunchKernelEx(&cfg, k_slices_reduce_gen<W>, part, S, NV, ea, gc);
}

}  // namespace gna
