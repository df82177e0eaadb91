// kernels_misc.cu -- everything on the device except the fused node loop:
// parameter preparation (step a0), the Gauss-Legendre rule and energy grids
// (step a1, configuration stage), the chi^2 epilogue (steps a7-a9), the plain
// FP64 one-kernel-per-transformation chain, the element-wise OscProb
// transformation and the Levenberg-Marquardt update.
#include <math.h>

#include "common.cuh"
#include "gnaosc.h"
#include <algorithm>

#include "misc.h"

namespace gna {

// --------------------------------------------------------------- step a0 --
// |U_e1|^2 = (1-s12)(1-s13), |U_e2|^2 = s12 (1-s13), |U_e3|^2 = s13 give
// A21 = 4 s12 (1-s12)(1-s13)^2, A31 = 4 (1-s12)(1-s13) s13, A32 = 4 s12 (1-s13) s13
// and their derivatives with respect to s12 = sin^2 theta12, s13 = sin^2 theta13;
// the phase constants are c_ij,r = K dm2_ij L_r.  One thread per (point, baseline slot).
// Also zeroes the evaluation's nz counters (the node kernel that follows is a
// programmatic dependent: it may be launched as soon as this kernel starts and
// waits in hardware for its completion before touching counters or constants).
__global__ void k_prepare_points(const gna_osc* __restrict__ prm, int npts, BaseConst bc, PointConst* __restrict__ out,
                                 int* __restrict__ zero, int64_t nz, int* __restrict__ status) {
    asm volatile("griddepcontrol.launch_dependents;");
    // launched as a programmatic dependent of the kernel before it (that
    // kernel's launch latency is hidden): wait until it has completed and its
    // writes are visible before touching the counters and constants it may use
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t k = tid; k < nz; k += (int64_t)gridDim.x * blockDim.x) zero[k] = 0;
    const int64_t idx = tid;
    const int p = (int)(idx / GNA_NLMAX), r = (int)(idx % GNA_NLMAX);
    if (p >= npts) return;
    const gna_osc o = prm[p];
    PointConst& pc = out[p];
    // the parameters live on the device: a point outside the physical domain
    // (s2 outside [0, 1], a mass splitting not finite) is reported through the
    // plan's status word (gna_plan_status); its results are not meaningful
    if (r == 0 && status &&
        !(o.s2_12 >= 0.0 && o.s2_12 <= 1.0 && o.s2_13 >= 0.0 && o.s2_13 <= 1.0 && isfinite(o.dm2_21) &&
          isfinite(o.dm2_32)))
        atomicExch(status, (int)GNA_EINVAL);
    const double kl = (r < bc.nL) ? bc.kld[r] : 0.0;
    const double c21 = o.dm2_21 * kl, c32 = o.dm2_32 * kl;
    pc.c21[r] = c21;
    pc.c32[r] = c32;
    split_ff(c21, pc.c21h[r], pc.c21l[r]);
    split_ff(c32, pc.c32h[r], pc.c32l[r]);
    if (r == 0) {
        const double s12 = o.s2_12, s13 = o.s2_13;
        const double c12 = 1.0 - s12, c13 = 1.0 - s13;
        double A[3], d12[3], d13[3];
        A[0] = 4.0 * s12 * c12 * c13 * c13;
        A[1] = 4.0 * c12 * c13 * s13;
        A[2] = 4.0 * s12 * c13 * s13;
        d12[0] = 4.0 * (1.0 - 2.0 * s12) * c13 * c13;
        d12[1] = -4.0 * c13 * s13;
        d12[2] = 4.0 * c13 * s13;
        d13[0] = -8.0 * s12 * c12 * c13;
        d13[1] = 4.0 * c12 * (1.0 - 2.0 * s13);
        d13[2] = 4.0 * s12 * (1.0 - 2.0 * s13);
        for (int j = 0; j < 3; j++) {
            pc.A[j] = A[j];
            pc.dA12[j] = d12[j];
            pc.dA13[j] = d13[j];
            pc.Af[j] = (float)A[j];
            pc.Alo[j] = (float)(A[j] - (double)(float)A[j]);
            pc.dA12f[j] = (float)d12[j];
            pc.dA13f[j] = (float)d13[j];
        }
    }
}

cudaError_t launch_prepare(const gna_osc* prm, int npts, const BaseConst& bc, PointConst* out, cudaStream_t s,
                           int* zero, int64_t nz, int* status) {
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
    return cudaLaunchKernelEx(&cfg, k_prepare_points, prm, npts, bc, out, zero, nz, status);
}

// --------------------------------------------------------------- step a1 --
// Gauss-Legendre rule of order n: Newton iteration on P_n evaluated by the
// three-term recurrence P_{j+1} = a_j x P_j - b_j P_{j-1}, a_j = (2j+1)/(j+1),
// b_j = j/(j+1) (tabulated once per order), from Tricomi's asymptotic
// estimate of the k-th root; P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1);
// w = 2 / ((1 - x^2) P_n'(x)^2), with 1 - x^2 formed as (1 - x)(1 + x).
// One thread per root pair (x, -x).
__global__ void k_legendre_coef(int n, double* __restrict__ a, double* __restrict__ b) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    a[j] = (2.0 * j + 1.0) / (j + 1.0);
    b[j] = (double)j / (j + 1.0);
}

__device__ __forceinline__ void legendre_pair(int n, double x, const double* __restrict__ a, const double* __restrict__ b,
                                              double& pn, double& pn1) {
    double p0 = 1.0, p1 = x;
    for (int j = 1; j < n; j++) {
        const double p2 = a[j] * x * p1 - b[j] * p0;
        p0 = p1;
        p1 = p2;
    }
    pn = (n == 0) ? 1.0 : p1;
    pn1 = (n == 0) ? 0.0 : p0;
}

__global__ void k_gl_roots(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ x,
                           double* __restrict__ w) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // k-th largest root, 0-based
    const int half = (n + 1) / 2;
    if (k >= half) return;
    const double nn = (double)n;
    const double theta = M_PI * (4.0 * k + 3.0) / (4.0 * nn + 2.0);
    double xk = (1.0 - (nn - 1.0) / (8.0 * nn * nn * nn)) * cos(theta);
    if ((n & 1) && k == half - 1) xk = 0.0;  // middle root of odd orders
    double pn = 0, pn1 = 0, dp = 1;
    for (int it = 0; it < 12; it++) {
        legendre_pair(n, xk, a, b, pn, pn1);
        dp = nn * (xk * pn - pn1) / ((xk - 1.0) * (xk + 1.0));
        const double dx = pn / dp;
        xk -= dx;
        if (fabs(dx) <= 2e-16 * fabs(xk) + 1e-300) break;
    }
    if ((n & 1) && k == half - 1) xk = 0.0;
    legendre_pair(n, xk, a, b, pn, pn1);
    dp = nn * (xk * pn - pn1) / ((xk - 1.0) * (xk + 1.0));
    const double wk = 2.0 / (((1.0 - xk) * (1.0 + xk)) * dp * dp);  // 1 - x^2 without cancellation near +-1
    x[n - 1 - k] = xk;
    w[n - 1 - k] = wk;
    x[k] = -xk;
    w[k] = wk;
}

cudaError_t launch_gl(int n, double* x, double* w, double* tmp_ab /*[2n]*/, cudaStream_t s) {
    k_legendre_coef<<<(n + 255) / 256, 256, 0, s>>>(n, tmp_ab, tmp_ab + n);
    const int half = (n + 1) / 2;
    k_gl_roots<<<(half + 63) / 64, 64, 0, s>>>(n, tmp_ab, tmp_ab + n, x, w);
    return cudaGetLastError();
}

// Energy grid of one point: E_ik = (a_i+b_i)/2 + (b_i-a_i)/2 x_k, stored as
// 1/E split into two floats, W = (b_i-a_i)/2 w_k S(E_ik e_scale) with the
// reactor shape S(E) = exp(0.87 - 0.16 E - 0.091 E^2), and W/E.  Layout 0:
// bin-major (node k of bin i at i*n + k); layout 1: groups of 32 bins,
// node k of bin i at ((i/32) n + k) 32 + i%32, padded bins have W = 0.
__global__ void k_build_grid(int nbins, int nbins_pad, const double* __restrict__ edges, int n, const double* __restrict__ x,
                             const double* __restrict__ w, double e_scale, int layout, float4* __restrict__ ff,
                             double2* __restrict__ d64, double2* __restrict__ plain64) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nbins_pad * n) return;
    const int i = (int)(idx / n);
    const int k = (int)(idx - (int64_t)i * n);
    double invE = 1.0, Wd = 0.0;
    if (i < nbins) {
        const double a = edges[i], b = edges[i + 1];
        const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
        const double E = mid + half * x[k];
        const double Es = E * e_scale;
        invE = 1.0 / E;
        Wd = half * w[k] * exp(0.87 - 0.16 * Es - 0.091 * Es * Es);
    }
    const int64_t pos = (layout == 0) ? idx : (((int64_t)(i >> 5) * n + k) * 32 + (i & 31));
    if (ff) {
        float hi, lo;
        split_ff(invE, hi, lo);
        ff[pos] = make_float4(hi, lo, (float)Wd, (float)(Wd * invE));
    }
    if (d64) d64[pos] = make_double2(invE, Wd);
    if (plain64 && i < nbins) plain64[idx] = make_double2(invE, Wd);
}

// Sum of the FP32 node weights of each bin, in double (for the epilogue's
// exact correction of the constant term): one warp per bin, lane l takes
// nodes l, l + 32, ... (coalesced in layout 0), then a fixed-order butterfly.
__global__ void k_sum_weights(const float4* __restrict__ grid, int nbins, int n, int layout, double* __restrict__ out) {
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nbins) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) {
        const int64_t pos = (layout == 0) ? (int64_t)i * n + k : (((int64_t)(i >> 5) * n + k) * 32 + (i & 31));
        s += (double)grid[pos].z;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

cudaError_t launch_sum_weights(const float4* grid, int nbins, int n, int layout, double* out, cudaStream_t s) {
    k_sum_weights<<<(unsigned)(((int64_t)nbins * 32 + 255) / 256), 256, 0, s>>>(grid, nbins, n, layout, out);
    return cudaGetLastError();
}

cudaError_t launch_build_grid(int nbins, int nbins_pad, const double* edges, int n, const double* x, const double* w,
                              double e_scale, int layout, float4* ff, double2* d64, double2* plain64, cudaStream_t s) {
    const int64_t total = (int64_t)nbins_pad * n;
    const int64_t blocks = (total + 255) / 256;
    k_build_grid<<<(unsigned)blocks, 256, 0, s>>>(nbins, nbins_pad, edges, n, x, w, e_scale, layout, ff, d64, plain64);
    return cudaGetLastError();
}

// ------------------------------------------------- plain FP64 chain -------
// One kernel per transformation of the paper's chain, intermediates in
// device memory: OscProb (+ tangents) -> weight -> bin integration -> chi^2.
// A launch covers a chunk of points, flattened over (point, baseline, node):
// element e of the chunk belongs to the point p with off[p] <= off[p0] + e <
// off[p + 1], whose grid has n_p nodes per bin; within the point, baseline
// r = local / (nbins n_p) and bin-major node k = local mod (nbins n_p).

// The point of flattened element e: the largest p in [p0, p0 + cnt) with off[p] <= e.
__device__ __forceinline__ int plain_point(const int64_t* __restrict__ off, int p0, int cnt, int64_t e) {
    int lo = p0, hi = p0 + cnt - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int plain_nodes(const PlainArgs& a, int p) { return a.gn[a.gid ? a.gid[p] : 0]; }

// node of flattened element idx (0 <= idx < len), and its point and baseline
__device__ __forceinline__ double2 plain_node(const PlainArgs& a, int64_t idx, int& p, int& r) {
    const int64_t e = a.off[a.p0] + idx;
    p = plain_point(a.off, a.p0, a.cnt, e);
    const int64_t nn = (int64_t)a.nbins * plain_nodes(a, p);
    const int64_t local = e - a.off[p];
    r = (int)(local / nn);
    const int64_t k = local - (int64_t)r * nn;
    return a.nodes[a.goff[a.gid ? a.gid[p] : 0] + k];
}

__global__ void k_plain_prob(PlainArgs a) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.len) return;
    int p, r;
    const double e = plain_node(a, idx, p, r).x;
    const PointConst& pc = a.pcs[p];
    const double x21 = pc.c21[r] * e, x32 = pc.c32[r] * e, x31 = (pc.c21[r] + pc.c32[r]) * e;
    double s21, c21, s31, c31, s32, c32;
    sincos(x21, &s21, &c21);
    sincos(x31, &s31, &c31);
    sincos(x32, &s32, &c32);
    const double S21 = s21 * s21, S31 = s31 * s31, S32 = s32 * s32;
    a.P[idx] = 1.0 - pc.A[0] * S21 - pc.A[1] * S31 - pc.A[2] * S32;
    if (a.grad) {
        const int64_t stride = a.len;
        const double kle = a.bc.kld[r] * e;
        a.dP[idx] = -(pc.dA12[0] * S21 + pc.dA12[1] * S31 + pc.dA12[2] * S32);
        a.dP[stride + idx] = -(pc.dA13[0] * S21 + pc.dA13[1] * S31 + pc.dA13[2] * S32);
        a.dP[2 * stride + idx] = -(pc.A[0] * 2.0 * s21 * c21 + pc.A[1] * 2.0 * s31 * c31) * kle;
        a.dP[3 * stride + idx] = -(pc.A[1] * 2.0 * s31 * c31 + pc.A[2] * 2.0 * s32 * c32) * kle;
    }
}

// V[q][idx] *= W of idx's node, for rows q of the chunk's len elements
__global__ void k_plain_weight(PlainArgs a, int rows, double* __restrict__ V) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.len * rows) return;
    int p, r;
    V[t] *= plain_node(a, t % a.len, p, r).y;
}

// one warp per (row q, point, baseline, bin): out[q][pl][r][i] = sum over the bin's nodes
__global__ void k_plain_binint(PlainArgs a, int rows, const double* __restrict__ V, double* __restrict__ out) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t per_row = (int64_t)a.cnt * a.nL * a.nbins;
    if (w >= rows * per_row) return;
    const int64_t q = w / per_row;
    const int64_t rem = w - q * per_row;
    const int pl = (int)(rem / ((int64_t)a.nL * a.nbins));
    const int rb = (int)(rem - (int64_t)pl * a.nL * a.nbins);  // r nbins + i
    const int p = a.p0 + pl;
    const int n = plain_nodes(a, p);
    const double* src = V + q * a.len + (a.off[p] - a.off[a.p0]) + (int64_t)rb * n;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += src[k];
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[w] = s;
}

// one CTA per point of the chunk; mu_r [cnt][nL][nbins], dmu [4][cnt][nL][nbins]
__global__ void k_plain_chi2(PlainChi2Args a) {
    __shared__ double sh[5][256];
    const int pl = blockIdx.x;
    const int p = a.p0 + pl;
    const double* mu_r = a.mu_r + (int64_t)pl * a.nL * a.nbins;
    const double* data = a.data + (a.dpp ? (int64_t)p * a.nbins : 0);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
        double M = 0, D[4] = {0, 0, 0, 0};
        for (int r = 0; r < a.nL; r++) {
            M += a.bc.omd[r] * mu_r[(int64_t)r * a.nbins + i];
            if (a.dmu)
                for (int q = 0; q < 4; q++)
                    D[q] += a.bc.omd[r] * a.dmu[(((int64_t)q * a.cnt + pl) * a.nL + r) * a.nbins + i];
        }
        const double e = a.eta ? a.eta[i] : 0.0;
        const double f = a.norm * (1.0 + e);
        const double mu = f * M;
        const double d = data[i];
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
        acc[0] += term;
        for (int q = 0; q < 4; q++) acc[1 + q] += g * f * D[q];
        if (a.mu_out) a.mu_out[(int64_t)p * a.nbins + i] = mu;
        if (a.grad_eta_out)
            a.grad_eta_out[(int64_t)p * a.nbins + i] = g * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
        if (a.spectra_out)
            for (int r = 0; r < a.nL; r++)
                a.spectra_out[((int64_t)p * a.nL + r) * a.nbins + i] = mu_r[(int64_t)r * a.nbins + i];
    }
    for (int v = 0; v < 5; v++) sh[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int v = 0; v < 5; v++) sh[v][threadIdx.x] += sh[v][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.chi2[p] = sh[0][0];
        if (a.grad)
            for (int q = 0; q < 4; q++) a.grad[(int64_t)p * 4 + q] = sh[1 + q][0];
    }
}

cudaError_t launch_plain_chunk(const PlainArgs& a, const PlainChi2Args& ca, cudaStream_t s) {
    const int64_t rows = a.grad ? 4 : 0;
    k_plain_prob<<<(unsigned)((a.len + 255) / 256), 256, 0, s>>>(a);
    k_plain_weight<<<(unsigned)((a.len + 255) / 256), 256, 0, s>>>(a, 1, a.P);
    if (a.grad) k_plain_weight<<<(unsigned)((rows * a.len + 255) / 256), 256, 0, s>>>(a, 4, a.dP);
    const int64_t w1 = (int64_t)a.cnt * a.nL * a.nbins * 32;
    k_plain_binint<<<(unsigned)((w1 + 255) / 256), 256, 0, s>>>(a, 1, a.P, a.mu_r);
    if (a.grad) k_plain_binint<<<(unsigned)((rows * w1 + 255) / 256), 256, 0, s>>>(a, 4, a.dP, a.dmu);
    k_plain_chi2<<<(unsigned)a.cnt, 256, 0, s>>>(ca);
    return cudaGetLastError();
}

// -------------------------------------------------- element-wise OscProb --
// FP64: P[r][k] = 1 - sum_ij A_ij sin^2(c_ij,r / E_k), CUDA double sin.
__global__ void k_oscprob64(const double* __restrict__ E, int64_t n, OscConst oc, double* __restrict__ P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double e = 1.0 / E[k];
    for (int r = 0; r < oc.nL; r++) {
        const double s21 = sin(oc.c21[r] * e), s32 = sin(oc.c32[r] * e), s31 = sin((oc.c21[r] + oc.c32[r]) * e);
        P[(int64_t)r * n + k] = 1.0 - oc.A[0] * s21 * s21 - oc.A[1] * s31 * s31 - oc.A[2] * s32 * s32;
    }
}

// Mixed: each phase reduced modulo pi/2 (quadrant parity q), sin r by the
// FP32 polynomial; sin^2(phase) = s^2 for even q, 1 - s^2 for odd q.  The
// dominant term is written as (1 - A21) + A21 s^2 for odd q so that P stays
// accurate to a few ulp where it is smallest.
template <int PH>
__device__ __forceinline__ float reduce_half_pi(float ch, float cl, double cd, float eh, float el, double ed, int& odd) {
    if (PH == 0) {
        float p = __fmul_rn(ch, eh);
        float e = __fmaf_rn(ch, eh, -p);
        float lo = __fmaf_rn(ch, el, __fmaf_rn(cl, eh, e));
        float qm = __fmaf_rn(p, 2.0f * GNA_INV_PI_F, GNA_ROUND_MAGIC);
        odd = __float_as_int(qm) & 1;
        float q = __fsub_rn(qm, GNA_ROUND_MAGIC);
        float r = __fmaf_rn(-q, 0.5f * GNA_PI_A, p);
        r = __fmaf_rn(-q, 0.5f * GNA_PI_B, r);
        r = __fmaf_rn(-q, 0.5f * GNA_PI_C, r);
        return __fadd_rn(r, lo);
    } else {
        double p = cd * ed;
        double q = rint(p * (2.0 * GNA_INV_PI_D));
        odd = ((long long)q) & 1;
        double r = fma(-q, 0.5 * GNA_PI_DA, p);
        r = fma(-q, 0.5 * GNA_PI_DB, r);
        r = fma(-q, 0.5 * GNA_PI_DC, r);
        return (float)r;
    }
}

template <int PH>
__global__ void k_oscprob_mixed(const double* __restrict__ E, int64_t n, OscConst oc, float* __restrict__ P) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float eh, el;
    ff_recip(E[k], eh, el);
    const double ed = (double)eh + (double)el;
    const float A21 = oc.Af[0], A31 = oc.Af[1], A32 = oc.Af[2];
    const float omA21 = oc.one_minus_A21f;
    for (int r = 0; r < oc.nL; r++) {
        int o21, o31, o32;
        const float r21 = reduce_half_pi<PH>(oc.c21h[r], oc.c21l[r], oc.c21[r], eh, el, ed, o21);
        const float r31 = reduce_half_pi<PH>(oc.c31h[r], oc.c31l[r], oc.c21[r] + oc.c32[r], eh, el, ed, o31);
        const float r32 = reduce_half_pi<PH>(oc.c32h[r], oc.c32l[r], oc.c32[r], eh, el, ed, o32);
        const float s21 = sin_poly(r21), s31 = sin_poly(r31), s32 = sin_poly(r32);
        const float q21 = s21 * s21, q31 = s31 * s31, q32 = s32 * s32;
        const float S31 = o31 ? 1.0f - q31 : q31;
        const float S32 = o32 ? 1.0f - q32 : q32;
        const float base = o21 ? fmaf(A21, q21, omA21) : fmaf(-A21, q21, 1.0f);
        P[(int64_t)r * n + k] = fmaf(-A32, S32, fmaf(-A31, S31, base));
    }
}

cudaError_t launch_oscprob(const double* E, int64_t n, const OscConst& oc, int prec, void* P, cudaStream_t s) {
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (prec == GNA_FP64)
        k_oscprob64<<<blocks, 256, 0, s>>>(E, n, oc, (double*)P);
    else if (prec == GNA_MIXED_F64PHASE)
        k_oscprob_mixed<1><<<blocks, 256, 0, s>>>(E, n, oc, (float*)P);
    else
        k_oscprob_mixed<0><<<blocks, 256, 0, s>>>(E, n, oc, (float*)P);
    return cudaGetLastError();
}

// ------------------------------------------------------------- step a11 --
// Batched Levenberg-Marquardt, one thread per data set, NP = 4 (survival
// chain: s2_12, s2_13, dm2_21, dm2_32) or 6 (any channel: s2_12, s2_13,
// s2_23, delta_cp, dm2_21, dm2_32).  The parameters are NP consecutive doubles
// per point (the layout of gna_osc and of gna_osc_full).
template <int NP>
__global__ void k_lm_init(LMStateT<NP>* __restrict__ st, int npts, double lam0) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    LMStateT<NP> s;
    for (int q = 0; q < NP; q++) {
        s.best[q] = 0.0;
        s.g[q] = 0.0;
    }
    for (int q = 0; q < NP * (NP + 1) / 2; q++) s.H[q] = 0.0;
    s.chi2 = HUGE_VAL;
    s.lam = lam0;
    st[p] = s;
}

// Box of the trials: mixing parameters (sin^2) in [1e-6, 1 - 1e-6], mass
// splittings >= 1e-7 eV^2, delta_cp free.
template <int NP>
__device__ __forceinline__ void lm_box(int q, double& lo, double& hi) {
    const bool mix = (NP == 4) ? q < 2 : q < 3;
    const bool cp = (NP == 6) && q == 3;
    lo = mix ? 1e-6 : cp ? -HUGE_VAL : 1e-7;
    hi = mix ? 1.0 - 1e-6 : HUGE_VAL;
}

// One iteration per data set: accept the trial just evaluated if its chi^2
// improved on the best (lambda / 10) else reject it (lambda x 10); solve
// (H + lambda diag H) delta = -g at the best point (Gaussian elimination with
// partial pivoting, FP64) and write the next trial, clamped into the box.
template <int NP>
__global__ void k_lm_update(int npts, const double* __restrict__ chi2, const double* __restrict__ grad,
                            const double* __restrict__ H, LMStateT<NP>* __restrict__ st, double* __restrict__ prm,
                            double* __restrict__ chi2_best) {
    constexpr int NH = NP * (NP + 1) / 2;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    LMStateT<NP> s = st[p];
    double* th = prm + (int64_t)p * NP;
    const double c = chi2[p];
    if (c < s.chi2) {
        s.chi2 = c;
        for (int q = 0; q < NP; q++) {
            s.best[q] = th[q];
            s.g[q] = grad[(int64_t)p * NP + q];
        }
        for (int q = 0; q < NH; q++) s.H[q] = H[(int64_t)p * NH + q];
        s.lam = s.lam / 10.0;
    } else {
        s.lam = s.lam * 10.0;
    }
    double A[NP][NP + 1];
    int t = 0;
    for (int q = 0; q < NP; q++)
        for (int r = q; r < NP; r++) {
            A[q][r] = s.H[t];
            A[r][q] = s.H[t];
            t++;
        }
    for (int q = 0; q < NP; q++) {
        A[q][q] += s.lam * A[q][q];
        A[q][NP] = -s.g[q];
    }
    bool ok = true;
    for (int col = 0; col < NP; col++) {
        int piv = col;
        for (int r = col + 1; r < NP; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (!(fabs(A[piv][col]) > 0.0)) {
            ok = false;
            break;
        }
        if (piv != col)
            for (int j = 0; j <= NP; j++) {
                const double tmp = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = tmp;
            }
        for (int r = col + 1; r < NP; r++) {
            const double m = A[r][col] / A[col][col];
            for (int j = col; j <= NP; j++) A[r][j] -= m * A[col][j];
        }
    }
    double delta[NP];
    for (int q = 0; q < NP; q++) delta[q] = 0.0;
    if (ok)
        for (int q = NP - 1; q >= 0; q--) {
            double acc = A[q][NP];
            for (int j = q + 1; j < NP; j++) acc -= A[q][j] * delta[j];
            delta[q] = acc / A[q][q];
        }
    for (int q = 0; q < NP; q++) {
        double lo, hi;
        lm_box<NP>(q, lo, hi);
        th[q] = fmin(fmax(s.best[q] + delta[q], lo), hi);
    }
    st[p] = s;
    if (chi2_best) chi2_best[p] = s.chi2;
}

template <int NP>
__global__ void k_lm_finish(int npts, const LMStateT<NP>* __restrict__ st, double* __restrict__ prm) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npts) return;
    for (int q = 0; q < NP; q++) prm[(int64_t)p * NP + q] = st[p].best[q];
}

template <int NP>
cudaError_t launch_lm_init(LMStateT<NP>* st, int npts, double lam0, cudaStream_t s) {
    k_lm_init<NP><<<(npts + 127) / 128, 128, 0, s>>>(st, npts, lam0);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_lm_update(int npts, const double* chi2, const double* grad, const double* H, LMStateT<NP>* st,
                             double* prm, double* chi2_best, cudaStream_t s) {
    k_lm_update<NP><<<(npts + 127) / 128, 128, 0, s>>>(npts, chi2, grad, H, st, prm, chi2_best);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_lm_finish(int npts, const LMStateT<NP>* st, double* prm, cudaStream_t s) {
    k_lm_finish<NP><<<(npts + 127) / 128, 128, 0, s>>>(npts, st, prm);
    return cudaGetLastError();
}

template cudaError_t launch_lm_init<4>(LMStateT<4>*, int, double, cudaStream_t);
template cudaError_t launch_lm_init<6>(LMStateT<6>*, int, double, cudaStream_t);
template cudaError_t launch_lm_update<4>(int, const double*, const double*, const double*, LMStateT<4>*, double*,
                                         double*, cudaStream_t);
template cudaError_t launch_lm_update<6>(int, const double*, const double*, const double*, LMStateT<6>*, double*,
                                         double*, cudaStream_t);
template cudaError_t launch_lm_finish<4>(int, const LMStateT<4>*, double*, cudaStream_t);
template cudaError_t launch_lm_finish<6>(int, const LMStateT<6>*, double*, cudaStream_t);

}  // namespace gna


namespace gna {

// -------------------------------------------------- FP32 rate probe -------
// Eight independent FMA chains per thread, `iters` steps each: the FP32 pipe
// rate that the node kernels are measured against (FMA = one operation).  The
// sum is stored only if it reaches a value the chains cannot reach, so the
// work is kept and nothing is written.
__global__ void __launch_bounds__(256) k_fma_probe(int iters, float* __restrict__ out) {
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; j++) a[j] = 1.0f + 1e-3f * (float)(j + (threadIdx.x & 7));
    const float m = 0.99999994f, c = 5.9604645e-8f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++) a[j] = fmaf(a[j], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; j++) s += a[j];
    if (s == -1.0f) out[0] = s;
}

cudaError_t launch_fma_probe(int blocks, int iters, float* out, cudaStream_t s) {
    k_fma_probe<<<blocks, 256, 0, s>>>(iters, out);
    return cudaGetLastError();
}

// a[i] *= *s (i < na), b[j] *= *s (j < nb): one grid-stride pass over both.
__global__ void __launch_bounds__(256) k_grad_scale(double* a, int64_t na, double* b, int64_t nb, const double* s) {
    const double f = *s;
    const int64_t n = na + nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < na) a[i] *= f;
        else b[i - na] *= f;
    }
}

cudaError_t launch_grad_scale(double* a, int64_t na, double* b, int64_t nb, const double* s, cudaStream_t st) {
    const int64_t n = na + nb;
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 1024);
    k_grad_scale<<<grid, 256, 0, st>>>(a, na, b, nb, s);
    return cudaGetLastError();
}

}  // namespace gna
