// general.cuh -- the chain for any channel P(alpha -> beta), neutrinos or
// antineutrinos, with the gradient in the six parameters (s2_12, s2_13,
// s2_23, delta_cp, dm2_21, dm2_32).
//
// Paper Sec. 4.1: P = delta_ab + sum_{i>j} [-4 Re X_ij sin^2 x_ij
// + 2 Im X_ij sin 2x_ij], X_ij = V*_ai V_bi V_aj V*_bj.  Writing
// a_ij = -4 Re X_ij, b_ij = 4 Im X_ij (sin 2x = 2 sin x cos x):
//   P = delta_ab + sum_ij (a_ij S_ij + b_ij C_ij),  S = sin^2 x, C = sin x cos x.
// The coefficients depend only on the mixing parameters and the channel, the
// phases only on the mass splittings, so the node pass accumulates
// channel-free sums and the epilogue contracts them with the point's
// coefficients:
//   U_ij = sum_k W_k sum_r omega_r S_ij,   V_ij = sum_k W_k sum_r omega_r C_ij,
//   Y_ij = sum_k W_k/E_k sum_r w_r C_ij,   Z_ij = sum_k W_k/E_k sum_r w_r (cos^2 - sin^2)_ij,
// w_r = 2 omega_r K L_r.  Then per bin
//   M = delta_ab sum_k W_k + sum_ij (a_ij U_ij + b_ij V_ij),
//   dM/dp = sum_ij (da_ij/dp U_ij + db_ij/dp V_ij) for the mixing parameters,
//   dM/d dm2_21 = sum_{ij = 21, 31} (a_ij Y_ij + b_ij Z_ij / 2),
//   dM/d dm2_32 = sum_{ij = 32, 31} (a_ij Y_ij + b_ij Z_ij / 2)
// (d S / dx = 2 C, d C / dx = cos^2 - sin^2, dx/d dm2 = K L / E).
//
// Survival channels cancel: P = 1 + sum a S with a = -4 |V_ai|^2 |V_aj|^2 of
// order -1, so where S -> 1 (a disappearance dip) M is a small difference of
// sum W and a U, and the FP32 rounding of S near 1 (~6e-8 absolute per node)
// becomes a large relative error of M.  Appearance channels cancel too, less:
// by unitarity a_31 S_31 + a_32 S_32 (terms of ~0.2 for nu_mu -> nu_e) nearly
// cancel as both S -> 1.  The mixed node pass therefore also accumulates
// Q_ij = sum_k W_k sum_r omega_r cos^2 x_ij, and the epilogue takes each
// pair's sine sum either as U_ij or, when Q_ij < U_ij, as
// sum_k W_k sum_r omega_r - Q_ij (sin^2 + cos^2 = 1, applied in double): both
// sums add positive terms, so the one used carries an error relative to the
// smaller of the two, and the large parts cancel in double.
// These kernels reuse the energy-grid layouts, the bin/slice task scheme and
// the group and point reductions of the nue_bar survival chain; they are
// separate kernels so that the survival chain's code stays as it is.
#pragma once

#include "epilogue.cuh"
#include "fused.cuh"
#include "fused64.cuh"

namespace gna {

// Per-point coefficients of the general channel (prepared on the device).
struct GenConst {
    double dab;        // delta_ab
    double a[3], b[3]; // pairs (21, 31, 32)
    double da[4][3];   // d a / d(s2_12, s2_13, s2_23, delta)
    double db[4][3];
    // FP32 copies for the gradient terms (FP64 instructions run at 1/64 of
    // the FP32 rate on this part; the gradient is held to 1e-4)
    float af[3], bf[3], daf[4][3], dbf[4][3];
    // sum_r omega_r as the mixed node pass applies the FP32 weights (hi + lo)
    double wsum;
};

// Values per (point, bin) of the mixed node pass: U(3), V(3), [Y(3), Z(3)], Q(3).
__host__ __device__ constexpr int gen_nv(bool grad) { return grad ? 15 : 9; }

// Per-bin epilogue values: chi^2 term (1), with the gradient six more, and
// for the fits the 21 entries of J^T W J (28 in all).
constexpr int kGenNBVFit = 28;

struct GenArgs {
    BinArgs b;
    const GenConst* gc;  // [npts]
};

struct GenArgs64 {
    BinArgs64 b;
    const GenConst* gc;  // [npts]
};

// Phase c * e (double-float) reduced modulo pi/2: phase = q pi/2 + r with
// |r| <= pi/4 (+ rounding); returns r and whether q is odd (bit 0 of the
// magic-rounded quotient).  pi/2 = (PI_A + PI_B + PI_C) / 2 with 12-bit PI_A
// and PI_B: for q < 2^12 (phases below 6434 rad) q PI_A / 2 and q PI_B / 2 are
// exact, so is r1 - q PI_B / 2, and r is rounded once, when the small part
// lo - q PI_C / 2 is added.  With |r| <= pi/4 neither polynomial cancels:
// cos x near a zero of cos is evaluated as a sine of a small r, to a relative
// error of a few ulp (near r = pi/2, 1 + u cos_tail(u) loses ~1e-7 absolute).
__device__ __forceinline__ float reduce_pi2_ff(float ch, float cl, float eh, float el, bool& odd) {
    const float p = __fmul_rn(ch, eh);
    const float e = __fmaf_rn(ch, eh, -p);
    const float lo = __fmaf_rn(ch, el, __fmaf_rn(cl, eh, e));
    const float qm = __fmaf_rn(p, 2.0f * GNA_INV_PI_F, GNA_ROUND_MAGIC);
    odd = (__float_as_uint(qm) & 1u) != 0u;
    const float q = __fsub_rn(qm, GNA_ROUND_MAGIC);
    float r = __fmaf_rn(-q, 0.5f * GNA_PI_A, p);
    r = __fmaf_rn(-q, 0.5f * GNA_PI_B, r);
    return __fadd_rn(r, __fmaf_rn(-q, 0.5f * GNA_PI_C, lo));
}

// The same with the phase formed and reduced in double (1.5 2^52 rounds to an integer).
__device__ __forceinline__ float reduce_pi2_f64(double c, double e, bool& odd) {
    const double p = c * e;
    const double qm = fma(p, 2.0 * GNA_INV_PI_D, 6755399441055744.0);
    odd = (__double2loint(qm) & 1) != 0;
    const double q = qm - 6755399441055744.0;
    double r = fma(-q, 0.5 * GNA_PI_DA, p);
    r = fma(-q, 0.5 * GNA_PI_DB, r);
    return (float)fma(-q, 0.5 * GNA_PI_DC, r);
}

// (sin x, cos x) up to a common sign (which sin^2, cos^2 and sin cos do not
// see) from x = q pi/2 + r: (sin r, cos r) for even q, (cos r, -sin r) for odd q.
__device__ __forceinline__ void sincos_quadrant(float r, bool odd, float& s, float& c) {
    float sr, cr;
    sincos_poly(r, sr, cr);
    s = odd ? cr : sr;
    c = odd ? -sr : cr;
}

// SURV: a survival channel (delta_ab = 1), whose P goes to ~0 at a
// disappearance minimum: the phases are then reduced modulo pi/2 with
// quadrant swaps, so that cos x near its zeros (the cos^2 sums there) keeps
// its relative accuracy; other channels reduce modulo pi (P stays well above
// the cos^2 errors there).
template <int PH, int NL, bool GRAD, bool SURV>
struct NodeMathGen {
    static constexpr int NV = gen_nv(GRAD);
    // with several baselines the weights enter as hi + lo (no bias from the
    // FP32 rounding of omega_r)
    static constexpr bool LO = NL > 1;

    PhaseConsts<PH, NL> ph;
    float om[NL], omlo[NL], wkl[NL];

    __device__ __forceinline__ void load(const PointConst* pc, const BaseConst& bc) {
        ph.load(pc);
#pragma unroll
        for (int r = 0; r < NL; r++) {
            om[r] = bc.om[r];
            omlo[r] = bc.omlo[r];
            wkl[r] = bc.wkl[r];
        }
    }

    // One energy node: g = {invE_hi, invE_lo, W, We}.
    __device__ __forceinline__ void update(float4 g, KahanF (&acc)[NV]) const {
        const float eh = g.x, el = g.y, W = g.z, We = g.w;
        double ed = 0.0;
        if (PH == 1) ed = (double)eh + (double)el;
        float U[3] = {0.f, 0.f, 0.f}, V[3] = {0.f, 0.f, 0.f}, Q[3] = {0.f, 0.f, 0.f};
        float Y[3] = {0.f, 0.f, 0.f}, Z[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int r = 0; r < NL; r++) {
            float s1, c1, s2, c2;
            if constexpr (SURV) {
                bool o21, o32;
                float r21, r32;
                if (PH == 0) {
                    r21 = reduce_pi2_ff(ph.ch21[r], ph.cl21[r], eh, el, o21);
                    r32 = reduce_pi2_ff(ph.ch32[r], ph.cl32[r], eh, el, o32);
                } else {
                    r21 = reduce_pi2_f64(ph.cd21[r], ed, o21);
                    r32 = reduce_pi2_f64(ph.cd32[r], ed, o32);
                }
                sincos_quadrant(r21, o21, s1, c1);
                sincos_quadrant(r32, o32, s2, c2);
            } else {
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
            }
            // x31 = x21 + x32 up to a multiple of pi: sin^2, sin cos and
            // cos^2 - sin^2 do not see it
            const float s3 = fmaf(s1, c2, c1 * s2);
            const float c3 = fmaf(c1, c2, -(s1 * s2));
            const float S[3] = {s1 * s1, s3 * s3, s2 * s2};
            const float C[3] = {s1 * c1, s3 * c3, s2 * c2};
            const float cc[3] = {c1, c3, c2};
            const float Cs[3] = {c1 * c1, c3 * c3, c2 * c2};
#pragma unroll
            for (int j = 0; j < 3; j++) {
                if constexpr (NL == 1) {
                    // one baseline: omega = w / w = 1 exactly, so the weighting is the identity
                    U[j] = S[j];
                    V[j] = C[j];
                    Q[j] = Cs[j];
                } else {
                    U[j] = fmaf(om[r], S[j], U[j]);
                    V[j] = fmaf(om[r], C[j], V[j]);
                    Q[j] = fmaf(om[r], Cs[j], Q[j]);
                }
                if constexpr (LO) {
                    U[j] = fmaf(omlo[r], S[j], U[j]);
                    V[j] = fmaf(omlo[r], C[j], V[j]);
                    Q[j] = fmaf(omlo[r], Cs[j], Q[j]);
                }
                if constexpr (GRAD) {
                    Y[j] = fmaf(wkl[r], C[j], Y[j]);
                    Z[j] = fmaf(wkl[r], fmaf(cc[j], cc[j], -S[j]), Z[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            kadd_prod(acc[j], W, U[j]);
            kadd_prod(acc[3 + j], W, V[j]);
            if constexpr (GRAD) {
                kadd_prod(acc[6 + j], We, Y[j]);
                kadd_prod(acc[9 + j], We, Z[j]);
            }
            kadd_prod(acc[NV - 3 + j], W, Q[j]);
        }
    }
};

// Bin i of point p from its summed values [U(3), V(3)] (+ [Y(3), Z(3)]) and
// Q(3): vd = {U, V, Q} (nine values) in double, vf the NV values in FP32, and
// the point's coefficients.  Each pair's sine sum is U, or sum W sum omega - Q where Q is
// the smaller sum (see the header); M is formed in double (its
// terms may cancel), its six derivatives in FP32, then the chi^2 term (from
// d - mu in double and the relative residual in FP32) and its gradient
// contributions into regs[0..6] (float pairs): [0] the chi^2 term,
// [1 + q] g_i N (1 + eta_i) dM/dp_q.
__device__ inline void gen_bin_epilogue(const EpiArgs& a, const GenConst& c, int p, int i, const double* vd,
                                        const float* vf, const BinIn& in, float2* regs) {
    const int64_t idx = (int64_t)p * a.nbins + i;
    double M = c.dab * in.sumw;
    const double wtot = in.sumw * c.wsum;
    float Sf[3];
    for (int j = 0; j < 3; j++) {
        const double Sj = (vd[6 + j] < vd[j]) ? wtot - vd[6 + j] : vd[j];
        Sf[j] = (float)Sj;
        M += c.a[j] * Sj + c.b[j] * vd[3 + j];
    }
    const double e = in.e;
    const double f = a.norm * (1.0 + e);
    const double mu = f * M;
    const double d = in.d;
    // as in the survival chain's mixed epilogue: d - mu in double (they are
    // close), the relative residual t = (d - mu) / mu, the Poisson term
    // 2 mu h(t) and the adjoint in FP32 (1e-7 relative per bin)
    const double dm = d - mu;
    const float tf = (float)dm / (float)mu;
    double term;
    float g;
    if (a.kind == GNA_PEARSON) {
        term = dm * (double)tf;                // (d - mu)^2 / mu
        g = 1.0f - (1.0f + tf) * (1.0f + tf);  // 1 - d^2 / mu^2
    } else {
        term = (d > 0.0) ? 2.0 * mu * (double)poisson_h(tf) : 2.0 * mu;
        g = -2.0f * tf;  // 2 (1 - d / mu)
    }
    const bool pen = a.eta && a.sigma > 0.0;
    if (pen) term += e * e / (a.sigma * a.sigma);
    regs[0] = to_ff(term);
    if (a.has_grad) {
        float dM[6];
        for (int q = 0; q < 4; q++) {
            dM[q] = 0.f;
            for (int j = 0; j < 3; j++) dM[q] = fmaf(c.daf[q][j], Sf[j], fmaf(c.dbf[q][j], vf[3 + j], dM[q]));
        }
        // pairs 0 = 21, 1 = 31, 2 = 32; x31 moves with both splittings
        const float t31 = fmaf(c.af[1], vf[7], 0.5f * c.bf[1] * vf[10]);
        dM[4] = fmaf(c.af[0], vf[6], fmaf(0.5f * c.bf[0], vf[9], t31));
        dM[5] = fmaf(c.af[2], vf[8], fmaf(0.5f * c.bf[2], vf[11], t31));
        const float gf = g * (float)f;
        for (int q = 0; q < 6; q++) regs[1 + q] = make_float2(gf * dM[q], 0.f);
        if (a.NBV >= kGenNBVFit) {
            // fits: this bin's part of J^T W J, J_q = d mu / d p_q, W = 2 / mu
            const float ff = (float)f, h = 2.0f / (float)mu;
            float J[6];
            for (int q = 0; q < 6; q++) J[q] = ff * dM[q];
            int t = 7;
            for (int q = 0; q < 6; q++)
                for (int r = q; r < 6; r++) regs[t++] = make_float2(h * J[q] * J[r], 0.f);
        }
    }
    if (a.mu_out) a.mu_out[idx] = mu;
    if (a.grad_eta_out)
        a.grad_eta_out[idx] = (double)g * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
}

// Group g of point p: lane l holds the values of bin 32 g + l in regs; up to
// kGenNBVFit values, summed 16 at a time by transposed reductions (value
// base + lane / 2 lands on the even lanes), stored per group.
__device__ inline void gen_group_reduce(const EpiArgs& a, int p, int g, int lane, const float2* regs) {
    const int i = (g << 5) + lane;
    for (int base = 0; base < a.NBV; base += 16) {
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; j++)
            v[j] = (base + j < a.NBV && i < a.nbins) ? regs[base + j] : make_float2(0.f, 0.f);
        warp_transpose_reduce<16>(v, lane);
        const int vi = base + (lane >> 1);
        if ((lane & 1) == 0 && vi < a.NBV) a.gvals[((int64_t)p * a.ngroups + g) * a.NBV + vi] = v[0];
    }
}

// Point p: lane l sums groups l, l + 32, ... in order, then transposed
// reductions, 16 values at a time; chi2, the six-parameter gradient and (fits)
// the 21 entries of J^T W J are written.
__device__ inline void gen_point_reduce(const EpiArgs& a, int p, int lane) {
    for (int base = 0; base < a.NBV; base += 16) {
        float2 v[16];
#pragma unroll
        for (int j = 0; j < 16; j++) v[j] = make_float2(0.f, 0.f);
        for (int g = lane; g < a.ngroups; g += 32) {
            const float2* gv = a.gvals + ((int64_t)p * a.ngroups + g) * a.NBV + base;
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (base + j < a.NBV) v[j] = ff_add(v[j], __ldcg(gv + j));
        }
        warp_transpose_reduce<16>(v, lane);
        const int vi = base + (lane >> 1);
        if ((lane & 1) == 0 && vi < a.NBV) {
            const double tot = (double)v[0].x + (double)v[0].y;
            if (vi == 0) a.chi2[p] = tot;
            else if (vi < 7) {
                if (a.grad) a.grad[(int64_t)p * 6 + vi - 1] = tot;
            } else if (a.H) {
                a.H[(int64_t)p * 21 + vi - 7] = tot;
            }
        }
    }
}

// The group g of point p has its per-bin values in regs (whole warp calls):
// sum the group, and the warp that completes the point's last group sums the
// groups.
static __device__ __noinline__ void gen_group_done(const EpiArgs& a, int p, int g, int lane, const float2* regs) {
    gen_group_reduce(a, p, g, lane, regs);
    __threadfence();
    __syncwarp();
    int lastp = 0;
    if (lane == 0) lastp = (atomicAdd(a.pt_cnt + p, 1) == a.ngroups - 1);
    lastp = __shfl_sync(0xffffffffu, lastp, 0);
    if (lastp) {
        __threadfence();
        gen_point_reduce(a, p, lane);
    }
}

// Node kernel of the general channel, bin and slice mappings: the task scheme
// and node loop of k_fused_bins with the channel-free sums above.
template <int PH, int NL, bool GRAD, bool SURV>
__global__ void __launch_bounds__(256) k_fused_bins_gen(GenArgs ga) {
    using M = NodeMathGen<PH, NL, GRAD, SURV>;
    constexpr int NV = M::NV;
    const BinArgs& a = ga.b;
    const int lane = threadIdx.x & 31;
    int last_p = -1;
    M m;
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
        const int kn = min(n, k0 + (a.S > 1 ? a.L : n)) - k0;
        if (p != last_p) {
            m.load(a.pcs + p, a.bc);
            last_p = p;
        }
        KahanF acc[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) kzero(acc[v]);
        const float4* g = a.grid + a.goff[gi] + ((int64_t)b * n + k0) * 32 + lane;
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
            continue;
        }
        const int i = b * 32 + lane;
        float2 regs[kGenNBVFit];
        if (i < a.nbins) {
            double vd[9];
            float vf[NV];
#pragma unroll
            for (int j = 0; j < 9; j++) {
                const int v = j < 6 ? j : NV - 9 + j;  // U, V, then Q
                vd[j] = (double)acc[v].s - (double)acc[v].c;
            }
#pragma unroll
            for (int j = 0; j < NV; j++) vf[j] = acc[j].s - acc[j].c;
            gen_bin_epilogue(a.ea, ga.gc[p], p, i, vd, vf, bin_inputs(a.ea, p, i), regs);
        }
        gen_group_done(a.ea, p, b, lane, regs);
    }
    asm volatile("griddepcontrol.launch_dependents;");
}

// Slice sums of the general channel (NV = 9 or 15 values), in slice order,
// then the epilogue and the group and point reductions: k_slices_reduce with
// the general epilogue.
template <int W>
__global__ void __launch_bounds__(W * 32) k_slices_reduce_gen(const float2* __restrict__ part, int S, int NV,
                                                               EpiArgs ea, const GenConst* __restrict__ gc) {
    constexpr int NVM = gen_nv(true);
    extern __shared__ float2 red[];  // [W][NV][32], then [NV][32] doubles
    double* fin = reinterpret_cast<double*>(red + W * NV * 32);
    const int pg = blockIdx.x;
    const int p = pg / ea.ngroups;
    const int g = pg - p * ea.ngroups;
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // the next evaluation's first kernel may be placed now (it waits for this one)
    asm volatile("griddepcontrol.launch_dependents;");
    float2 acc[NVM];
#pragma unroll
    for (int v = 0; v < NVM; v++) acc[v] = make_float2(0.f, 0.f);
    const int i = g * 32 + lane;
    BinIn in{0.0, 0.0, 0.0};
    if (w == 0 && i < ea.nbins) in = bin_inputs(ea, p, i);
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
    float2* fin2 = reinterpret_cast<float2*>(fin);
    for (int v = w; v < NV; v += W) {
        float2 sum = red[v * 32 + lane];
        for (int k = 1; k < W; k++) sum = ff_add(sum, red[(k * NV + v) * 32 + lane]);
        fin2[v * 32 + lane] = sum;
    }
    __syncthreads();
    if (w == 0) {
        double vd[9];
        float vf[NVM];
        for (int v = 0; v < NV; v++) {
            const float2 t = fin2[v * 32 + lane];
            vf[v] = t.x + t.y;
            if (v < 6) vd[v] = (double)t.x + (double)t.y;
            else if (v >= NV - 3) vd[v - NV + 9] = (double)t.x + (double)t.y;  // Q
        }
        float2 regs[kGenNBVFit];
        if (i < ea.nbins) gen_bin_epilogue(ea, gc[p], p, i, vd, vf, in, regs);
        gen_group_done(ea, p, g, lane, regs);
    }
}

// ------------------------------------------------------------- GNA_FP64 ----
// The same sums with every step in double (phases reduced modulo pi in
// double, CUDA's double sincos), for the bin mapping on the double grids
// {1/E, W}.
template <int NL, bool GRAD>
struct NodeMathGen64 {
    // the sums of the mixed variant, then sum_k W_k (the delta_ab term; the
    // mixed precisions take it from the plan's per-bin weight sums)
    static constexpr int NV = GRAD ? 13 : 7;
    double c21[NL], c32[NL], om[NL], wk[NL];

    __device__ __forceinline__ void load(const PointConst* pc, const BaseConst& bc) {
#pragma unroll
        for (int r = 0; r < NL; r++) {
            c21[r] = pc->c21[r];
            c32[r] = pc->c32[r];
            om[r] = bc.omd[r];
            wk[r] = 2.0 * bc.omd[r] * bc.kld[r];
        }
    }

    __device__ __forceinline__ void update(double2 g, double (&acc)[NV]) const {
        const double e = g.x, W = g.y;
        double U[3] = {0, 0, 0}, V[3] = {0, 0, 0}, Y[3] = {0, 0, 0}, Z[3] = {0, 0, 0};
#pragma unroll
        for (int r = 0; r < NL; r++) {
            double s1, c1, s2, c2;
            sincos(reduce_pi_d(c21[r] * e), &s1, &c1);
            sincos(reduce_pi_d(c32[r] * e), &s2, &c2);
            const double s3 = s1 * c2 + c1 * s2, c3 = c1 * c2 - s1 * s2;
            const double S[3] = {s1 * s1, s3 * s3, s2 * s2};
            const double C[3] = {s1 * c1, s3 * c3, s2 * c2};
            const double cc[3] = {c1, c3, c2};
#pragma unroll
            for (int j = 0; j < 3; j++) {
                U[j] += om[r] * S[j];
                V[j] += om[r] * C[j];
                if constexpr (GRAD) {
                    Y[j] += wk[r] * C[j];
                    Z[j] += wk[r] * (cc[j] * cc[j] - S[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 3; j++) {
            acc[j] += W * U[j];
            acc[3 + j] += W * V[j];
            if constexpr (GRAD) {
                acc[6 + j] += W * e * Y[j];
                acc[9 + j] += W * e * Z[j];
            }
        }
        acc[NV - 1] += W;
    }
};

// Epilogue of one bin with all sums and the contraction in double; v[nv - 1]
// is the bin's sum of node weights.
__device__ inline void gen_bin_epilogue64(const EpiArgs& a, const GenConst& c, int p, int i, const double* v,
                                          int nv, const BinIn& in, float2* regs) {
    const int64_t idx = (int64_t)p * a.nbins + i;
    double M = c.dab * v[nv - 1];
    for (int j = 0; j < 3; j++) M += c.a[j] * v[j] + c.b[j] * v[3 + j];
    const double e = in.e;
    const double f = a.norm * (1.0 + e);
    const double mu = f * M;
    const double d = in.d;
    double term, gd;
    if (a.kind == GNA_PEARSON) {
        term = (d - mu) * (d - mu) / mu;
        gd = 1.0 - (d * d) / (mu * mu);
    } else {
        term = (d > 0.0) ? 2.0 * (mu - d + d * log(d / mu)) : 2.0 * mu;
        gd = 2.0 * (1.0 - d / mu);
    }
    const bool pen = a.eta && a.sigma > 0.0;
    if (pen) term += e * e / (a.sigma * a.sigma);
    regs[0] = to_ff(term);
    if (a.has_grad) {
        double dM[6];
        for (int q = 0; q < 4; q++) {
            dM[q] = 0.0;
            for (int j = 0; j < 3; j++) dM[q] += c.da[q][j] * v[j] + c.db[q][j] * v[3 + j];
        }
        const double t31 = c.a[1] * v[7] + 0.5 * c.b[1] * v[10];
        dM[4] = c.a[0] * v[6] + 0.5 * c.b[0] * v[9] + t31;
        dM[5] = c.a[2] * v[8] + 0.5 * c.b[2] * v[11] + t31;
        for (int q = 0; q < 6; q++) regs[1 + q] = to_ff(gd * f * dM[q]);
        if (a.NBV >= kGenNBVFit) {  // fits: J^T W J, J_q = d mu / d p_q = f dM_q, W = 2 / mu
            const double h = 2.0 / mu;
            int t = 7;
            for (int q = 0; q < 6; q++)
                for (int r = q; r < 6; r++) regs[t++] = to_ff(h * (f * dM[q]) * (f * dM[r]));
        }
    }
    if (a.mu_out) a.mu_out[idx] = mu;
    if (a.grad_eta_out) a.grad_eta_out[idx] = gd * a.norm * M + (pen ? 2.0 * e / (a.sigma * a.sigma) : 0.0);
}

template <int NL, bool GRAD>
__global__ void __launch_bounds__(256) k_fused64_bins_gen(GenArgs64 ga) {
    using M = NodeMathGen64<NL, GRAD>;
    constexpr int NV = M::NV;
    const BinArgs64& a = ga.b;
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
        float2 regs[kGenNBVFit];
        if (i < a.nbins) gen_bin_epilogue64(a.ea, ga.gc[p], p, i, acc, NV, bin_inputs(a.ea, p, i), regs);
        gen_group_done(a.ea, p, b, lane, regs);
    }
}

// Launchers (general.cu).
cudaError_t launch_prepare_general(const gna_osc_full* prm, int npts, const BaseConst& bc, int alpha, int beta,
                                   int anti, PointConst* out, GenConst* gout, int* zero, int64_t nz, int* status,
                                   cudaStream_t s);
cudaError_t dispatch_general(int ph, int nl, bool grad, bool surv, const GenArgs& a, int grid, int block,
                             cudaStream_t s);
int general_resident_ctas(int ph, int nl, bool grad, bool surv, int block);
cudaError_t dispatch_general64(int nl, bool grad, const GenArgs64& a, int grid, int block, cudaStream_t s);
cudaError_t launch_slices_reduce_general(const float2* part, int S, int NV, const EpiArgs& ea, const GenConst* gc,
                                         int npts, cudaStream_t s);

}  // namespace gna
