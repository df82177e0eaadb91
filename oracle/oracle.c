/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the three-flavour vacuum
 * oscillation chain (probability -> spectrum x weight -> Gauss-Legendre bin
 * integration -> chi^2 and its gradient).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * links it, and it shares no code, header or constant with the CUDA side.
 *
 * Every function states the passage it follows.  "Paper" is "CUDA Support in
 * GNA Data Analysis Framework" (arXiv:1804.07682).  Steps that the paper does
 * not define (spectrum, Gauss-Legendre rule, chi^2, nuisances, gradient) are
 * written out from their textbook definitions and say so.
 *
 * Units: E in MeV, L in km, mass splittings in eV^2.  The phase is formed in
 * natural units from hbar*c, not from a pre-multiplied constant.
 *
 * Precision: double everywhere, sums in plain index order.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* hbar*c = 197.3269804 MeV fm (CODATA 2018) = 197.3269804e-9 eV m. */
static const double OR_HBARC_EV_M = 197.3269804e-9;

int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* PMNS matrix, standard parameterisation U = R23 * U13(delta) * R12         */
/* (paper Sec. 4.1 names V the PMNS matrix; the parameterisation is the      */
/* textbook one and is not printed in the paper).                            */
/* Output: U_re/U_im row-major, U[alpha][i], alpha = e, mu, tau; i = 1,2,3.  */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double complex A[3][3], const double complex B[3][3],
                     double complex C[3][3]) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double complex s = 0;
            for (int k = 0; k < 3; k++) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static void pmns_complex(double s12sq, double s13sq, double s23sq, double delta,
                         double complex U[3][3]) {
    double s12 = sqrt(s12sq), c12 = sqrt(1.0 - s12sq);
    double s13 = sqrt(s13sq), c13 = sqrt(1.0 - s13sq);
    double s23 = sqrt(s23sq), c23 = sqrt(1.0 - s23sq);
    double complex em = cexp(-I * delta), ep = cexp(I * delta);
    double complex R23[3][3] = {{1, 0, 0}, {0, c23, s23}, {0, -s23, c23}};
    double complex R13[3][3] = {{c13, 0, s13 * em}, {0, 1, 0}, {-s13 * ep, 0, c13}};
    double complex R12[3][3] = {{c12, s12, 0}, {-s12, c12, 0}, {0, 0, 1}};
    double complex T[3][3];
    mat3_mul(R23, R13, T);
    mat3_mul(T, R12, U);
}

void or_pmns(double s12sq, double s13sq, double s23sq, double delta,
             double* U_re, double* U_im) {
    double complex U[3][3];
    pmns_complex(s12sq, s13sq, s23sq, delta, U);
    for (int a = 0; a < 3; a++)
        for (int i = 0; i < 3; i++) {
            U_re[3 * a + i] = creal(U[a][i]);
            U_im[3 * a + i] = cimag(U[a][i]);
        }
}

/* ------------------------------------------------------------------------ */
/* General vacuum oscillation probability, paper Sec. 4.1 (the unnumbered   */
/* multline equation):                                                       */
/*   P(a->b) = delta_ab - 4 sum_{i>j} Re(V*_ai V_bi V_aj V*_bj) sin^2(x_ij)  */
/*                      + 2 sum_{i>j} Im(V*_ai V_bi V_aj V*_bj) sin(2 x_ij)  */
/* with x_ij = dm2_ij L / (4E) in natural units.  Antineutrinos use V*.      */
/* Mass splittings: dm2_21, dm2_32 given; dm2_31 = dm2_21 + dm2_32.          */
/* ------------------------------------------------------------------------ */
static double half_phase(double dm2_eV2, double L_km, double E_MeV) {
    /* dm2 L / (4E): L in 1/eV is L_m / (hbar c), E in eV. */
    double L_inv_eV = (L_km * 1e3) / OR_HBARC_EV_M;
    double E_eV = E_MeV * 1e6;
    return dm2_eV2 * L_inv_eV / (4.0 * E_eV);
}

static double prob_general(int a, int b, const double complex U[3][3], double dm21,
                           double dm32, double L_km, double E_MeV, int anti) {
    double complex V[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) V[r][c] = anti ? conj(U[r][c]) : U[r][c];
    /* m2[i] = m_i^2 - m_1^2 */
    double m2[3] = {0.0, dm21, dm21 + dm32};
    double P = (a == b) ? 1.0 : 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < i; j++) {
            double complex X = conj(V[a][i]) * V[b][i] * V[a][j] * conj(V[b][j]);
            double x = half_phase(m2[i] - m2[j], L_km, E_MeV);
            double sx = sin(x);
            P += -4.0 * creal(X) * sx * sx + 2.0 * cimag(X) * sin(2.0 * x);
        }
    return P;
}

double or_prob(int alpha, int beta, double s12sq, double s13sq, double s23sq,
               double delta, double dm21, double dm32, double L_km, double E_MeV,
               int anti) {
    double complex U[3][3];
    pmns_complex(s12sq, s13sq, s23sq, delta, U);
    return prob_general(alpha, beta, U, dm21, dm32, L_km, E_MeV, anti);
}

/* Electron-antineutrino survival P(nue_bar -> nue_bar) on an array of        */
/* energies: the alpha = beta = e entry of the general formula above.        */
/* theta23 and delta do not enter it; fixed values are used.                 */
void or_pee(const double* E_MeV, int64_t n, double L_km, const double* osc,
            double* P) {
    double complex U[3][3];
    pmns_complex(osc[0], osc[1], 0.5, 0.0, U);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++)
        P[k] = prob_general(0, 0, U, osc[2], osc[3], L_km, E_MeV[k], 1);
}

/* dP_ee/d(theta) for theta = (s12^2, s13^2, dm2_21, dm2_32), from the same   */
/* literal formula.  For a = b = e the coefficient is |U_ei|^2 |U_ej|^2,      */
/* |U_e1|^2 = (1-s12^2)(1-s13^2), |U_e2|^2 = s12^2 (1-s13^2), |U_e3|^2 =      */
/* s13^2 (textbook moduli of the standard parameterisation); the derivative  */
/* is the product rule on those moduli and d sin^2(x)/dx = sin(2x).          */
static void pee_and_grad(double s12, double s13, double dm21, double dm32, double L_km,
                         double E_MeV, double* P, double* dP) {
    double ue[3] = {(1 - s12) * (1 - s13), s12 * (1 - s13), s13};
    double due_ds12[3] = {-(1 - s13), (1 - s13), 0.0};
    double due_ds13[3] = {-(1 - s12), -s12, 1.0};
    double m2[3] = {0.0, dm21, dm21 + dm32};
    /* d(m2[i]-m2[j])/d(dm21), d/d(dm32) */
    double dm2_d21[3] = {0.0, 1.0, 1.0};
    double dm2_d32[3] = {0.0, 0.0, 1.0};
    double p = 1.0, g12 = 0, g13 = 0, g21 = 0, g32 = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < i; j++) {
            double x = half_phase(m2[i] - m2[j], L_km, E_MeV);
            double dx_ddm2 = half_phase(1.0, L_km, E_MeV);
            double s2 = sin(x) * sin(x);
            double coef = ue[i] * ue[j];
            p -= 4.0 * coef * s2;
            g12 -= 4.0 * (due_ds12[i] * ue[j] + ue[i] * due_ds12[j]) * s2;
            g13 -= 4.0 * (due_ds13[i] * ue[j] + ue[i] * due_ds13[j]) * s2;
            double dsin2 = sin(2.0 * x) * dx_ddm2;
            g21 -= 4.0 * coef * dsin2 * (dm2_d21[i] - dm2_d21[j]);
            g32 -= 4.0 * coef * dsin2 * (dm2_d32[i] - dm2_d32[j]);
        }
    *P = p;
    if (dP) {
        dP[0] = g12;
        dP[1] = g13;
        dP[2] = g21;
        dP[3] = g32;
    }
}

void or_pee_grad(const double* E_MeV, int64_t n, double L_km, const double* osc,
                 double* P, double* dP /* [n][4] */) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; k++)
        pee_and_grad(osc[0], osc[1], osc[2], osc[3], L_km, E_MeV[k], &P[k],
                     dP ? &dP[4 * k] : NULL);
}

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [-1,1] (not in the paper; textbook definition):    */
/* nodes are the roots of P_n, found by Newton's method on the three-term    */
/* recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}, started from          */
/* cos(pi (k - 1/4) / (n + 1/2)); weights w = 2 / ((1 - x^2) P_n'(x)^2) with  */
/* P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1).  Nodes returned ascending.      */
/* (x^2 - 1 is evaluated as (x - 1)(x + 1) to avoid cancellation at the      */
/* outermost nodes.)                                                          */
/* Returns 0, or -1 for n < 1.                                                */
/* ------------------------------------------------------------------------ */
static void legendre_eval(int n, double x, double* pn, double* pn1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        *pn = 1.0;
        *pn1 = 0.0;
        return;
    }
    for (int j = 1; j < n; j++) {
        double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

int or_gl(int n, double* x, double* w) {
    if (n < 1) return -1;
    const double pi = 3.14159265358979323846;
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 1; k <= n; k++) {
        double xk = cos(pi * (k - 0.25) / (n + 0.5));
        double pn = 0, pn1 = 0, dp = 0;
        for (int it = 0; it < 100; it++) {
            legendre_eval(n, xk, &pn, &pn1);
            dp = n * (xk * pn - pn1) / ((xk - 1.0) * (xk + 1.0));
            double dx = pn / dp;
            xk -= dx;
            if (fabs(dx) <= 1e-16 * (1.0 + fabs(xk))) break;
        }
        legendre_eval(n, xk, &pn, &pn1);
        dp = n * (xk * pn - pn1) / ((xk - 1.0) * (xk + 1.0));
        /* k = 1 is the largest root; store ascending.  1 - x^2 is formed as
         * (1 - x)(1 + x): near x = +-1 the difference is then exact. */
        x[n - k] = xk;
        w[n - k] = 2.0 / (((1.0 - xk) * (1.0 + xk)) * dp * dp);
    }
    return 0;
}

/* Reactor spectrum shape S(E) = exp(0.87 - 0.16 E - 0.091 E^2) (not in the   */
/* paper; the workload definition).  E is in MeV unless e_scale rescales it   */
/* (1e-3 evaluates the same shape with E in GeV).                             */
double or_spectrum(double E_MeV, double e_scale) {
    double E = E_MeV * e_scale;
    return exp(0.87 - 0.16 * E - 0.091 * E * E);
}

/* ------------------------------------------------------------------------ */
/* Binned prediction per baseline (the JUNO-like graph of paper Fig. 3:      */
/* one OscProb per baseline on a shared energy vector) integrated per bin    */
/* with an n-point Gauss-Legendre rule:                                      */
/*   mu[r][i] = sum_k (b_i - a_i)/2 w_k S(E_ik) P_r(E_ik),                   */
/*   E_ik = (a_i + b_i)/2 + (b_i - a_i)/2 x_k.                               */
/* dmu[r][i][4] (optional) holds d mu[r][i] / d theta.                       */
/* x, w: the rule (from or_gl).  Returns 0.                                  */
/* ------------------------------------------------------------------------ */
int or_binned(int nbins, const double* edges, int n, const double* x, const double* w,
              int nL, const double* L_km, const double* osc, double e_scale,
              double* mu, double* dmu) {
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int r = 0; r < nL; r++)
        for (int i = 0; i < nbins; i++) {
            double a = edges[i], b = edges[i + 1];
            double half = 0.5 * (b - a), mid = 0.5 * (a + b);
            double s = 0, g[4] = {0, 0, 0, 0};
            for (int k = 0; k < n; k++) {
                double E = mid + half * x[k];
                double wt = half * w[k] * or_spectrum(E, e_scale);
                double P, dP[4];
                pee_and_grad(osc[0], osc[1], osc[2], osc[3], L_km[r], E, &P, dmu ? dP : NULL);
                s += wt * P;
                if (dmu)
                    for (int q = 0; q < 4; q++) g[q] += wt * dP[q];
            }
            mu[(int64_t)r * nbins + i] = s;
            if (dmu)
                for (int q = 0; q < 4; q++) dmu[((int64_t)r * nbins + i) * 4 + q] = g[q];
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Any channel with its gradient (beyond the nue_bar survival chain).        */
/* dU/dp for p = (s12^2, s13^2, s23^2, delta): the product rule on           */
/* U = R23 U13(delta) R12, each rotation differentiated in its own variable   */
/* (d sin(theta)/d sin^2(theta) = 1 / (2 sin(theta)), d cos(theta) /          */
/* d sin^2(theta) = -1 / (2 cos(theta)); d e^(-+i delta)/d delta = -+i        */
/* e^(-+i delta)).  Interior points only (0 < s^2 < 1).                      */
/* ------------------------------------------------------------------------ */
static void pmns_dU(double s12sq, double s13sq, double s23sq, double delta,
                    double complex dU[4][3][3]) {
    double s12 = sqrt(s12sq), c12 = sqrt(1.0 - s12sq);
    double s13 = sqrt(s13sq), c13 = sqrt(1.0 - s13sq);
    double s23 = sqrt(s23sq), c23 = sqrt(1.0 - s23sq);
    double complex em = cexp(-I * delta), ep = cexp(I * delta);
    double complex R23[3][3] = {{1, 0, 0}, {0, c23, s23}, {0, -s23, c23}};
    double complex R13[3][3] = {{c13, 0, s13 * em}, {0, 1, 0}, {-s13 * ep, 0, c13}};
    double complex R12[3][3] = {{c12, s12, 0}, {-s12, c12, 0}, {0, 0, 1}};
    double ds12 = 0.5 / s12, dc12 = -0.5 / c12;
    double ds13 = 0.5 / s13, dc13 = -0.5 / c13;
    double ds23 = 0.5 / s23, dc23 = -0.5 / c23;
    double complex D12[3][3] = {{dc12, ds12, 0}, {-ds12, dc12, 0}, {0, 0, 0}};
    double complex D13[3][3] = {{dc13, 0, ds13 * em}, {0, 0, 0}, {-ds13 * ep, 0, dc13}};
    double complex D23[3][3] = {{0, 0, 0}, {0, dc23, ds23}, {0, -ds23, dc23}};
    double complex Dd[3][3] = {{0, 0, -I * s13 * em}, {0, 0, 0}, {-I * s13 * ep, 0, 0}};
    double complex T[3][3];
    mat3_mul(R23, R13, T);
    mat3_mul(T, D12, dU[0]);
    mat3_mul(R23, D13, T);
    mat3_mul(T, R12, dU[1]);
    mat3_mul(D23, R13, T);
    mat3_mul(T, R12, dU[2]);
    mat3_mul(R23, Dd, T);
    mat3_mul(T, R12, dU[3]);
}

/* P(a->b) of the Sec. 4.1 formula (as prob_general) and its derivatives     */
/* dP[6] with respect to (s12^2, s13^2, s23^2, delta, dm2_21, dm2_32):        */
/* for the mixing parameters the product rule on X_ij = V*_ai V_bi V_aj V*_bj */
/* with dV = dU (or its conjugate for antineutrinos); for the mass           */
/* splittings d/dx [-4 Re X sin^2 x + 2 Im X sin 2x] = -4 Re X sin 2x +      */
/* 4 Im X cos 2x times dx/d(dm2).                                             */
static void prob_general_grad(int a, int b, const double complex U[3][3],
                              const double complex dU[4][3][3], double dm21, double dm32,
                              double L_km, double E_MeV, int anti, double* P, double* dP) {
    double complex V[3][3], dV[4][3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) {
            V[r][c] = anti ? conj(U[r][c]) : U[r][c];
            for (int q = 0; q < 4; q++) dV[q][r][c] = anti ? conj(dU[q][r][c]) : dU[q][r][c];
        }
    double m2[3] = {0.0, dm21, dm21 + dm32};
    double dm2_d21[3] = {0.0, 1.0, 1.0};
    double dm2_d32[3] = {0.0, 0.0, 1.0};
    double p = (a == b) ? 1.0 : 0.0;
    for (int q = 0; q < 6; q++) dP[q] = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < i; j++) {
            double complex X = conj(V[a][i]) * V[b][i] * V[a][j] * conj(V[b][j]);
            double x = half_phase(m2[i] - m2[j], L_km, E_MeV);
            double sx = sin(x), s2x = sin(2.0 * x), c2x = cos(2.0 * x);
            p += -4.0 * creal(X) * sx * sx + 2.0 * cimag(X) * s2x;
            for (int q = 0; q < 4; q++) {
                double complex dX = conj(dV[q][a][i]) * V[b][i] * V[a][j] * conj(V[b][j]) +
                                    conj(V[a][i]) * dV[q][b][i] * V[a][j] * conj(V[b][j]) +
                                    conj(V[a][i]) * V[b][i] * dV[q][a][j] * conj(V[b][j]) +
                                    conj(V[a][i]) * V[b][i] * V[a][j] * conj(dV[q][b][j]);
                dP[q] += -4.0 * creal(dX) * sx * sx + 2.0 * cimag(dX) * s2x;
            }
            double dterm_dx = -4.0 * creal(X) * s2x + 4.0 * cimag(X) * c2x;
            double dx = half_phase(1.0, L_km, E_MeV);
            dP[4] += dterm_dx * dx * (dm2_d21[i] - dm2_d21[j]);
            dP[5] += dterm_dx * dx * (dm2_d32[i] - dm2_d32[j]);
        }
    *P = p;
}

/* osc6 = (s12^2, s13^2, s23^2, delta, dm2_21, dm2_32); dP[6] as above.      */
void or_prob_grad(int alpha, int beta, const double* osc6, double L_km, double E_MeV, int anti,
                  double* P, double* dP) {
    double complex U[3][3], dU[4][3][3];
    pmns_complex(osc6[0], osc6[1], osc6[2], osc6[3], U);
    pmns_dU(osc6[0], osc6[1], osc6[2], osc6[3], dU);
    prob_general_grad(alpha, beta, U, dU, osc6[4], osc6[5], L_km, E_MeV, anti, P, dP);
}

/* Binned prediction per baseline for P(alpha -> beta), as or_binned, with   */
/* dmu[r][i][6] (optional) the derivatives in the six parameters above.      */
int or_binned_general(int nbins, const double* edges, int n, const double* x, const double* w,
                      int nL, const double* L_km, const double* osc6, int alpha, int beta, int anti,
                      double e_scale, double* mu, double* dmu) {
    double complex U[3][3], dU[4][3][3];
    pmns_complex(osc6[0], osc6[1], osc6[2], osc6[3], U);
    pmns_dU(osc6[0], osc6[1], osc6[2], osc6[3], dU);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int r = 0; r < nL; r++)
        for (int i = 0; i < nbins; i++) {
            double a = edges[i], b = edges[i + 1];
            double half = 0.5 * (b - a), mid = 0.5 * (a + b);
            double s = 0, g[6] = {0, 0, 0, 0, 0, 0};
            for (int k = 0; k < n; k++) {
                double E = mid + half * x[k];
                double wt = half * w[k] * or_spectrum(E, e_scale);
                double P, dP[6];
                prob_general_grad(alpha, beta, U, dU, osc6[4], osc6[5], L_km[r], E, anti, &P, dP);
                s += wt * P;
                for (int q = 0; q < 6; q++) g[q] += wt * dP[q];
            }
            mu[(int64_t)r * nbins + i] = s;
            if (dmu)
                for (int q = 0; q < 6; q++) dmu[((int64_t)r * nbins + i) * 6 + q] = g[q];
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Detector prediction, chi^2 and gradient (not in the paper; textbook).     */
/*   M_i  = sum_r omega_r mu[r][i]                    (baseline combination) */
/*   mu_i = N (1 + eta_i) M_i                          (normalisation, nuis.) */
/*   Pearson: chi2 = sum_i (d_i - mu_i)^2 / mu_i                             */
/*   Poisson: chi2 = 2 sum_i [mu_i - d_i + d_i ln(d_i / mu_i)], d_i = 0 -> 2mu */
/*   + sum_i eta_i^2 / sigma^2 when eta is given and sigma > 0.             */
/* grad (optional): [4 + nbins] = d chi2 / d(theta, eta).                    */
/* J (optional): [nbins][4] = d mu_i / d theta.  mu_out (optional): mu_i.    */
/* kind: 0 Pearson, 1 Poisson.  Returns chi2.                                */
/* ------------------------------------------------------------------------ */
double or_chi2(int nbins, int nL, const double* omega, const double* mu_rb,
               const double* dmu_rb, double N, const double* eta, double sigma,
               const double* data, int kind, double* grad, double* J, double* mu_out) {
    double chi2 = 0.0;
    if (grad)
        for (int q = 0; q < 4 + nbins; q++) grad[q] = 0.0;
    for (int i = 0; i < nbins; i++) {
        double M = 0, dM[4] = {0, 0, 0, 0};
        for (int r = 0; r < nL; r++) {
            M += omega[r] * mu_rb[(int64_t)r * nbins + i];
            if (dmu_rb)
                for (int q = 0; q < 4; q++)
                    dM[q] += omega[r] * dmu_rb[((int64_t)r * nbins + i) * 4 + q];
        }
        double e = eta ? eta[i] : 0.0;
        double m = N * (1.0 + e) * M;
        double d = data[i];
        double term, gi;
        if (kind == 0) {
            term = (d - m) * (d - m) / m;
            gi = 1.0 - (d * d) / (m * m);
        } else {
            term = (d > 0) ? 2.0 * (m - d + d * log(d / m)) : 2.0 * m;
            gi = 2.0 * (1.0 - d / m);
        }
        chi2 += term;
        if (mu_out) mu_out[i] = m;
        if (J)
            for (int q = 0; q < 4; q++) J[4 * i + q] = N * (1.0 + e) * dM[q];
        if (grad) {
            for (int q = 0; q < 4; q++) grad[q] += gi * N * (1.0 + e) * dM[q];
            grad[4 + i] = gi * N * M;
        }
    }
    if (eta && sigma > 0) {
        for (int i = 0; i < nbins; i++) {
            chi2 += eta[i] * eta[i] / (sigma * sigma);
            if (grad) grad[4 + i] += 2.0 * eta[i] / (sigma * sigma);
        }
    }
    return chi2;
}

/* ------------------------------------------------------------------------ */
/* Pseudo-data (beyond the paper: the pseudo-experiments of the batched     */
/* fits).  Philox4x32-10, the counter-based generator of Salmon, Moraes,    */
/* Dror and Shaw (SC'11), from its published definition: ten rounds of      */
/*   (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (32 x 32 -> 64 bits),       */
/*   c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),                          */
/* with the key bumped by (W0, W1) before every round but the first.        */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    for (int i = 0; i < 4; i++) out[i] = c[i];
}

/* Poisson(mu) by inversion from one uniform u in [0, 1): the smallest k   */
/* with F(k) = sum_{j<=k} p_j >= u, p_0 = e^-mu (given: em), p_j =          */
/* p_{j-1} mu / j; at most kmax = 10 mu + 100 steps.  Only +, *, / in      */
/* double, each rounded once (no contraction), so that another             */
/* implementation with the same operations draws the same integers.       */
int64_t or_poisson_inv(double mu, double em, double u) {
    const int64_t kmax = (int64_t)(10.0 * mu) + 100;
    int64_t k = 0;
    double p = em, F = em;
    while (u > F && k < kmax) {
        k++;
        p = (p * mu) / (double)k;
        F = F + p;
    }
    return k;
}

/* Data set j, bin i: the sum of M_i parts, part m ~ Poisson(mu_i / M_i)   */
/* from the counter (i, j_lo, j_hi, m) under the key (seed_lo, seed_hi)     */
/* (M_i = ceil(mu_i / 500), so that e^-(mu_i / M_i) stays a normal number); */
/* u = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53 from the first two outputs.       */
/* mu_part, em_part and parts are formed by the caller.                     */
void or_pseudo_data(const double* mu_part, const double* em_part, const int* parts, int nbins, int64_t j0,
                    int64_t nds, uint64_t seed, double* out) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t j = j0; j < j0 + nds; j++)
        for (int i = 0; i < nbins; i++) {
            int64_t k = 0;
            for (int m = 0; m < parts[i]; m++) {
                const uint32_t ctr[4] = {(uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)m};
                uint32_t x[4];
                or_philox4x32_10(ctr, key, x);
                const double u = ((double)(x[0] >> 5) * 67108864.0 + (double)(x[1] >> 6)) * (1.0 / 9007199254740992.0);
                k += or_poisson_inv(mu_part[i], em_part[i], u);
            }
            out[(j - j0) * nbins + i] = (double)k;
        }
}
