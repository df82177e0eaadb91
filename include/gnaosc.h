/*
 * gnaosc.h -- C ABI of the GB300 oscillation-chain library (libgnaosc.so).
 *
 * The library evaluates the three-flavour vacuum electron-antineutrino
 * survival probability on large energy arrays and the chain that consumes
 * it: spectrum x oscillation weight, Gauss-Legendre integration per bin over
 * one or more baselines, Pearson or Poisson chi^2 against data, the gradient
 * of chi^2 with respect to (sin^2 theta12, sin^2 theta13, dm2_21, dm2_32,
 * per-bin nuisances), batched parameter points with uneven grids, and batched
 * Levenberg-Marquardt fits.  The same chain for any channel P(alpha -> beta),
 * neutrinos or antineutrinos, with the gradient in (sin^2 theta12,
 * sin^2 theta13, sin^2 theta23, delta_cp, dm2_21, dm2_32); the element-wise
 * probability for any channel, from device or pinned host memory; Poisson
 * pseudo-data on the device.
 *
 * Paper: "CUDA Support in GNA Data Analysis Framework" (arXiv:1804.07682).
 * The probability is the paper's Sec. 4.1 vacuum formula with alpha = beta = e;
 * the calls follow its transformation model (Sec. 2.1: read-only array
 * inputs, scalar "variables", outputs allocated at the configuration stage,
 * Sec. 4.2: all memory preallocated, inputs are views, the status of a GPU
 * function is available on the host after the computation).
 *
 * Conventions for every call:
 *   - Units: E in MeV, L in km, dm2 in eV^2.  The phase of pair (i,j) is
 *     1266.932679419849 * dm2_ij * L / E rad (hbar c = 197.3269804 MeV fm);
 *     dm2_31 = dm2_21 + dm2_32 (normal ordering).
 *   - "device" pointers are CUDA global-memory pointers on the current
 *     device, owned by the caller; "host" pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it and return;
 *     argument errors are returned at once, device-side failures (CUDA
 *     errors, parameter points outside the physical domain) are reported by
 *     gna_plan_status().
 *   - Evaluation calls use only the memory gna_plan_create() allocated.
 *     Outside plans, gna_gl_nodes uses a temporary of 16 n bytes (freed
 *     before it returns), gna_poisson_datasets a stream-ordered temporary,
 *     and gna_oscprob_ee_staged keeps its staging buffers per device for the
 *     life of the process.
 *   - No exception crosses the ABI.  Errors are gna_status codes; the text of
 *     the last error of a plan is gna_plan_error(plan).
 *   - Layouts are row-major C arrays; [a][b] means b varies fastest.
 */
#ifndef GNAOSC_H
#define GNAOSC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GNA_OK = 0,
    GNA_EINVAL = 1,   /* bad argument value or NULL pointer */
    GNA_ESHAPE = 2,   /* sizes inconsistent with the plan or out of range */
    GNA_ENOMEM = 3,   /* device or pinned-host allocation failed (plan creation only) */
    GNA_ECUDA = 4,    /* a CUDA runtime call failed */
    GNA_ETIMEOUT = 5, /* reserved: no call waits on a device flag */
    GNA_ESTATE = 6    /* call not valid in the plan's current state */
} gna_status;

typedef enum {
    GNA_FP64 = 0,           /* all arithmetic in double */
    GNA_MIXED_F64PHASE = 1, /* phase and its reduction mod pi in double, the rest FP32 + Kahan */
    GNA_MIXED_FFPHASE = 2   /* phase as an unevaluated sum of two floats (double-FP32), rest FP32 + Kahan;
                               the reduction is exact for phases below 2^12 pi = 12,868 rad (K dm2 L / E),
                               beyond that its error grows with the phase: use GNA_MIXED_F64PHASE there */
} gna_precision;

typedef enum { GNA_PEARSON = 0, GNA_POISSON = 1 } gna_chi2_kind;

/* Oscillation parameters of one point: the transformation's "variables". */
typedef struct {
    double s2_12;  /* sin^2 theta12 */
    double s2_13;  /* sin^2 theta13 */
    double dm2_21; /* eV^2 */
    double dm2_32; /* eV^2 */
} gna_osc;

/* Configuration of a plan (host memory; copied by gna_plan_create). */
typedef struct {
    int nbins;                  /* >= 1 */
    const double* edges;        /* host [nbins+1], MeV, strictly increasing, > 0 */
    int nodes_per_bin;          /* Gauss-Legendre order of every point when node_counts == NULL; 1..65536 */
    int npts;                   /* parameter points evaluated per call; >= 1 */
    const int32_t* node_counts; /* host [npts] per-point order (points of equal order share a grid), or NULL */
    int nL;                     /* baselines, 1..16 */
    const double* L;            /* host [nL], km, > 0 */
    const double* Lweight;      /* host [nL] combination weights (finite, >= 0, positive finite sum; normalised to sum 1), or NULL for 1/L^2 */
    double norm;                /* N: mu_i = N (1 + eta_i) sum_r omega_r mu_r,i */
    double e_scale;             /* spectrum S(E * e_scale): 1 for MeV, 1e-3 for GeV */
    gna_precision prec;
    gna_chi2_kind kind;
    int max_datasets;           /* >= npts when each point has its own data row (fits); 0 = npts */
    int flags;                  /* GNA_PLAN_* bits below */
    int alpha, beta;            /* with GNA_PLAN_GENERAL: the channel P(alpha -> beta), 0 = e, 1 = mu, 2 = tau */
    int anti;                   /* with GNA_PLAN_GENERAL: 1 for antineutrinos, 0 for neutrinos */
} gna_plan_desc;

#define GNA_PLAN_WITH_PLAIN 1  /* also build the FP64 arrays and scratch of gna_chain_eval_plain */
#define GNA_PLAN_FORCE_SPLIT 2 /* equal node ranges per warp across bins (default in FP64 for >= 1024 nodes/bin) */
#define GNA_PLAN_FORCE_BINS 4  /* one thread per bin (default for small or per-point grids) */
#define GNA_PLAN_FORCE_SLICES 8 /* one thread per bin and slice of its nodes, slices summed by a
                                   second kernel (default for uniform grids in the mixed
                                   precisions when points x bin groups are too few to fill the GPU) */
#define GNA_PLAN_GENERAL 16     /* the chain for any channel (alpha, beta, anti above), evaluated by
                                   gna_chain_eval_general: up to 8 baselines; in the mixed
                                   precisions the slice mapping on equal node counts and the bin
                                   mapping otherwise, in GNA_FP64 the bin mapping; the
                                   survival-chain calls return GNA_ESTATE on such a plan */

/* Outputs of one evaluation (device pointers; any may be NULL except chi2). */
typedef struct {
    double* chi2;    /* [npts] */
    double* grad;    /* [npts][4] d chi2 / d(s2_12, s2_13, dm2_21, dm2_32) */
    double* grad_eta;/* [npts][nbins] d chi2 / d eta_i (needs eta) */
    double* mu;      /* [npts][nbins] mu_i = N (1 + eta_i) M_i */
    double* spectra; /* [npts][nL][nbins] per-baseline integrals mu_r,i = int_bin S(E) P_r(E) dE */
} gna_outputs;

/* Parameters of the general three-flavour formula (gna_oscprob, gna_pmns). */
typedef struct {
    double s2_12, s2_13, s2_23; /* sin^2 theta12, theta13, theta23 */
    double delta_cp;            /* CP phase, rad */
    double dm2_21, dm2_32;      /* eV^2; dm2_31 = dm2_21 + dm2_32 (normal ordering) */
} gna_osc_full;

typedef struct gna_plan gna_plan;

/* ---------------------------------------------------------------------------
 * gna_strerror: static text for a status code.  Never NULL.
 */
const char* gna_strerror(gna_status s);

/* ---------------------------------------------------------------------------
 * gna_gl_nodes: n-point Gauss-Legendre rule on [-1, 1] (nodes ascending,
 * weights), computed by a device kernel (Newton iteration on the Legendre
 * recurrence, FP64).  The rule is not in the paper; it is the integration
 * step of the chain.  x, w: device [n].  n in 1..65536 else GNA_ESHAPE.
 * Synchronises `stream` before it returns (its 16 n-byte temporary is freed
 * then).
 */
gna_status gna_gl_nodes(int n, double* x, double* w, void* stream);

/* ---------------------------------------------------------------------------
 * gna_poisson_datasets: Poisson pseudo-data for batched fits (the
 * pseudo-experiments of the fits workload; not a step of the paper's chain),
 * generated on the device: data_out[j][i] ~ Poisson(mu[i]) for data sets
 * j < ndatasets.  Counter-based and reproducible: a mean is drawn as the sum
 * of M = ceil(mu / 500) parts of mean m = mu / M; part q of bin i in data set
 * j uses Philox4x32-10 (Salmon et al., SC'11) of the counter (i, j mod 2^32,
 * j / 2^32, q) under the key (seed mod 2^32, seed / 2^32), one 53-bit
 * uniform u = ((x0 >> 5) 2^26 + (x1 >> 6)) 2^-53, and inversion: the
 * smallest k with F(k) >= u, p_0 = e^-m (computed on the host), p_k =
 * p_{k-1} m / k, k at most 10 m + 100, each operation rounded once.  The
 * cumulative F is tabulated once per bin and bisected per sample, so the
 * cost is O(m) per bin plus O(log m) per sample.  Draws do not depend on the
 * launch shape.
 *   mu:       host [nbins], each in [0, 1e7] (GNA_EINVAL otherwise)
 *   data_out: device [ndatasets][nbins] double (integer values)
 * Uses a stream-ordered temporary: 3 nbins doubles and ints, and the tables
 * (10 m + 101 doubles per bin, bin ranges of at most 2^24 entries at a time).
 */
gna_status gna_poisson_datasets(const double* mu, int nbins, int64_t ndatasets, uint64_t seed, double* data_out,
                                void* stream);

/* ---------------------------------------------------------------------------
 * gna_oscprob_ee: element-wise OscProb transformation, paper Sec. 4.1
 * (P(nue_bar -> nue_bar), i.e. alpha = beta = e of the general formula, for
 * which the Im term vanishes): P[r][k] = 1 - sum_{i>j} A_ij sin^2(phase_ij)
 * at E[k], L[r].
 *   E:     device [n] double, MeV, > 0 -- or pinned host memory: the kernel
 *          reads it in place over the host link (unified addressing), so a
 *          host-to-host evaluation needs no staging copies
 *   L:     host [nL] double, km; nL in 1..16
 *   p:     host, one parameter point
 *   prec:  GNA_FP64 writes double P; the mixed modes write float P
 *   P_out: device (or pinned host) [nL][n] of double (GNA_FP64) or float (mixed)
 * n = 0 is valid and launches nothing.  Returns GNA_EINVAL for NULL
 * pointers, for E or P_out that the device cannot address (host memory that
 * is neither page-locked nor coherently accessible) or that is not aligned to
 * its element type, or an unknown precision; GNA_ESHAPE for n < 0 or bad nL.
 */
gna_status gna_oscprob_ee(const double* E, int64_t n, const double* L, int nL, const gna_osc* p,
                          gna_precision prec, void* P_out, void* stream);

/* ---------------------------------------------------------------------------
 * gna_oscprob_ee_staged: gna_oscprob_ee from host memory to host memory
 * through device staging buffers, in chunks whose transfers overlap the
 * evaluation (paper Sec. 4.2: CUDA streams, data in chunks, asynchronous
 * copies).  Chunk c goes to stage c mod 3, each stage an internal stream:
 * upload of E[chunk], evaluation, download of the nL rows of P[chunk]; so the
 * upload of one chunk, the evaluation of the next and the download of the one
 * before run at the same time.
 *   E_host: page-locked host [n] double, MeV, > 0
 *   P_host: page-locked host [nL][n] of double (GNA_FP64) or float (mixed)
 *   chunk:  energies per chunk; 0 = max(65536, ceil(n / 8))
 *   L, nL, p, prec: as for gna_oscprob_ee
 * Asynchronous: the stages start after the work queued on `stream` and
 * `stream` waits for all of them, so P_host is complete once `stream` has
 * synchronised.  The stages' streams and staging buffers are kept per device
 * for the life of the process (a buffer grows to the largest chunk asked
 * for); calls are serialised.  The result equals gna_oscprob_ee's bit for
 * bit.  GNA_EINVAL for NULL pointers, host memory that is not page-locked
 * (device memory included) or not aligned to its element type, or an unknown
 * precision; GNA_ESHAPE for n < 0,
 * chunk < 0 or bad nL; GNA_ECUDA if a copy or launch could not be queued.
 */
gna_status gna_oscprob_ee_staged(const double* E_host, int64_t n, const double* L, int nL, const gna_osc* p,
                                 gna_precision prec, void* P_host, int64_t chunk, void* stream);

/* ---------------------------------------------------------------------------
 * gna_pmns: the mixing matrix U[alpha][i] (alpha = e, mu, tau; i = 1, 2, 3)
 * in the standard parameterisation (paper Sec. 4.1 uses its elements),
 * U = R23 U13(delta) R12, as row-major real and imaginary parts [9] each.
 * Host only (no device work).  GNA_EINVAL for NULL pointers or s2 outside [0, 1].
 */
gna_status gna_pmns(const gna_osc_full* p, double* U_re, double* U_im);

/* ---------------------------------------------------------------------------
 * gna_oscprob: element-wise OscProb for any channel, paper Sec. 4.1 (the
 * general formula with its Im term):
 *   P[r][k] = delta_ab + sum_{i>j} [-4 Re X_ij sin^2 x_ij + 2 Im X_ij sin 2x_ij],
 *   X_ij = V*_ai V_bi V_aj V*_bj, V = U for neutrinos (anti = 0) and U* for
 *   antineutrinos (anti = 1), x_ij = K dm2_ij L[r] / E[k].
 *   alpha, beta: 0 = e, 1 = mu, 2 = tau
 *   E, L, prec, P_out, n, nL: as for gna_oscprob_ee
 * The mixed precisions reduce each phase modulo pi (both sin^2 x and sin 2x
 * have that period) and evaluate FP32 polynomials; P is then accurate to
 * ~1e-7 absolute.  GNA_EINVAL for a flavour outside 0..2, NULL pointers or
 * an unknown precision; GNA_ESHAPE for n < 0 or bad nL.
 */
gna_status gna_oscprob(const double* E, int64_t n, const double* L, int nL, int alpha, int beta, int anti,
                       const gna_osc_full* p, gna_precision prec, void* P_out, void* stream);

/* ---------------------------------------------------------------------------
 * gna_plan_create: configuration stage (paper Sec. 2, Sec. 4.2): validates
 * the description, builds every point's Gauss-Legendre energy grid on the
 * device (nodes E_ik, 1/E_ik and the weights (b-a)/2 w_k S(E_ik)), and
 * allocates all scratch.  Nothing is allocated by the evaluation calls.
 * *out receives the plan (NULL on failure).  Work is enqueued on `stream`
 * and the call synchronises it before returning.
 */
gna_status gna_plan_create(gna_plan** out, const gna_plan_desc* desc, void* stream);

/* gna_plan_destroy: frees everything the plan owns.  NULL is a no-op. */
gna_status gna_plan_destroy(gna_plan* plan);

/* gna_plan_error: text of the plan's last error ("" if none).  Owned by the plan. */
const char* gna_plan_error(const gna_plan* plan);

/* gna_plan_status: synchronises the stream of the plan's last call and
 * returns GNA_ECUDA if an asynchronous CUDA error was raised, else the device
 * status word: GNA_EINVAL when an evaluation met a parameter point outside
 * the physical domain (s2 outside [0, 1], a mass splitting not finite; the
 * parameters live on the device, so this is found there), else GNA_OK.
 * Clears the status word.  (No kernel waits on a flag, so GNA_ETIMEOUT is
 * never returned; the code is kept for the ABI.) */
gna_status gna_plan_status(gna_plan* plan);

/* gna_plan_info: sizes of the plan (host pointers; any may be NULL):
 * total energy nodes over all points, probability evaluations per call
 * (nodes x baselines), and device bytes owned. */
gna_status gna_plan_info(const gna_plan* plan, int64_t* nodes, int64_t* points_per_eval, int64_t* device_bytes);

/* ---------------------------------------------------------------------------
 * gna_chain_eval: computational stage, one fused evaluation of all npts
 * points: phase -> sin^2 -> P -> W P -> Gauss-Legendre bin sums (and the four
 * tangents when out->grad or out->grad_eta is set) -> baseline combination
 * -> nuisance normalisation -> chi^2 -> gradient contraction.
 *   params: device [npts] gna_osc
 *   eta:    device [nbins] nuisances (shared by all points) or NULL
 *   sigma_eta: nuisance sigma; the penalty sum eta_i^2 / sigma^2 is added
 *           when eta != NULL and sigma_eta > 0
 *   data:   device [npts][nbins] if data_per_point else [nbins]
 *   out:    host struct of device pointers
 * Precision follows the plan.  Asynchronous on `stream`.
 */
gna_status gna_chain_eval(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                          const double* data, int data_per_point, const gna_outputs* out, void* stream);

/* ---------------------------------------------------------------------------
 * gna_chain_eval_general: the same chain for any channel P(alpha -> beta)
 * of a plan created with GNA_PLAN_GENERAL (paper Sec. 4.1, the general
 * formula with its Im term; neutrinos use U, antineutrinos U*).
 *   params: device [npts] gna_osc_full (s2_12, s2_13, s2_23, delta_cp,
 *           dm2_21, dm2_32); the mixing parameters must lie inside (0, 1)
 *           (the gradient is singular on the boundary): a point outside is
 *           reported by gna_plan_status as GNA_EINVAL
 *   eta, sigma_eta, data, data_per_point: as for gna_chain_eval
 *   out:    chi2 [npts]; grad [npts][6] = d chi2 / d(s2_12, s2_13, s2_23,
 *           delta_cp, dm2_21, dm2_32) or NULL; grad_eta and mu as for
 *           gna_chain_eval; spectra must be NULL (GNA_EINVAL)
 * Every precision of the plan is available (GNA_FP64 uses the bin mapping).
 * The node pass accumulates channel-free sums per bin (sin^2 and sin cos of
 * the three phases, and their derivatives in the phases); the epilogue
 * contracts them with the point's coefficients -4 Re X_ij, 4 Im X_ij and
 * their derivatives, X_ij = V*_ai V_bi V_aj V*_bj.  Asynchronous on
 * `stream` (launched directly: graph mode applies to gna_chain_eval);
 * GNA_ESTATE on a survival-chain plan.
 */
gna_status gna_chain_eval_general(gna_plan* plan, const gna_osc_full* params, const double* eta, double sigma_eta,
                                  const double* data, int data_per_point, const gna_outputs* out, void* stream);

/* gna_chain_eval_cached: the epilogue only (steps a7-a9: nuisance
 * normalisation, chi^2, gradient contraction) on the per-bin node sums that
 * the plan's last gna_chain_eval / host-buffer evaluation kept, with new
 * eta, sigma_eta and data: the oscillation parameters are that
 * evaluation's.  This is the paper's recompute-only-what-changed rule for
 * the transformations downstream of the node pass (Sec. 2: a transformation
 * is recomputed only when its inputs change); a nuisance or data change costs
 * O(npts x nbins) work instead of a pass over the nodes.  Outputs as for
 * gna_chain_eval; grad / grad_eta need a kept evaluation with a gradient,
 * spectra one with spectra (else GNA_ESTATE, also when none was kept yet);
 * GNA_ESHAPE when the plan keeps no sums (npts x nbins x values > 2^25).
 * Stream order: enqueue after the evaluation that kept the sums (same stream,
 * or synchronise). */
gna_status gna_chain_eval_cached(gna_plan* plan, const double* eta, double sigma_eta, const double* data,
                                 int data_per_point, const gna_outputs* out, void* stream);

/* gna_chain_eval_host: the same evaluation from HOST buffers (the paper's
 * Sec. 4.2 sub-chain with one transfer in and one out): packs params [npts],
 * data and eta [nbins] (or NULL) into the plan's pinned staging, copies them
 * to the device in one transfer, evaluates, copies chi2 [npts], grad
 * [npts][4] (if grad != NULL) and spectra [npts][nL][nbins] (if spectra !=
 * NULL; GNA_ESHAPE when that exceeds 2^24 values) back in one transfer,
 * waits for it and unpacks them into the caller's buffers.  The evaluation
 * runs on `stream` (replayed as one graph with graph mode on,
 * gna_plan_set_graph); the two transfers run on two plan-owned copy streams,
 * joined to it by events.  Any host memory is accepted. */
gna_status gna_chain_eval_host(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                               const double* data, int data_per_point, double* chi2, double* grad, double* spectra,
                               void* stream);

/* gna_chain_eval_host_async / gna_chain_eval_host_wait: gna_chain_eval_host
 * in two halves, so that consecutive evaluations overlap the host's packing,
 * launching and unpacking with the device's work.  _async packs the inputs
 * into one of the plan's two pinned staging slots (each with its own device
 * inputs and outputs), enqueues the upload on a plan-owned copy stream, the
 * evaluation on `stream` after it, and the download on a second copy stream
 * after the evaluation (outputs: chi2, and the gradient and the spectra when
 * grad / spectra != 0), and returns a ticket at once: the upload of one
 * evaluation and the download of the other overlap the evaluation running on
 * `stream`.  _wait
 * blocks until that evaluation is done and unpacks its results into the
 * caller's buffers (any of them may be NULL).  At most two evaluations may be
 * outstanding: _async returns GNA_ESTATE while the slot it needs holds a
 * result not yet waited for, and _wait returns GNA_ESTATE for a ticket that
 * is not outstanding.  The input buffers may be reused as soon as _async
 * returns. */
gna_status gna_chain_eval_host_async(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                                     const double* data, int data_per_point, int grad, int spectra, void* stream,
                                     int64_t* ticket);
gna_status gna_chain_eval_host_wait(gna_plan* plan, int64_t ticket, double* chi2, double* grad, double* spectra);

/* gna_chain_eval_general_host, gna_chain_eval_general_host_async: the
 * host-buffer evaluation (one transfer in, one out; paper Sec. 4.2) of an
 * any-channel plan (GNA_PLAN_GENERAL; paper Sec. 4.1, the general formula):
 * params host [npts] gna_osc_full, eta and data as for gna_chain_eval_host,
 * outputs chi2 [npts] and, when grad != NULL (async: grad != 0),
 * d chi2 / d(s2_12, s2_13, s2_23, delta_cp, dm2_21, dm2_32) [npts][6].
 * The same staging slots, copy streams, graph mode and ticket rules as the
 * survival chain's calls; gna_chain_eval_host_wait takes the results (its
 * spectra argument is ignored).  GNA_ESTATE on a survival-chain plan (and
 * the survival calls return GNA_ESTATE on an any-channel plan). */
gna_status gna_chain_eval_general_host(gna_plan* plan, const gna_osc_full* params, const double* eta,
                                       double sigma_eta, const double* data, int data_per_point, double* chi2,
                                       double* grad, void* stream);
gna_status gna_chain_eval_general_host_async(gna_plan* plan, const gna_osc_full* params, const double* eta,
                                             double sigma_eta, const double* data, int data_per_point, int grad,
                                             void* stream, int64_t* ticket);

/* gna_chain_eval_plain: the same outputs computed by the plain FP64 chain,
 * one kernel per transformation as in the paper (Sec. 4.1: OscProb and its
 * tangents -> weight -> bin integration -> chi^2), intermediates in device
 * memory, CUDA's double sin/cos, no graph.  Needs a plan created with
 * GNA_PLAN_WITH_PLAIN; any node counts, per-point data and nuisances.  The
 * points are processed in chunks of at most 2^27 (point, baseline, node)
 * elements (a point is never split), each chunk flattened over its points:
 * 4 launches per chunk, 6 with a gradient.  The plan then also holds
 * 40 bytes per chunk element of scratch and 16 bytes per energy node.  The
 * reference against which the fused path is measured. */
gna_status gna_chain_eval_plain(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                                const double* data, int data_per_point, const gna_outputs* out, void* stream);

/* ---------------------------------------------------------------------------
 * gna_fit_batch: batched Levenberg-Marquardt fits of the four oscillation
 * parameters, one per point/dataset (the paper has no fitter; its Sec. 2.1
 * describes minimisation as the consumer of the prediction).  Each of the
 * `iters` iterations is one fused chi^2 + gradient + J^T W J evaluation of
 * all npts points followed by one device kernel that accepts or rejects the
 * trial (lambda /10 or x10), solves (H + lambda diag H) delta = -g (4x4,
 * FP64) and clamps the next trial into s2 in [1e-6, 1-1e-6], dm2 >= 1e-7.
 *   params: device [npts] gna_osc; in: start points; out: best points
 *   data:   device [npts][nbins]
 *   chi2_out: device [npts] best chi^2
 *   lambda0: initial damping (e.g. 1e-3)
 * With use_graph != 0 one iteration is captured once into a CUDA graph and
 * replayed `iters` times.  Asynchronous on `stream`.
 */
gna_status gna_fit_batch(gna_plan* plan, gna_osc* params, const double* data, int iters, double lambda0,
                         double* chi2_out, int use_graph, void* stream);

/* gna_fit_batch_general: the same batched Levenberg-Marquardt fits for an
 * any-channel plan, in the six parameters (s2_12, s2_13, s2_23, delta_cp,
 * dm2_21, dm2_32): each iteration is one evaluation of chi^2, its gradient
 * and J^T W J (21 entries, W = 2 / mu) followed by the 6x6 damped solve;
 * trials are clamped into s2 in [1e-6, 1 - 1e-6] for the three mixing
 * parameters and dm2 >= 1e-7, delta_cp is free.
 *   params: device [npts] gna_osc_full (in: start points, out: best points)
 *   data, iters, lambda0, chi2_out, use_graph: as for gna_fit_batch
 * GNA_ESTATE on a survival-chain plan. */
gna_status gna_fit_batch_general(gna_plan* plan, gna_osc_full* params, const double* data, int iters, double lambda0,
                                 double* chi2_out, int use_graph, void* stream);

/* ---------------------------------------------------------------------------
 * Launch shape, autotuning and graphs.
 * gna_plan_autotune: times the candidate mappings and launch shapes (node
 * mapping, threads per block, nodes per lane, slice length) for this plan on
 * `stream` with CUDA events over `reps` evaluations each and keeps the
 * fastest.  The evaluations write the outputs `out` names (device pointers,
 * as for gna_chain_eval: the kernels differ with the outputs requested), or,
 * with out == NULL, chi^2 and the gradient into plan scratch.  The choice can
 * be read back and restored as text ("mapping=slices block=256 nodes=16
 * grid=0 slice=216") for caching between runs.
 */
gna_status gna_plan_autotune(gna_plan* plan, const gna_osc* params, const double* data, int data_per_point,
                             const gna_outputs* out, int reps, void* stream);
/* gna_plan_autotune_general: the same for an any-channel plan (params:
 * device [npts] gna_osc_full; out required, as for gna_chain_eval_general):
 * threads per block and, with the slice mapping, the slice length. */
gna_status gna_plan_autotune_general(gna_plan* plan, const gna_osc_full* params, const double* data,
                                     int data_per_point, const gna_outputs* out, int reps, void* stream);
gna_status gna_plan_get_tuning(const gna_plan* plan, char* buf, int buflen);
gna_status gna_plan_set_tuning(gna_plan* plan, const char* text);

/* gna_plan_set_graph: with on != 0, gna_chain_eval captures its launches
 * into a CUDA graph the first time it sees a given set of argument pointers
 * and replays that graph afterwards (device contents may change between
 * calls; pointers may not without a new capture). */
gna_status gna_plan_set_graph(gna_plan* plan, int on);

/* gna_plan_kernel_launches: kernels launched by the most recent evaluation
 * call (graph replays count the kernels inside the graph). */
int gna_plan_kernel_launches(const gna_plan* plan);

/* gna_plan_profile: with on = k >= 1, every k-th evaluation outside graph
 * capture (the first, then every k-th after it) records a pair of CUDA events
 * on its stream around the fused node kernel (with the slice mapping: the
 * node kernel and the slice reduction; up to 8192 pairs); on = 0 switches it
 * off, on < 0 is GNA_EINVAL.  Events between two kernels keep the second from
 * starting while the first drains, so a period above 1 leaves most
 * evaluations undisturbed.  gna_plan_profile_read synchronises those events and
 * returns the summed kernel time in ms and the number of timed launches,
 * then clears them. */
gna_status gna_plan_profile(gna_plan* plan, int on);
gna_status gna_plan_profile_read(gna_plan* plan, double* total_ms, int* launches);

/* gna_fp32_probe: a measurement aid, not a step of the chain (the paper has no
 * counterpart): launches `blocks` blocks of 256 threads, each thread running 8
 * independent FP32 FMA chains for `iters` steps, i.e. blocks x 2048 x iters
 * FMAs, on `stream`.  Timed by the caller with events, it gives the FP32 pipe
 * rate against which the node kernels' operation counts are compared.
 * out: device [1] float, never written in practice (it keeps the work alive).
 * GNA_EINVAL for out == NULL, blocks < 1 or iters < 1. */
gna_status gna_fp32_probe(int blocks, int iters, float* out, void* stream);

/* gna_grad_scale: the chain rule's last step for a caller that differentiates
 * a function of chi^2 (an autograd engine): with s = d loss / d chi^2 on the
 * device, a[i] *= *s for i < na and b[j] *= *s for j < nb, in place, in one
 * launch on `stream` (a = d chi2 / d theta, b = d chi2 / d eta as an
 * evaluation wrote them).  a, b, s: memory the current device can access,
 * float64 (8-byte aligned), owned by the caller; a (b) may be NULL when na
 * (nb) is 0; na = nb = 0 launches nothing.  GNA_EINVAL for s == NULL,
 * negative counts, a NULL array with a positive count, or memory the
 * device cannot access; GNA_ECUDA if the launch fails. */
gna_status gna_grad_scale(double* a, int64_t na, double* b, int64_t nb, const double* s, void* stream);


/* ---------------------------------------------------------------------------
 * gna_chain_eval_noalloc: chi^2 (and optionally its gradient and the binned
 * prediction) of ONE parameter point for callers that cannot allocate device
 * memory -- code that runs inside a memory pool or arena it does not own,
 * plug-ins whose host framework forbids cudaMalloc, or processes that must
 * keep their device footprint fixed once they have started.  It needs no
 * plan, and it calls no cudaMalloc, no cudaFree and no allocating library
 * routine.  Its working memory is one fixed array of about 0.9 MB inside this
 * library, held by every GPU that loads the library until the process exits.
 * The paper has no counterpart to this call; it is an addition of the library.
 *   E, W:   device [nbins][n] double, bin-major: node energies (MeV, > 0) and
 *           node weights (spectrum x integration weight x half bin width)
 *   L, Lweight, nL: host, as in gna_plan_desc (Lweight NULL = 1/L^2)
 *   params: device [1] gna_osc
 *   norm, kind: as in gna_plan_desc
 *   data:   device [nbins]
 *   chi2:   device [1]; grad: device [4] or NULL; mu: device [nbins] or NULL
 * Arithmetic as GNA_MIXED_FFPHASE.  Limits: nbins <= 2048, nL <= 8 and
 * nbins * ceil(n / 1024) <= 16384; beyond them the call returns GNA_ESHAPE
 * and launches nothing.  GNA_EINVAL (nothing launched) for a NULL required
 * pointer, a device pointer that is not global memory of the current device
 * (or managed memory) or not aligned to 8 bytes, norm <= 0, an unknown chi^2
 * kind, L <= 0 or a negative weight.  The parameters live on the device and
 * are not range-checked by this call (there is no status word to report
 * through): a point outside the physical domain (s2 outside [0, 1], a mass
 * splitting not finite) gives a meaningless chi^2.  The first call on a device looks up the device
 * address of the array (cudaGetSymbolAddress) once for that device; make that
 * first call before any stream capture on the device.  Each call clears the
 * counters it needs; the rest of the array keeps the previous call's
 * contents.  Every call uses the same array, so calls whose work overlaps on
 * the GPU (other streams, other host threads) race and give wrong results:
 * serialise them on one stream.  Asynchronous on `stream`.
 */
gna_status gna_chain_eval_noalloc(int nbins, int n, const double* E, const double* W, const double* L, int nL,
                                  const double* Lweight, const gna_osc* params, double norm, gna_chi2_kind kind,
                                  const double* data, double* chi2, double* grad, double* mu, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GNAOSC_H */
