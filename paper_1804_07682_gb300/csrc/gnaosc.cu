// gnaosc.cu -- the C ABI: plans (configuration stage), evaluations
// (computational stage), the plain FP64 chain, batched fits, autotuning and
// CUDA-graph replay.  Paper Sec. 2 (transformations, configuration vs
// computational stage) and Sec. 4.2 (all memory preallocated at configuration,
// inputs are views, two host/device transfers per sub-chain, GPU status
// readable on the host).
#include <algorithm>
#include <complex>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "dispatch.h"
#include "fused.cuh"
#include "fused64.cuh"
#include "general.cuh"
#include "gnaosc.h"
#include "misc.h"

using namespace gna;

namespace gna {
cudaError_t dispatch_split_ph0(int, bool, bool, const void*, int, int, cudaStream_t);
cudaError_t dispatch_bins_ph0(int, bool, bool, const void*, int, int, cudaStream_t);
cudaError_t dispatch_split_ph1(int, bool, bool, const void*, int, int, cudaStream_t);
cudaError_t dispatch_bins_ph1(int, bool, bool, const void*, int, int, cudaStream_t);
cudaError_t dispatch_split_ph2(int, bool, bool, const void*, int, int, cudaStream_t);
cudaError_t dispatch_bins_ph2(int, bool, bool, const void*, int, int, cudaStream_t);
int split_regs_ph0(int, bool, bool);
int split_regs_ph1(int, bool, bool);
int split_regs_ph2(int, bool, bool);

cudaError_t dispatch_split(int ph, int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    if (ph == 0) return dispatch_split_ph0(nl, grad, spec, args, grid, block, s);
    if (ph == 1) return dispatch_split_ph1(nl, grad, spec, args, grid, block, s);
    return dispatch_split_ph2(nl, grad, spec, args, grid, block, s);
}
cudaError_t dispatch_bins(int ph, int nl, bool grad, bool spec, const void* args, int grid, int block, cudaStream_t s) {
    if (ph == 0) return dispatch_bins_ph0(nl, grad, spec, args, grid, block, s);
    if (ph == 1) return dispatch_bins_ph1(nl, grad, spec, args, grid, block, s);
    return dispatch_bins_ph2(nl, grad, spec, args, grid, block, s);
}
int split_regs(int ph, int nl, bool grad, bool spec) {
    if (ph == 0) return split_regs_ph0(nl, grad, spec);
    if (ph == 1) return split_regs_ph1(nl, grad, spec);
    return split_regs_ph2(nl, grad, spec);
}
}  // namespace gna

namespace {

enum { MAP_SPLIT = 0, MAP_BINS = 1, MAP_SLICES = 2 };
const int kDefaultBlock = 256;
const int kDefaultNodesPerThread = 16;

int inst_nl(int nl, int ph) {
    if (ph == 0) {
        if (nl <= 1) return 1;
        if (nl <= 2) return 2;
        if (nl <= 4) return 4;
        if (nl <= 8) return 8;
        return 16;
    }
    if (nl <= 1) return 1;
    if (nl <= 8) return 8;
    return 16;
}

struct GraphKey {
    std::vector<uintptr_t> v;
    bool operator==(const GraphKey& o) const { return v == o.v; }
};

}  // namespace

struct gna_plan {
    // configuration
    int nbins = 0, npts = 0, nL = 0, nl_inst = 0, ph = 0;
    std::vector<double> edges, L, omega;
    std::vector<int> counts;
    bool uniform = true;
    int n_uniform = 0;
    double norm = 1.0, e_scale = 1.0;
    int prec = GNA_MIXED_FFPHASE, kind = GNA_PEARSON, flags = 0, max_datasets = 0;
    int mapping = MAP_SPLIT;
    int sm_count = 0;
    // any-channel plans (GNA_PLAN_GENERAL): P(g_alpha -> g_beta), antineutrinos
    // when g_anti; their coefficients are prepared per point into d_gc
    bool general = false;
    int g_alpha = 0, g_beta = 0, g_anti = 0;
    GenConst* d_gc = nullptr;
    // grids: the split layout (bin-major, uniform grids) and/or the bins layout
    // ([group][node][lane] per grid); small uniform grids keep both so that the
    // autotuner can choose the mapping
    bool has_split = false, has_bins = false;
    float4* grid_split = nullptr;
    float4* grid_bins = nullptr;
    double2* grid64_split = nullptr;
    double2* grid64_bins = nullptr;
    double2* plain64 = nullptr;
    int64_t grid_len = 0, total_nodes = 0;
    int64_t* d_goff = nullptr;
    int* d_gn = nullptr;
    int* d_gid = nullptr;  // [npts] grid of each point (NULL: one grid for all)
    int ngrids = 0, ngroups = 0;
    int* d_tasks = nullptr;
    int ntasks = 0;
    // [1 + npts + npts*ngroups (+ npts*nbins, split)]: work counter, groups
    // finished per point, bins finished per group, segments finished per bin
    int* d_counters = nullptr;
    int64_t ncounters = 0;
    int maxseg_cap = 2;  // split mapping: partial slots per (point, bin) the plan allocated
    int slices_cap = 0;  // slice mapping: slices per group the plan allocated (0: unavailable)
    float2* d_slices = nullptr;  // [npts][ngroups][slices][NV][32]
    double* d_edges = nullptr;
    // constants
    BaseConst bc{};
    PointConst* d_pc = nullptr;
    // scratch
    void* d_part = nullptr;
    size_t part_cap = 0;  // elements of 8 bytes
    float2* d_binvals = nullptr;
    float2* d_gvals = nullptr;  // [npts][ngroups][15] group sums
    // per-bin node sums of the last evaluation, for epilogue-only re-evaluations
    double* d_binsums = nullptr;  // [npts][nbins][nv_max], or NULL (too large)
    bool cache_valid = false, cache_grad = false, cache_spec = false;
    double* d_H = nullptr;
    double* d_chi2_tmp = nullptr;
    double* d_grad_tmp = nullptr;
    // plain chain: element offsets per point, grid offsets, chunks of points
    // (first point of each chunk, then npts), scratch for one chunk
    std::vector<int64_t> plain_off;
    std::vector<int> plain_chunks;
    int64_t* d_plain_off = nullptr;
    int64_t* d_plain_goff = nullptr;
    double* d_plainP = nullptr;
    double* d_plainD = nullptr;
    double* d_plainMu = nullptr;
    double* d_plainDmu = nullptr;
    // fitter
    LMState* d_lm = nullptr;
    LMStateT<6>* d_lm6 = nullptr;  // any-channel plans: six parameters
    // launch shape
    int block = kDefaultBlock, npt = kDefaultNodesPerThread, grid_mult = 0;
    int slice_len = 0;  // slice mapping: nodes per slice (0: chosen from the GPU size)
    // graphs
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    int graph_launches = 0;
    // bookkeeping
    std::string err;
    cudaStream_t last_stream = nullptr;
    int last_launches = 0;
    int64_t dev_bytes = 0;
    int* d_status = nullptr;
    std::vector<void*> allocs;
    // kernel timing
    bool profile = false;
    std::vector<cudaEvent_t> prof_ev;  // pairs
    int prof_n = 0;
    int prof_every = 1;      // time every prof_every-th evaluation
    int64_t prof_seen = 0;   // evaluations seen since profiling was switched on
    // packed staging of the host-buffer call: inputs [params | data | eta],
    // outputs [chi2 | grad | spectra], pinned on the host, contiguous on the device
    // host-buffer evaluations: two pinned staging slots (an evaluation packs
    // slot k while the one before it may still be copying from slot k ^ 1),
    // one device staging pair (the stream serialises its use)
    // Host-buffer evaluations: two slots, each with pinned host staging and its
    // own device inputs and outputs, so that the upload of one evaluation (on
    // cp_in) and the download of another (on cp_out) overlap the evaluation
    // running on the caller's stream.
    struct HostSlot {
        double* h_in = nullptr;
        double* h_out = nullptr;
        double* d_in = nullptr;
        double* d_out = nullptr;
        cudaGraphExec_t exec = nullptr;
        GraphKey key;
        cudaEvent_t in_ready = nullptr;  // upload complete (cp_in)
        cudaEvent_t computed = nullptr;  // evaluation complete (caller's stream)
        cudaEvent_t done = nullptr;      // download complete (cp_out)
        int64_t ticket = -1;  // evaluation whose results the slot holds
        bool pending = false; // enqueued, results not yet taken
        bool grad = false, spectra = false;
    } hs[2];
    int64_t next_ticket = 0;
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    size_t in_cap = 0, out_cap = 0;
    double* d_sumW = nullptr;  // [ngrids][nbins]
    double wsum_all_lo = 0.0;  // sum_r (om_r + omlo_r) - wsum: constant term when the weights enter as hi + lo
    // graphs are captured on a plan-owned stream joined to the caller's by events
    cudaStream_t cap_stream = nullptr;
};

namespace {

gna_status fail(gna_plan* p, gna_status s, const char* fmt, ...) {
    if (p) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        p->err = buf;
    }
    return s;
}

#define CU(call)                                                                                      \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            cudaGetLastError(); /* consume the (non-sticky) error so later calls start clean */       \
            return fail(plan, GNA_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                    \
        }                                                                                             \
    } while (0)

template <typename T>
gna_status dalloc(gna_plan* plan, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) return GNA_OK;
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(plan, GNA_ENOMEM, "cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    }
    plan->allocs.push_back(v);
    plan->dev_bytes += (int64_t)(count * sizeof(T));
    *ptr = static_cast<T*>(v);
    return GNA_OK;
}

#define TRY(x)                          \
    do {                                \
        gna_status s_ = (x);            \
        if (s_ != GNA_OK) return s_;    \
    } while (0)

// Split mapping: equal node ranges, one per warp.  The warp count is the
// resident capacity (occupancy from the register count), but no warp gets
// fewer than 32 x npt nodes; the range length keeps every bin's segment count
// within the partial slots the plan allocated.
struct SplitShape {
    int grid;
    int64_t per;
    int maxseg;
};

int resident_ctas_per_sm(const gna_plan* p, bool grad, bool spec);

SplitShape split_shape(const gna_plan* p, bool grad, bool spec) {
    const int64_t total = (int64_t)p->npts * p->nbins * p->n_uniform;
    const int64_t resident = (int64_t)p->sm_count * resident_ctas_per_sm(p, grad, spec) * (p->block / 32);
    const int64_t min_per = 32LL * p->npt;
    int64_t warps = std::max<int64_t>(1, std::min<int64_t>(resident, (total + min_per - 1) / min_per));
    int64_t per = (total + warps - 1) / warps;
    // a bin of n nodes meets at most ceil(n / per) + 1 ranges
    const int64_t per_floor = (p->n_uniform + (p->maxseg_cap - 1) - 1) / (p->maxseg_cap - 1);
    if (per < per_floor) {
        per = per_floor;
        warps = (total + per - 1) / per;
    }
    SplitShape sh;
    sh.per = per;
    sh.grid = (int)std::max<int64_t>(1, (warps * 32 + p->block - 1) / p->block);
    sh.maxseg = (int)((p->n_uniform + per - 1) / per + 1);
    return sh;
}


int value_count(const gna_plan* p, bool grad, bool spec) { return fused_nv(p->nl_inst, grad, spec); }

int resident_ctas_per_sm(const gna_plan* p, bool grad, bool spec) {
    int per_sm = std::max(1, 1024 / p->block);
    if (p->mapping == MAP_SPLIT) {
        const int regs = split_regs(p->ph, p->nl_inst, grad, spec);
        if (regs > 0) {
            const int alloc = ((std::max(regs, 32) + 7) / 8) * 8;  // registers are allocated in units of 8
            per_sm = std::max(1, std::min(65536 / (alloc * p->block), 2048 / p->block));
        }
    }
    if (p->grid_mult > 0) per_sm = p->grid_mult;
    return per_sm;
}

// Persistent grid size of the bin mapping (warp-sized work items).
int grid_size(const gna_plan* p, bool grad, bool spec, int64_t work_items) {
    int64_t g = (int64_t)p->sm_count * resident_ctas_per_sm(p, grad, spec);
    g = std::min<int64_t>(g, (work_items * 32 + p->block - 1) / p->block);
    return (int)std::max<int64_t>(1, g);
}

// Slice mapping: S slices of L nodes per group of 32 bins.  The default L
// gives about two tasks per resident warp (estimate: 16 warps per SM), so
// that the task counter can even out the warps the schedulers favour.
struct SliceShape {
    int S, L, ntasks;
};

SliceShape slice_shape(const gna_plan* p) {
    const int n = p->n_uniform;
    const int64_t pg = (int64_t)p->npts * p->ngroups;
    int64_t L = p->slice_len;
    if (L <= 0) {
        const int64_t target = 2LL * 16 * p->sm_count;
        const int64_t S = std::max<int64_t>(1, (target + pg - 1) / pg);
        L = (n + S - 1) / S;
    }
    if (p->slices_cap <= 1) L = n;
    else L = std::max<int64_t>(L, (n + p->slices_cap - 1) / p->slices_cap);
    L = std::min<int64_t>(std::max<int64_t>(L, 1), n);
    SliceShape sh;
    sh.L = (int)L;
    sh.S = (int)((n + L - 1) / L);
    sh.ntasks = (int)(pg * sh.S);
    return sh;
}

struct EvalReq {
    const gna_osc* params;
    const double* eta;
    double sigma;
    const double* data;
    int dpp;
    double* chi2;
    double* grad;      // [npts][4] or NULL
    double* grad_eta;  // [npts][nbins] or NULL
    double* mu;
    double* spectra;
    double* H;  // [npts][10] (survival chain) or [npts][21] (any channel), or NULL (fitter)
    const gna_osc_full* pfull = nullptr;  // any-channel plans: [npts] parameters
};

// Epilogue arguments of one evaluation (outputs of q; NV node sums per bin
// laid out for the grad / spec flags).
EpiArgs make_epi(const gna_plan* plan, const EvalReq& q, bool grad, bool spec, int NV) {
    EpiArgs ea{};
    ea.is64 = plan->ph == 2;
    ea.NV = NV;
    ea.has_grad = grad;
    ea.nspec = spec ? plan->nl_inst : 0;
    ea.nL_out = plan->nL;
    ea.npts = plan->npts;
    ea.nbins = plan->nbins;
    ea.norm = plan->norm;
    ea.kind = plan->kind;
    ea.eta = q.eta;
    ea.sigma = q.sigma;
    ea.data = q.data;
    ea.data_per_point = q.dpp;
    ea.mu_out = q.mu;
    ea.spectra_out = q.spectra;
    ea.grad_eta_out = q.grad_eta;
    ea.binvals = plan->d_binvals;
    ea.NBV = q.H ? 15 : (grad ? 5 : 1);
    ea.sumW = plan->d_sumW;
    ea.gid = plan->d_gid;
    // the kernel's constant term is wsum; the exact one is sum_r om_r when the
    // per-baseline sums carry the weight correction (or one baseline), else
    // sum_r (om_r + omlo_r)
    ea.wsum_lo = (float)((spec || plan->nl_inst == 1) ? plan->bc.wsum_lo : plan->wsum_all_lo);
    for (int r = 0; r < GNA_NLMAX; r++)
        ea.om_delta[r] = (r < plan->nL) ? (float)(plan->bc.omd[r] - (double)plan->bc.om[r]) : 0.f;
    ea.chi2 = q.chi2;
    ea.grad = q.grad;
    ea.H = q.H;
    ea.gvals = plan->d_gvals;
    ea.ngroups = plan->ngroups;
    ea.pt_cnt = plan->d_counters + 1;
    ea.grp_cnt = plan->d_counters + 1 + plan->npts;
    ea.bin_cnt = plan->d_counters + 1 + plan->npts + (int64_t)plan->npts * plan->ngroups;
    return ea;
}

// Enqueue one fused evaluation; counts kernel launches into *launches.
gna_status enqueue_eval(gna_plan* plan, const EvalReq& q, cudaStream_t s, int* launches) {
    const bool grad = q.grad || q.grad_eta || q.H;
    const bool spec = q.spectra != nullptr;
    int nl = 0;
    const int NV = value_count(plan, grad, spec);
    SplitShape sh{};
    if (plan->mapping == MAP_SPLIT) {
        sh = split_shape(plan, grad, spec);
        if ((size_t)plan->npts * plan->nbins * sh.maxseg * NV > plan->part_cap)
            return fail(plan, GNA_ESHAPE, "launch shape needs %lld partials, capacity %zu",
                        (long long)plan->npts * plan->nbins * sh.maxseg * NV, plan->part_cap);
    }
    SliceShape ssh{1, 0, plan->ntasks};
    if (plan->mapping == MAP_SLICES) {
        ssh = slice_shape(plan);
        if ((int64_t)plan->npts * plan->ngroups * ssh.S >= (1LL << 31)) return fail(plan, GNA_ESHAPE, "too many slice tasks");
    }
    // work counter, per-point and per-bin arrival counters: zeroed by the
    // kernel that prepares the per-point constants
    const int64_t ncnt = 1 + (int64_t)plan->npts * (1 + plan->ngroups) +
                         (plan->mapping == MAP_SPLIT ? (int64_t)plan->npts * plan->nbins : 0);
    CU(launch_prepare(q.params, plan->npts, plan->bc, plan->d_pc, s, plan->d_counters, ncnt, plan->d_status));
    nl++;
    EpiArgs ea = make_epi(plan, q, grad, spec, NV);
    // keep the node sums for epilogue-only re-evaluations (not in fits)
    ea.binsums = q.H ? nullptr : plan->d_binsums;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cap));
    bool timed = false;
    if (plan->profile && cap == cudaStreamCaptureStatusNone)
        timed = (plan->prof_seen++ % plan->prof_every) == 0 && plan->prof_n < (int)plan->prof_ev.size() / 2;
    if (timed) CU(cudaEventRecord(plan->prof_ev[2 * plan->prof_n], s));
    if (plan->mapping == MAP_SPLIT) {
        if (plan->ph < 2) {
            const int gstep = (int)(32 % ((int64_t)plan->nbins * plan->n_uniform));
            SplitArgs a{plan->grid_split, plan->nbins, plan->n_uniform, plan->npts, sh.per, sh.maxseg, gstep,
                        plan->d_pc, plan->bc, (float2*)plan->d_part, ea};
            CU(dispatch_split(plan->ph, plan->nl_inst, grad, spec, &a, sh.grid, plan->block, s));
        } else {
            SplitArgs64 a{plan->grid64_split, plan->nbins, plan->n_uniform, plan->npts, sh.per, sh.maxseg,
                          plan->d_pc, plan->bc, (double*)plan->d_part, ea};
            CU(dispatch_split(2, plan->nl_inst, grad, spec, &a, sh.grid, plan->block, s));
        }
    } else if (plan->mapping == MAP_SLICES) {
        const int g = grid_size(plan, grad, spec, ssh.ntasks);
        const bool sliced = ssh.S > 1;
        BinArgs a{plan->grid_bins, plan->d_goff, plan->d_gn, plan->d_gid, plan->d_tasks, ssh.ntasks,
                  plan->ngroups, plan->nbins, plan->d_pc, plan->bc, plan->d_counters, ea,
                  ssh.S, ssh.L, sliced ? plan->d_slices : nullptr};
        CU(dispatch_bins(plan->ph, plan->nl_inst, grad, spec, &a, g, plan->block, s));
        if (sliced) {
            CU(launch_slices_reduce(plan->d_slices, ssh.S, NV, ea, plan->npts, s));
            nl++;
        }
    } else {
        const int g = grid_size(plan, grad, spec, plan->ntasks);
        if (plan->ph < 2) {
            BinArgs a{plan->grid_bins, plan->d_goff, plan->d_gn, plan->d_gid, plan->d_tasks, plan->ntasks,
                      plan->ngroups, plan->nbins, plan->d_pc, plan->bc, plan->d_counters, ea, 1, 0, nullptr};
            CU(dispatch_bins(plan->ph, plan->nl_inst, grad, spec, &a, g, plan->block, s));
        } else {
            BinArgs64 a{plan->grid64_bins, plan->d_goff, plan->d_gn, plan->d_gid, plan->d_tasks, plan->ntasks,
                        plan->ngroups, plan->nbins, plan->d_pc, plan->bc, plan->d_counters, ea};
            CU(dispatch_bins(2, plan->nl_inst, grad, spec, &a, g, plan->block, s));
        }
    }
    nl++;
    if (timed) {
        CU(cudaEventRecord(plan->prof_ev[2 * plan->prof_n + 1], s));
        plan->prof_n++;
    }
    if (ea.binsums) {
        plan->cache_valid = true;
        plan->cache_grad = grad;
        plan->cache_spec = spec;
    }
    *launches = nl;
    return GNA_OK;
}

// Enqueue one evaluation of an any-channel plan (q.pfull: the parameters;
// q.H set for the fits' J^T W J); counts kernel launches into *launches.
gna_status enqueue_eval_general(gna_plan* plan, const EvalReq& q, cudaStream_t s, int* launches) {
    const bool grad = q.grad || q.grad_eta || q.H;
    const bool surv = plan->g_alpha == plan->g_beta;  // survival channel: phases modulo pi/2 (general.cuh)
    const int NV = gen_nv(grad);
    SliceShape ssh{1, 0, plan->ntasks};
    if (plan->mapping == MAP_SLICES) {
        ssh = slice_shape(plan);
        if ((int64_t)plan->npts * plan->ngroups * ssh.S >= (1LL << 31)) return fail(plan, GNA_ESHAPE, "too many slice tasks");
    }
    const int64_t ncnt = 1 + (int64_t)plan->npts * (1 + plan->ngroups);
    CU(launch_prepare_general(q.pfull, plan->npts, plan->bc, plan->g_alpha, plan->g_beta, plan->g_anti, plan->d_pc,
                              plan->d_gc, plan->d_counters, ncnt, plan->d_status, s));
    EpiArgs ea = make_epi(plan, q, grad, false, NV);
    ea.NBV = q.H ? kGenNBVFit : (grad ? 7 : 1);  // chi2, the six-parameter gradient terms, J^T W J
    ea.binsums = nullptr;
    const bool sliced = ssh.S > 1;
    int64_t g = (int64_t)plan->sm_count * general_resident_ctas(plan->ph, plan->nl_inst, grad, surv, plan->block);
    g = std::max<int64_t>(1, std::min<int64_t>(g, ((int64_t)ssh.ntasks * 32 + plan->block - 1) / plan->block));
    if (plan->ph == 2) {
        GenArgs64 ga64{BinArgs64{plan->grid64_bins, plan->d_goff, plan->d_gn, plan->d_gid, plan->d_tasks, plan->ntasks,
                                 plan->ngroups, plan->nbins, plan->d_pc, plan->bc, plan->d_counters, ea},
                       plan->d_gc};
        CU(dispatch_general64(plan->nl_inst, grad, ga64, (int)g, plan->block, s));
        *launches = 2;
        return GNA_OK;
    }
    GenArgs ga{BinArgs{plan->grid_bins, plan->d_goff, plan->d_gn, plan->d_gid, plan->d_tasks, ssh.ntasks,
                       plan->ngroups, plan->nbins, plan->d_pc, plan->bc, plan->d_counters, ea, ssh.S, ssh.L,
                       sliced ? plan->d_slices : nullptr},
               plan->d_gc};
    CU(dispatch_general(plan->ph, plan->nl_inst, grad, surv, ga, (int)g, plan->block, s));
    *launches = 2;
    if (sliced) {
        CU(launch_slices_reduce_general(plan->d_slices, ssh.S, NV, ea, plan->d_gc, plan->npts, s));
        *launches = 3;
    }
    return GNA_OK;
}

gna_status check_eval_args(gna_plan* plan, const gna_osc* params, const double* data, const gna_outputs* out, int dpp) {
    if (!plan) return GNA_EINVAL;
    if (plan->general) return fail(plan, GNA_ESTATE, "an any-channel plan is evaluated by gna_chain_eval_general");
    if (!params || !data || !out || !out->chi2) return fail(plan, GNA_EINVAL, "params, data, out and out->chi2 are required");
    if (dpp && plan->max_datasets < plan->npts)
        return fail(plan, GNA_ESHAPE, "data_per_point needs max_datasets >= npts");
    return GNA_OK;
}

void destroy_profile(gna_plan* p) {
    for (cudaEvent_t e : p->prof_ev) cudaEventDestroy(e);
    p->prof_ev.clear();
    p->prof_n = 0;
    p->profile = false;
}

void destroy_graph(gna_plan* p) {
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
    p->gkey.v.clear();
    for (auto& h : p->hs) {
        if (h.exec) cudaGraphExecDestroy(h.exec);
        h.exec = nullptr;
        h.key.v.clear();
    }
}

}  // namespace

// ============================================================ C ABI ======
extern "C" {

const char* gna_strerror(gna_status s) {
    switch (s) {
        case GNA_OK: return "ok";
        case GNA_EINVAL: return "invalid argument";
        case GNA_ESHAPE: return "inconsistent or out-of-range size";
        case GNA_ENOMEM: return "allocation failed";
        case GNA_ECUDA: return "CUDA runtime error";
        case GNA_ETIMEOUT: return "bounded device wait timed out";
        case GNA_ESTATE: return "call not valid in the current state";
    }
    return "unknown status";
}

gna_status gna_gl_nodes(int n, double* x, double* w, void* stream) {
    if (!x || !w) return GNA_EINVAL;
    if (n < 1 || n > GNA_MAX_ORDER) return GNA_ESHAPE;
    cudaStream_t s = (cudaStream_t)stream;
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, 2 * sizeof(double) * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return GNA_ENOMEM;
    }
    cudaError_t e = launch_gl(n, x, w, tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    return e == cudaSuccess ? GNA_OK : GNA_ECUDA;
}

static bool aligned(const void* ptr, size_t a) { return (reinterpret_cast<uintptr_t>(ptr) % a) == 0; }

// Whether a kernel on the current device may dereference ptr: memory of this
// device, managed memory, page-locked host memory mapped at the same address
// (unified addressing), or ordinary host memory where the device reports
// coherent access to pageable memory.  Anything else (another device's
// memory included) is refused before a launch could fault.
static bool device_accessible(const void* ptr) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    switch (at.type) {
        case cudaMemoryTypeDevice: return at.device == dev;
        case cudaMemoryTypeManaged: return true;
        case cudaMemoryTypeHost: return at.devicePointer == ptr;
        default: {
            int pageable = 0;
            if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) return false;
            return pageable != 0;
        }
    }
}

// Constants of the nue_bar survival probability for one parameter point and nL
// baselines (Sec. 4.1 with alpha = beta = e): amplitudes A_ij and the phase
// coefficients K dm2 L, also as float pairs for the double-float modes.
static gna_status ee_constants(const double* L, int nL, const gna_osc* p, OscConst& oc) {
    oc = OscConst{};
    oc.nL = nL;
    const double s12 = p->s2_12, s13 = p->s2_13;
    oc.A[0] = 4.0 * s12 * (1 - s12) * (1 - s13) * (1 - s13);
    oc.A[1] = 4.0 * (1 - s12) * (1 - s13) * s13;
    oc.A[2] = 4.0 * s12 * (1 - s13) * s13;
    for (int j = 0; j < 3; j++) oc.Af[j] = (float)oc.A[j];
    oc.one_minus_A21f = (float)(1.0 - oc.A[0]);
    for (int r = 0; r < nL; r++) {
        if (!(L[r] >= 0.0)) return GNA_EINVAL;
        const double kl = GNA_K_PHASE * L[r];
        oc.c21[r] = p->dm2_21 * kl;
        oc.c32[r] = p->dm2_32 * kl;
        split_ff(oc.c21[r], oc.c21h[r], oc.c21l[r]);
        split_ff(oc.c32[r], oc.c32h[r], oc.c32l[r]);
        split_ff(oc.c21[r] + oc.c32[r], oc.c31h[r], oc.c31l[r]);
    }
    return GNA_OK;
}

gna_status gna_oscprob_ee(const double* E, int64_t n, const double* L, int nL, const gna_osc* p, gna_precision prec,
                          void* P_out, void* stream) {
    if (n < 0 || nL < 1 || nL > GNA_NLMAX) return GNA_ESHAPE;
    if (!L || !p) return GNA_EINVAL;
    if (prec != GNA_FP64 && prec != GNA_MIXED_F64PHASE && prec != GNA_MIXED_FFPHASE) return GNA_EINVAL;
    if (n == 0) return GNA_OK;
    if (!E || !P_out) return GNA_EINVAL;
    if (!device_accessible(E) || !device_accessible(P_out)) return GNA_EINVAL;
    if (!aligned(E, sizeof(double)) || !aligned(P_out, prec == GNA_FP64 ? sizeof(double) : sizeof(float)))
        return GNA_EINVAL;
    OscConst oc;
    if (ee_constants(L, nL, p, oc) != GNA_OK) return GNA_EINVAL;
    cudaError_t e = launch_oscprob(E, n, oc, prec, P_out, (cudaStream_t)stream);
    return e == cudaSuccess ? GNA_OK : GNA_ECUDA;
}

namespace {
// State of the staged transfer pipeline, one per device and kept for the
// process: a stream per stage, the events that fork the stages from and join
// them back into the caller's stream, and each stage's staging buffer.  A
// buffer is only touched by work on its own stage's stream, so stream order
// alone keeps one call's chunks from overwriting another's; growing it frees
// the old one in that same order.  The mutex serialises enqueueing.
constexpr int kStages = 3;
struct StageState {
    cudaStream_t s[kStages] = {};
    cudaEvent_t fork = nullptr, join[kStages] = {};
    char* buf[kStages] = {};
    size_t cap[kStages] = {};
};
std::mutex g_stage_mu;
std::map<int, StageState> g_stage;

cudaError_t stage_state(StageState*& out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    auto it = g_stage.find(dev);
    if (it == g_stage.end()) {
        StageState st;
        e = cudaEventCreateWithFlags(&st.fork, cudaEventDisableTiming);
        for (int j = 0; e == cudaSuccess && j < kStages; j++) {
            e = cudaStreamCreateWithFlags(&st.s[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.join[j], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            if (st.fork) cudaEventDestroy(st.fork);
            for (int j = 0; j < kStages; j++) {
                if (st.s[j]) cudaStreamDestroy(st.s[j]);
                if (st.join[j]) cudaEventDestroy(st.join[j]);
            }
            return e;
        }
        it = g_stage.emplace(dev, st).first;
    }
    out = &it->second;
    return cudaSuccess;
}
}  // namespace

gna_status gna_oscprob_ee_staged(const double* E_host, int64_t n, const double* L, int nL, const gna_osc* p,
                                 gna_precision prec, void* P_host, int64_t chunk, void* stream) {
    if (n < 0 || nL < 1 || nL > GNA_NLMAX || chunk < 0) return GNA_ESHAPE;
    if (!L || !p) return GNA_EINVAL;
    if (prec != GNA_FP64 && prec != GNA_MIXED_F64PHASE && prec != GNA_MIXED_FFPHASE) return GNA_EINVAL;
    if (n == 0) return GNA_OK;
    if (!E_host || !P_host) return GNA_EINVAL;
    for (const void* q : {(const void*)E_host, (const void*)P_host}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
            cudaGetLastError();
            return GNA_EINVAL;
        }
        if (at.type != cudaMemoryTypeHost) return GNA_EINVAL;  // page-locked host memory only
    }
    if (!aligned(E_host, sizeof(double)) || !aligned(P_host, prec == GNA_FP64 ? sizeof(double) : sizeof(float)))
        return GNA_EINVAL;
    OscConst oc;
    if (ee_constants(L, nL, p, oc) != GNA_OK) return GNA_EINVAL;
    if (chunk == 0) chunk = std::max<int64_t>(int64_t(1) << 16, (n + 7) / 8);
    chunk = std::min(chunk, n);
    const size_t esz = prec == GNA_FP64 ? sizeof(double) : sizeof(float);
    const int64_t nchunks = (n + chunk - 1) / chunk;
    const int nslots = (int)std::min<int64_t>(kStages, nchunks);
    // each staging buffer, and P's part of it, starts on a 256-byte boundary
    // (element alignment of the kernels' loads and stores, whatever chunk and nL are)
    auto round256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t e_bytes = round256(size_t(chunk) * sizeof(double)), p_bytes = round256(size_t(chunk) * nL * esz);
    std::lock_guard<std::mutex> lk(g_stage_mu);
    StageState* st = nullptr;
    if (stage_state(st) != cudaSuccess) return GNA_ECUDA;
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaEventRecord(st->fork, cs) != cudaSuccess) return GNA_ECUDA;
    bool ok = true;
    int forked = 0;
    for (int j = 0; ok && j < nslots; j++) {
        ok = cudaStreamWaitEvent(st->s[j], st->fork, 0) == cudaSuccess;
        if (!ok) break;
        forked = j + 1;
        if (st->cap[j] < e_bytes + p_bytes) {
            if (st->buf[j]) cudaFreeAsync(st->buf[j], st->s[j]);
            st->buf[j] = nullptr;
            st->cap[j] = 0;
            ok = cudaMallocAsync((void**)&st->buf[j], e_bytes + p_bytes, st->s[j]) == cudaSuccess;
            if (ok) st->cap[j] = e_bytes + p_bytes;
        }
    }
    // chunk c on stage c mod nslots: upload its energies, evaluate, download its
    // nL probability rows; the stages overlap the upload of one chunk with the
    // evaluation of the next and the download of the one before
    for (int64_t c = 0; ok && c < nchunks; c++) {
        const int j = (int)(c % nslots);
        const int64_t k0 = c * chunk, len = std::min(chunk, n - k0);
        double* dE = (double*)st->buf[j];
        char* dP = st->buf[j] + e_bytes;
        ok = cudaMemcpyAsync(dE, E_host + k0, len * sizeof(double), cudaMemcpyHostToDevice, st->s[j]) == cudaSuccess &&
             launch_oscprob(dE, len, oc, prec, dP, st->s[j]) == cudaSuccess &&
             cudaMemcpy2DAsync((char*)P_host + k0 * esz, n * esz, dP, len * esz, len * esz, nL,
                               cudaMemcpyDeviceToHost, st->s[j]) == cudaSuccess;
    }
    // join the stages back into the caller's stream (also after a failed enqueue)
    for (int j = 0; j < forked; j++)
        if (cudaEventRecord(st->join[j], st->s[j]) != cudaSuccess || cudaStreamWaitEvent(cs, st->join[j], 0) != cudaSuccess)
            ok = false;
    return ok ? GNA_OK : GNA_ECUDA;
}

gna_status gna_pmns(const gna_osc_full* p, double* U_re, double* U_im) {
    if (!p || !U_re || !U_im) return GNA_EINVAL;
    const double q[3] = {p->s2_12, p->s2_13, p->s2_23};
    for (double v : q)
        if (!(v >= 0.0 && v <= 1.0)) return GNA_EINVAL;
    // elements of R23 U13(delta) R12 written out (s_ij = sin, c_ij = cos)
    const double s12 = std::sqrt(q[0]), c12 = std::sqrt(1.0 - q[0]);
    const double s13 = std::sqrt(q[1]), c13 = std::sqrt(1.0 - q[1]);
    const double s23 = std::sqrt(q[2]), c23 = std::sqrt(1.0 - q[2]);
    const std::complex<double> ed = std::polar(1.0, p->delta_cp);  // e^{i delta}
    const std::complex<double> U[3][3] = {
        {c12 * c13, s12 * c13, s13 * std::conj(ed)},
        {-s12 * c23 - c12 * s23 * s13 * ed, c12 * c23 - s12 * s23 * s13 * ed, s23 * c13},
        {s12 * s23 - c12 * c23 * s13 * ed, -c12 * s23 - s12 * c23 * s13 * ed, c23 * c13}};
    for (int a = 0; a < 3; a++)
        for (int i = 0; i < 3; i++) {
            U_re[3 * a + i] = U[a][i].real();
            U_im[3 * a + i] = U[a][i].imag();
        }
    return GNA_OK;
}

gna_status gna_oscprob(const double* E, int64_t n, const double* L, int nL, int alpha, int beta, int anti,
                       const gna_osc_full* p, gna_precision prec, void* P_out, void* stream) {
    if (n < 0 || nL < 1 || nL > GNA_NLMAX) return GNA_ESHAPE;
    if (!L || !p || alpha < 0 || alpha > 2 || beta < 0 || beta > 2) return GNA_EINVAL;
    if (prec != GNA_FP64 && prec != GNA_MIXED_F64PHASE && prec != GNA_MIXED_FFPHASE) return GNA_EINVAL;
    double ure[9], uim[9];
    if (gna_pmns(p, ure, uim) != GNA_OK) return GNA_EINVAL;
    if (n == 0) return GNA_OK;
    if (!E || !P_out) return GNA_EINVAL;
    if (!device_accessible(E) || !device_accessible(P_out)) return GNA_EINVAL;
    if (!aligned(E, sizeof(double)) || !aligned(P_out, prec == GNA_FP64 ? sizeof(double) : sizeof(float)))
        return GNA_EINVAL;
    // V = U or U*; X_ij = V*_ai V_bi V_aj V*_bj for (i, j) = (2, 1), (3, 1), (3, 2)
    auto V = [&](int a, int i) {
        return std::complex<double>(ure[3 * a + i], anti ? -uim[3 * a + i] : uim[3 * a + i]);
    };
    const int pi_[3] = {1, 2, 2}, pj_[3] = {0, 0, 1};
    OscGenConst oc{};
    oc.nL = nL;
    oc.dab = (alpha == beta) ? 1.0 : 0.0;
    for (int q = 0; q < 3; q++) {
        const int i = pi_[q], j = pj_[q];
        const std::complex<double> X = std::conj(V(alpha, i)) * V(beta, i) * V(alpha, j) * std::conj(V(beta, j));
        oc.cr[q] = -4.0 * X.real();
        oc.ci[q] = 2.0 * X.imag();
        oc.crf[q] = (float)oc.cr[q];
        oc.cif[q] = (float)oc.ci[q];
    }
    for (int r = 0; r < nL; r++) {
        if (!(L[r] >= 0.0)) return GNA_EINVAL;
        const double kl = GNA_K_PHASE * L[r];
        const double c21 = p->dm2_21 * kl, c32 = p->dm2_32 * kl;
        const double cq[3] = {c21, c21 + c32, c32};
        for (int q = 0; q < 3; q++) {
            oc.c[q][r] = cq[q];
            split_ff(cq[q], oc.ch[q][r], oc.cl[q][r]);
        }
    }
    cudaError_t e = launch_oscgen(E, n, oc, prec, P_out, (cudaStream_t)stream);
    return e == cudaSuccess ? GNA_OK : GNA_ECUDA;
}

gna_status gna_plan_destroy(gna_plan* plan) {
    if (!plan) return GNA_OK;
    destroy_graph(plan);
    destroy_profile(plan);
    for (cudaStream_t cs : {plan->cp_in, plan->cp_out})
        if (cs) cudaStreamSynchronize(cs);
    for (auto& h : plan->hs) {
        if (h.exec) cudaGraphExecDestroy(h.exec);
        for (cudaEvent_t ev : {h.in_ready, h.computed, h.done})
            if (ev) cudaEventDestroy(ev);
        if (h.h_in) cudaFreeHost(h.h_in);
        if (h.h_out) cudaFreeHost(h.h_out);
    }
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    if (plan->cp_in) cudaStreamDestroy(plan->cp_in);
    if (plan->cp_out) cudaStreamDestroy(plan->cp_out);
    for (void* v : plan->allocs) cudaFree(v);
    delete plan;
    return GNA_OK;
}

const char* gna_plan_error(const gna_plan* plan) { return plan ? plan->err.c_str() : "no plan"; }

gna_status gna_plan_info(const gna_plan* plan, int64_t* nodes, int64_t* points, int64_t* bytes) {
    if (!plan) return GNA_EINVAL;
    if (nodes) *nodes = plan->total_nodes;
    if (points) *points = plan->total_nodes * plan->nL * (plan->uniform ? plan->npts : 1);
    if (bytes) *bytes = plan->dev_bytes;
    return GNA_OK;
}

static gna_status plan_build(gna_plan* plan, const gna_plan_desc* d, cudaStream_t s) {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&plan->sm_count, cudaDevAttrMultiProcessorCount, dev));
    plan->nbins = d->nbins;
    plan->npts = d->npts;
    plan->nL = d->nL;
    plan->norm = d->norm;
    plan->e_scale = d->e_scale > 0 ? d->e_scale : 1.0;
    plan->prec = d->prec;
    plan->kind = d->kind;
    plan->flags = d->flags;
    plan->max_datasets = std::max(d->max_datasets, d->npts);
    plan->ph = (d->prec == GNA_MIXED_FFPHASE) ? 0 : (d->prec == GNA_MIXED_F64PHASE) ? 1 : 2;
    plan->nl_inst = inst_nl(d->nL, plan->ph);
    plan->general = (d->flags & GNA_PLAN_GENERAL) != 0;
    if (plan->general) {  // the descriptor was checked by gna_plan_create
        plan->g_alpha = d->alpha;
        plan->g_beta = d->beta;
        plan->g_anti = d->anti;
    }
    plan->edges.assign(d->edges, d->edges + d->nbins + 1);
    plan->L.assign(d->L, d->L + d->nL);
    // baseline weights
    plan->omega.resize(d->nL);
    double wsum = 0.0;
    for (int r = 0; r < d->nL; r++) {
        plan->omega[r] = d->Lweight ? d->Lweight[r] : 1.0 / (d->L[r] * d->L[r]);
        wsum += plan->omega[r];
    }
    for (int r = 0; r < d->nL; r++) plan->omega[r] /= wsum;
    // node counts
    plan->counts.resize(d->npts);
    for (int p = 0; p < d->npts; p++) plan->counts[p] = d->node_counts ? d->node_counts[p] : d->nodes_per_bin;
    plan->uniform = true;
    for (int p = 1; p < d->npts; p++)
        if (plan->counts[p] != plan->counts[0]) plan->uniform = false;
    plan->n_uniform = plan->counts[0];
    // base constants
    BaseConst& bc = plan->bc;
    memset(&bc, 0, sizeof(bc));
    bc.nL = d->nL;
    double fsum = 0.0;
    for (int r = 0; r < d->nL; r++) {
        bc.omd[r] = plan->omega[r];
        bc.kld[r] = GNA_K_PHASE * d->L[r];
        bc.om[r] = (float)plan->omega[r];
        bc.omlo[r] = (float)(plan->omega[r] - (double)bc.om[r]);
        bc.wkl[r] = (float)(2.0 * plan->omega[r] * bc.kld[r]);
        fsum += (double)bc.om[r];  // exact: a handful of floats summed in double
    }
    bc.wsum = (float)fsum;
    bc.wsum_lo = fsum - (double)bc.wsum;
    double fall = 0.0;
    for (int r = 0; r < d->nL; r++) fall += (double)bc.om[r] + (double)bc.omlo[r];
    plan->wsum_all_lo = fall - (double)bc.wsum;
    // mapping and layouts
    const int ngroups = (d->nbins + 31) / 32;
    plan->ngroups = ngroups;
    if ((d->flags & (GNA_PLAN_FORCE_SPLIT | GNA_PLAN_FORCE_SLICES)) && !plan->uniform)
        return fail(plan, GNA_EINVAL, "the split and slice mappings need equal node counts for all points");
    if ((d->flags & GNA_PLAN_FORCE_SLICES) && plan->ph == 2)
        return fail(plan, GNA_EINVAL, "the slice mapping is for the mixed precisions");
    // slices of a group's nodes give enough warp tasks when the points x
    // groups alone do not (estimate: 16 resident warps per SM)
    const int64_t warps_est = 16LL * plan->sm_count;
    const bool slices_ok = plan->uniform && plan->ph < 2;
    if (plan->general)
        plan->mapping = (plan->uniform && plan->ph < 2 && !(d->flags & GNA_PLAN_FORCE_BINS)) ? MAP_SLICES : MAP_BINS;
    else if (d->flags & GNA_PLAN_FORCE_SPLIT) plan->mapping = MAP_SPLIT;
    else if (d->flags & GNA_PLAN_FORCE_BINS) plan->mapping = MAP_BINS;
    else if (d->flags & GNA_PLAN_FORCE_SLICES) plan->mapping = MAP_SLICES;
    else if (slices_ok && (int64_t)d->npts * ngroups < 4 * warps_est) plan->mapping = MAP_SLICES;
    else if (plan->uniform && (plan->n_uniform >= 1024 || (int64_t)d->npts * ngroups < 16LL * plan->sm_count))
        plan->mapping = MAP_SPLIT;
    else plan->mapping = MAP_BINS;
    const bool forced = plan->general ||
                        (d->flags & (GNA_PLAN_FORCE_SPLIT | GNA_PLAN_FORCE_BINS | GNA_PLAN_FORCE_SLICES)) != 0;
    const bool small = plan->uniform && (int64_t)d->nbins * plan->n_uniform <= (1LL << 20) &&
                       (int64_t)d->npts * d->nbins <= (1LL << 16);
    // a default slice mapping keeps the split layout too (grids up to 2^26
    // nodes), so that the autotuner can compare the two
    const bool keep_split = plan->mapping == MAP_SLICES && !forced &&
                            (int64_t)d->nbins * plan->n_uniform <= (1LL << 26);
    plan->has_split = plan->mapping == MAP_SPLIT || (!forced && small) || keep_split;
    plan->has_bins = plan->mapping == MAP_BINS || plan->mapping == MAP_SLICES || (!forced && small);
    // one grid per distinct node count: the bins and weights depend on nothing
    // else, so points with the same count share one grid (read once from HBM
    // and from L2 by the points that follow it in the task order)
    std::vector<int> gn(plan->counts.begin(), plan->counts.end());
    std::sort(gn.begin(), gn.end());
    gn.erase(std::unique(gn.begin(), gn.end()), gn.end());
    plan->ngrids = (int)gn.size();
    std::vector<int> gid(d->npts);
    for (int p = 0; p < d->npts; p++)
        gid[p] = (int)(std::lower_bound(gn.begin(), gn.end(), plan->counts[p]) - gn.begin());
    const int nbins_pad = ngroups * 32;
    // grid offsets of the bins layout (the split layout is one bin-major grid)
    std::vector<int64_t> goff(plan->ngrids);
    int64_t off = 0;
    for (int g = 0; g < plan->ngrids; g++) {
        goff[g] = off;
        off += (int64_t)nbins_pad * gn[g];
    }
    const int64_t len_bins = off;
    const int64_t len_split = (int64_t)d->nbins * plan->n_uniform;
    plan->grid_len = plan->has_bins ? len_bins : len_split;
    plan->total_nodes = 0;  // node evaluations per evaluation of all points (per point if uniform)
    if (plan->uniform) plan->total_nodes = (int64_t)d->nbins * plan->n_uniform;
    else
        for (int p = 0; p < d->npts; p++) plan->total_nodes += (int64_t)d->nbins * plan->counts[p];
    const bool want64 = plan->ph == 2;
    const bool want_plain = (d->flags & GNA_PLAN_WITH_PLAIN) != 0;
    TRY(dalloc(plan, &plan->d_edges, d->nbins + 1));
    CU(cudaMemcpyAsync(plan->d_edges, d->edges, sizeof(double) * (d->nbins + 1), cudaMemcpyHostToDevice, s));
    if (plan->has_split) {
        if (plan->ph < 2) TRY(dalloc(plan, &plan->grid_split, len_split));
        if (want64) TRY(dalloc(plan, &plan->grid64_split, len_split));
    }
    if (plan->has_bins) {
        if (plan->ph < 2) TRY(dalloc(plan, &plan->grid_bins, len_bins));
        if (want64) TRY(dalloc(plan, &plan->grid64_bins, len_bins));
    }
    // plain chain: one bin-major {1/E, W} grid per distinct node count (the
    // FP64 split grid when the plan has one: the same layout)
    const bool plain_alias = want_plain && plan->grid64_split;
    std::vector<int64_t> plain_goff(plan->ngrids);
    int64_t plain_len = 0;
    for (int g = 0; g < plan->ngrids; g++) {
        plain_goff[g] = plain_len;
        plain_len += (int64_t)d->nbins * gn[g];
    }
    if (want_plain && !plain_alias) TRY(dalloc(plan, &plan->plain64, plain_len));
    TRY(dalloc(plan, &plan->d_goff, plan->ngrids));
    TRY(dalloc(plan, &plan->d_gn, plan->ngrids));
    CU(cudaMemcpyAsync(plan->d_goff, goff.data(), sizeof(int64_t) * plan->ngrids, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(plan->d_gn, gn.data(), sizeof(int) * plan->ngrids, cudaMemcpyHostToDevice, s));
    if (plan->ngrids > 1) {
        TRY(dalloc(plan, &plan->d_gid, d->npts));
        CU(cudaMemcpyAsync(plan->d_gid, gid.data(), sizeof(int) * d->npts, cudaMemcpyHostToDevice, s));
    }
    // Gauss-Legendre rules per distinct order
    std::vector<int> orders(gn.begin(), gn.end());
    std::sort(orders.begin(), orders.end());
    orders.erase(std::unique(orders.begin(), orders.end()), orders.end());
    int64_t gl_total = 0;
    for (int n : orders) gl_total += n;
    double *glx = nullptr, *glw = nullptr, *tmp = nullptr;
    TRY(dalloc(plan, &glx, gl_total));
    TRY(dalloc(plan, &glw, gl_total));
    TRY(dalloc(plan, &tmp, 2 * (size_t)orders.back()));
    std::map<int, int64_t> gl_off;
    int64_t go = 0;
    for (int n : orders) {
        gl_off[n] = go;
        CU(launch_gl(n, glx + go, glw + go, tmp, s));
        go += n;
    }
    // energy grids
    if (plan->has_split) {
        const int n = plan->n_uniform;
        CU(launch_build_grid(d->nbins, d->nbins, plan->d_edges, n, glx + gl_off[n], glw + gl_off[n], plan->e_scale, 0,
                             plan->grid_split, plan->grid64_split, plan->plain64, s));
    }
    if (plan->has_bins)
        for (int g = 0; g < plan->ngrids; g++) {
            const int n = gn[g];
            CU(launch_build_grid(d->nbins, nbins_pad, plan->d_edges, n, glx + gl_off[n], glw + gl_off[n],
                                 plan->e_scale, 1, plan->grid_bins ? plan->grid_bins + goff[g] : nullptr,
                                 plan->grid64_bins ? plan->grid64_bins + goff[g] : nullptr,
                                 (plan->plain64 && !plan->has_split) ? plan->plain64 + plain_goff[g] : nullptr, s));
        }
    if (plain_alias) plan->plain64 = plan->grid64_split;
    if (plan->ph < 2) {
        TRY(dalloc(plan, &plan->d_sumW, (size_t)plan->ngrids * d->nbins));
        for (int g = 0; g < plan->ngrids; g++) {
            if (plan->has_split)
                CU(launch_sum_weights(plan->grid_split, d->nbins, gn[g], 0, plan->d_sumW + (size_t)g * d->nbins, s));
            else
                CU(launch_sum_weights(plan->grid_bins + goff[g], d->nbins, gn[g], 1, plan->d_sumW + (size_t)g * d->nbins, s));
        }
    }
    CU(cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking));
    // task list (bins mapping): (point, group) ordered by decreasing node count
    if (plan->has_bins) {
        if ((int64_t)d->npts * ngroups >= (1LL << 31)) return fail(plan, GNA_ESHAPE, "too many bin groups");
        std::vector<int> order(d->npts);
        for (int p = 0; p < d->npts; p++) order[p] = p;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return plan->counts[a] > plan->counts[b]; });
        std::vector<int> tasks;
        tasks.reserve((size_t)d->npts * ngroups);
        for (int p : order)
            for (int b = 0; b < ngroups; b++) tasks.push_back(p * ngroups + b);
        plan->ntasks = (int)tasks.size();
        TRY(dalloc(plan, &plan->d_tasks, tasks.size()));
        CU(cudaMemcpyAsync(plan->d_tasks, tasks.data(), sizeof(int) * tasks.size(), cudaMemcpyHostToDevice, s));
    }
    plan->ncounters = 1 + (int64_t)d->npts * (1 + ngroups) + (plan->has_split ? (int64_t)d->npts * d->nbins : 0);
    TRY(dalloc(plan, &plan->d_counters, plan->ncounters));
    // scratch
    TRY(dalloc(plan, &plan->d_pc, d->npts));
    if (plan->general) TRY(dalloc(plan, &plan->d_gc, d->npts));
    const int nv_max = std::max(fused_nv(plan->nl_inst, true, true), plan->general ? gen_nv(true) : 0);
    if (plan->has_split) {
        // ranges are at least 128 nodes long, so a bin meets at most ceil(n / 128) + 1 of
        // them; the slot count is capped so that the partials stay within 256 M values
        const int64_t pairs = (int64_t)d->npts * d->nbins;
        const int64_t by_len = (plan->n_uniform + 127) / 128 + 1;
        const int64_t by_mem = std::max<int64_t>(2, (256LL << 20) / (pairs * nv_max));
        plan->maxseg_cap = (int)std::min(by_len, by_mem);
        plan->part_cap = (size_t)pairs * plan->maxseg_cap * nv_max;
        TRY(dalloc(plan, (double**)&plan->d_part, plan->part_cap));
    }
    if (slices_ok && plan->has_bins) {
        // slices per group: up to 8 tasks per resident warp, at least 16 nodes per slice
        const int64_t pg = (int64_t)d->npts * ngroups;
        const int64_t by_tasks = (8 * warps_est + pg - 1) / pg;
        const int64_t by_len = std::max<int64_t>(1, plan->n_uniform / 16);
        plan->slices_cap = (int)std::max<int64_t>(1, std::min(by_tasks, by_len));
        if (plan->slices_cap > 1)
            TRY(dalloc(plan, &plan->d_slices, (size_t)pg * plan->slices_cap * nv_max * 32));
    }
    const int nbv_max = plan->general ? kGenNBVFit : 15;
    TRY(dalloc(plan, &plan->d_binvals, (size_t)d->npts * d->nbins * nbv_max));
    TRY(dalloc(plan, &plan->d_gvals, (size_t)d->npts * ngroups * nbv_max));
    if (!plan->general && (int64_t)d->npts * d->nbins * nv_max <= (32LL << 20))  // up to 256 MB
        TRY(dalloc(plan, &plan->d_binsums, (size_t)d->npts * d->nbins * nv_max));
    const int npar = plan->general ? 6 : 4;
    TRY(dalloc(plan, &plan->d_H, (size_t)d->npts * (npar * (npar + 1) / 2)));
    TRY(dalloc(plan, &plan->d_chi2_tmp, d->npts));
    TRY(dalloc(plan, &plan->d_grad_tmp, (size_t)d->npts * npar));
    plan->in_cap = (size_t)d->npts * npar + (size_t)plan->max_datasets * d->nbins + d->nbins;
    plan->out_cap = (size_t)d->npts * (1 + npar);
    if (!plan->general && (int64_t)d->npts * d->nL * d->nbins <= (1LL << 24))
        plan->out_cap += (size_t)d->npts * d->nL * d->nbins;
    CU(cudaStreamCreateWithFlags(&plan->cp_in, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&plan->cp_out, cudaStreamNonBlocking));
    for (auto& h : plan->hs) {
        TRY(dalloc(plan, &h.d_in, plan->in_cap));
        TRY(dalloc(plan, &h.d_out, plan->out_cap));
        cudaError_t e1 = cudaMallocHost(&h.h_in, plan->in_cap * sizeof(double));
        cudaError_t e2 = cudaMallocHost(&h.h_out, plan->out_cap * sizeof(double));
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            cudaGetLastError();
            return fail(plan, GNA_ENOMEM, "pinned staging of %zu + %zu doubles", plan->in_cap, plan->out_cap);
        }
        for (cudaEvent_t* ev : {&h.in_ready, &h.computed, &h.done})
            CU(cudaEventCreateWithFlags(ev, cudaEventDisableTiming));
    }
    if (plan->general) TRY(dalloc(plan, &plan->d_lm6, d->npts));
    else TRY(dalloc(plan, &plan->d_lm, d->npts));
    TRY(dalloc(plan, &plan->d_status, 1));
    CU(cudaMemsetAsync(plan->d_status, 0, sizeof(int), s));
    if (want_plain) {
        // points in chunks of at most 2^27 (point, baseline, node) elements
        // (P 1 GB, tangents 4 GB), a point never split across chunks
        std::vector<int64_t>& off = plan->plain_off;
        off.assign(d->npts + 1, 0);
        int64_t max_pt = 0;
        for (int p = 0; p < d->npts; p++) {
            off[p + 1] = off[p] + (int64_t)d->nbins * plan->counts[p] * d->nL;
            max_pt = std::max(max_pt, off[p + 1] - off[p]);
        }
        const int64_t cap = std::max(max_pt, std::min<int64_t>(1LL << 27, off[d->npts]));
        plan->plain_chunks.clear();
        int max_cnt = 0;
        for (int p = 0; p < d->npts;) {
            int q = p + 1;
            while (q < d->npts && off[q + 1] - off[p] <= cap) q++;
            plan->plain_chunks.push_back(p);
            max_cnt = std::max(max_cnt, q - p);
            p = q;
        }
        plan->plain_chunks.push_back(d->npts);
        TRY(dalloc(plan, &plan->d_plain_off, off.size()));
        CU(cudaMemcpyAsync(plan->d_plain_off, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, s));
        TRY(dalloc(plan, &plan->d_plain_goff, plain_goff.size()));
        CU(cudaMemcpyAsync(plan->d_plain_goff, plain_goff.data(), sizeof(int64_t) * plain_goff.size(),
                           cudaMemcpyHostToDevice, s));
        TRY(dalloc(plan, &plan->d_plainP, cap));
        TRY(dalloc(plan, &plan->d_plainD, 4 * cap));
        TRY(dalloc(plan, &plan->d_plainMu, (size_t)max_cnt * d->nL * d->nbins));
        TRY(dalloc(plan, &plan->d_plainDmu, 4 * (size_t)max_cnt * d->nL * d->nbins));
    }
    CU(cudaStreamSynchronize(s));
    CU(cudaGetLastError());
    plan->last_stream = s;
    return GNA_OK;
}

gna_status gna_plan_create(gna_plan** out, const gna_plan_desc* d, void* stream) {
    if (!out) return GNA_EINVAL;
    *out = nullptr;
    if (!d || !d->edges || !d->L) return GNA_EINVAL;
    if (d->nbins < 1 || d->npts < 1 || d->nL < 1 || d->nL > GNA_NLMAX) return GNA_ESHAPE;
    if (d->prec != GNA_FP64 && d->prec != GNA_MIXED_F64PHASE && d->prec != GNA_MIXED_FFPHASE) return GNA_EINVAL;
    if (d->kind != GNA_PEARSON && d->kind != GNA_POISSON) return GNA_EINVAL;
    for (int i = 0; i < d->nbins; i++)
        if (!(d->edges[i] > 0.0) || !(d->edges[i + 1] > d->edges[i])) return GNA_EINVAL;
    double lw_sum = 0.0;
    for (int r = 0; r < d->nL; r++) {
        if (!(d->L[r] > 0.0) || !std::isfinite(d->L[r])) return GNA_EINVAL;
        if (d->Lweight) {
            if (!(d->Lweight[r] >= 0.0) || !std::isfinite(d->Lweight[r])) return GNA_EINVAL;
            lw_sum += d->Lweight[r];
        }
    }
    // the weights are normalised by their sum: it must be positive and finite
    if (d->Lweight && !(lw_sum > 0.0 && std::isfinite(lw_sum))) return GNA_EINVAL;
    for (int p = 0; p < d->npts; p++) {
        const int n = d->node_counts ? d->node_counts[p] : d->nodes_per_bin;
        if (n < 1 || n > GNA_MAX_ORDER) return GNA_ESHAPE;
        if (!d->node_counts) break;
    }
    if (!(d->norm > 0.0)) return GNA_EINVAL;
    if (d->flags & GNA_PLAN_GENERAL) {
        if (d->flags & (GNA_PLAN_FORCE_SPLIT | GNA_PLAN_WITH_PLAIN)) return GNA_EINVAL;
        if (d->alpha < 0 || d->alpha > 2 || d->beta < 0 || d->beta > 2 || (d->anti != 0 && d->anti != 1))
            return GNA_EINVAL;
        if (d->nL > 8) return GNA_ESHAPE;
    }
    gna_plan* plan = new gna_plan();
    gna_status st = plan_build(plan, d, (cudaStream_t)stream);
    if (st != GNA_OK) {
        fprintf(stderr, "gna_plan_create: %s\n", plan->err.c_str());
        cudaStreamSynchronize((cudaStream_t)stream);
        gna_plan_destroy(plan);
        return st;
    }
    *out = plan;
    return GNA_OK;
}

gna_status gna_plan_status(gna_plan* plan) {
    if (!plan) return GNA_EINVAL;
    cudaError_t e = cudaStreamSynchronize(plan->last_stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(plan, GNA_ECUDA, "asynchronous CUDA error: %s", cudaGetErrorString(e));
    int st = 0;
    e = cudaMemcpy(&st, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(plan, GNA_ECUDA, "status read: %s", cudaGetErrorString(e));
    if (st != 0) {
        cudaMemset(plan->d_status, 0, sizeof(int));
        return fail(plan, (gna_status)st, "device status %d", st);
    }
    return GNA_OK;
}

gna_status gna_chain_eval(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta, const double* data,
                          int data_per_point, const gna_outputs* out, void* stream) {
    TRY(check_eval_args(plan, params, data, out, data_per_point));
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    EvalReq q{params, eta, sigma_eta, data, data_per_point, out->chi2, out->grad, out->grad_eta, out->mu, out->spectra,
              nullptr};
    if (!plan->use_graph) return enqueue_eval(plan, q, s, &plan->last_launches);
    double sig = sigma_eta;
    uintptr_t sigbits;
    memcpy(&sigbits, &sig, sizeof(sigbits));
    GraphKey key{{(uintptr_t)params, (uintptr_t)eta, sigbits, (uintptr_t)data, (uintptr_t)data_per_point,
                  (uintptr_t)out->chi2, (uintptr_t)out->grad, (uintptr_t)out->grad_eta, (uintptr_t)out->mu,
                  (uintptr_t)out->spectra, (uintptr_t)plan->block, (uintptr_t)plan->npt, (uintptr_t)plan->grid_mult}};
    cudaStream_t cs = plan->cap_stream;
    if (!plan->gexec || !(key == plan->gkey)) {
        destroy_graph(plan);
        CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        gna_status st = enqueue_eval(plan, q, cs, &nl);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st != GNA_OK || e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            if (st != GNA_OK) return st;
            return fail(plan, GNA_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&plan->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            plan->gexec = nullptr;
            return fail(plan, GNA_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        plan->gkey = key;
        plan->graph_launches = nl;
    }
    // captured on the plan's own stream, replayed on the caller's
    CU(cudaGraphLaunch(plan->gexec, s));
    plan->last_launches = plan->graph_launches;
    return GNA_OK;
}

gna_status gna_chain_eval_general(gna_plan* plan, const gna_osc_full* params, const double* eta, double sigma_eta,
                                  const double* data, int data_per_point, const gna_outputs* out, void* stream) {
    if (!plan) return GNA_EINVAL;
    if (!plan->general) return fail(plan, GNA_ESTATE, "the plan was created for the nue_bar survival chain");
    if (!params || !data || !out || !out->chi2) return fail(plan, GNA_EINVAL, "params, data, out and out->chi2 are required");
    if (out->spectra) return fail(plan, GNA_EINVAL, "the any-channel chain has no per-baseline spectra");
    if (data_per_point && plan->max_datasets < plan->npts)
        return fail(plan, GNA_ESHAPE, "data_per_point needs max_datasets >= npts");
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    EvalReq q{nullptr, eta, sigma_eta, data, data_per_point, out->chi2, out->grad, out->grad_eta, out->mu, nullptr,
              nullptr, params};
    return enqueue_eval_general(plan, q, s, &plan->last_launches);
}

gna_status gna_chain_eval_cached(gna_plan* plan, const double* eta, double sigma_eta, const double* data,
                                 int data_per_point, const gna_outputs* out, void* stream) {
    if (!plan || !out || !out->chi2 || !data) return GNA_EINVAL;
    if (plan->general) return fail(plan, GNA_ESTATE, "not available for an any-channel plan");
    if (data_per_point && plan->max_datasets < plan->npts) return fail(plan, GNA_ESHAPE, "data_per_point needs max_datasets >= npts");
    if (!plan->d_binsums) return fail(plan, GNA_ESHAPE, "the plan keeps no node sums (points x bins too large)");
    if (!plan->cache_valid) return fail(plan, GNA_ESTATE, "no evaluation has kept node sums yet");
    if ((out->grad || out->grad_eta) && !plan->cache_grad)
        return fail(plan, GNA_ESTATE, "the kept node sums have no tangents (evaluate with a gradient first)");
    if (out->spectra && !plan->cache_spec)
        return fail(plan, GNA_ESTATE, "the kept node sums have no per-baseline spectra");
    if (out->grad_eta && !eta) return fail(plan, GNA_EINVAL, "grad_eta needs eta");
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    const int NV = value_count(plan, plan->cache_grad, plan->cache_spec);
    EvalReq q{nullptr, eta, sigma_eta, data, data_per_point, out->chi2, out->grad, out->grad_eta, out->mu, out->spectra,
              nullptr};
    EpiArgs ea = make_epi(plan, q, plan->cache_grad, plan->cache_spec, NV);
    ea.NBV = out->grad ? 5 : 1;  // the tangent terms are summed over bins only when asked for
    ea.binsums = nullptr;
    CU(cudaMemsetAsync(plan->d_counters, 0, sizeof(int) * (1 + (size_t)plan->npts * (1 + plan->ngroups)), s));
    CU(launch_cached_epilogue(plan->d_binsums, ea, s));
    plan->last_launches = 1;
    return GNA_OK;
}

}  // extern "C"

namespace {

// Host-buffer evaluation of either chain: params are npar doubles per point
// (gna_osc, or gna_osc_full on an any-channel plan).
gna_status host_async(gna_plan* plan, const double* params, const double* eta, double sigma_eta, const double* data,
                      int data_per_point, int grad, int spectra, void* stream, int64_t* ticket) {
    const int npar = plan->general ? 6 : 4;
    if (!params || !data || !ticket) return fail(plan, GNA_EINVAL, "params, data and ticket are required");
    if (data_per_point && plan->max_datasets < plan->npts) return fail(plan, GNA_ESHAPE, "data_per_point needs max_datasets >= npts");
    const size_t n_spec = (size_t)plan->npts * plan->nL * plan->nbins;
    const size_t n_head = (size_t)plan->npts * (1 + npar);  // chi2, gradient
    if (spectra && plan->out_cap < n_head + n_spec) return fail(plan, GNA_ESHAPE, "spectra staging exceeds 2^24 values");
    const int64_t t = plan->next_ticket;
    auto& h = plan->hs[t & 1];
    if (h.pending) return fail(plan, GNA_ESTATE, "two host evaluations are outstanding: wait for ticket %lld first", (long long)h.ticket);
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    // the slot's previous evaluation was taken; its copy from h_in is complete
    CU(cudaEventSynchronize(h.done));
    // pack the inputs into pinned staging: [params | data | eta]
    const size_t n_par = (size_t)plan->npts * npar;
    const size_t n_dat = (data_per_point ? (size_t)plan->npts : 1) * plan->nbins;
    const size_t n_eta = eta ? (size_t)plan->nbins : 0;
    memcpy(h.h_in, params, n_par * sizeof(double));
    memcpy(h.h_in + n_par, data, n_dat * sizeof(double));
    if (eta) memcpy(h.h_in + n_par + n_dat, eta, n_eta * sizeof(double));
    const size_t n_in = n_par + n_dat + n_eta;
    const size_t n_out = n_head + (spectra ? n_spec : 0);
    double* d_par = h.d_in;
    double* d_dat = h.d_in + n_par;
    double* d_eta = eta ? h.d_in + n_par + n_dat : nullptr;
    EvalReq q{plan->general ? nullptr : (const gna_osc*)d_par, d_eta, sigma_eta, d_dat, data_per_point, h.d_out,
              grad ? h.d_out + plan->npts : nullptr, nullptr, nullptr, spectra ? h.d_out + n_head : nullptr, nullptr,
              plan->general ? (const gna_osc_full*)d_par : nullptr};
    // upload on cp_in once the evaluation that last read this slot's inputs
    // is done; it overlaps whatever the caller's stream is running
    CU(cudaStreamWaitEvent(plan->cp_in, h.computed, 0));
    CU(cudaMemcpyAsync(h.d_in, h.h_in, n_in * sizeof(double), cudaMemcpyHostToDevice, plan->cp_in));
    CU(cudaEventRecord(h.in_ready, plan->cp_in));
    // the evaluation on the caller's stream, after the upload and after the
    // download of this slot's previous results
    CU(cudaStreamWaitEvent(s, h.in_ready, 0));
    CU(cudaStreamWaitEvent(s, h.done, 0));
    auto enqueue_all = [&](cudaStream_t st, int* nl) -> gna_status {
        return plan->general ? enqueue_eval_general(plan, q, st, nl) : enqueue_eval(plan, q, st, nl);
    };
    if (plan->use_graph) {
        double sig = sigma_eta;
        uintptr_t sigbits;
        memcpy(&sigbits, &sig, sizeof(sigbits));
        GraphKey key{{(uintptr_t)data_per_point, (uintptr_t)(eta != nullptr), sigbits, (uintptr_t)(grad != 0),
                      (uintptr_t)(spectra != 0), (uintptr_t)plan->block, (uintptr_t)plan->npt,
                      (uintptr_t)plan->grid_mult, (uintptr_t)plan->mapping, (uintptr_t)plan->slice_len}};
        cudaStream_t cs = plan->cap_stream;
        if (!h.exec || !(key == h.key)) {
            if (h.exec) cudaGraphExecDestroy(h.exec);
            h.exec = nullptr;
            CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            int nl = 0;
            gna_status st = enqueue_all(cs, &nl);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cs, &g);
            if (st != GNA_OK || e != cudaSuccess) {
                cudaGetLastError();
                if (g) cudaGraphDestroy(g);
                if (st != GNA_OK) return st;
                return fail(plan, GNA_ECUDA, "host graph capture: %s", cudaGetErrorString(e));
            }
            e = cudaGraphInstantiate(&h.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h.exec = nullptr;
                return fail(plan, GNA_ECUDA, "host graph instantiate: %s", cudaGetErrorString(e));
            }
            h.key = key;
            plan->graph_launches = nl;
        }
        CU(cudaGraphLaunch(h.exec, s));
        plan->last_launches = plan->graph_launches;
    } else {
        TRY(enqueue_all(s, &plan->last_launches));
    }
    CU(cudaEventRecord(h.computed, s));
    // download on cp_out after the evaluation; it overlaps the next one
    CU(cudaStreamWaitEvent(plan->cp_out, h.computed, 0));
    CU(cudaMemcpyAsync(h.h_out, h.d_out, n_out * sizeof(double), cudaMemcpyDeviceToHost, plan->cp_out));
    CU(cudaEventRecord(h.done, plan->cp_out));
    h.ticket = t;
    h.pending = true;
    h.grad = grad != 0;
    h.spectra = spectra != 0;
    plan->next_ticket = t + 1;
    *ticket = t;
    return GNA_OK;
}

}  // namespace

extern "C" {

gna_status gna_chain_eval_host_async(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                                     const double* data, int data_per_point, int grad, int spectra, void* stream,
                                     int64_t* ticket) {
    if (!plan) return GNA_EINVAL;
    if (plan->general) return fail(plan, GNA_ESTATE, "an any-channel plan is evaluated by gna_chain_eval_general_host_async");
    return host_async(plan, (const double*)params, eta, sigma_eta, data, data_per_point, grad, spectra, stream, ticket);
}

gna_status gna_chain_eval_general_host_async(gna_plan* plan, const gna_osc_full* params, const double* eta,
                                             double sigma_eta, const double* data, int data_per_point, int grad,
                                             void* stream, int64_t* ticket) {
    if (!plan) return GNA_EINVAL;
    if (!plan->general) return fail(plan, GNA_ESTATE, "the plan was created for the nue_bar survival chain");
    return host_async(plan, (const double*)params, eta, sigma_eta, data, data_per_point, grad, 0, stream, ticket);
}

gna_status gna_chain_eval_host_wait(gna_plan* plan, int64_t ticket, double* chi2, double* grad, double* spectra) {
    if (!plan) return GNA_EINVAL;
    if (ticket < 0) return fail(plan, GNA_EINVAL, "bad ticket");
    auto& h = plan->hs[ticket & 1];
    if (h.ticket != ticket || !h.pending) return fail(plan, GNA_ESTATE, "no outstanding host evaluation %lld", (long long)ticket);
    CU(cudaEventSynchronize(h.done));
    h.pending = false;
    const int npar = plan->general ? 6 : 4;
    if (chi2) memcpy(chi2, h.h_out, sizeof(double) * plan->npts);
    if (grad && h.grad) memcpy(grad, h.h_out + plan->npts, sizeof(double) * npar * plan->npts);
    if (spectra && h.spectra)
        memcpy(spectra, h.h_out + (size_t)plan->npts * (1 + npar), sizeof(double) * plan->npts * plan->nL * plan->nbins);
    return GNA_OK;
}

gna_status gna_chain_eval_general_host(gna_plan* plan, const gna_osc_full* params, const double* eta,
                                       double sigma_eta, const double* data, int data_per_point, double* chi2,
                                       double* grad, void* stream) {
    if (!plan) return GNA_EINVAL;
    if (!chi2) return fail(plan, GNA_EINVAL, "params, data and chi2 are required");
    int64_t t = -1;
    TRY(gna_chain_eval_general_host_async(plan, params, eta, sigma_eta, data, data_per_point, grad != nullptr, stream,
                                          &t));
    return gna_chain_eval_host_wait(plan, t, chi2, grad, nullptr);
}

gna_status gna_chain_eval_host(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                               const double* data, int data_per_point, double* chi2, double* grad, double* spectra,
                               void* stream) {
    if (!plan) return GNA_EINVAL;
    if (!chi2) return fail(plan, GNA_EINVAL, "params, data and chi2 are required");
    int64_t t = -1;
    TRY(gna_chain_eval_host_async(plan, params, eta, sigma_eta, data, data_per_point, grad != nullptr, spectra != nullptr,
                                  stream, &t));
    return gna_chain_eval_host_wait(plan, t, chi2, grad, spectra);
}

gna_status gna_chain_eval_plain(gna_plan* plan, const gna_osc* params, const double* eta, double sigma_eta,
                                const double* data, int data_per_point, const gna_outputs* out, void* stream) {
    TRY(check_eval_args(plan, params, data, out, data_per_point));
    if (!plan->plain64 || !plan->d_plainP)
        return fail(plan, GNA_ESTATE, "plan was created without GNA_PLAN_WITH_PLAIN");
    cudaStream_t s = (cudaStream_t)stream;
    plan->last_stream = s;
    const bool grad = out->grad || out->grad_eta;
    CU(launch_prepare(params, plan->npts, plan->bc, plan->d_pc, s, nullptr, 0, plan->d_status));
    int nl = 1;
    for (size_t c = 0; c + 1 < plan->plain_chunks.size(); c++) {
        const int p0 = plan->plain_chunks[c], p1 = plan->plain_chunks[c + 1];
        PlainArgs a{};
        a.nodes = plan->plain64;
        a.goff = plan->d_plain_goff;
        a.gn = plan->d_gn;
        a.gid = plan->d_gid;
        a.off = plan->d_plain_off;
        a.pcs = plan->d_pc;
        a.bc = plan->bc;
        a.nbins = plan->nbins;
        a.nL = plan->nL;
        a.p0 = p0;
        a.cnt = p1 - p0;
        a.grad = grad;
        a.len = plan->plain_off[p1] - plan->plain_off[p0];
        a.P = plan->d_plainP;
        a.dP = plan->d_plainD;
        a.mu_r = plan->d_plainMu;
        a.dmu = plan->d_plainDmu;
        PlainChi2Args ca{};
        ca.mu_r = plan->d_plainMu;
        ca.dmu = grad ? plan->d_plainDmu : nullptr;
        ca.bc = plan->bc;
        ca.nL = plan->nL;
        ca.nbins = plan->nbins;
        ca.p0 = p0;
        ca.cnt = p1 - p0;
        ca.norm = plan->norm;
        ca.kind = plan->kind;
        ca.eta = eta;
        ca.sigma = sigma_eta;
        ca.data = data;
        ca.dpp = data_per_point;
        ca.chi2 = out->chi2;
        ca.grad = out->grad;
        ca.mu_out = out->mu;
        ca.grad_eta_out = out->grad_eta;
        ca.spectra_out = out->spectra;
        CU(launch_plain_chunk(a, ca, s));
        nl += grad ? 6 : 4;
    }
    plan->last_launches = nl;
    return GNA_OK;
}

}  // extern "C"

namespace {

// Batched Levenberg-Marquardt fits of either chain: NP parameters per data set
// (NP doubles per point: gna_osc, or gna_osc_full on an any-channel plan).
template <int NP>
gna_status fit_impl(gna_plan* plan, double* params, const double* data, int iters, double lambda0, double* chi2_out,
                    int use_graph, cudaStream_t s, LMStateT<NP>* lm) {
    if (!params || !data || !chi2_out) return fail(plan, GNA_EINVAL, "params, data and chi2_out are required");
    if (iters < 1) return fail(plan, GNA_EINVAL, "iters must be >= 1");
    if (plan->max_datasets < plan->npts) return fail(plan, GNA_ESHAPE, "fits need one data row per point");
    plan->last_stream = s;
    CU(launch_lm_init<NP>(lm, plan->npts, lambda0, s));
    EvalReq q{NP == 4 ? (const gna_osc*)params : nullptr, nullptr, 0.0, data, 1, plan->d_chi2_tmp, plan->d_grad_tmp,
              nullptr, nullptr, nullptr, plan->d_H, NP == 6 ? (const gna_osc_full*)params : nullptr};
    auto enqueue = [&](cudaStream_t st, int* nl) -> gna_status {
        return NP == 6 ? enqueue_eval_general(plan, q, st, nl) : enqueue_eval(plan, q, st, nl);
    };
    int launches = 1;
    if (use_graph) {
        cudaStream_t cs = plan->cap_stream;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int nl = 0;
        gna_status st = enqueue(cs, &nl);
        cudaError_t e1 = launch_lm_update<NP>(plan->npts, plan->d_chi2_tmp, plan->d_grad_tmp, plan->d_H, lm, params,
                                              chi2_out, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (st != GNA_OK || e1 != cudaSuccess || e != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            if (st != GNA_OK) return st;
            return fail(plan, GNA_ECUDA, "fit graph capture: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e));
        }
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(plan, GNA_ECUDA, "fit graph instantiate: %s", cudaGetErrorString(e));
        }
        for (int it = 0; it < iters && e == cudaSuccess; it++) e = cudaGraphLaunch(ex, s);
        cudaGraphExecDestroy(ex);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(plan, GNA_ECUDA, "fit graph launch: %s", cudaGetErrorString(e));
        }
        launches += iters * (nl + 1);
    } else {
        for (int it = 0; it < iters; it++) {
            int nl = 0;
            TRY(enqueue(s, &nl));
            CU(launch_lm_update<NP>(plan->npts, plan->d_chi2_tmp, plan->d_grad_tmp, plan->d_H, lm, params, chi2_out, s));
            launches += nl + 1;
        }
    }
    CU(launch_lm_finish<NP>(plan->npts, lm, params, s));
    plan->last_launches = launches + 1;
    return GNA_OK;
}

}  // namespace

extern "C" {

gna_status gna_fit_batch(gna_plan* plan, gna_osc* params, const double* data, int iters, double lambda0, double* chi2_out,
                         int use_graph, void* stream) {
    if (!plan) return GNA_EINVAL;
    if (plan->general) return fail(plan, GNA_ESTATE, "an any-channel plan is fitted by gna_fit_batch_general");
    return fit_impl<4>(plan, (double*)params, data, iters, lambda0, chi2_out, use_graph, (cudaStream_t)stream,
                       plan->d_lm);
}

gna_status gna_fit_batch_general(gna_plan* plan, gna_osc_full* params, const double* data, int iters, double lambda0,
                                 double* chi2_out, int use_graph, void* stream) {
    if (!plan) return GNA_EINVAL;
    if (!plan->general) return fail(plan, GNA_ESTATE, "the plan was created for the nue_bar survival chain");
    return fit_impl<6>(plan, (double*)params, data, iters, lambda0, chi2_out, use_graph, (cudaStream_t)stream,
                       plan->d_lm6);
}

gna_status gna_plan_get_tuning(const gna_plan* plan, char* buf, int buflen) {
    if (!plan || !buf || buflen < 1) return GNA_EINVAL;
    static const char* names[3] = {"split", "bins", "slices"};
    snprintf(buf, buflen, "mapping=%s block=%d nodes=%d grid=%d slice=%d", names[plan->mapping], plan->block, plan->npt,
             plan->grid_mult, plan->slice_len);
    return GNA_OK;
}

gna_status gna_plan_set_tuning(gna_plan* plan, const char* text) {
    if (!plan || !text) return GNA_EINVAL;
    int block = plan->block, npt = plan->npt, gm = plan->grid_mult, mapping = plan->mapping, sl = plan->slice_len;
    const char* b = strstr(text, "block=");
    const char* n = strstr(text, "nodes=");
    const char* g = strstr(text, "grid=");
    const char* m = strstr(text, "mapping=");
    const char* c = strstr(text, "slice=");
    if (b) block = atoi(b + 6);
    if (n) npt = atoi(n + 6);
    if (g) gm = atoi(g + 5);
    if (c) sl = atoi(c + 6);
    if (m) {
        if (!strncmp(m + 8, "split", 5)) mapping = MAP_SPLIT;
        else if (!strncmp(m + 8, "bins", 4)) mapping = MAP_BINS;
        else if (!strncmp(m + 8, "slices", 6)) mapping = MAP_SLICES;
        else return fail(plan, GNA_EINVAL, "bad mapping in '%s'", text);
    }
    if (block < 32 || block > 256 || (block & 31) || npt < 1 || npt > 1024 || gm < 0 || gm > 64 || sl < 0)
        return fail(plan, GNA_EINVAL, "bad tuning '%s'", text);
    if (plan->general && mapping != plan->mapping)
        return fail(plan, GNA_EINVAL, "an any-channel plan keeps the mapping it was created with");
    if ((mapping == MAP_SPLIT && !plan->has_split) || (mapping == MAP_BINS && !plan->has_bins) ||
        (mapping == MAP_SLICES && (!plan->has_bins || !plan->uniform || plan->ph == 2)))
        return fail(plan, GNA_EINVAL, "the plan has no grid for the %s mapping",
                    mapping == MAP_SPLIT ? "split" : mapping == MAP_BINS ? "bins" : "slices");
    if (mapping == MAP_SPLIT && npt < 4) return fail(plan, GNA_EINVAL, "nodes per lane must be >= 4");
    plan->block = block;
    plan->npt = npt;
    plan->grid_mult = gm;
    plan->mapping = mapping;
    plan->slice_len = sl;
    destroy_graph(plan);
    return GNA_OK;
}

// Times each tuning candidate (a warm-up call, then reps calls between two
// events on the stream) and keeps the fastest; the plan's tuning is restored
// when no candidate runs.
extern "C++" template <typename Eval>
gna_status time_candidates(gna_plan* plan, const std::vector<std::string>& cand, int reps, cudaStream_t s, Eval eval) {
    char best_t[128];
    gna_plan_get_tuning(plan, best_t, sizeof(best_t));
    float best = 1e30f;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    for (const std::string& c : cand) {
        if (gna_plan_set_tuning(plan, c.c_str()) != GNA_OK) continue;
        if (eval() != GNA_OK) continue;  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; r++) eval();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            snprintf(best_t, sizeof(best_t), "%s", c.c_str());
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gna_status st = gna_plan_set_tuning(plan, best_t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(plan, GNA_ECUDA, "autotune: %s", cudaGetErrorString(e));
    return st;
}

gna_status gna_plan_autotune(gna_plan* plan, const gna_osc* params, const double* data, int data_per_point,
                             const gna_outputs* out, int reps, void* stream) {
    if (!plan || !params || !data) return GNA_EINVAL;
    if (plan->general) return fail(plan, GNA_ESTATE, "not available for an any-channel plan");
    if (reps < 1) reps = 3;
    cudaStream_t s = (cudaStream_t)stream;
    // candidates are timed the way the plan will run them (graph replay when
    // the plan uses graphs: each candidate's first call captures its graph)
    std::vector<std::string> cand;
    const int blocks[3] = {64, 128, 256};
    char t[96];
    if (plan->has_split) {
        // block size only changes how the equal ranges sit on the SMs; the
        // minimum range length matters only for workloads smaller than the GPU
        const int npts_c[3] = {4, 16, 64};
        for (int b : blocks)
            for (int m : npts_c) {
                snprintf(t, sizeof(t), "mapping=split block=%d nodes=%d", b, m);
                cand.push_back(t);
            }
    }
    if (plan->has_bins)
        for (int b : blocks) {
            snprintf(t, sizeof(t), "mapping=bins block=%d nodes=1", b);
            cand.push_back(t);
        }
    if (plan->has_bins && plan->uniform && plan->ph < 2 && plan->slices_cap > 1) {
        // slice lengths for about 1, 2 and 4 tasks per resident warp
        const int64_t pg = (int64_t)plan->npts * plan->ngroups;
        for (int b : {128, 256})
            for (int tpw : {1, 2, 4}) {
                const int64_t S = std::max<int64_t>(1, ((int64_t)tpw * 16 * plan->sm_count + pg - 1) / pg);
                const int64_t L = (plan->n_uniform + S - 1) / S;
                snprintf(t, sizeof(t), "mapping=slices block=%d slice=%lld", b, (long long)L);
                cand.push_back(t);
            }
    }
    const gna_outputs o = out ? *out : gna_outputs{plan->d_chi2_tmp, plan->d_grad_tmp, nullptr, nullptr, nullptr};
    return time_candidates(plan, cand, reps, s, [&]() {
        return gna_chain_eval(plan, params, nullptr, 0.0, data, data_per_point, &o, stream);
    });
}

gna_status gna_plan_autotune_general(gna_plan* plan, const gna_osc_full* params, const double* data,
                                     int data_per_point, const gna_outputs* out, int reps, void* stream) {
    if (!plan || !params || !data || !out || !out->chi2) return GNA_EINVAL;
    if (!plan->general) return fail(plan, GNA_ESTATE, "the plan was created for the nue_bar survival chain");
    if (reps < 1) reps = 3;
    std::vector<std::string> cand;
    char t[96];
    for (int b : {64, 128, 256}) {
        if (plan->mapping == MAP_BINS) {
            snprintf(t, sizeof(t), "mapping=bins block=%d", b);
            cand.push_back(t);
        } else {
            const int64_t pg = (int64_t)plan->npts * plan->ngroups;
            for (int tpw : {1, 2, 4}) {
                const int64_t S = std::max<int64_t>(1, ((int64_t)tpw * 16 * plan->sm_count + pg - 1) / pg);
                const int64_t L = std::min<int64_t>(plan->n_uniform, (plan->n_uniform + S - 1) / S);
                snprintf(t, sizeof(t), "mapping=slices block=%d slice=%lld", b, (long long)L);
                cand.push_back(t);
            }
        }
    }
    return time_candidates(plan, cand, reps, (cudaStream_t)stream, [&]() {
        return gna_chain_eval_general(plan, params, nullptr, 0.0, data, data_per_point, out, stream);
    });
}

gna_status gna_plan_set_graph(gna_plan* plan, int on) {
    if (!plan) return GNA_EINVAL;
    plan->use_graph = on != 0;
    if (!plan->use_graph) destroy_graph(plan);
    return GNA_OK;
}

int gna_plan_kernel_launches(const gna_plan* plan) { return plan ? plan->last_launches : 0; }

gna_status gna_fp32_probe(int blocks, int iters, float* out, void* stream) {
    if (!out || blocks < 1 || iters < 1) return GNA_EINVAL;
    return launch_fma_probe(blocks, iters, out, (cudaStream_t)stream) == cudaSuccess ? GNA_OK : GNA_ECUDA;
}

gna_status gna_grad_scale(double* a, int64_t na, double* b, int64_t nb, const double* s, void* stream) {
    if (!s || na < 0 || nb < 0 || (na > 0 && !a) || (nb > 0 && !b) || na > INT64_MAX / 2 || nb > INT64_MAX / 2)
        return GNA_EINVAL;
    if (na + nb == 0) return GNA_OK;
    // memory the current device cannot read or write is refused before a launch could fault
    if (!device_accessible(s) || !aligned(s, sizeof(double))) return GNA_EINVAL;
    if (na > 0 && (!device_accessible(a) || !aligned(a, sizeof(double)))) return GNA_EINVAL;
    if (nb > 0 && (!device_accessible(b) || !aligned(b, sizeof(double)))) return GNA_EINVAL;
    return launch_grad_scale(a, na, b, nb, s, (cudaStream_t)stream) == cudaSuccess ? GNA_OK : GNA_ECUDA;
}

gna_status gna_plan_profile(gna_plan* plan, int on) {
    if (!plan) return GNA_EINVAL;
    destroy_profile(plan);
    if (on < 0) return fail(plan, GNA_EINVAL, "profile period must be >= 0");
    if (on) {
        plan->prof_ev.resize(2 * 8192);
        for (auto& e : plan->prof_ev) CU(cudaEventCreate(&e));
        plan->profile = true;
        plan->prof_every = on;
        plan->prof_seen = 0;
    }
    return GNA_OK;
}

gna_status gna_plan_profile_read(gna_plan* plan, double* total_ms, int* launches) {
    if (!plan || !total_ms || !launches) return GNA_EINVAL;
    double tot = 0.0;
    for (int i = 0; i < plan->prof_n; i++) {
        CU(cudaEventSynchronize(plan->prof_ev[2 * i + 1]));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, plan->prof_ev[2 * i], plan->prof_ev[2 * i + 1]));
        tot += ms;
    }
    *total_ms = tot;
    *launches = plan->prof_n;
    plan->prof_n = 0;
    return GNA_OK;
}

}  // extern "C"
