// noalloc.cu -- chi^2 + gradient of one parameter point without any device
// allocation: for callers that cannot call cudaMalloc (code that runs inside
// a memory pool they do not own, sandboxed plug-ins of a host framework, or
// processes that must not grow their device footprint after start-up).
//
// The working memory is one file-scope device array of fixed size.  Every GPU
// that loads this library holds it until the process exits.  All calls share
// it: two calls whose work overlaps on the GPU (different streams, or
// different host threads on the same device) race on it and give wrong
// results; serialise them.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "epilogue.cuh"
#include "fused.cuh"
#include "gnaosc.h"
#include "misc.h"

namespace {

// Limits of the allocation-free evaluation.
constexpr int kMaxBins = 2048;
constexpr int kMaxGroups = kMaxBins / 32;
constexpr int kMaxTiles = 16384;  // warp tiles of kTileNodes nodes over all bins
constexpr int kTileNodes = 1024;  // 32 lanes x 32 nodes
constexpr int kMaxNL = 8;
constexpr int kNVT = 6;  // combined prediction, four tangents, sum of the FP32 node weights

// Byte layout of the scratch array (each part 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffPc = 0;
constexpr size_t kOffCnt = align256(kOffPc + sizeof(PointConst));
constexpr size_t kOffSumW = align256(kOffCnt + sizeof(int) * (2 + kMaxGroups + kMaxBins));
constexpr size_t kOffPart = align256(kOffSumW + sizeof(double) * kMaxBins);
constexpr size_t kOffBin = align256(kOffPart + sizeof(float2) * kMaxTiles * kNVT);
constexpr size_t kOffGrp = align256(kOffBin + sizeof(float2) * kMaxBins * 5);
constexpr size_t kScratchBytes = align256(kOffGrp + sizeof(float2) * kMaxGroups * 5);
static_assert(kScratchBytes < (1u << 20), "scratch must stay below 1 MiB");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
void* g_scratch_dev[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];

struct NoAllocArgs {
    const double* E;  // [nbins][n]
    const double* W;  // [nbins][n]
    int nbins, n, nchunks;
    const PointConst* pc;
    BaseConst bc;
    int* counters;  // [0] tile counter, [1] groups finished, [2 + g] bins of group g finished,
                    // [2 + kMaxGroups + i] chunks of bin i finished
    float2* part;   // [nbins][nchunks][kNVT]
    double* sumW;   // [nbins]
    gna::EpiArgs ea;
};

// Same warp-tile structure as the plan's split kernel; the node values are
// formed from the caller's E and W on the fly (1/E in double, split into two
// floats), and the bin's sum of the FP32 weights is accumulated alongside for
// the epilogue's exact correction of the constant term.
template <int NL>
__global__ void __launch_bounds__(256, 2) k_noalloc_chi2(NoAllocArgs a) {
    using M = gna::NodeMath<0, NL, true, false>;
    constexpr int NV = M::NV;
    constexpr int NVP = gna::pow2ceil(kNVT);
    constexpr int SH = 5 - gna::ilog2(NVP);
    const int lane = threadIdx.x & 31;
    const int ntiles = a.nbins * a.nchunks;
    M m;
    m.load(a.pc, a.bc);
    while (true) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counters, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const int c = t % a.nchunks;
        const int i = t / a.nchunks;
        KahanF acc[NV];
        KahanF accw;
#pragma unroll
        for (int v = 0; v < NV; v++) kzero(acc[v]);
        kzero(accw);
        const int k1 = min(a.n, (c + 1) * kTileNodes);
        const double* Ei = a.E + (int64_t)i * a.n;
        const double* Wi = a.W + (int64_t)i * a.n;
        for (int k = c * kTileNodes + lane; k < k1; k += 32) {
            const double inv = 1.0 / Ei[k];
            const double w = Wi[k];
            float hi, lo;
            split_ff(inv, hi, lo);
            const float4 g = make_float4(hi, lo, (float)w, (float)(w * inv));
            m.update(g, acc);
            kadd_prod(accw, g.z, 1.0f);
        }
        float2 v[NVP];
#pragma unroll
        for (int j = 0; j < NVP; j++)
            v[j] = (j < NV) ? kahan_to_ff(acc[j < NV ? j : 0]) : (j == NV ? kahan_to_ff(accw) : make_float2(0.f, 0.f));
        warp_transpose_reduce<NVP>(v, lane);
        float2* pp = a.part + ((int64_t)i * a.nchunks) * kNVT;
        const int vi = lane >> SH;
        if ((lane & ((1 << SH) - 1)) == 0 && vi < kNVT) {
            pp[c * kNVT + vi] = v[0];
            __threadfence();
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) last = (atomicAdd(a.counters + 2 + kMaxGroups + i, 1) == a.nchunks - 1);
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double val = 0.0;
            if (lane < kNVT) {
                float2 s = __ldcg(pp + lane);
                for (int cc = 1; cc < a.nchunks; cc++) s = ff_add(s, __ldcg(pp + cc * kNVT + lane));
                val = (double)s.x + (double)s.y;
            }
            double sv[kNVT];
#pragma unroll
            for (int j = 0; j < kNVT; j++) sv[j] = __shfl_sync(0xffffffffu, val, j);
            if (lane == 0) {
                a.sumW[i] = sv[NV];
                gna::bin_epilogue(a.ea, 0, i, sv, gna::bin_inputs(a.ea, 0, i));
            }
            gna::bin_done(a.ea, 0, i, lane);
        }
    }
}

// Device address of the scratch array on the current device; looked up once
// per device (cudaGetSymbolAddress) on that device's first call.
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_once[dev], [dev]() {
        void* p = nullptr;
        g_setup_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_dev[dev] = p;
    });
    if (g_setup_err[dev] != cudaSuccess) return g_setup_err[dev];
    *out = static_cast<unsigned char*>(g_scratch_dev[dev]);
    return cudaSuccess;
}

// Whether ptr is global memory a kernel on the current device may use:
// memory of this device or managed memory, aligned to `align` bytes.  Another
// device's memory and host memory are refused before anything is launched.
bool on_this_device(const void* ptr, size_t align) {
    if (reinterpret_cast<uintptr_t>(ptr) % align) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return (at.type == cudaMemoryTypeDevice && at.device == dev) || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" gna_status gna_chain_eval_noalloc(int nbins, int n, const double* E, const double* W, const double* L, int nL,
                                             const double* Lweight, const gna_osc* params, double norm,
                                             gna_chi2_kind kind, const double* data, double* chi2, double* grad,
                                             double* mu, void* stream) {
    if (!E || !W || !L || !params || !data || !chi2) return GNA_EINVAL;
    if (kind != GNA_PEARSON && kind != GNA_POISSON) return GNA_EINVAL;
    if (!(norm > 0.0)) return GNA_EINVAL;
    if (nbins < 1 || n < 1 || nL < 1) return GNA_ESHAPE;
    const int64_t nchunks64 = ((int64_t)n + kTileNodes - 1) / kTileNodes;
    if (nbins > kMaxBins || nL > kMaxNL || (int64_t)nbins * nchunks64 > kMaxTiles) return GNA_ESHAPE;
    const int nchunks = (int)nchunks64;
    if (!on_this_device(E, 8) || !on_this_device(W, 8) || !on_this_device(params, 8) || !on_this_device(data, 8) ||
        !on_this_device(chi2, 8) || (grad && !on_this_device(grad, 8)) || (mu && !on_this_device(mu, 8)))
        return GNA_EINVAL;
    // baseline weights and their FP32 parts, as in a plan
    BaseConst bc;
    memset(&bc, 0, sizeof(bc));
    bc.nL = nL;
    double wsum = 0.0;
    double om[kMaxNL];
    for (int r = 0; r < nL; r++) {
        if (!(L[r] > 0.0) || !std::isfinite(L[r]) || (Lweight && !(Lweight[r] >= 0.0 && std::isfinite(Lweight[r]))))
            return GNA_EINVAL;
        om[r] = Lweight ? Lweight[r] : 1.0 / (L[r] * L[r]);
        wsum += om[r];
    }
    if (!(wsum > 0.0) || !std::isfinite(wsum)) return GNA_EINVAL;
    double fall = 0.0;
    for (int r = 0; r < nL; r++) {
        om[r] /= wsum;
        bc.omd[r] = om[r];
        bc.kld[r] = GNA_K_PHASE * L[r];
        bc.om[r] = (float)om[r];
        bc.omlo[r] = (float)(om[r] - (double)bc.om[r]);
        bc.wkl[r] = (float)(2.0 * om[r] * bc.kld[r]);
        fall += (double)bc.om[r] + (double)bc.omlo[r];
    }
    double fsum = 0.0;
    for (int r = 0; r < nL; r++) fsum += (double)bc.om[r];
    bc.wsum = (float)fsum;
    bc.wsum_lo = fsum - (double)bc.wsum;
    const int nl_inst = nL <= 1 ? 1 : nL <= 2 ? 2 : nL <= 4 ? 4 : 8;

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GNA_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    NoAllocArgs a{};
    a.E = E;
    a.W = W;
    a.nbins = nbins;
    a.n = n;
    a.nchunks = nchunks;
    a.pc = reinterpret_cast<const PointConst*>(base + kOffPc);
    a.bc = bc;
    a.counters = reinterpret_cast<int*>(base + kOffCnt);
    a.part = reinterpret_cast<float2*>(base + kOffPart);
    a.sumW = reinterpret_cast<double*>(base + kOffSumW);
    gna::EpiArgs& ea = a.ea;
    ea.is64 = 0;
    ea.NV = 5;
    ea.has_grad = 1;
    ea.nspec = 0;
    ea.nL_out = nL;
    ea.npts = 1;
    ea.nbins = nbins;
    ea.norm = norm;
    ea.kind = kind;
    ea.data = data;
    ea.mu_out = mu;
    ea.binvals = reinterpret_cast<float2*>(base + kOffBin);
    ea.NBV = 5;
    ea.sumW = a.sumW;
    ea.gid = nullptr;
    ea.wsum_lo = (float)((nl_inst == 1) ? bc.wsum_lo : fall - (double)bc.wsum);
    ea.chi2 = chi2;
    ea.grad = grad;
    ea.gvals = reinterpret_cast<float2*>(base + kOffGrp);
    ea.ngroups = (nbins + 31) / 32;
    ea.pt_cnt = a.counters + 1;
    ea.grp_cnt = a.counters + 2;
    ea.bin_cnt = a.counters + 2 + kMaxGroups;

    // the counters are the only scratch that must start at zero
    e = cudaMemsetAsync(a.counters, 0, sizeof(int) * (2 + kMaxGroups + nbins), s);
    if (e == cudaSuccess) e = gna::launch_prepare(params, 1, bc, reinterpret_cast<PointConst*>(base + kOffPc), s);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t need = ((int64_t)nbins * nchunks * 32 + 255) / 256;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(2LL * sms, need));
        switch (nl_inst) {
            case 1: k_noalloc_chi2<1><<<grid, 256, 0, s>>>(a); break;
            case 2: k_noalloc_chi2<2><<<grid, 256, 0, s>>>(a); break;
            case 4: k_noalloc_chi2<4><<<grid, 256, 0, s>>>(a); break;
            default: k_noalloc_chi2<8><<<grid, 256, 0, s>>>(a); break;
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GNA_ECUDA;
    }
    return GNA_OK;
}
