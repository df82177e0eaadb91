// pseudo.cu -- Poisson pseudo-data on the device (the pseudo-experiments of
// the batched fits; not a step of the paper's chain).  Counter-based:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) of the counter
// (bin, data set lo, data set hi, part) under the key (seed lo, seed hi); one
// 53-bit uniform per part; Poisson by inversion of the cumulative
// probabilities, formed with only +, *, / in double, each rounded once, from
// p_0 = e^-mu computed by the host (a table per bin, shared by all data sets);
// a mean is drawn as the sum of ceil(mu / 500) parts.  The draws do not depend
// on the launch shape.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gnaosc.h"

namespace {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// The cumulative Poisson probabilities of one bin's part mean m, F_k for
// k = 0..kmax (kmax = floor(10 m) + 100): p_0 = e^-m (from the host),
// p_k = p_(k-1) m / k and F_k = F_(k-1) + p_k, each operation rounded once.
// Past the mode (k > m) p_k no longer grows, so once adding it leaves F
// unchanged no later term changes F either: the table stops there, at ks, and
// F_k = F_ks for k > ks.  One thread per bin; the table serves all data sets.
__global__ void k_poisson_cdf(const double* __restrict__ mu_part, const double* __restrict__ em_part,
                              const int64_t* __restrict__ off, int i0, int i1, double* __restrict__ F,
                              int64_t* __restrict__ kstop) {
    const int i = i0 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= i1) return;
    const double m = mu_part[i];
    const int64_t kmax = off[i + 1] - off[i] - 1;
    double* f = F + (off[i] - off[i0]);
    double p = em_part[i], c = em_part[i];
    f[0] = c;
    int64_t k = 1;
    for (; k <= kmax; k++) {
        p = __ddiv_rn(__dmul_rn(p, m), (double)k);
        const double cn = __dadd_rn(c, p);
        f[k] = cn;
        if (cn == c && (double)k > m) break;
        c = cn;
    }
    kstop[i] = k > kmax ? kmax : k;
}

// Inversion: the draw for uniform u is the least k in [0, kmax] with u <= F_k,
// else kmax -- the count at which a sequential search from k = 0 stops, found
// here by bisection of the non-decreasing table.
__global__ void k_pseudo_data(const int* __restrict__ parts, const int64_t* __restrict__ off,
                              const int64_t* __restrict__ kstop, int nbins, int i0, int i1, int64_t nds, uint32_t k0,
                              uint32_t k1, const double* __restrict__ F, double* __restrict__ out) {
    const int nb = i1 - i0;
    const int64_t total = nds * nb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nb;
        const int i = i0 + (int)(t - j * nb);
        const double* f = F + (off[i] - off[i0]);
        const int64_t kmax = off[i + 1] - off[i] - 1, ks = kstop[i];
        int64_t k = 0;
        for (int part = 0; part < parts[i]; part++) {
            uint32_t c[4] = {(uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)part};
            philox4x32_10(c, k0, k1);
            const double u = __dmul_rn(__dadd_rn(__dmul_rn((double)(c[0] >> 5), 67108864.0), (double)(c[1] >> 6)),
                                       1.0 / 9007199254740992.0);
            int64_t lo = 0, hi = kmax;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (u > __ldg(f + (mid < ks ? mid : ks)))
                    lo = mid + 1;
                else
                    hi = mid;
            }
            k += lo;
        }
        out[j * nbins + i] = (double)k;
    }
}

}  // namespace

extern "C" gna_status gna_poisson_datasets(const double* mu, int nbins, int64_t ndatasets, uint64_t seed,
                                           double* data_out, void* stream) {
    if (nbins < 1 || ndatasets < 0) return GNA_ESHAPE;
    if (!mu || (ndatasets > 0 && !data_out)) return GNA_EINVAL;
    // a mean is drawn as the sum of M = ceil(mu / 500) parts of mean mu / M
    // (e^-(mu / M) stays a normal number); the host forms mu / M and its
    // exponential so that every implementation starts from the same bits
    std::vector<double> host(2 * (size_t)nbins);
    std::vector<int> parts(nbins);
    std::vector<int64_t> off(nbins + 1, 0);
    for (int i = 0; i < nbins; i++) {
        if (!(mu[i] >= 0.0 && mu[i] <= 1e7)) return GNA_EINVAL;
        parts[i] = std::max(1, (int)std::ceil(mu[i] / 500.0));
        host[i] = mu[i] / (double)parts[i];
        host[nbins + i] = std::exp(-host[i]);
        off[i + 1] = off[i] + (int64_t)(10.0 * host[i]) + 101;  // table F_0..F_kmax
    }
    if (ndatasets == 0) return GNA_OK;
    // tables of consecutive bin ranges of at most kTableMax entries (a bin
    // needs at most 5101); each range is built, then drawn from
    constexpr int64_t kTableMax = int64_t(1) << 24;
    int64_t table = 0;
    for (int i0 = 0; i0 < nbins;) {
        int i1 = i0 + 1;
        while (i1 < nbins && off[i1 + 1] - off[i0] <= kTableMax) i1++;
        table = std::max(table, off[i1] - off[i0]);
        i0 = i1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    char* d = nullptr;
    const size_t b_host = sizeof(double) * host.size(), b_off = sizeof(int64_t) * off.size(),
                 b_parts = sizeof(int) * parts.size(), b_ks = sizeof(int64_t) * (size_t)nbins;
    const size_t o_off = (b_host + 255) & ~size_t(255), o_parts = (o_off + b_off + 255) & ~size_t(255),
                 o_ks = (o_parts + b_parts + 255) & ~size_t(255), o_F = (o_ks + b_ks + 255) & ~size_t(255);
    cudaError_t e = cudaMallocAsync((void**)&d, o_F + sizeof(double) * (size_t)table, s);
    double* dhost = reinterpret_cast<double*>(d);
    int64_t* doff = reinterpret_cast<int64_t*>(d + o_off);
    int* dparts = reinterpret_cast<int*>(d + o_parts);
    int64_t* dks = reinterpret_cast<int64_t*>(d + o_ks);
    double* dF = reinterpret_cast<double*>(d + o_F);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dhost, host.data(), b_host, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(doff, off.data(), b_off, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dparts, parts.data(), b_parts, cudaMemcpyHostToDevice, s);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int i0 = 0; e == cudaSuccess && i0 < nbins;) {
        int i1 = i0 + 1;
        while (i1 < nbins && off[i1 + 1] - off[i0] <= kTableMax) i1++;
        // one warp per 32 bins: the sequential builds spread over the SMs
        k_poisson_cdf<<<(unsigned)((i1 - i0 + 31) / 32), 32, 0, s>>>(dhost, dhost + nbins, doff, i0, i1, dF, dks);
        const int64_t total = ndatasets * (i1 - i0);
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
        k_pseudo_data<<<(unsigned)blocks, 256, 0, s>>>(dparts, doff, dks, nbins, i0, i1, ndatasets, (uint32_t)seed,
                                                       (uint32_t)(seed >> 32), dF, data_out);
        e = cudaGetLastError();
        i0 = i1;
    }
    if (d) {
        cudaError_t e2 = cudaFreeAsync(d, s);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GNA_ECUDA;
    }
    return GNA_OK;
}
