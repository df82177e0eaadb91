// pseudo.cu -- Poisson pseudo-data on the device (the pseudo-experiments of
// the batched fits; not a step of the paper's chain).  Counter-based:
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) of the counter
// (bin, data set lo, data set hi, part) under the key (seed lo, seed hi); one
// 53-bit uniform per part; Poisson by inversion with only +, *, / in double,
// each rounded once, from p_0 = e^-mu computed by the host; a mean is drawn as
// the sum of ceil(mu / 500) parts.  The draws do not depend on the launch shape.
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

__global__ void k_pseudo_data(const double* __restrict__ mu_part, const double* __restrict__ em_part,
                              const int* __restrict__ parts, int nbins, int64_t nds, uint32_t k0, uint32_t k1,
                              double* __restrict__ out) {
    const int64_t total = nds * nbins;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / nbins;
        const int i = (int)(t - j * nbins);
        const double m = mu_part[i];
        const int64_t kmax = (int64_t)(__dmul_rn(10.0, m)) + 100;
        int64_t k = 0;
        for (int part = 0; part < parts[i]; part++) {
            uint32_t c[4] = {(uint32_t)i, (uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)part};
            philox4x32_10(c, k0, k1);
            const double u = __dmul_rn(__dadd_rn(__dmul_rn((double)(c[0] >> 5), 67108864.0), (double)(c[1] >> 6)),
                                       1.0 / 9007199254740992.0);
            int64_t kp = 0;
            double p = em_part[i], F = em_part[i];
            while (u > F && kp < kmax) {
                kp++;
                p = __ddiv_rn(__dmul_rn(p, m), (double)kp);
                F = __dadd_rn(F, p);
            }
            k += kp;
        }
        out[t] = (double)k;
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
    for (int i = 0; i < nbins; i++) {
        if (!(mu[i] >= 0.0 && mu[i] <= 1e7)) return GNA_EINVAL;
        parts[i] = std::max(1, (int)std::ceil(mu[i] / 500.0));
        host[i] = mu[i] / (double)parts[i];
        host[nbins + i] = std::exp(-host[i]);
    }
    if (ndatasets == 0) return GNA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    double* d = nullptr;
    const size_t bytes = sizeof(double) * host.size() + sizeof(int) * parts.size();
    cudaError_t e = cudaMallocAsync(&d, bytes, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, s);
    int* dparts = reinterpret_cast<int*>(d + host.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(dparts, parts.data(), sizeof(int) * parts.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t total = ndatasets * nbins;
        const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8);
        k_pseudo_data<<<(unsigned)blocks, 256, 0, s>>>(d, d + nbins, dparts, nbins, ndatasets, (uint32_t)seed,
                                                       (uint32_t)(seed >> 32), data_out);
        e = cudaGetLastError();
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
