// Polarization energy without any device allocation, for callers that cannot allocate.
//
// Same quantity as the energy of polarization_energy_forces(): E_pol = -(f/2) sum_i mu_i . E_i.
// The context-based path reduces through workspace that ap_create() allocated; this variant
// needs no context: its scratch (one partial sum per block) is a file-scope __device__ array
// that every GPU loading the library holds until the process exits. The reduction is two
// fixed-shape passes (block partials, then one block summing them in order), so the result
// is deterministic for a given n.
#include "common.cuh"

#include <mutex>

#define AP_NOALLOC_BLOCKS 4096     // partial sums (= maximum grid); 32 KB of scratch
#define AP_NOALLOC_THREADS 256
#define AP_NOALLOC_MAX_ATOMS (1 << 24)

static __device__ __align__(256) double g_noalloc_partials[AP_NOALLOC_BLOCKS];

namespace {

__device__ __forceinline__ double block_sum(double v, double *sm) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    }
    return v;
}

// pass 1: every block writes its partial of sum mu.E (no accumulation into old contents)
__global__ void k_energy_partials(const double *__restrict__ mu, const double *__restrict__ E, long m,
                                  double *__restrict__ partials) {
    __shared__ double sm[AP_NOALLOC_THREADS / 32];
    double v = 0.0;
    for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long)gridDim.x * blockDim.x)
        v += mu[k] * E[k];
    v = block_sum(v, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// pass 2: one block sums the partials of this call in a fixed order
__global__ void k_energy_final(const double *__restrict__ partials, int nparts, double scale,
                               double *__restrict__ out) {
    __shared__ double sm[AP_NOALLOC_THREADS / 32];
    double v = 0.0;
    for (int k = threadIdx.x; k < nparts; k += blockDim.x) v += partials[k];
    v = block_sum(v, sm);
    if (threadIdx.x == 0) *out = scale * v;
}

std::mutex g_mtx;
double *g_dev_ptr[256] = {nullptr};

// device address of the scratch array on the current device, looked up once per device and
// kept for the process (a cudaDeviceReset() would reload the module elsewhere: the header
// tells callers not to use this entry point on a device after resetting it)
int scratch_address(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_mtx);
    if (dev < 0 || dev >= 256) return ap_fail(nullptr, AP_ERR_ARG, "device ordinal out of range");
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            return ap_fail(nullptr, AP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_dev_ptr[dev] = (double *)p;
    }
    *out = g_dev_ptr[dev];
    return AP_OK;
}

}  // namespace

extern "C" int polarization_energy_noalloc(const double *d_mu, const double *d_field, int n, double *d_energy,
                                           void *stream) {
    if (!d_mu || !d_field || !d_energy) return ap_fail(nullptr, AP_ERR_ARG, "null pointer");
    if (n <= 0 || n > AP_NOALLOC_MAX_ATOMS)
        return ap_fail(nullptr, AP_ERR_ARG, "n must be in [1, 16777216] for polarization_energy_noalloc");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    double *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    const long m = 3L * n;
    int blocks = (int)std::min<long>(AP_NOALLOC_BLOCKS, (m + AP_NOALLOC_THREADS - 1) / AP_NOALLOC_THREADS);
    cudaStream_t s = (cudaStream_t)stream;
    k_energy_partials<<<blocks, AP_NOALLOC_THREADS, 0, s>>>(d_mu, d_field, m, scratch);
    k_energy_final<<<1, AP_NOALLOC_THREADS, 0, s>>>(scratch, blocks, -0.5 * AP_COULOMB, d_energy);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ap_fail(nullptr, AP_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return AP_OK;
}
