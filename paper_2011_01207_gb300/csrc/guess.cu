// Trajectory extrapolation of the initial guess (classical predictor beside the learned
// guess): out = base + 2 (mu1 - base1) - (mu2 - base2), element by element.
#include "common.cuh"

namespace {

__global__ void k_extrapolate(long m, const double *__restrict__ base, const double *__restrict__ mu1,
                              const double *__restrict__ base1, const double *__restrict__ mu2,
                              const double *__restrict__ base2, double *__restrict__ out) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double b = base ? base[i] : 0.0, b1 = base1 ? base1[i] : 0.0, b2 = base2 ? base2[i] : 0.0;
    out[i] = b + 2.0 * (mu1[i] - b1) - (mu2[i] - b2);
}

}  // namespace

extern "C" int ap_extrapolate_guess(int n, const double *d_base, const double *d_mu1, const double *d_base1,
                                    const double *d_mu2, const double *d_base2, double *d_out, void *stream) {
    if (n < 1 || !d_mu1 || !d_mu2 || !d_out) return AP_ERR_ARG;
    const long m = 3L * n;
    k_extrapolate<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(m, d_base, d_mu1, d_base1, d_mu2,
                                                                                 d_base2, d_out);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}
