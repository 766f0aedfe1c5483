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

// history h = [mu(t-1), mu(t-2), g(t-1), g(t-2)] of m entries each: out = g + 2 (mu1 - g1)
// - (mu2 - g2) once two steps are held, else g
__global__ void k_hist_guess(long m, const double *__restrict__ g, const double *__restrict__ h,
                             const int *__restrict__ count, double *__restrict__ out) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    out[i] = *count >= 2 ? g[i] + 2.0 * (h[i] - h[2 * m + i]) - (h[m + i] - h[3 * m + i]) : g[i];
}

// shift the history by one step: mu(t-2) <- mu(t-1) <- mu, g(t-2) <- g(t-1) <- g
__global__ void k_hist_push(long m, const double *__restrict__ g, const double *__restrict__ mu,
                            double *__restrict__ h, int *__restrict__ count) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        h[m + i] = h[i];
        h[i] = mu[i];
        h[3 * m + i] = h[2 * m + i];
        h[2 * m + i] = g[i];
    }
    if (i == 0) *count = min(*count + 1, 2);
}

}  // namespace

int hist_guess_launch(ap_ctx *ctx, const double *g, const double *h, double *out, cudaStream_t s) {
    const long m = 3L * ctx->n;
    k_hist_guess<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, g, h, ctx->hist_count, out);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

int hist_push_launch(ap_ctx *ctx, const double *g, const double *mu, double *h, cudaStream_t s) {
    const long m = 3L * ctx->n;
    k_hist_push<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, g, mu, h, ctx->hist_count);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

extern "C" int ap_extrapolate_guess(int n, const double *d_base, const double *d_mu1, const double *d_base1,
                                    const double *d_mu2, const double *d_base2, double *d_out, void *stream) {
    if (n < 1 || !d_mu1 || !d_mu2 || !d_out) return AP_ERR_ARG;
    const long m = 3L * n;
    k_extrapolate<<<(unsigned)((m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(m, d_base, d_mu1, d_base1, d_mu2,
                                                                                 d_base2, d_out);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}
