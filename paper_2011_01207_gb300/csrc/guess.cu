// Trajectory extrapolation of the initial guess (classical predictors beside the learned
// guess): out = base + 2 (mu1 - base1) - (mu2 - base2), element by element; and the
// adaptive form out = base + e1 + c (e1 - e2), e_k = mu_k - base_k, with c the
// least-squares fit of the previous step's change of e from the one before.
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

// adaptive extrapolation: c = (e1 - e2).(e2 - e3) / |e2 - e3|^2 (clamped to [0, 1]) from block
// partials over a grid-stride loop; the last block (ticket counter in the scratch) sums them
// in a fixed order and stores c in scratch[0]
constexpr int AD_BLOCKS = 256, AD_THREADS = 256;
static_assert(AD_BLOCKS <= AD_THREADS, "the last block loads one partial per thread");

__global__ void __launch_bounds__(AD_THREADS) k_adaptive_coef(long m, const double *__restrict__ mu1,
                                                              const double *__restrict__ b1,
                                                              const double *__restrict__ mu2,
                                                              const double *__restrict__ b2,
                                                              const double *__restrict__ mu3,
                                                              const double *__restrict__ b3,
                                                              double *__restrict__ scratch,
                                                              const int *__restrict__ count) {
    __shared__ double sa[AD_THREADS / 32], sb[AD_THREADS / 32];
    __shared__ bool last;
    double num = 0.0, den = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long)gridDim.x * blockDim.x) {
        const double e1 = mu1[i] - (b1 ? b1[i] : 0.0), e2 = mu2[i] - (b2 ? b2[i] : 0.0),
                     e3 = mu3[i] - (b3 ? b3[i] : 0.0);
        const double d12 = e1 - e2, d23 = e2 - e3;
        num += d12 * d23;
        den += d23 * d23;
    }
    for (int off = 16; off; off >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sa[w] = num; sb[w] = den; }
    __syncthreads();
    double *part = scratch + 2;   // [2][AD_BLOCKS]
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + 1);
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < AD_THREADS / 32; ++q) { a += sa[q]; b += sb[q]; }
        part[blockIdx.x] = a;
        part[AD_BLOCKS + blockIdx.x] = b;
        __threadfence();
        const unsigned int ticket = atomicAdd(counter, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // last block: thread k loads partial k (gridDim.x <= AD_THREADS), then the same fixed
    // warp-and-block tree as above, so the result does not depend on block order
    __threadfence();
    num = threadIdx.x < gridDim.x ? __ldcg(part + threadIdx.x) : 0.0;
    den = threadIdx.x < gridDim.x ? __ldcg(part + AD_BLOCKS + threadIdx.x) : 0.0;
    for (int off = 16; off; off >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, off);
        den += __shfl_xor_sync(0xffffffffu, den, off);
    }
    if (l == 0) { sa[w] = num; sb[w] = den; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int q = 0; q < AD_THREADS / 32; ++q) { a += sa[q]; b += sb[q]; }
    double c = b > 0.0 ? a / b : 0.0;
    c = isfinite(c) ? fmin(1.0, fmax(0.0, c)) : 0.0;
    if (count && *count < 3) c = 0.0;   // history too short: hold the last error
    scratch[0] = c;
    *counter = 0u;
}

// out = base + e1 + c (e1 - e2)
__global__ void k_adaptive_apply(long m, const double *__restrict__ base, const double *__restrict__ mu1,
                                 const double *__restrict__ b1, const double *__restrict__ mu2,
                                 const double *__restrict__ b2, const double *__restrict__ scratch,
                                 double *__restrict__ out, const int *__restrict__ count) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (count && *count == 0) {   // no history yet: the base guess alone
        out[i] = base ? base[i] : 0.0;
        return;
    }
    const double c = scratch[0];
    const double e1 = mu1[i] - (b1 ? b1[i] : 0.0), e2 = mu2[i] - (b2 ? b2[i] : 0.0);
    out[i] = (base ? base[i] : 0.0) + e1 + c * (e1 - e2);
}

// three-level history h = [mu1, mu2, mu3, g1, g2, g3] (m entries each): shift by one step
__global__ void k_hist_push3(long m, const double *__restrict__ g, const double *__restrict__ mu,
                             double *__restrict__ h, int *__restrict__ count) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) {
        h[2 * m + i] = h[m + i];
        h[m + i] = h[i];
        h[i] = mu[i];
        h[5 * m + i] = h[4 * m + i];
        h[4 * m + i] = h[3 * m + i];
        h[3 * m + i] = g[i];
    }
    if (i == 0) *count = min(*count + 1, 3);
}

// mu0 (caller order) = alpha E from the sorted slots
__global__ void k_direct_guess(const double *__restrict__ E, const double *__restrict__ alpha,
                               const int *__restrict__ iperm, int n, int n_pad, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = iperm[i];
    const double a = alpha[s];
    for (int c = 0; c < 3; ++c) out[3 * i + c] = a * E[(size_t)c * n_pad + s];
}

}  // namespace

// adaptive guess from the three-level history (layout of ap_batch_step.d_hist_lsq)
int hist_adaptive_launch(ap_ctx *ctx, const double *g, double *h, double *out, cudaStream_t s) {
    const long m = 3L * ctx->n;
    double *scratch = h + 7 * m;
    k_adaptive_coef<<<AD_BLOCKS, AD_THREADS, 0, s>>>(m, h, h + 3 * m, h + m, h + 4 * m, h + 2 * m, h + 5 * m, scratch,
                                                     ctx->hist_count);
    k_adaptive_apply<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, g, h, h + 3 * m, h + m, h + 4 * m, scratch, out,
                                                                 ctx->hist_count);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

int hist_push3_launch(ap_ctx *ctx, const double *g, const double *mu, double *h, cudaStream_t s) {
    const long m = 3L * ctx->n;
    k_hist_push3<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, g, mu, h, ctx->hist_count);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

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

extern "C" int ap_adaptive_guess(int n, const double *d_base, const double *d_mu1, const double *d_base1,
                                 const double *d_mu2, const double *d_base2, const double *d_mu3,
                                 const double *d_base3, double *d_out, double *d_scratch, void *stream) {
    if (n < 1 || !d_mu1 || !d_mu2 || !d_mu3 || !d_out || !d_scratch) return AP_ERR_ARG;
    const long m = 3L * n;
    cudaStream_t st = (cudaStream_t)stream;
    k_adaptive_coef<<<AD_BLOCKS, AD_THREADS, 0, st>>>(m, d_mu1, d_base1, d_mu2, d_base2, d_mu3, d_base3, d_scratch,
                                                      nullptr);
    k_adaptive_apply<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(m, d_base, d_mu1, d_base1, d_mu2, d_base2, d_scratch,
                                                                  d_out, nullptr);
    return cudaGetLastError() == cudaSuccess ? AP_OK : AP_ERR_CUDA;
}

extern "C" int ap_direct_guess(ap_ctx *ctx, double *d_mu0) {
    if (!ctx || !d_mu0) return AP_ERR_ARG;
    ctx->err.clear();
    if (!ctx->config_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field() must come first");
    k_direct_guess<<<ap_grid_for(ctx->n, 256), 256, 0, ctx->s0>>>(ctx->E, ctx->alpha, ctx->iperm, ctx->n, ctx->n_pad,
                                                                  d_mu0);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}
