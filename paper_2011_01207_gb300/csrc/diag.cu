// Diagnostics: an FP32 issue-rate microbenchmark (the denominator of the pair kernels'
// roofline fraction) and an evaluation of the pair kernels' FP32 erfc beside CUDA's erfcf.
//
// FP32 peak: the pair kernels (permanent field, dipole matvec, forces) are bound by plain FP32 ALU work
// (no dense contraction, so no tensor cores). Their peak is the FP32 fused multiply-add rate
// of the device: SMs x FP32 lanes per SM x 2 flops x SM clock. Rather than assume the lane
// count and clock, this kernel measures it: every thread runs 8 independent FMA chains (enough
// in flight to cover the FMA latency with 8 warps per scheduler), the grid is a multiple of
// the SM count queried at run time, and CUDA events time the launches.
#include "common.cuh"
#include "pair_math.cuh"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_fma_peak(int iters, float a, float b, float *__restrict__ sink) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
    // every chain stays positive (x0 >= 0, a > 0, b > 0), so this never holds; it keeps the
    // chains live without a store per thread
    if (s < -1.0f) sink[0] = s;
}

// erfc(x) as the pair kernels form it (erfc_e2 with e^{-x^2} from the same fast exponential
// as the screened-function recursion) and CUDA's erfcf, for x >= 0
__global__ void k_erfc_pair(const float *__restrict__ x, int n, float *__restrict__ approx, float *__restrict__ lib) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    approx[i] = erfc_e2(v, ap_fexp(-v * v));
    lib[i] = erfcf(v);
}

}  // namespace

extern "C" int ap_eval_erfc(const float *d_x, int n, float *d_approx, float *d_lib, void *stream) {
    ap_ctx *ctx = nullptr;   // errors are reported through ap_last_error(NULL)
    if (!d_x || !d_approx || !d_lib || n < 1) return ap_fail(nullptr, AP_ERR_ARG, "null pointer or n < 1");
    k_erfc_pair<<<ap_grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(d_x, n, d_approx, d_lib);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

extern "C" int ap_fp32_peak(int reps, double *h_tflops, int *h_sm_count) {
    ap_ctx *ctx = nullptr;   // errors are reported through ap_last_error(NULL)
    if (!h_tflops || reps < 1) return ap_fail(nullptr, AP_ERR_ARG, "h_tflops is NULL or reps < 1");
    int dev = 0, sms = 0, per_sm = 0;
    AP_CUDA(cudaGetDevice(&dev));
    AP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak, PK_THREADS, 0));
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    const int iters = 2048;
    cudaStream_t s = nullptr;
    AP_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    AP_CUDA(cudaEventCreate(&e0));
    AP_CUDA(cudaEventCreate(&e1));
    // a = 1 - 2^-20, b = 2^-12: every chain stays positive and finite (it tends to b / (1 - a))
    const float a = 0.99999905f, b = 2.44140625e-4f;
    float *sink = nullptr;
    AP_CUDA(cudaMalloc((void **)&sink, sizeof(float)));
    k_fma_peak<<<grid, PK_THREADS, 0, s>>>(iters, a, b, sink);   // warm-up (clocks ramp)
    AP_CUDA(cudaGetLastError());
    double best = 1e30;
    for (int r = 0; r < reps; ++r) {
        AP_CUDA(cudaEventRecord(e0, s));
        k_fma_peak<<<grid, PK_THREADS, 0, s>>>(iters, a, b, sink);
        AP_CUDA(cudaEventRecord(e1, s));
        AP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        AP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms > 0.f && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    cudaFree(sink);
    const double flops = 2.0 * PK_CHAINS * 16.0 * iters * (double)grid * PK_THREADS;
    *h_tflops = flops / (best * 1e-3) / 1e12;
    if (h_sm_count) *h_sm_count = sms;
    return AP_OK;
}
