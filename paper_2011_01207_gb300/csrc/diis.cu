// f3 - Jacobi iteration with DIIS extrapolation, the other iterative solver of the same
// polarization system (paper Sec. 1.3: the induced dipoles solve A mu = E with
// A = alpha^-1 - T; the Tinker-HP solvers it builds on offer Jacobi/DIIS beside PCG).
//
//   x_0 = guess (default alpha E)
//   step k:  y_k = alpha (E + T x_k)         (the Jacobi map of the splitting alpha^-1 - T)
//            e_k = y_k - x_k = alpha r_k     (so eps is the PCG's Debye RMS of alpha r)
//            stop if eps_k <= tol, returning x_k
//            B_ij = e_i . e_j over the last `depth` steps; c minimises |sum c_i e_i| with
//            sum c_i = 1 (Pulay's bordered normal equations)
//            x_{k+1} = sum_i c_i y_i
//
// One T application per step (the same real-space and PME kernels as the PCG, on p = x_k in
// the pair/PME precision). The step kernel forms y and e in FP64 into rings of `depth`
// vectors and reduces e_k against every error in the window; its last block finishes the
// dots in a fixed order, updates B, tests convergence and solves the bordered system on one
// thread. The combine kernel forms x_{k+1}. The loop is a conditional WHILE node, as for
// the PCG, never run beyond max_iter + 1 times.
#include "common.cuh"

#include <cmath>
#include <cstdlib>

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s);
int dipole_operator_into(ap_ctx *ctx, cudaStream_t main, cudaStream_t aux);

struct DiisState {
    double B[AP_DIIS_MAX_DEPTH * AP_DIIS_MAX_DEPTH];   // e_i . e_j by ring position
    double c[AP_DIIS_MAX_DEPTH];                 // extrapolation coefficients by ring position
    double tol, eps, eps0;
    int iter;          // extrapolated updates taken
    int max_iter;
    int depth;         // window length
    int count;         // steps held in the rings (<= depth)
    int head;          // ring position of the next step
    int guard;         // loop-body executions (bounds the WHILE node)
    int done, status, nonfinite, window;   // window: entries the last solve used
    unsigned int blocks_done;
};

namespace {

constexpr int NT = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// x_0 (caller-order guess gathered into slots, or alpha E) into mu (FP64) and p (T4)
template <class T>
__global__ void k_diis_guess(const double *__restrict__ guess, const double *__restrict__ E,
                             const double *__restrict__ alpha, const int *__restrict__ perm, int n, int n_pad,
                             double *__restrict__ mu, typename V4<T>::type *__restrict__ p) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    double m[3] = {0.0, 0.0, 0.0};
    if (s < n) {
        if (guess) {
            const int i = perm[s];
            for (int c = 0; c < 3; ++c) m[c] = guess[3 * i + c];
        } else {
            for (int c = 0; c < 3; ++c) m[c] = alpha[s] * E[c * n_pad + s];
        }
    }
    for (int c = 0; c < 3; ++c) mu[c * n_pad + s] = m[c];
    typename V4<T>::type v;
    v.x = (T)m[0]; v.y = (T)m[1]; v.z = (T)m[2]; v.w = (T)0;
    p[s] = v;
}

__global__ void k_diis_init(DiisState *st, double tol, int max_iter, int depth) {
    if (threadIdx.x != 0) return;
    for (int k = 0; k < AP_DIIS_MAX_DEPTH * AP_DIIS_MAX_DEPTH; ++k) st->B[k] = 0.0;
    for (int k = 0; k < AP_DIIS_MAX_DEPTH; ++k) st->c[k] = 0.0;
    st->tol = tol;
    st->eps = st->eps0 = 0.0;
    st->iter = 0;
    st->max_iter = max_iter;
    st->depth = depth;
    st->count = 0;
    st->head = 0;
    st->guard = 0;
    st->done = 0;
    st->status = AP_OK;
    st->nonfinite = 0;
    st->window = 0;
    st->blocks_done = 0u;
}

__global__ void k_diis_set_cond(cudaGraphConditionalHandle h, const DiisState *st) {
    cudaGraphSetConditional(h, st->done ? 0u : 1u);
}

// Solves the bordered system over the `w` newest ring entries (ages 0..w-1, age 0 at ring
// position j), with B scaled by its largest diagonal entry (c does not change):
//   [ B  -1 ] [c     ]   [ 0 ]
//   [ -1  0 ] [lambda] = [-1 ]
// Gaussian elimination with partial pivoting. Returns false on a zero pivot or a
// non-finite coefficient.
__device__ bool bordered_solve(const DiisState *st, int j, int w, double *c) {
    constexpr int M = AP_DIIS_MAX_DEPTH + 1;
    double a[M][M + 1];
    int pos[AP_DIIS_MAX_DEPTH];
    const int depth = st->depth;
    for (int t = 0; t < w; ++t) pos[t] = (j - t + depth) % depth;
    double scale = 0.0;
    for (int t = 0; t < w; ++t) scale = fmax(scale, st->B[pos[t] * AP_DIIS_MAX_DEPTH + pos[t]]);
    if (!(scale > 0.0)) return false;
    const double inv = 1.0 / scale;
    const int m = w + 1;
    for (int r = 0; r < w; ++r) {
        for (int q = 0; q < w; ++q) a[r][q] = st->B[pos[r] * AP_DIIS_MAX_DEPTH + pos[q]] * inv;
        a[r][w] = -1.0;
        a[r][m] = 0.0;
    }
    for (int q = 0; q < w; ++q) a[w][q] = -1.0;
    a[w][w] = 0.0;
    a[w][m] = -1.0;
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return false;
        if (piv != col)
            for (int q = col; q <= m; ++q) {
                const double t = a[col][q];
                a[col][q] = a[piv][q];
                a[piv][q] = t;
            }
        for (int r = col + 1; r < m; ++r) {
            const double f = a[r][col] / a[col][col];
            for (int q = col; q <= m; ++q) a[r][q] -= f * a[col][q];
        }
    }
    double sol[M];
    for (int r = m - 1; r >= 0; --r) {
        double v = a[r][m];
        for (int q = r + 1; q < m; ++q) v -= a[r][q] * sol[q];
        sol[r] = v / a[r][r];
    }
    for (int k = 0; k < AP_DIIS_MAX_DEPTH; ++k) c[k] = 0.0;
    for (int t = 0; t < w; ++t) {
        if (!isfinite(sol[t])) return false;
        c[pos[t]] = sol[t];
    }
    return true;
}

// y = alpha (E + T x), e = y - x into ring position j; partial e . e_i for the window; clears
// acc for the next operator application. The last block finishes the iteration.
template <class T>
__global__ void __launch_bounds__(NT) k_diis_step(const double *__restrict__ x, double *__restrict__ acc,
                                                  const T *__restrict__ rec, const double *__restrict__ E,
                                                  const double *__restrict__ alpha, double self_coef, int n_pad,
                                                  int n, double *__restrict__ ys, double *__restrict__ es,
                                                  double *__restrict__ part, DiisState *st,
                                                  cudaGraphConditionalHandle h, int use_cond, int fixed) {
    __shared__ double sred[NT / 32][AP_DIIS_MAX_DEPTH];
    __shared__ bool last;
    const int j = st->head;
    const int m = min(st->count + 1, st->depth);   // window including this step
    const size_t stride = (size_t)3 * n_pad;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double dots[AP_DIIS_MAX_DEPTH];
#pragma unroll
    for (int i = 0; i < AP_DIIS_MAX_DEPTH; ++i) dots[i] = 0.0;
    if (s < n_pad) {
        const double a = alpha[s];
        for (int c = 0; c < 3; ++c) {
            const int k = c * n_pad + s;
            const double xv = x[k];
            const double y = a * (E[k] + acc_value(acc, k, fixed) + (double)rec[k] + self_coef * xv);
            const double e = y - xv;
            acc[k] = 0.0;
            ys[j * stride + k] = y;
            es[j * stride + k] = e;
#pragma unroll
            for (int i = 0; i < AP_DIIS_MAX_DEPTH; ++i)
                if (i < m) dots[i] += e * (i == j ? e : es[i * stride + k]);
        }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < AP_DIIS_MAX_DEPTH; ++i) {
        if (i < m) {
            const double v = warp_sum(dots[i]);
            if (l == 0) sred[w][i] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double v = 0.0;
        for (int q = 0; q < NT / 32; ++q) v += sred[q][threadIdx.x];
        part[threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicAdd(&st->blocks_done, 1u);
        last = ticket == gridDim.x - 1;
        if (last) st->blocks_done = 0u;
    }
    __syncthreads();
    if (!last) return;
    // fixed-order sums of the partials: warp i sums dot i
    __shared__ double tot[AP_DIIS_MAX_DEPTH];
    for (int i = w; i < m; i += NT / 32) {
        double v = 0.0;
        for (int b = l; b < (int)gridDim.x; b += 32) v += __ldcg(part + i * gridDim.x + b);
        v = warp_sum(v);
        if (l == 0) tot[i] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double eps = AP_DEBYE * sqrt(tot[j] / n);
    if (st->guard == 0) st->eps0 = eps;
    st->guard += 1;
    st->eps = eps;
    st->count = m;
    st->head = (j + 1) % st->depth;
    for (int i = 0; i < m; ++i) {
        st->B[j * AP_DIIS_MAX_DEPTH + i] = tot[i];
        st->B[i * AP_DIIS_MAX_DEPTH + j] = tot[i];
    }
    if (!isfinite(eps)) {
        st->nonfinite = 1;
        st->done = 1;
        st->status = AP_ERR_NONFINITE;
    } else if (eps <= st->tol) {
        st->done = 1;
        st->status = AP_OK;
    } else if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = AP_NOT_CONVERGED;
    } else {
        // the newest entries whose bordered system is regular (one entry always is: c = 1)
        double c[AP_DIIS_MAX_DEPTH];
        int wn = m;
        while (wn > 1 && !bordered_solve(st, j, wn, c)) --wn;
        if (wn == 1) {
            for (int k = 0; k < AP_DIIS_MAX_DEPTH; ++k) c[k] = 0.0;
            c[j] = 1.0;
        }
        for (int k = 0; k < AP_DIIS_MAX_DEPTH; ++k) st->c[k] = c[k];
        st->window = wn;
        st->iter += 1;
    }
    if (use_cond) cudaGraphSetConditional(h, (!st->done && st->guard <= st->max_iter) ? 1u : 0u);
}

// x_{k+1} = sum_i c_i y_i into mu (FP64) and p (T4); nothing once the solve is done
template <class T>
__global__ void k_diis_combine(const double *__restrict__ ys, const DiisState *__restrict__ st, int n_pad,
                               double *__restrict__ mu, typename V4<T>::type *__restrict__ p) {
    if (st->done) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    const int m = st->count;
    const size_t stride = (size_t)3 * n_pad;
    double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < AP_DIIS_MAX_DEPTH; ++i) {
        if (i < m) {
            const double ci = st->c[i];
            if (ci != 0.0)
                for (int c = 0; c < 3; ++c) v[c] += ci * ys[i * stride + c * n_pad + s];
        }
    }
    for (int c = 0; c < 3; ++c) mu[c * n_pad + s] = v[c];
    typename V4<T>::type q;
    q.x = (T)v[0]; q.y = (T)v[1]; q.z = (T)v[2]; q.w = (T)0;
    p[s] = q;
}

double diis_self_coef(const ap_ctx *ctx) {
    return 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI);
}

template <class T>
int enqueue_step(ap_ctx *ctx, cudaGraphConditionalHandle h, int use_cond, cudaStream_t main, cudaStream_t aux) {
    typedef typename V4<T>::type T4;
    const int nb = ap_grid_for(ctx->n_pad, NT);
    int rc = dipole_operator_into(ctx, main, aux);
    if (rc) return rc;
    k_diis_step<T><<<nb, NT, 0, main>>>(ctx->mu, ctx->acc, (const T *)ctx->rec, ctx->E, ctx->alpha,
                                         diis_self_coef(ctx), ctx->n_pad, ctx->n, ctx->diis_y, ctx->diis_e,
                                         ctx->diis_part, (DiisState *)ctx->diis_st, h, use_cond, ctx->fixed);
    k_diis_combine<T><<<nb, NT, 0, main>>>(ctx->diis_y, (const DiisState *)ctx->diis_st, ctx->n_pad, ctx->mu,
                                            (T4 *)ctx->p);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

// [set condition] -> WHILE { T x; step; combine }; the window length is read from the state,
// so one graph serves every depth the rings hold
template <class T>
int build_diis_graph(ap_ctx *ctx) {
    cudaGraph_t g = nullptr;
    AP_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 0, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return AP_OK;
    }
    cudaKernelNodeParams kp = {};
    const DiisState *stp = (const DiisState *)ctx->diis_st;
    void *args[2] = {(void *)&h, (void *)&stp};
    kp.func = (void *)k_diis_set_cond;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    cudaGraphNode_t n_set, n_while;
    AP_CUDA(cudaGraphAddKernelNode(&n_set, g, nullptr, 0, &kp));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    AP_CUDA(cudaGraphAddNode(&n_while, g, &n_set, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = nullptr;
    AP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    AP_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step<T>(ctx, h, 1, cs, ctx->s1);
    cudaGraph_t captured = nullptr;
    cudaError_t ec = cudaStreamEndCapture(cs, &captured);
    cudaStreamDestroy(cs);
    if (rc || ec != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        ctx->err.clear();
        return AP_OK;   // the host loop
    }
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        return AP_OK;
    }
    cudaGraphDestroy(g);
    ctx->diis_exec = ex;
    return AP_OK;
}

// rings for `depth` steps, partial sums and state; drops a graph made for smaller rings
int diis_reserve(ap_ctx *ctx, int depth) {
    if (!ctx->diis_st || !ctx->diis_st_host || !ctx->diis_part) {
        // state, its pinned mirror and the partial sums together, or none
        const int nb = ap_grid_for(ctx->n_pad, NT);
        cudaError_t e = cudaSuccess;
        if (!ctx->diis_st) e = cudaMalloc(&ctx->diis_st, sizeof(DiisState));
        if (e == cudaSuccess && !ctx->diis_st_host) e = cudaMallocHost(&ctx->diis_st_host, sizeof(DiisState));
        if (e == cudaSuccess && !ctx->diis_part)
            e = cudaMalloc((void **)&ctx->diis_part, sizeof(double) * AP_DIIS_MAX_DEPTH * nb);
        if (e != cudaSuccess) {
            if (ctx->diis_st) cudaFree(ctx->diis_st);
            if (ctx->diis_st_host) cudaFreeHost(ctx->diis_st_host);
            if (ctx->diis_part) cudaFree(ctx->diis_part);
            ctx->diis_st = ctx->diis_st_host = nullptr;
            ctx->diis_part = nullptr;
            return ap_fail(ctx, AP_ERR_CUDA, std::string("DIIS state allocation: ") + cudaGetErrorString(e));
        }
    }
    if (depth > ctx->diis_cap) {
        if (ctx->diis_exec) cudaGraphExecDestroy(ctx->diis_exec);
        ctx->diis_exec = nullptr;
        if (ctx->diis_y) cudaFree(ctx->diis_y);
        if (ctx->diis_e) cudaFree(ctx->diis_e);
        ctx->diis_y = ctx->diis_e = nullptr;
        ctx->diis_cap = 0;
        const size_t bytes = sizeof(double) * 3 * (size_t)ctx->n_pad * depth;
        cudaError_t e = cudaMalloc((void **)&ctx->diis_y, bytes);
        if (e == cudaSuccess) e = cudaMalloc((void **)&ctx->diis_e, bytes);
        if (e != cudaSuccess) {
            if (ctx->diis_y) cudaFree(ctx->diis_y);
            ctx->diis_y = nullptr;
            ctx->diis_e = nullptr;
            return ap_fail(ctx, AP_ERR_CUDA, std::string("DIIS ring allocation: ") + cudaGetErrorString(e));
        }
        ctx->diis_cap = depth;
    }
    return AP_OK;
}

template <class T>
int diis_t(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, int depth, double *d_mu,
           ap_solve_info *info) {
    typedef typename V4<T>::type T4;
    cudaStream_t s = ctx->s0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    AP_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return ap_fail(ctx, AP_ERR_ARG, "induced_dipoles_diis cannot be captured into a graph");
    int rc = diis_reserve(ctx, depth);
    if (rc) return rc;
    const int nb = ap_grid_for(ctx->n_pad, NT);
    DiisState *st = (DiisState *)ctx->diis_st;
    k_diis_init<<<1, 32, 0, s>>>(st, tol, max_iter, depth);
    AP_CUDA(cudaMemsetAsync(ctx->acc, 0, sizeof(double) * 3 * ctx->n_pad, s));
    k_diis_guess<T><<<nb, NT, 0, s>>>(d_guess, ctx->E, ctx->alpha, ctx->perm, ctx->n, ctx->n_pad, ctx->mu,
                                       (T4 *)ctx->p);
    AP_CUDA(cudaGetLastError());
    const char *env = getenv("AP_SOLVE_GRAPH");
    const bool graphs = !(env && env[0] == '0');
    if (graphs && ctx->diis_exec == nullptr) {
        rc = build_diis_graph<T>(ctx);
        if (rc) return rc;
    }
    DiisState *hs = (DiisState *)ctx->diis_st_host;
    if (graphs && ctx->diis_exec) {
        AP_CUDA(cudaGraphLaunch(ctx->diis_exec, s));
    } else {
        for (int it = 0; it <= max_iter; ++it) {
            rc = enqueue_step<T>(ctx, 0, 0, ctx->s0, ctx->s1);
            if (rc) return rc;
            AP_CUDA(cudaMemcpyAsync(hs, st, sizeof(DiisState), cudaMemcpyDeviceToHost, s));
            AP_CUDA(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
    }
    unsort3(ctx, ctx->mu, d_mu, s);
    AP_CUDA(cudaGetLastError());
    if (info) return diis_info(ctx, info);
    return AP_OK;
}

}  // namespace

int diis_info(ap_ctx *ctx, ap_solve_info *info) {
    if (!ctx->diis_st) return ap_fail(ctx, AP_ERR_STATE, "no DIIS solve on this context");
    DiisState *hs = (DiisState *)ctx->diis_st_host;
    AP_CUDA(cudaMemcpyAsync(hs, ctx->diis_st, sizeof(DiisState), cudaMemcpyDeviceToHost, ctx->s0));
    AP_CUDA(cudaStreamSynchronize(ctx->s0));
    info->iterations = hs->iter;
    info->eps_debye = hs->eps;
    info->eps_initial = hs->eps0;
    info->status = hs->status;
    if (hs->nonfinite) return ap_fail(ctx, AP_ERR_NONFINITE, "non-finite value in the DIIS reductions");
    return hs->status;
}

int diis_solve(ap_ctx *ctx, const double *d_guess, double tol, int max_iter, int depth, double *d_mu,
               ap_solve_info *info) {
    return ctx->prec == AP_FP64 ? diis_t<double>(ctx, d_guess, tol, max_iter, depth, d_mu, info)
                                : diis_t<float>(ctx, d_guess, tol, max_iter, depth, d_mu, info);
}

void diis_release(ap_ctx *ctx) {
    if (ctx->diis_exec) cudaGraphExecDestroy(ctx->diis_exec);
    if (ctx->diis_st) cudaFree(ctx->diis_st);
    if (ctx->diis_st_host) cudaFreeHost(ctx->diis_st_host);
    if (ctx->diis_part) cudaFree(ctx->diis_part);
    if (ctx->diis_y) cudaFree(ctx->diis_y);
    if (ctx->diis_e) cudaFree(ctx->diis_e);
}
