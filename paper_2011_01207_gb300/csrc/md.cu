// A minimal rigid-water integrator and its extra force term (row f3's trajectories).
//
// An MD step is one call of an integrator that moves positions and velocities from one time
// step to the next under the forces (paper Sec. 1.1); velocity Verlet is the paper's default
// (Sec. 2.5, 2.6) and its benchmarks step at 2 fs (Sec. 2.7). Here:
//   * ap_md_kick_drift / ap_md_kick: velocity Verlet in the kick-drift-kick form for rigid
//     three-site molecules, the three distances of each molecule held by SHAKE after the
//     drift and by RATTLE on the velocities after the second kick, optionally followed by a
//     uniform velocity scale (a Berendsen thermostat, which the paper lists among its
//     features, Sec. 2.6; 1 for constant energy); one thread per molecule, FP64 (a few
//     hundred flops per molecule and step);
//   * ap_lj_forces: a Lennard-Jones term, force-shifted at the real-space cutoff (energy and
//     force continuous there), over the current configuration's in-range pair bits (each
//     pair once) with the exclusions removed: one warp per work item, the j side through
//     shared memory, FP64 atomics. The polarization energy is attractive, so a liquid under
//     it alone collapses; this term supplies the repulsion of a van der Waals potential.
// Units: A, fs, amu, kcal/mol; 1 kcal/mol/A on 1 amu accelerates by 4.184e-4 A/fs^2.
#include "common.cuh"
#include "pair_math.cuh"

#include <cmath>

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s);

namespace {

constexpr double MD_ACC = 4.184e-4;
constexpr int MD_MAXIT = 1000;
constexpr double MD_TOL = 1e-12;

__device__ __forceinline__ double md_dot(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// (atom a, atom b, length index) of the three constraints, in the order the sweeps take them
__constant__ int c_pairs[3][3] = {{0, 1, 0}, {0, 2, 1}, {1, 2, 2}};

__global__ void k_md_kick_drift(int n_mol, const int *__restrict__ mol, double3 L2, const double *__restrict__ mass,
                                double dt, const double *__restrict__ f, double *__restrict__ x,
                                double *__restrict__ v, int *__restrict__ status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_mol) return;
    const double len2[3] = {L2.x, L2.y, L2.z};
    int at[3];
    double xo[3][3], xn[3][3], im[3];
    for (int a = 0; a < 3; ++a) {
        at[a] = mol[3 * k + a];
        im[a] = 1.0 / mass[at[a]];
        for (int c = 0; c < 3; ++c) {
            const double vh = v[3 * at[a] + c] + 0.5 * dt * MD_ACC * f[3 * at[a] + c] * im[a];
            xo[a][c] = x[3 * at[a] + c];
            xn[a][c] = xo[a][c] + dt * vh;
        }
    }
    bool ok = false;
    for (int it = 0; it < MD_MAXIT && !ok; ++it) {
        double worst = 0.0;
        for (int p = 0; p < 3; ++p) {
            const int a = c_pairs[p][0], b = c_pairs[p][1];
            const double d2 = len2[c_pairs[p][2]];
            double r[3], ro[3];
            for (int c = 0; c < 3; ++c) {
                r[c] = xn[a][c] - xn[b][c];
                ro[c] = xo[a][c] - xo[b][c];
            }
            const double diff = md_dot(r, r) - d2;
            worst = fmax(worst, fabs(diff) / d2);
            const double g = diff / (2.0 * (im[a] + im[b]) * md_dot(r, ro));
            for (int c = 0; c < 3; ++c) {
                xn[a][c] -= g * im[a] * ro[c];
                xn[b][c] += g * im[b] * ro[c];
            }
        }
        ok = worst < MD_TOL;
    }
    if (!ok && status) atomicOr(status, 1);
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            v[3 * at[a] + c] = (xn[a][c] - xo[a][c]) / dt;
            x[3 * at[a] + c] = xn[a][c];
        }
}

__global__ void k_md_kick(int n_mol, const int *__restrict__ mol, double3 L2, const double *__restrict__ mass,
                          double dt, const double *__restrict__ f, const double *__restrict__ x,
                          double *__restrict__ v, double lambda, double *__restrict__ kinetic,
                          int *__restrict__ status) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (k < n_mol) {
        const double len2[3] = {L2.x, L2.y, L2.z};
        int at[3];
        double xx[3][3], vv[3][3], im[3];
        for (int a = 0; a < 3; ++a) {
            at[a] = mol[3 * k + a];
            im[a] = 1.0 / mass[at[a]];
            for (int c = 0; c < 3; ++c) {
                xx[a][c] = x[3 * at[a] + c];
                vv[a][c] = v[3 * at[a] + c] + 0.5 * dt * MD_ACC * f[3 * at[a] + c] * im[a];
            }
        }
        bool ok = false;
        for (int it = 0; it < MD_MAXIT && !ok; ++it) {
            double worst = 0.0;
            for (int p = 0; p < 3; ++p) {
                const int a = c_pairs[p][0], b = c_pairs[p][1];
                const double d2 = len2[c_pairs[p][2]];
                double r[3], dv[3];
                for (int c = 0; c < 3; ++c) {
                    r[c] = xx[a][c] - xx[b][c];
                    dv[c] = vv[a][c] - vv[b][c];
                }
                const double rv = md_dot(r, dv);
                worst = fmax(worst, fabs(rv) / d2);
                const double g = rv / ((im[a] + im[b]) * d2);
                for (int c = 0; c < 3; ++c) {
                    vv[a][c] -= g * im[a] * r[c];
                    vv[b][c] += g * im[b] * r[c];
                }
            }
            ok = worst < MD_TOL;
        }
        if (!ok && status) atomicOr(status, 2);
        for (int a = 0; a < 3; ++a) {
            for (int c = 0; c < 3; ++c) {
                vv[a][c] *= lambda;                // a uniform scale keeps r . v_rel = 0
                v[3 * at[a] + c] = vv[a][c];
            }
            ke += 0.5 * md_dot(vv[a], vv[a]) / (im[a] * MD_ACC);
        }
    }
    if (kinetic) {
        __shared__ double sm[8];
        for (int off = 16; off; off >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, off);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = ke;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
            atomicAdd(kinetic, t);
        }
    }
}

// force-shifted Lennard-Jones pair: energy and F(r)/r (F = -dV/dr), both zero at rc
template <class T>
__device__ __forceinline__ void lj_fs(T r2, T eps, T sig, T rc, T &V, T &f_over_r) {
    const T r = sqrt(r2);
    const T s2 = sig * sig / r2, s6 = s2 * s2 * s2;
    const T c2 = sig * sig / (rc * rc), c6 = c2 * c2 * c2;
    const T Fc = T(24) * eps * (T(2) * c6 * c6 - c6) / rc;
    V = T(4) * eps * (s6 * s6 - s6) - T(4) * eps * (c6 * c6 - c6) + (r - rc) * Fc;
    f_over_r = (T(24) * eps * (T(2) * s6 * s6 - s6) / r - Fc) / r;
}

// one warp per work item (grid-stride): lane i of block I takes the pairs (i, j) of its row
// word (each in-range pair of the configuration appears in exactly one row word), minus its
// exclusion bits; j's position, parameters and slot come from shared memory. Forces into acc
// [3][n_pad] (slot order, FP64 atomics), energy into *energy.
template <class T, bool MINIMG>
__global__ void __launch_bounds__(128) k_lj_forces(WorkArgs wa, const typename V4<T>::type *__restrict__ posq,
                                                   const int *__restrict__ perm, const double *__restrict__ lj,
                                                   int n, int n_pad, T rc, T Lx, T Ly, T Lz,
                                                   double *__restrict__ acc, double *__restrict__ energy) {
    typedef typename V4<T>::type T4;
    __shared__ T4 sp[4][32];
    __shared__ T se[4][32], ss[4][32];
    __shared__ int sl[4][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long gw = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    const long nitems = *wa.n_work;
    const T4 *cpos = (const T4 *)wa.chunk_pos;
    double e_sum = 0.0;
    for (long t = gw; t < nitems; t += nw) {
        const int2 it = wa.work[t];
        const int si = it.x * 32 + lane;
        const bool vi = si < n;
        const T4 pi = posq[si];
        const T ei = vi ? (T)lj[2 * perm[si]] : T(0), sgi = vi ? (T)lj[2 * perm[si] + 1] : T(1);
        int sj;
        T4 pj;
        unsigned ex;
        if (it.y < 0) {
            sj = si;
            pj = pi;
            const int e = wa.tile_excl[wa.tile_off[it.x]];
            ex = e >= 0 ? wa.excl_mask[(size_t)e * 32 + lane] : 0u;
        } else {
            const size_t cs = (size_t)it.y * 32 + lane;
            sj = wa.chunk_j[cs];
            pj = cpos[cs];
            ex = wa.chunk_flag[it.y] ? wa.chunk_mask[cs] : 0u;
        }
        const bool vj = sj >= 0 && sj < n;
        __syncwarp();
        sp[w][lane] = pj;
        se[w][lane] = vj ? (T)lj[2 * perm[sj]] : T(0);
        ss[w][lane] = vj ? (T)lj[2 * perm[sj] + 1] : T(1);
        sl[w][lane] = vj ? sj : -1;
        __syncwarp();
        unsigned m = wa.pmask[(size_t)t * 32 + lane] & ~ex;
        double fi[3] = {0.0, 0.0, 0.0};
        while (m && vi && ei > T(0)) {
            const int j = __ffs(m) - 1;
            m &= m - 1u;
            const T ej = se[w][j];
            if (!(ej > T(0)) || sl[w][j] < 0) continue;
            const T4 q = sp[w][j];
            T dx = pi.x - q.x, dy = pi.y - q.y, dz = pi.z - q.z;
            if (MINIMG) {
                dx -= Lx * ap_rint(dx / Lx);
                dy -= Ly * ap_rint(dy / Ly);
                dz -= Lz * ap_rint(dz / Lz);
            }
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < rc * rc)) continue;
            // the pair function in FP64 (few pairs: oxygens only): the force-shifted terms of
            // close and far pairs cancel in the sum, which FP32 would resolve to ~1e-5 only
            const double ddx = dx, ddy = dy, ddz = dz;
            double V, fr;
            lj_fs<double>(ddx * ddx + ddy * ddy + ddz * ddz, sqrt((double)ei * (double)ej),
                          0.5 * ((double)sgi + (double)ss[w][j]), (double)rc, V, fr);
            e_sum += V;
            const double f3[3] = {fr * ddx, fr * ddy, fr * ddz};
            for (int c = 0; c < 3; ++c) {
                fi[c] += f3[c];
                atomicAdd(acc + (size_t)c * n_pad + sl[w][j], -f3[c]);
            }
        }
        if (vi)
            for (int c = 0; c < 3; ++c)
                if (fi[c] != 0.0) atomicAdd(acc + (size_t)c * n_pad + si, fi[c]);
    }
    for (int off = 16; off; off >>= 1) e_sum += __shfl_xor_sync(0xffffffffu, e_sum, off);
    if (lane == 0 && e_sum != 0.0) atomicAdd(energy, e_sum);
}

// out[i] (caller order) += acc[slot of i]
__global__ void k_add_unsort3(const double *__restrict__ acc, const int *__restrict__ iperm, int n, int n_pad,
                              double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = iperm[i];
    for (int c = 0; c < 3; ++c) out[3 * i + c] += acc[(size_t)c * n_pad + s];
}

template <class T>
int lj_t(ap_ctx *ctx, const double *d_lj, double *d_energy, double *d_forces) {
    typedef typename V4<T>::type T4;
    cudaStream_t s = ctx->s0;
    const ap_params &P = ctx->prm;
    double *acc = ctx->qv;   // scratch [3][n_pad] (the PCG's q vector, free between solves)
    AP_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * ctx->n_pad, s));
    AP_CUDA(cudaMemsetAsync(d_energy, 0, sizeof(double), s));
    auto kern = ctx->minimg ? k_lj_forces<T, true> : k_lj_forces<T, false>;
    kern<<<4 * ctx->sm_count, 128, 0, s>>>(work_args(ctx), (const T4 *)ctx->posq, ctx->perm, d_lj, ctx->n, ctx->n_pad,
                                          (T)P.cutoff, (T)P.box[0], (T)P.box[1], (T)P.box[2], acc, d_energy);
    AP_CUDA(cudaGetLastError());
    k_add_unsort3<<<ap_grid_for(ctx->n, 256), 256, 0, s>>>(acc, ctx->iperm, ctx->n, ctx->n_pad, d_forces);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

bool lengths_ok(const double *h) {
    for (int k = 0; k < 3; ++k)
        if (!(h[k] > 0.0) || !std::isfinite(h[k])) return false;
    return true;
}

}  // namespace

extern "C" int ap_lj_forces(ap_ctx *ctx, const double *d_lj, double *d_energy, double *d_forces) {
    if (!ctx) return AP_ERR_ARG;
    ctx->err.clear();
    if (!d_lj || !d_energy || !d_forces) return ap_fail(ctx, AP_ERR_ARG, "null pointer");
    if (!ctx->config_valid) return ap_fail(ctx, AP_ERR_STATE, "permanent_field() must come first");
    return ctx->prec == AP_FP64 ? lj_t<double>(ctx, d_lj, d_energy, d_forces)
                                : lj_t<float>(ctx, d_lj, d_energy, d_forces);
}

extern "C" int ap_md_kick_drift(int n_mol, const int *d_mol, const double *h_lengths, const double *d_mass,
                                double dt_fs, const double *d_forces, double *d_xyz, double *d_vel, int *d_status,
                                void *stream) {
    ap_ctx *ctx = nullptr;   // errors through ap_last_error(NULL)
    if (n_mol < 1 || !d_mol || !h_lengths || !d_mass || !d_forces || !d_xyz || !d_vel || !(dt_fs > 0.0))
        return ap_fail(nullptr, AP_ERR_ARG, "bad argument to ap_md_kick_drift");
    if (!lengths_ok(h_lengths)) return ap_fail(nullptr, AP_ERR_ARG, "constraint lengths must be positive");
    const double3 L2 = make_double3(h_lengths[0] * h_lengths[0], h_lengths[1] * h_lengths[1],
                                    h_lengths[2] * h_lengths[2]);
    k_md_kick_drift<<<ap_grid_for(n_mol, 128), 128, 0, (cudaStream_t)stream>>>(n_mol, d_mol, L2, d_mass, dt_fs,
                                                                              d_forces, d_xyz, d_vel, d_status);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

extern "C" int ap_md_kick(int n_mol, const int *d_mol, const double *h_lengths, const double *d_mass, double dt_fs,
                          const double *d_forces, const double *d_xyz, double *d_vel, double lambda,
                          double *d_kinetic, int *d_status, void *stream) {
    ap_ctx *ctx = nullptr;
    if (n_mol < 1 || !d_mol || !h_lengths || !d_mass || !d_forces || !d_xyz || !d_vel || !(dt_fs > 0.0))
        return ap_fail(nullptr, AP_ERR_ARG, "bad argument to ap_md_kick");
    if (!lengths_ok(h_lengths)) return ap_fail(nullptr, AP_ERR_ARG, "constraint lengths must be positive");
    if (!(lambda > 0.0) || !std::isfinite(lambda)) return ap_fail(nullptr, AP_ERR_ARG, "lambda must be positive");
    const double3 L2 = make_double3(h_lengths[0] * h_lengths[0], h_lengths[1] * h_lengths[1],
                                    h_lengths[2] * h_lengths[2]);
    cudaStream_t s = (cudaStream_t)stream;
    if (d_kinetic) AP_CUDA(cudaMemsetAsync(d_kinetic, 0, sizeof(double), s));
    k_md_kick<<<ap_grid_for(n_mol, 128), 128, 0, s>>>(n_mol, d_mol, L2, d_mass, dt_fs, d_forces, d_xyz, d_vel,
                                                     lambda, d_kinetic, d_status);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}
