// Configuration loading: caller-order positions and local-frame multipoles -> sorted slots,
// global-frame multipoles (frame rotation, AMOEBA local frames: Z-then-X and bisector),
// and the assembly of the permanent field E = real + reciprocal + self.
#include "common.cuh"

#include <cmath>

namespace {

// FP64 division and sqrt are slow on this part: minimum image with 1/L, normalisation with rsqrt
__device__ __forceinline__ double mi(double v, double L, double iL) { return v - L * rint(v * iL); }

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <class C>
__device__ __forceinline__ void unit3(C *v) {
    const C in = rsq(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] *= in; v[1] *= in; v[2] *= in;
}

// columns of R are the local x, y, z axes in global coordinates; the minimum-image
// vectors to the frame atoms (kept in fv) in FP64, the axes in C
template <class C>
__device__ void frame_matrix(const double *__restrict__ xyz, int i, int type, int za, int xa, double3 L,
                             double3 iL, C R[3][3], double *fv) {
    for (int a = 0; a < 6; ++a) fv[a] = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) R[a][b] = (a == b) ? C(1) : C(0);
    if (type != AP_FRAME_Z_THEN_X && type != AP_FRAME_BISECTOR) return;
    const double Ls[3] = {L.x, L.y, L.z}, iLs[3] = {iL.x, iL.y, iL.z};
    C vz[3], vx[3], z[3], x[3];
    for (int a = 0; a < 3; ++a) {
        const double dz = mi(xyz[3 * za + a] - xyz[3 * i + a], Ls[a], iLs[a]);
        const double dx = mi(xyz[3 * xa + a] - xyz[3 * i + a], Ls[a], iLs[a]);
        fv[a] = dz;
        fv[3 + a] = dx;
        vz[a] = (C)dz;
        vx[a] = (C)dx;
    }
    if (type == AP_FRAME_Z_THEN_X) {
        for (int a = 0; a < 3; ++a) z[a] = vz[a];
        unit3(z);
        C d = vx[0] * z[0] + vx[1] * z[1] + vx[2] * z[2];
        for (int a = 0; a < 3; ++a) x[a] = vx[a] - d * z[a];
    } else {
        unit3(vz);
        unit3(vx);
        for (int a = 0; a < 3; ++a) z[a] = vz[a] + vx[a];
        unit3(z);
        C d = vx[0] * z[0] + vx[1] * z[1] + vx[2] * z[2];
        for (int a = 0; a < 3; ++a) x[a] = vx[a] - d * z[a];
    }
    unit3(x);
    C y[3] = {z[1] * x[2] - z[2] * x[1], z[2] * x[0] - z[0] * x[2], z[0] * x[1] - z[1] * x[0]};
    for (int a = 0; a < 3; ++a) {
        R[a][0] = x[a];
        R[a][1] = y[a];
        R[a][2] = z[a];
    }
}

template <class T>
__global__ void k_load(const double *__restrict__ xyz, const double *__restrict__ mpole,
                       const int *__restrict__ frame, const double *__restrict__ alpha,
                       const int *__restrict__ iperm, const float4 *__restrict__ bcenter, int n, double3 L, double3 iL,
                       typename V4<T>::type *__restrict__ posq, typename V4<T>::type *__restrict__ dipd,
                       typename V4<T>::type *__restrict__ quad0, typename V4<T>::type *__restrict__ quad1,
                       double *__restrict__ alpha_s, double *__restrict__ rot, double *__restrict__ mpl,
                       int *__restrict__ frame_s, double *__restrict__ fvec, int *__restrict__ bad, int3 K,
                       double3 sK, int4 *__restrict__ stb, typename V4<T>::type *__restrict__ stw) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = iperm[i];
    const float4 c = bcenter[s >> 5];
    double p[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    const double Ls[3] = {L.x, L.y, L.z}, iLs[3] = {iL.x, iL.y, iL.z};
    const double cc[3] = {c.x, c.y, c.z};
    for (int a = 0; a < 3; ++a) p[a] -= Ls[a] * rint((p[a] - cc[a]) * iLs[a]);   // image nearest the block
    int type = frame[3 * i];
    const int za = frame[3 * i + 1], xa = frame[3 * i + 2];
    bool frame_ok = true;
    if (type == AP_FRAME_Z_THEN_X || type == AP_FRAME_BISECTOR) {
        frame_ok = za >= 0 && za < n && xa >= 0 && xa < n && za != i && xa != i && za != xa;
    } else {
        frame_ok = type == AP_FRAME_NONE;
    }
    if (!frame_ok) type = AP_FRAME_NONE;   // never index with a bad frame atom; reported below
    // frames and rotations in the pair arithmetic's type (FP32 in the mixed and fixed modes:
    // FP64 is a small fraction of the FP32 rate on this part, and the rotated multipoles are
    // stored in that type anyway)
    typedef T C;
    C R[3][3];
    frame_matrix<C>(xyz, i, type, za, xa, L, iL, R, fvec + 6 * s);
    const double *m = mpole + 10 * i;
    const C dl[3] = {(C)m[1], (C)m[2], (C)m[3]};
    const C Ql[3][3] = {{(C)m[4], (C)m[5], (C)m[6]}, {(C)m[5], (C)m[7], (C)m[8]}, {(C)m[6], (C)m[8], (C)m[9]}};
    C dg[3], Qg[3][3], tmp[3][3];
    for (int a = 0; a < 3; ++a) dg[a] = R[a][0] * dl[0] + R[a][1] * dl[1] + R[a][2] * dl[2];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) tmp[a][b] = R[a][0] * Ql[0][b] + R[a][1] * Ql[1][b] + R[a][2] * Ql[2][b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Qg[a][b] = tmp[a][0] * R[b][0] + tmp[a][1] * R[b][1] + tmp[a][2] * R[b][2];
    const double al = alpha[i];
    bool ok = isfinite(p[0]) && isfinite(p[1]) && isfinite(p[2]) && isfinite(al) && al > 0.0;
    for (int k = 0; k < 10; ++k) ok = ok && isfinite(m[k]);
    if (!ok || !frame_ok) atomicExch(bad, 1);
    typedef typename V4<T>::type T4;
    T4 v;
    v.x = (T)(p[0] - cc[0]); v.y = (T)(p[1] - cc[1]); v.z = (T)(p[2] - cc[2]); v.w = (T)m[0];
    posq[s] = v;
    // smooth-PME stencil from the FP64 position: u = K x / L, origin floor(u) mod K, fraction
    {
        const int Ks[3] = {K.x, K.y, K.z};
        const double sk[3] = {sK.x, sK.y, sK.z};
        int ib[3];
        double w[3];
        for (int a = 0; a < 3; ++a) {
            const double u = p[a] * sk[a];
            const double b = floor(u);
            w[a] = u - b;
            long long k = (long long)b % Ks[a];
            if (k < 0) k += Ks[a];
            ib[a] = (k >= 0 && k < Ks[a]) ? (int)k : 0;
        }
        stb[s] = make_int4(ib[0], ib[1], ib[2], 0);
        v.x = (T)w[0]; v.y = (T)w[1]; v.z = (T)w[2]; v.w = (T)0;
        stw[s] = v;
    }
    v.x = (T)dg[0]; v.y = (T)dg[1]; v.z = (T)dg[2]; v.w = (T)(al > 0.0 ? rsqrt(al) : 1e4);
    dipd[s] = v;
    v.x = (T)Qg[0][0]; v.y = (T)Qg[0][1]; v.z = (T)Qg[0][2]; v.w = (T)Qg[1][1];
    quad0[s] = v;
    v.x = (T)Qg[1][2]; v.y = (T)Qg[2][2]; v.z = (T)al; v.w = (T)0;
    quad1[s] = v;
    alpha_s[s] = al;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) rot[9 * s + 3 * a + b] = R[a][b];
    for (int k = 0; k < 10; ++k) mpl[10 * s + k] = m[k];
    frame_s[3 * s] = type;
    frame_s[3 * s + 1] = (type != AP_FRAME_NONE && za >= 0) ? iperm[za] : -1;
    frame_s[3 * s + 2] = (type != AP_FRAME_NONE && xa >= 0) ? iperm[xa] : -1;
}

// padding slots: NaN positions make every pair test false; zero multipoles and alpha
template <class T>
__global__ void k_pad(int n, int n_pad, typename V4<T>::type *posq, typename V4<T>::type *dipd,
                      typename V4<T>::type *quad0, typename V4<T>::type *quad1, double *alpha_s, int *frame_s) {
    int s = n + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    typedef typename V4<T>::type T4;
    T nanv = (T)NAN;
    T4 z;
    z.x = z.y = z.z = z.w = (T)0;
    T4 pp = z;
    pp.x = pp.y = pp.z = nanv;
    posq[s] = pp;
    dipd[s] = z;
    quad0[s] = z;
    quad1[s] = z;
    alpha_s[s] = 0.0;
    frame_s[3 * s] = 0;
    frame_s[3 * s + 1] = -1;
    frame_s[3 * s + 2] = -1;
}

template <class T>
__global__ void k_field_finish(const double *__restrict__ acc, const T *__restrict__ rec,
                               const typename V4<T>::type *__restrict__ dipd, double self_coef, int n, int n_pad,
                               double *__restrict__ E, const int *__restrict__ iperm, double *__restrict__ out, int fixed) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_pad) return;
    if (s >= n) {
        for (int c = 0; c < 3; ++c) E[c * n_pad + s] = 0.0;
        return;
    }
    typename V4<T>::type d = dipd[s];
    double dd[3] = {(double)d.x, (double)d.y, (double)d.z};
    for (int c = 0; c < 3; ++c)
        E[c * n_pad + s] = acc_value(acc, (size_t)c * n_pad + s, fixed) + (double)rec[c * n_pad + s] + self_coef * dd[c];
}

__global__ void k_unsort3(const double *__restrict__ src, int n_pad, const int *__restrict__ iperm, int n,
                          double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = iperm[i];
    out[3 * i] = src[s];
    out[3 * i + 1] = src[n_pad + s];
    out[3 * i + 2] = src[2 * n_pad + s];
}

template <class T>
int load_t(ap_ctx *ctx, const double *d_xyz, const double *d_mpole, const int *d_frame, const double *d_alpha) {
    typedef typename V4<T>::type T4;
    const ap_params &P = ctx->prm;
    double3 L = make_double3(P.box[0], P.box[1], P.box[2]);
    double3 iL = make_double3(1.0 / P.box[0], 1.0 / P.box[1], 1.0 / P.box[2]);
    int *bad = (int *)ctx->red;   // scratch int at the start of the reduction buffer
    AP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->s0));
    k_load<T><<<ap_grid_for(ctx->n, 128), 128, 0, ctx->s0>>>(
        d_xyz, d_mpole, d_frame, d_alpha, ctx->iperm, ctx->bcenter, ctx->n, L, iL, (T4 *)ctx->posq, (T4 *)ctx->dipd,
        (T4 *)ctx->quad0, (T4 *)ctx->quad1, ctx->alpha, ctx->rot, ctx->mpl, ctx->frame_s, ctx->fvec, bad,
        make_int3(ctx->K[0], ctx->K[1], ctx->K[2]),
        make_double3(ctx->K[0] / P.box[0], ctx->K[1] / P.box[1], ctx->K[2] / P.box[2]), ctx->stb, (T4 *)ctx->stw);
    if (ctx->n_pad > ctx->n)
        k_pad<T><<<1, 32, 0, ctx->s0>>>(ctx->n, ctx->n_pad, (T4 *)ctx->posq, (T4 *)ctx->dipd, (T4 *)ctx->quad0,
                                        (T4 *)ctx->quad1, ctx->alpha, ctx->frame_s);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

template <class T>
int finish_t(ap_ctx *ctx, double *out) {
    typedef typename V4<T>::type T4;
    double self_coef = 4.0 * std::pow(ctx->prm.ewald_beta, 3) / (3.0 * AP_SQRT_PI);
    k_field_finish<T><<<ap_grid_for(ctx->n_pad, 256), 256, 0, ctx->s0>>>(
        ctx->acc, (const T *)ctx->rec, (const T4 *)ctx->dipd, self_coef, ctx->n, ctx->n_pad, ctx->E, ctx->iperm, out,
        ctx->fixed);
    if (out) k_unsort3<<<ap_grid_for(ctx->n, 256), 256, 0, ctx->s0>>>(ctx->E, ctx->n_pad, ctx->iperm, ctx->n, out);
    AP_CUDA(cudaGetLastError());
    return AP_OK;
}

}  // namespace

int cfg_load(ap_ctx *ctx, const double *d_xyz, const double *d_mpole, const int *d_frame, const double *d_alpha) {
    return ctx->prec == AP_FP64 ? load_t<double>(ctx, d_xyz, d_mpole, d_frame, d_alpha)
                                : load_t<float>(ctx, d_xyz, d_mpole, d_frame, d_alpha);
}

int field_finish(ap_ctx *ctx, double *d_field_out) {
    return ctx->prec == AP_FP64 ? finish_t<double>(ctx, d_field_out) : finish_t<float>(ctx, d_field_out);
}

void unsort3(ap_ctx *ctx, const double *src, double *out, cudaStream_t s) {
    k_unsort3<<<ap_grid_for(ctx->n, 256), 256, 0, s>>>(src, ctx->n_pad, ctx->iperm, ctx->n, out);
}
