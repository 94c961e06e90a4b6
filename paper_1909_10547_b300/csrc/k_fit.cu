// Gradient-descent support for the fit (fk_pdf_eval, fk_pdf_grad,
// fk_adam_step): the PDF parametrisation f = exp(t0 + t1 ln x + t2 ln(1 - x))
// evaluated on the master grid, its adjoint, and the Adam update.  The fit of
// the paper is gradient descent on the PDF parameters (Sec. 2); the chain
// dchi2/dtheta = (dchi2/dF)(dF/dtheta) closes it over the fit step's
// dchi2/dF.
#include "fk_internal.h"

#include <cmath>

namespace fk {
namespace {

// F[r][a][m] = exp(t0 + t1 ln x_m + t2 ln(1 - x_m)); one thread per value
template <typename T>
__global__ void k_pdf_eval(const T *__restrict__ theta, int R, const double *__restrict__ x, int nxg,
                           T *__restrict__ F) {
    const long long n = (long long)R * NFL * nxg;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e % nxg);
        const long long ra = e / nxg;  // r * 14 + a
        const T *t = theta + ra * 3;
        const T lx = (T)log(x[m]), l1x = (T)log1p(-x[m]);
        F[e] = exp(t[0] + t[1] * lx + t[2] * l1x);
    }
}

// gtheta[r][a][k] = sum_m gF * F * (1, ln x_m, ln(1 - x_m))[k]: one warp per
// (r, a), lanes over the grid, butterfly sums (a fixed order)
template <typename T>
__global__ void k_pdf_grad(const T *__restrict__ F, const T *__restrict__ gF, int R,
                           const double *__restrict__ x, int nxg, T *__restrict__ gtheta) {
    const long long ra = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ra >= (long long)R * NFL) return;
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int m = lane; m < nxg; m += 32) {
        const T w = gF[ra * nxg + m] * F[ra * nxg + m];
        s0 += w;
        s1 += w * (T)log(x[m]);
        s2 += w * (T)log1p(-x[m]);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) {
        gtheta[ra * 3 + 0] = s0;
        gtheta[ra * 3 + 1] = s1;
        gtheta[ra * 3 + 2] = s2;
    }
}

template <typename T>
__global__ void k_adam(T *__restrict__ p, const T *__restrict__ g, T *__restrict__ m, T *__restrict__ v,
                       long long n, T lr, T b1, T b2, T eps, T c1, T c2) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const T ge = g[e];
        const T me = b1 * m[e] + (T(1) - b1) * ge;
        const T ve = b2 * v[e] + (T(1) - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        p[e] -= lr * (me / c1) / (sqrt(ve / c2) + eps);
    }
}

unsigned blocks_for(long long n) {
    return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148LL * 16));
}

}  // namespace
}  // namespace fk

using namespace fk;

int fk_pdf_eval(const void *theta, int R, const double *x_grid, int nx_grid, void *F, int prec,
                fk_stream stream) {
    if (!theta || !x_grid || !F || R < 1 || nx_grid < 1 || nx_grid > MAX_NXG)
        return fail(FK_EINVAL, "fk_pdf_eval: bad arguments");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "fk_pdf_eval: unknown precision");
    const long long n = (long long)R * NFL * nx_grid;
    const cudaStream_t s = (cudaStream_t)stream;
    if (FK_IO64(prec))
        k_pdf_eval<double><<<blocks_for(n), 256, 0, s>>>((const double *)theta, R, x_grid, nx_grid, (double *)F);
    else
        k_pdf_eval<float><<<blocks_for(n), 256, 0, s>>>((const float *)theta, R, x_grid, nx_grid, (float *)F);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

int fk_pdf_grad(const void *F, const void *gF, int R, const double *x_grid, int nx_grid, void *gtheta,
                int prec, fk_stream stream) {
    if (!F || !gF || !x_grid || !gtheta || R < 1 || nx_grid < 1 || nx_grid > MAX_NXG)
        return fail(FK_EINVAL, "fk_pdf_grad: bad arguments");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "fk_pdf_grad: unknown precision");
    const long long warps = (long long)R * NFL;
    const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
    const cudaStream_t s = (cudaStream_t)stream;
    if (FK_IO64(prec))
        k_pdf_grad<double><<<blocks, 256, 0, s>>>((const double *)F, (const double *)gF, R, x_grid, nx_grid,
                                                  (double *)gtheta);
    else
        k_pdf_grad<float><<<blocks, 256, 0, s>>>((const float *)F, (const float *)gF, R, x_grid, nx_grid,
                                                 (float *)gtheta);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

int fk_adam_step(void *p, const void *g, void *m, void *v, long long n, int t, double lr, double b1,
                 double b2, double eps, int prec, fk_stream stream) {
    if (!p || !g || !m || !v || n < 0 || t < 1 || !(lr > 0) || !(b1 >= 0 && b1 < 1) || !(b2 >= 0 && b2 < 1) ||
        !(eps > 0))
        return fail(FK_EINVAL, "fk_adam_step: bad arguments");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "fk_adam_step: unknown precision");
    if (n == 0) return FK_OK;
    const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
    const cudaStream_t s = (cudaStream_t)stream;
    if (FK_IO64(prec))
        k_adam<double><<<blocks_for(n), 256, 0, s>>>((double *)p, (const double *)g, (double *)m, (double *)v, n, lr,
                                                     b1, b2, eps, c1, c2);
    else
        k_adam<float><<<blocks_for(n), 256, 0, s>>>((float *)p, (const float *)g, (float *)m, (float *)v, n,
                                                    (float)lr, (float)b1, (float)b2, (float)eps, (float)c1,
                                                    (float)c2);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}
