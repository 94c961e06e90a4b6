/*
 * FP64 CPU oracle for the FK-table convolution (arXiv:1909.10547, Sec. 3).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow definition of what the
 * CUDA library computes.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it; the library itself never does, and the two
 * share no code, headers or constants.
 *
 * Every sum is written in the order of its definition (data point, channel,
 * x_i, x_j), in double precision, with Neumaier-compensated accumulation of the
 * terms so that the oracle's own rounding error stays near one unit in the last
 * place of the result.  Each entry point cites the passage it follows.
 *
 * Layouts (row-major, C order):
 *   DIS table      fk[ndata][14][nx]           (dense over all 14 flavours)
 *   hadronic table fk[ndata][nc][nx][nx]       channel c = (ca[c], cb[c])
 *   PDF replicas   F[R][14][nxg]               xmap[i] in [0, nxg) is the PDF
 *                                              grid point of the table's x_i
 *   observables    O[R][ndata]
 *
 * All entry points return 0 on success and a negative value on bad arguments.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define NFL 14

/* Neumaier's improvement of Kahan summation. */
typedef struct { double s, c; } acc_t;

static inline void acc_add(acc_t *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static inline double acc_get(const acc_t *a) { return a->s + a->c; }

static inline int xidx(const int *xmap, int i) { return xmap ? xmap[i] : i; }

static int check_xmap(const int *xmap, int nx, int nxg)
{
    if (!xmap) return nx <= nxg ? 0 : -1;
    for (int i = 0; i < nx; ++i)
        if (xmap[i] < 0 || xmap[i] >= nxg) return -1;
    return 0;
}

/*
 * DIS observable (named in Table 1 of the paper; the linear analogue of Eq. 1):
 *   O[r][d] = sum_a sum_i FK[d][a][i] * f_a(x_i)   for replica r.
 * S[r][d] (optional) = sum of |term|, the scale that the tolerance of the GPU
 * comparison is relative to.
 */
int fk_oracle_dis(int ndata, int nx, const double *fk, const int *xmap, int nxg,
                  int R, const double *F, double *O, double *S)
{
    if (ndata < 0 || nx < 0 || R < 0 || check_xmap(xmap, nx, nxg)) return -1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int r = 0; r < R; ++r)
        for (int d = 0; d < ndata; ++d) {
            const double *f = F + (size_t)r * NFL * nxg;
            acc_t o = {0, 0}, s = {0, 0};
            for (int a = 0; a < NFL; ++a)
                for (int i = 0; i < nx; ++i) {
                    double term = fk[((size_t)d * NFL + a) * nx + i] * f[a * nxg + xidx(xmap, i)];
                    acc_add(&o, term);
                    acc_add(&s, fabs(term));
                }
            O[(size_t)r * ndata + d] = acc_get(&o);
            if (S) S[(size_t)r * ndata + d] = acc_get(&s);
        }
    return 0;
}

/*
 * Hadronic observable, Eq. 1 of the paper written per active channel:
 *   O[r][d] = sum_c sum_i sum_j f_{ca[c]}(x_i) f_{cb[c]}(x_j) FK[d][c][i][j].
 * Each term is formed as FK * f_a * f_b and accumulated in (c, i, j) order.
 */
int fk_oracle_had(int ndata, int nc, const int *ca, const int *cb, int nx,
                  const double *fk, const int *xmap, int nxg, int R,
                  const double *F, double *O, double *S)
{
    if (ndata < 0 || nc < 0 || nx < 0 || R < 0 || check_xmap(xmap, nx, nxg)) return -1;
    for (int c = 0; c < nc; ++c)
        if (ca[c] < 0 || ca[c] >= NFL || cb[c] < 0 || cb[c] >= NFL) return -1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int r = 0; r < R; ++r)
        for (int d = 0; d < ndata; ++d) {
            const double *f = F + (size_t)r * NFL * nxg;
            acc_t o = {0, 0}, s = {0, 0};
            for (int c = 0; c < nc; ++c) {
                const double *fa = f + ca[c] * nxg;
                const double *fb = f + cb[c] * nxg;
                const double *blk = fk + ((size_t)d * nc + c) * nx * nx;
                for (int i = 0; i < nx; ++i)
                    for (int j = 0; j < nx; ++j) {
                        double term = blk[(size_t)i * nx + j] * fa[xidx(xmap, i)] * fb[xidx(xmap, j)];
                        acc_add(&o, term);
                        acc_add(&s, fabs(term));
                    }
            }
            O[(size_t)r * ndata + d] = acc_get(&o);
            if (S) S[(size_t)r * ndata + d] = acc_get(&s);
        }
    return 0;
}

/*
 * Gradient of the DIS observables contracted with gO (the custom operator's
 * gradient, Sec. 3 and Table 1 of the paper):
 *   gF[r][a][xmap[i]] = sum_d gO[r][d] * dO[r][d]/df_a(x_i) = sum_d gO[r][d] FK[d][a][i].
 * gF is overwritten; PDF grid points the table does not use get 0.
 */
int fk_oracle_dis_grad(int ndata, int nx, const double *fk, const int *xmap, int nxg,
                       int R, const double *gO, double *gF)
{
    if (ndata < 0 || nx < 0 || R < 0 || check_xmap(xmap, nx, nxg)) return -1;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r) {
        double *g = gF + (size_t)r * NFL * nxg;
        memset(g, 0, sizeof(double) * NFL * nxg);
        for (int a = 0; a < NFL; ++a)
            for (int i = 0; i < nx; ++i) {
                acc_t s = {0, 0};
                for (int d = 0; d < ndata; ++d)
                    acc_add(&s, gO[(size_t)r * ndata + d] * fk[((size_t)d * NFL + a) * nx + i]);
                g[a * nxg + xidx(xmap, i)] += acc_get(&s);
            }
    }
    return 0;
}

/*
 * Gradient of the hadronic observables contracted with gO.  Each term of Eq. 1,
 * FK[d][c][i][j] f_a(x_i) f_b(x_j), is differentiated by the product rule:
 *   d/df_a(x_i) gives FK * f_b(x_j),   d/df_b(x_j) gives FK * f_a(x_i),
 * so a diagonal channel (a == b) receives both parts.  Every partial derivative
 * is weighted by gO[r][d] and summed into gF[r][flavour][grid point], which is
 * overwritten.
 */
int fk_oracle_had_grad(int ndata, int nc, const int *ca, const int *cb, int nx,
                       const double *fk, const int *xmap, int nxg, int R,
                       const double *F, const double *gO, double *gF)
{
    if (ndata < 0 || nc < 0 || nx < 0 || R < 0 || check_xmap(xmap, nx, nxg)) return -1;
    for (int c = 0; c < nc; ++c)
        if (ca[c] < 0 || ca[c] >= NFL || cb[c] < 0 || cb[c] >= NFL) return -1;
    const size_t ng = (size_t)NFL * nxg;
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < R; ++r) {
        const double *f = F + (size_t)r * ng;
        acc_t *g = (acc_t *)calloc(ng, sizeof(acc_t));
        for (int d = 0; d < ndata; ++d) {
            double w = gO[(size_t)r * ndata + d];
            for (int c = 0; c < nc; ++c) {
                const double *blk = fk + ((size_t)d * nc + c) * nx * nx;
                for (int i = 0; i < nx; ++i) {
                    int xi = xidx(xmap, i);
                    for (int j = 0; j < nx; ++j) {
                        int xj = xidx(xmap, j);
                        double k = blk[(size_t)i * nx + j];
                        acc_add(&g[ca[c] * nxg + xi], w * k * f[cb[c] * nxg + xj]);
                        acc_add(&g[cb[c] * nxg + xj], w * k * f[ca[c] * nxg + xi]);
                    }
                }
            }
        }
        double *out = gF + (size_t)r * ng;
        for (size_t e = 0; e < ng; ++e) out[e] = acc_get(&g[e]);
        free(g);
    }
    return 0;
}

/*
 * Cholesky factorisation C = L L^T (Cholesky-Banachiewicz, row by row) of one
 * dense SPD covariance block, as the chi^2 of the fit needs.  L is written
 * lower-triangular with zeros above the diagonal.  Returns k+1 if the k-th
 * pivot is not positive (C not SPD).
 */
int fk_oracle_cholesky(int n, const double *C, double *L)
{
    if (n < 0) return -1;
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            acc_t s = {C[(size_t)i * n + j], 0};
            for (int k = 0; k < j; ++k)
                acc_add(&s, -L[(size_t)i * n + k] * L[(size_t)j * n + k]);
            double v = acc_get(&s);
            if (i == j) {
                if (!(v > 0.0)) return i + 1;
                L[(size_t)i * n + i] = sqrt(v);
            } else {
                L[(size_t)i * n + j] = v / L[(size_t)j * n + j];
            }
        }
    return 0;
}

/*
 * chi^2 of one covariance block for R replicas:
 *   res = O_r - D,  solve L z = res (forward substitution),  chi2[r] = z . z,
 * which equals res^T C^{-1} res.  If gO is not NULL it receives
 * d chi2 / d O_r = 2 C^{-1} res, obtained by solving L^T y = z (back
 * substitution) and doubling y.
 */
int fk_oracle_chi2(int n, const double *L, int R, const double *O, const double *D,
                   double *chi2, double *gO)
{
    if (n < 0 || R < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r) {
        double *z = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
        const double *o = O + (size_t)r * n;
        for (int i = 0; i < n; ++i) {
            acc_t s = {o[i], 0};
            acc_add(&s, -D[i]);
            for (int k = 0; k < i; ++k) acc_add(&s, -L[(size_t)i * n + k] * z[k]);
            z[i] = acc_get(&s) / L[(size_t)i * n + i];
        }
        acc_t q = {0, 0};
        for (int i = 0; i < n; ++i) acc_add(&q, z[i] * z[i]);
        chi2[r] = acc_get(&q);
        if (gO) {
            double *y = gO + (size_t)r * n;
            for (int i = n - 1; i >= 0; --i) {
                acc_t s = {z[i], 0};
                for (int k = i + 1; k < n; ++k) acc_add(&s, -L[(size_t)k * n + i] * y[k]);
                y[i] = acc_get(&s) / L[(size_t)i * n + i];
            }
            for (int i = 0; i < n; ++i) y[i] *= 2.0;
        }
        free(z);
    }
    return 0;
}

/*
 * The "PDF matrix" of the paper's timing study (Sec. 3, Table 3): for a
 * hadronic channel list, one column per replica holding the products
 * f_a(x_i) f_b(x_j) in the table's (channel, x_i, x_j) element order, so that
 * Eq. 1 becomes a plain product of the flattened table with this matrix.
 * Stored replica-major: L[r][(c * nx + i) * nx + j] = F[r][ca[c]][xmap[i]] * F[r][cb[c]][xmap[j]].
 */
int fk_oracle_luminosity(int nc, const int *ca, const int *cb, int nx, const int *xmap, int nxg,
                         int R, const double *F, double *L)
{
    if (nc < 0 || nx < 0 || R < 0 || check_xmap(xmap, nx, nxg)) return -1;
    for (int c = 0; c < nc; ++c)
        if (ca[c] < 0 || ca[c] >= NFL || cb[c] < 0 || cb[c] >= NFL) return -1;
    const size_t K = (size_t)nc * nx * nx;
    for (int r = 0; r < R; ++r) {
        const double *f = F + (size_t)r * NFL * nxg;
        for (int c = 0; c < nc; ++c)
            for (int i = 0; i < nx; ++i)
                for (int j = 0; j < nx; ++j)
                    L[(size_t)r * K + ((size_t)c * nx + i) * nx + j] =
                        f[ca[c] * nxg + xidx(xmap, i)] * f[cb[c] * nxg + xidx(xmap, j)];
    }
    return 0;
}

/*
 * The dense product timed in the paper's Table 3: an FK table flattened to
 * [ndata][K] times a PDF matrix [K][R] (given replica-major, L[r][k]):
 *   O[r][d] = sum_k fk[d][k] * L[r][k],  S[r][d] = sum_k |fk[d][k] * L[r][k]|.
 */
int fk_oracle_dense(int ndata, long long K, const double *fk, int R, const double *L,
                    double *O, double *S)
{
    if (ndata < 0 || K < 0 || R < 0) return -1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int r = 0; r < R; ++r)
        for (int d = 0; d < ndata; ++d) {
            const double *row = fk + (size_t)d * K;
            const double *l = L + (size_t)r * K;
            acc_t o = {0, 0}, s = {0, 0};
            for (long long k = 0; k < K; ++k) {
                const double term = row[k] * l[k];
                acc_add(&o, term);
                acc_add(&s, fabs(term));
            }
            O[(size_t)r * ndata + d] = acc_get(&o);
            if (S) S[(size_t)r * ndata + d] = acc_get(&s);
        }
    return 0;
}

/* Threads the OpenMP runtime will use (for reporting the CPU baseline). */
int fk_oracle_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the OpenMP thread count of later calls (n >= 1); returns the count in
 * effect afterwards.  Timing only: results do not depend on it (each output
 * is computed by one thread in a fixed order). */
int fk_oracle_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#endif
    return fk_oracle_threads();
}
