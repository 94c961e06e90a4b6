// chi^2 of the fit, FP64: chi2[r] = (O_r - D)^T C^{-1} (O_r - D) for a
// block-diagonal covariance (one dense SPD block per dataset), and its
// gradient d chi2 / d O_r = 2 C^{-1} (O_r - D), which the adjoint of the
// convolution turns into the gradient with respect to the PDF (the fit of
// Sec. 2 is gradient descent).
//
// Set-up (fk_cov_create, once): C_k = L_k L_k^T by a column-wise (left-looking)
// Cholesky, then X_k = L_k^{-1} by forward substitution against the identity.
// Per call: z = X_k (O_r - D) (the triangular solve L_k z = O_r - D, applied as
// a product with the precomputed inverse so that every row is independent),
// chi2 = |z|^2, gO = 2 X_k^T z.  Sums over rows use fixed-order partials.
#include "fk_internal.h"

#include <algorithm>
#include <cmath>

struct fk_cov {
    int nblocks = 0, n = 0;
    std::vector<int> sizes, offs;
    std::vector<long long> loff;
    int *d_sizes = nullptr, *d_offs = nullptr;
    long long *d_loff = nullptr;
    int ntiles = 0;
    int *d_tile_blk = nullptr, *d_tile_i0 = nullptr;
    int nzu = 0, ngu = 0;                          // work units of the two passes
    int *d_zu = nullptr, *d_gu = nullptr, *d_zt = nullptr, *d_gt = nullptr;
    double *L = nullptr;     // per block n_k x n_k row-major, lower factor
    double *Linv = nullptr;  // same layout, L^{-1} (lower)
    size_t bytes = 0;
};

namespace fk {
namespace {

constexpr int CT = 32;  // tile of rows / replicas

// One CTA per block.  In: A = C_k.  Out: A = L_k (zeros above the diagonal).
__global__ void __launch_bounds__(256) k_chol(const long long *__restrict__ loff,
                                              const int *__restrict__ sizes, double *__restrict__ L,
                                              int *__restrict__ info) {
    const int k = blockIdx.x, n = sizes[k];
    double *A = L + loff[k];
    __shared__ double red[256];
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int q = threadIdx.x; q < j; q += 256) s = fma(A[(size_t)j * n + q], A[(size_t)j * n + q], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double v = A[(size_t)j * n + j] - red[0];
            if (!(v > 0.0)) {
                bad = j + 1;
                piv = 1.0;
            } else {
                piv = sqrt(v);
            }
            A[(size_t)j * n + j] = piv;
        }
        __syncthreads();
        if (bad) break;
        const double p = piv;
        for (int i = j + 1 + threadIdx.x; i < n; i += 256) {
            double t = A[(size_t)i * n + j];
            for (int q = 0; q < j; ++q) t = fma(-A[(size_t)i * n + q], A[(size_t)j * n + q], t);
            A[(size_t)i * n + j] = t / p;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) info[k] = bad;
    if (bad) return;
    for (size_t idx = threadIdx.x; idx < (size_t)n * n; idx += 256) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        if (j > i) A[idx] = 0.0;
    }
}

// grid (nblocks, ceil(maxn/128)); thread = one column m of X = L^{-1}.
__global__ void __launch_bounds__(128) k_trinv(const long long *__restrict__ loff,
                                               const int *__restrict__ sizes,
                                               const double *__restrict__ L, double *__restrict__ X) {
    const int k = blockIdx.x, n = sizes[k];
    const int m = blockIdx.y * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double *Lk = L + loff[k];
    double *Xk = X + loff[k];
    for (int i = 0; i < m; ++i) Xk[(size_t)i * n + m] = 0.0;
    Xk[(size_t)m * n + m] = 1.0 / Lk[(size_t)m * n + m];
    for (int i = m + 1; i < n; ++i) {
        double s = 0.0;
        for (int q = m; q < i; ++q) s = fma(Lk[(size_t)i * n + q], Xk[(size_t)q * n + m], s);
        Xk[(size_t)i * n + m] = -s / Lk[(size_t)i * n + i];
    }
}

// A tile is 32 rows i0.. of one block.  Its contraction range is cut into
// work units of at most UNIT_COLS columns so that no CTA carries a long chain
// (the FP64 pipe is shared by the CTAs of an SM; one long tile would set the
// kernel's length); the units' partial sums are added in unit order.
constexpr int UNIT_COLS = 4 * CT;

struct CovView {
    int n;
    const int *sizes, *offs, *tile_blk, *tile_i0;
    const long long *loff;
    const double *Linv;
    const int *zu, *gu;     // units [u][3]: tile, m0, m1 (z pass, gradient pass)
    const int *zt, *gt;     // per tile [t][2]: first unit, unit count
};

// grid (nunits, ceil(R/32)), 256 threads: thread (ty, tx) -> rows i0+ty*4+p, replica r0+tx.
// Zp[(u*32 + row)*R + r] = sum_{m in [m0, m1)} X[i][m] (O[r][off+m] - D[off+m])
template <typename TO>
__global__ void __launch_bounds__(256) k_chi2_zpart(CovView cv, const TO *__restrict__ O,
                                                    const double *__restrict__ D, int R,
                                                    double *__restrict__ Zp) {
    const int u = blockIdx.x, tile = cv.zu[3 * u], m0u = cv.zu[3 * u + 1], m1u = cv.zu[3 * u + 2];
    const int k = cv.tile_blk[tile], i0 = cv.tile_i0[tile];
    const int nk = cv.sizes[k], off = cv.offs[k];
    const double *X = cv.Linv + cv.loff[k];
    const int r0 = blockIdx.y * CT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    __shared__ double Ls[CT][CT + 1], Rs[CT][CT + 1];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m0 = m0u; m0 < m1u; m0 += CT) {
        for (int idx = threadIdx.x; idx < CT * CT; idx += 256) {
            const int a = idx / CT, b = idx % CT;
            const int i = i0 + a, m = m0 + b;
            Ls[a][b] = (i < nk && m < m1u) ? X[(size_t)i * nk + m] : 0.0;
            const int r = r0 + a;
            Rs[b][a] = (r < R && m < m1u) ? (double)O[(size_t)r * cv.n + off + m] - D[off + m] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int mm = 0; mm < CT; ++mm) {
            const double rv = Rs[mm][tx];
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[p] = fma(Ls[ty * 4 + p][mm], rv, acc[p]);
        }
        __syncthreads();
    }
    const int r = r0 + tx;
    if (r < R) {
#pragma unroll
        for (int p = 0; p < 4; ++p) Zp[((size_t)u * CT + ty * 4 + p) * R + r] = acc[p];
    }
}

// grid (ntiles, ceil(R/32)): Z = sum of the tile's unit partials (in order),
// zsq[tile*R + r] = sum over the tile's rows of Z^2.
__global__ void __launch_bounds__(256) k_chi2_zred(CovView cv, const double *__restrict__ Zp, int R,
                                                   double *__restrict__ Z, double *__restrict__ zsq) {
    const int tile = blockIdx.x, k = cv.tile_blk[tile], i0 = cv.tile_i0[tile];
    const int nk = cv.sizes[k], off = cv.offs[k];
    const int u0 = cv.zt[2 * tile], nu = cv.zt[2 * tile + 1];
    const int r = blockIdx.y * CT + (threadIdx.x & 31), ty = threadIdx.x >> 5;
    __shared__ double sq[8][CT];
    double s = 0.0;
    if (r < R) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int row = ty * 4 + p, i = i0 + row;
            double z = 0.0;
            for (int u = 0; u < nu; ++u) z += Zp[((size_t)(u0 + u) * CT + row) * R + r];
            if (i < nk) {
                Z[(size_t)(off + i) * R + r] = z;
                s = fma(z, z, s);
            }
        }
    }
    sq[ty][threadIdx.x & 31] = s;
    __syncthreads();
    if (ty == 0 && r < R) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += sq[q][threadIdx.x];
        zsq[(size_t)tile * R + r] = t;
    }
}

// chi2[r] = sum_tile zsq[tile][r], tiles in order.
__global__ void k_chi2_sum(const double *__restrict__ zsq, int ntiles, int R, double *__restrict__ chi2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int t = 0; t < ntiles; ++t) s += zsq[(size_t)t * R + r];
    chi2[r] = s;
}

// grid (nunits, ceil(R/32)): Gp[(u*32 + row)*R + r] = sum_{m in [m0, m1)} X[m][i] Z[off+m][r]
__global__ void __launch_bounds__(256) k_chi2_gpart(CovView cv, const double *__restrict__ Z, int R,
                                                    double *__restrict__ Gp) {
    const int u = blockIdx.x, tile = cv.gu[3 * u], m0u = cv.gu[3 * u + 1], m1u = cv.gu[3 * u + 2];
    const int k = cv.tile_blk[tile], i0 = cv.tile_i0[tile];
    const int nk = cv.sizes[k], off = cv.offs[k];
    const double *X = cv.Linv + cv.loff[k];
    const int r0 = blockIdx.y * CT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    __shared__ double Ls[CT][CT + 1], Zs[CT][CT + 1];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int m0 = m0u; m0 < m1u; m0 += CT) {
        for (int idx = threadIdx.x; idx < CT * CT; idx += 256) {
            const int a = idx / CT, b = idx % CT;
            const int m = m0 + a, i = i0 + b;
            Ls[a][b] = (m < m1u && i < nk) ? X[(size_t)m * nk + i] : 0.0;
            const int r = r0 + b;
            Zs[a][b] = (m < m1u && r < R) ? Z[(size_t)(off + m) * R + r] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int mm = 0; mm < CT; ++mm) {
            const double zv = Zs[mm][tx];
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[p] = fma(Ls[mm][ty * 4 + p], zv, acc[p]);
        }
        __syncthreads();
    }
    const int r = r0 + tx;
    if (r < R) {
#pragma unroll
        for (int p = 0; p < 4; ++p) Gp[((size_t)u * CT + ty * 4 + p) * R + r] = acc[p];
    }
}

// grid (ntiles, ceil(R/32)): gO[r][off+i] = 2 * sum of the tile's unit partials (in order)
template <typename TO>
__global__ void __launch_bounds__(256) k_chi2_gred(CovView cv, const double *__restrict__ Gp, int R,
                                                   TO *__restrict__ gO) {
    const int tile = blockIdx.x, k = cv.tile_blk[tile], i0 = cv.tile_i0[tile];
    const int nk = cv.sizes[k], off = cv.offs[k];
    const int u0 = cv.gt[2 * tile], nu = cv.gt[2 * tile + 1];
    const int r0 = blockIdx.y * CT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    __shared__ double out[CT][CT + 1];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int row = ty * 4 + p;
        double g = 0.0;
        if (r0 + tx < R)
            for (int u = 0; u < nu; ++u) g += Gp[((size_t)(u0 + u) * CT + row) * R + r0 + tx];
        out[tx][row] = 2.0 * g;
    }
    __syncthreads();
    // stage for coalesced stores along i
    for (int idx = threadIdx.x; idx < CT * CT; idx += 256) {
        const int rr = idx / CT, ii = idx % CT;
        const int r = r0 + rr, i = i0 + ii;
        if (r < R && i < nk) gO[(size_t)r * cv.n + off + i] = (TO)out[rr][ii];
    }
}

CovView cview(const fk_cov *c) {
    return CovView{c->n, c->d_sizes, c->d_offs, c->d_tile_blk, c->d_tile_i0, c->d_loff, c->Linv,
                   c->d_zu, c->d_gu, c->d_zt, c->d_gt};
}

void cov_free(fk_cov *c) {
    if (!c) return;
    cudaFree(c->d_sizes);
    cudaFree(c->d_offs);
    cudaFree(c->d_loff);
    cudaFree(c->d_tile_blk);
    cudaFree(c->d_tile_i0);
    cudaFree(c->d_zu);
    cudaFree(c->d_gu);
    cudaFree(c->d_zt);
    cudaFree(c->d_gt);
    cudaFree(c->L);
    cudaFree(c->Linv);
    delete c;
}

// Work units of the two passes: z needs columns [0, min(i0+32, n)) of the
// tile's rows, the gradient columns [i0, n); each range cut every UNIT_COLS.
void make_units(const std::vector<int> &tb, const std::vector<int> &ti, const std::vector<int> &sizes,
                bool grad, std::vector<int> &units, std::vector<int> &per_tile) {
    for (size_t t = 0; t < tb.size(); ++t) {
        const int n = sizes[tb[t]], i0 = ti[t];
        const int b = grad ? i0 : 0, e = grad ? n : std::min(i0 + CT, n);
        per_tile.push_back((int)(units.size() / 3));
        int cnt = 0;
        for (int m = b; m < e; m += UNIT_COLS, ++cnt) {
            units.push_back((int)t);
            units.push_back(m);
            units.push_back(std::min(m + UNIT_COLS, e));
        }
        per_tile.push_back(cnt);
    }
}

int cov_create(const double *C, const int *bs, int nb, fk_cov **out) {
    if (!C || !bs || !out || nb < 1) return fail(FK_EINVAL, "fk_cov_create: null pointer or nblocks < 1");
    *out = nullptr;
    fk_cov *c = new fk_cov();
    c->nblocks = nb;
    long long tot = 0, el = 0;
    int maxn = 0;
    std::vector<int> tb, ti;
    for (int k = 0; k < nb; ++k) {
        if (bs[k] < 1) {
            delete c;
            return fail(FK_EINVAL, "fk_cov_create: block size < 1");
        }
        c->sizes.push_back(bs[k]);
        c->offs.push_back((int)tot);
        c->loff.push_back(el);
        for (int i0 = 0; i0 < bs[k]; i0 += CT) {
            tb.push_back(k);
            ti.push_back(i0);
        }
        tot += bs[k];
        el += (long long)bs[k] * bs[k];
        maxn = std::max(maxn, bs[k]);
    }
    if (tot > (1LL << 30)) {
        delete c;
        return fail(FK_EINVAL, "fk_cov_create: dimension too large");
    }
    c->n = (int)tot;
    c->ntiles = (int)tb.size();
    c->bytes = sizeof(double) * 2 * el;
    auto cleanup = [&](int st) {
        cov_free(c);
        return st;
    };
    if (cudaMalloc(&c->d_sizes, sizeof(int) * nb) || cudaMalloc(&c->d_offs, sizeof(int) * nb) ||
        cudaMalloc(&c->d_loff, sizeof(long long) * nb) ||
        cudaMalloc(&c->d_tile_blk, sizeof(int) * c->ntiles) ||
        cudaMalloc(&c->d_tile_i0, sizeof(int) * c->ntiles) || cudaMalloc(&c->L, sizeof(double) * el) ||
        cudaMalloc(&c->Linv, sizeof(double) * el))
        return cleanup(fail(FK_ENOMEM, "fk_cov_create: device allocation failed"));
    int *d_info = nullptr;
    if (cudaMalloc(&d_info, sizeof(int) * nb)) return cleanup(fail(FK_ENOMEM, "fk_cov_create: info"));
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpy(c->d_sizes, c->sizes.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_offs, c->offs.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_loff, c->loff.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_tile_blk, tb.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_tile_i0, ti.data(), sizeof(int) * c->ntiles, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->L, C, sizeof(double) * el, cudaMemcpyHostToDevice);
    std::vector<int> zu, zt, gu, gt;
    make_units(tb, ti, c->sizes, false, zu, zt);
    make_units(tb, ti, c->sizes, true, gu, gt);
    c->nzu = (int)zu.size() / 3;
    c->ngu = (int)gu.size() / 3;
    if (!e && (cudaMalloc(&c->d_zu, sizeof(int) * zu.size()) || cudaMalloc(&c->d_gu, sizeof(int) * gu.size()) ||
               cudaMalloc(&c->d_zt, sizeof(int) * zt.size()) || cudaMalloc(&c->d_gt, sizeof(int) * gt.size()))) {
        cudaFree(d_info);
        return cleanup(fail(FK_ENOMEM, "fk_cov_create: work units"));
    }
    e = e ? e : cudaMemcpy(c->d_zu, zu.data(), sizeof(int) * zu.size(), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_gu, gu.data(), sizeof(int) * gu.size(), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_zt, zt.data(), sizeof(int) * zt.size(), cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_gt, gt.data(), sizeof(int) * gt.size(), cudaMemcpyHostToDevice);
    if (e) {
        cudaFree(d_info);
        return cleanup(cuda_fail(e, "fk_cov_create: copy"));
    }
    k_chol<<<nb, 256>>>(c->d_loff, c->d_sizes, c->L, d_info);
    count_launch();
    e = cudaGetLastError();
    dim3 g2(nb, (maxn + 127) / 128);
    if (!e) {
        k_trinv<<<g2, 128>>>(c->d_loff, c->d_sizes, c->L, c->Linv);
        count_launch();
    }
    e = e ? e : cudaGetLastError();
    std::vector<int> info(nb, 0);
    e = e ? e : cudaMemcpy(info.data(), d_info, sizeof(int) * nb, cudaMemcpyDeviceToHost);
    cudaFree(d_info);
    if (e) return cleanup(cuda_fail(e, "fk_cov_create: factorisation"));
    for (int k = 0; k < nb; ++k)
        if (info[k])
            return cleanup(fail(FK_EINVAL, "fk_cov_create: block " + std::to_string(k) +
                                               " is not positive definite (pivot " +
                                               std::to_string(info[k] - 1) + ")"));
    *out = c;
    return FK_OK;
}

template <typename TO>
int chi2_t(const fk_cov *c, const TO *O, const double *D, int R, double *out, TO *gO,
           cudaStream_t s) {
    Scratch scr(s);
    double *Z = nullptr, *zsq = nullptr, *part = nullptr;
    FK_CUDA(scr.get(&Z, (size_t)c->n * R));
    FK_CUDA(scr.get(&zsq, (size_t)c->ntiles * R));
    FK_CUDA(scr.get(&part, (size_t)std::max(c->nzu, c->ngu) * CT * R));
    CovView cv = cview(c);
    const int rt = (R + CT - 1) / CT;
    k_chi2_zpart<TO><<<dim3(c->nzu, rt), 256, 0, s>>>(cv, O, D, R, part);
    count_launch();
    FK_CUDA(cudaGetLastError());
    k_chi2_zred<<<dim3(c->ntiles, rt), 256, 0, s>>>(cv, part, R, Z, zsq);
    count_launch();
    FK_CUDA(cudaGetLastError());
    k_chi2_sum<<<(R + 127) / 128, 128, 0, s>>>(zsq, c->ntiles, R, out);
    count_launch();
    FK_CUDA(cudaGetLastError());
    if (gO) {
        k_chi2_gpart<<<dim3(c->ngu, rt), 256, 0, s>>>(cv, Z, R, part);
        count_launch();
        FK_CUDA(cudaGetLastError());
        k_chi2_gred<TO><<<dim3(c->ntiles, rt), 256, 0, s>>>(cv, part, R, gO);
        count_launch();
        FK_CUDA(cudaGetLastError());
    }
    return FK_OK;
}

}  // namespace
}  // namespace fk

extern "C" {

int fk_cov_create(const double *C_blocks, const int *block_sizes, int nblocks, fk_cov **out) {
    return fk::cov_create(C_blocks, block_sizes, nblocks, out);
}

int fk_cov_destroy(fk_cov *cov) {
    fk::cov_free(cov);
    return FK_OK;
}

int fk_cov_size(const fk_cov *cov) { return cov ? cov->n : 0; }

int fk_chi2(const fk_cov *cov, const void *O, const double *D, int R, double *chi2, void *gO,
            int io_prec, fk_stream stream) {
    if (!cov || !O || !D || !chi2 || R < 1) return fk::fail(FK_EINVAL, "fk_chi2: null pointer or R < 1");
    if (io_prec < FK_FP64 || io_prec > FK_TF32) return fk::fail(FK_EINVAL, "fk_chi2: unknown precision");
    if (io_prec == FK_FP64)
        return fk::chi2_t<double>(cov, (const double *)O, D, R, chi2, (double *)gO, (cudaStream_t)stream);
    return fk::chi2_t<float>(cov, (const float *)O, D, R, chi2, (float *)gO, (cudaStream_t)stream);
}

}  // extern "C"
