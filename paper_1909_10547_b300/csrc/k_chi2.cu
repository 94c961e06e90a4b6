// chi^2 of the fit, FP64: chi2[r] = (O_r - D)^T C^{-1} (O_r - D) for a
// block-diagonal covariance (one dense SPD block per dataset), and its
// gradient d chi2 / d O_r = 2 C^{-1} (O_r - D), which the adjoint of the
// convolution turns into the gradient with respect to the PDF (the fit of
// Sec. 2 is gradient descent).
//
// Set-up (fk_cov_create, once per covariance):
//   C_k = L_k L_k^T by a column-wise (left-looking) Cholesky, kept row-major
//   and transposed (LT = L^T, row-major: column m of L is contiguous);
//   the inverses of the 32 x 32 diagonal blocks of L_k and of its "reversed
//   transpose" U[i][m] = L[n-1-m][n-1-i] (lower triangular), each by
//   substitution against the identity.
// Per call (one kernel, k_chi2_solve): blocked forward substitution
// L z = O_r - D over panels of 32 rows (the usual TRSM arrangement): the
// panel's rows first take the contributions of every earlier row,
// t_i = r_i - sum_{m < i0} L[i][m] z_m, then its own triangle is applied
// through its inverted diagonal block.  chi2 = |z|^2.  The back substitution
// L^T w = z is the same forward substitution on U with reversed vectors
// (w'_i = w_{n-1-i}), and gO = 2 w.  In the update one lane owns one row of
// the panel and the CTA's warps split the columns m, so every load of L is a
// coalesced row of LT (or, reversed, of L) and each lane's partial sums stay
// in registers; the eight warp partials are added in warp order.  One CTA owns
// one covariance block and a few replicas, keeps their vectors in shared
// memory and writes chi^2 and gO directly: every sum runs in an order that
// depends only on the block size, never on R or on the replica tile.
#include "fk_internal.h"

#include <algorithm>
#include <cmath>

struct fk_cov {
    int nblocks = 0, n = 0, maxn = 0;
    std::vector<int> sizes, offs;
    std::vector<long long> loff, doff;
    int *d_sizes = nullptr, *d_offs = nullptr;
    long long *d_loff = nullptr, *d_doff = nullptr;
    double *L = nullptr;   // per block n_k x n_k row-major, lower factor
    double *LT = nullptr;  // per block, L^T row-major
    double *DL = nullptr;  // per block, per 32-row panel: inverse of L's diagonal block, column-major 32 x 32
    double *DU = nullptr;  // the same for U
    size_t bytes = 0;
};

namespace fk {
namespace {

constexpr int PB = 32;          // rows per panel
constexpr int SOLVE_THREADS = 256;
constexpr int SOLVE_WARPS = SOLVE_THREADS / 32;
// a block's vectors stay in shared memory up to this many doubles per CTA
constexpr int SMEM_VEC_DOUBLES = 3072;  // 24 KB (with the 8 + 16 KB of static panel buffers, within 48 KB)

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

// grid (nblocks, 64): LT[m][i] = L[i][m]
__global__ void __launch_bounds__(256) k_transpose(const long long *__restrict__ loff, const int *__restrict__ sizes,
                                                   const double *__restrict__ L, double *__restrict__ LT) {
    const int k = blockIdx.x, n = sizes[k];
    const double *Lk = L + loff[k];
    double *Tk = LT + loff[k];
    const size_t nn = (size_t)n * n;
    for (size_t idx = (size_t)blockIdx.y * 256 + threadIdx.x; idx < nn; idx += (size_t)gridDim.y * 256) {
        const int m = (int)(idx / n), i = (int)(idx % n);
        Tk[idx] = Lk[(size_t)i * n + m];
    }
}

// grid (nblocks, max panels, 2), 32 threads: thread c solves B x = e_c for the
// panel's diagonal block B (rows and columns i0 .. i0 + rows - 1 of L, or for
// blockIdx.z = 1 of U[i][m] = L[n-1-m][n-1-i]) and stores column c of B^{-1}
// at Dinv[p][c][0..32) (zeros above the diagonal and outside the block).
__global__ void __launch_bounds__(32) k_dinv(const long long *__restrict__ loff, const long long *__restrict__ doff,
                                             const int *__restrict__ sizes, const double *__restrict__ L,
                                             double *__restrict__ DL, double *__restrict__ DU) {
    const int k = blockIdx.x, p = blockIdx.y, n = sizes[k];
    const int i0 = p * PB;
    if (i0 >= n) return;
    const int rows = min(PB, n - i0);
    const double *Lk = L + loff[k];
    const bool rev = blockIdx.z != 0;
    auto el = [&](int i, int m) {  // element (i, m) of L or of U
        return rev ? Lk[(size_t)(n - 1 - m) * n + (n - 1 - i)] : Lk[(size_t)i * n + m];
    };
    double *out = (rev ? DU : DL) + doff[k] + (size_t)p * PB * PB;
    const int c = threadIdx.x;
    double x[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i) x[i] = 0.0;
    if (c < rows) {
        for (int i = c; i < rows; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = c; q < i; ++q) s = fma(-el(i0 + i, i0 + q), x[q], s);
            x[i] = s / el(i0 + i, i0 + i);
        }
    }
#pragma unroll
    for (int i = 0; i < PB; ++i) out[c * PB + i] = x[i];
}

struct CovView {
    int n;
    const int *sizes, *offs;
    const long long *loff, *doff;
    const double *L, *LT, *DL, *DU;
};

__device__ __forceinline__ double warp_sum(double v) {
    // xor butterfly: every lane ends with the same value (each level adds the
    // same two numbers in every lane, and addition is commutative)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Solves M y = b in place for RT right-hand sides, M lower triangular n x n
// with element (i, m) at P[m * sm + i * si], b / y in v[rr * n + idx(i)]
// (idx(i) = i, or n - 1 - i when REV: the reversed vectors of the back
// substitution).  Dinv holds the inverted diagonal blocks of M.  Shared
// memory: part [SOLVE_WARPS][RT][32] for the warp partials, Ds [32 * 32] for
// the panel's inverted diagonal block.
template <int RT, bool REV>
__device__ void blocked_solve(const double *__restrict__ P, long long sm, long long si,
                              const double *__restrict__ Dinv, int n, double *v,
                              double (*part)[RT][PB], double *Ds) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    auto at = [&](int rr, int i) -> double & {
        const int j = REV ? n - 1 - i : i;
        return v[FK_DBG(j >= 0 && j < n && rr < RT, 20, j) ? rr * n + j : 0];
    };
    for (int i0 = 0; i0 < n; i0 += PB) {
        const int rows = min(PB, n - i0);
        const bool own = lane < rows;  // lane owns row i0 + lane
        // the panel's Dinv block to shared memory; its loads overlap the update
        const double *Dp = Dinv + (size_t)(i0 / PB) * PB * PB;
        for (int e = threadIdx.x; e < PB * PB; e += SOLVE_THREADS) Ds[e] = __ldg(Dp + e);
        const double *Pi = P + (long long)(i0 + (own ? lane : 0)) * si;
        // columns [0, i0) in SOLVE_WARPS chunks of `per`; four interleaved
        // accumulators per replica keep the dependent chains short
        const int per = (i0 + SOLVE_WARPS - 1) / SOLVE_WARPS;
        const int m0 = warp * per, m1 = min(i0, m0 + per);
        double acc[RT][4];
#pragma unroll
        for (int rr = 0; rr < RT; ++rr)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[rr][u] = 0.0;
        int m = m0;
        for (; m + 4 <= m1; m += 4) {
            double a[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = own ? __ldg(Pi + (long long)(m + u) * sm) : 0.0;
#pragma unroll
            for (int rr = 0; rr < RT; ++rr)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[rr][u] = fma(a[u], at(rr, m + u), acc[rr][u]);
        }
        for (; m < m1; ++m) {
            const double a = own ? __ldg(Pi + (long long)m * sm) : 0.0;
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) acc[rr][0] = fma(a, at(rr, m), acc[rr][0]);
        }
#pragma unroll
        for (int rr = 0; rr < RT; ++rr) part[warp][rr][lane] = (acc[rr][0] + acc[rr][1]) + (acc[rr][2] + acc[rr][3]);
        __syncthreads();
        // warp rr: t = b - (sum of the warp partials, in warp order), then
        // y_panel = Dinv_p t (Dinv_p column-major, zero above its diagonal and
        // outside the panel, so all 32 columns can be summed)
        for (int rr = warp; rr < RT; rr += SOLVE_WARPS) {
            double sum = part[0][rr][lane];
#pragma unroll
            for (int w = 1; w < SOLVE_WARPS; ++w) sum += part[w][rr][lane];
            const double t = own ? at(rr, i0 + lane) - sum : 0.0;
            double s4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < PB; ++c) s4[c & 3] = fma(Ds[c * PB + lane], __shfl_sync(0xffffffffu, t, c), s4[c & 3]);
            if (own) at(rr, i0 + lane) = (s4[0] + s4[1]) + (s4[2] + s4[3]);
        }
        __syncthreads();
    }
}

// grid (nblocks, replica tiles of RT from rfirst), SOLVE_THREADS threads.  vg: global scratch for
// the vectors when a block is too large for shared memory (else NULL).
// chi2 of the block goes to out[k * R + r] (or straight to chi2[r] when the
// covariance has one block: out = chi2).
template <typename TO, int RT>
__global__ void __launch_bounds__(SOLVE_THREADS) k_chi2_solve(CovView cv, const TO *__restrict__ O,
                                                              const double *__restrict__ D, int R, int rfirst,
                                                              double *__restrict__ out, TO *__restrict__ gO,
                                                              double *__restrict__ vg) {
    const int k = blockIdx.x, n = cv.sizes[k], off = cv.offs[k];
    const int r0 = rfirst + blockIdx.y * RT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ double smem_v[];
    __shared__ double part[SOLVE_WARPS][RT][PB];
    __shared__ double Ds[PB * PB];
    double *v = vg ? vg + ((size_t)blockIdx.y * gridDim.x + k) * RT * (size_t)n : smem_v;
    for (int idx = threadIdx.x; idx < RT * n; idx += SOLVE_THREADS) {
        const int rr = idx / n, i = idx - rr * n, r = r0 + rr;
        v[idx] = r < R ? (double)O[(size_t)r * cv.n + off + i] - D[off + i] : 0.0;
    }
    __syncthreads();
    const double *Lk = cv.L + cv.loff[k];
    // forward: L[i][m] = LT[m * n + i]
    blocked_solve<RT, false>(cv.LT + cv.loff[k], n, 1, cv.DL + cv.doff[k], n, v, part, Ds);
    for (int rr = warp; rr < RT; rr += SOLVE_WARPS) {
        double s = 0.0;
        for (int i = lane; i < n; i += 32) s = fma(v[rr * n + i], v[rr * n + i], s);
        s = warp_sum(s);
        if (lane == 0 && r0 + rr < R) out[(size_t)k * R + r0 + rr] = s;
    }
    if (!gO) return;
    // back: U[i][m] = L[n-1-m][n-1-i] = Lk[(n-1)(n+1) - m n - i]
    blocked_solve<RT, true>(Lk + (long long)(n - 1) * (n + 1), -(long long)n, -1, cv.DU + cv.doff[k], n, v, part, Ds);
    for (int idx = threadIdx.x; idx < RT * n; idx += SOLVE_THREADS) {
        const int rr = idx / n, i = idx - rr * n, r = r0 + rr;
        if (r < R && FK_DBG(off + i < cv.n, 21, off + i)) gO[(size_t)r * cv.n + off + i] = (TO)(2.0 * v[idx]);
    }
}

// Whitened chi^2: with the tables and data already multiplied by L^{-1} (once,
// when a fit is set up), Z = L^{-1} O and Dw = L^{-1} D, so z = Z - Dw,
// chi2[r] = |z_r|^2 and d chi2 / d Z_r = 2 z_r, which the adjoint of the
// whitened tables turns into the gradient with respect to the PDF.  FP64
// arithmetic; one warp per replica, lane l adding i = l, l + 32, ... and a
// butterfly sum, an order that depends on n only.  Grid ceil(R / 8), 256 threads.
template <typename TO>
__global__ void __launch_bounds__(256) k_chi2_white(const TO *__restrict__ Z, int ldz, const double *__restrict__ Dw,
                                                    int n, int R, double *__restrict__ chi2, TO *__restrict__ gO,
                                                    int ldg) {
    const int r = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (r >= R) return;  // whole warps leave together
    const TO *z = Z + (size_t)r * ldz;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double d = (double)z[i] - Dw[i];
        s = fma(d, d, s);
        if (gO) gO[(size_t)r * ldg + i] = (TO)(2.0 * d);
    }
    s = warp_sum(s);
    if (lane == 0) chi2[r] = s;
}

// chi2[r] = sum_k zsq[k][r], blocks in order.
__global__ void k_chi2_sum(const double *__restrict__ zsq, int nblocks, int R, double *__restrict__ chi2) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double s = 0.0;
    for (int k = 0; k < nblocks; ++k) s += zsq[(size_t)k * R + r];
    chi2[r] = s;
}

}  // namespace

FK_DBG_READER(dbg_chi2)

namespace {

CovView cview(const fk_cov *c) {
    return CovView{c->n, c->d_sizes, c->d_offs, c->d_loff, c->d_doff, c->L, c->LT, c->DL, c->DU};
}

void cov_free(fk_cov *c) {
    if (!c) return;
    cudaFree(c->d_sizes);
    cudaFree(c->d_offs);
    cudaFree(c->d_loff);
    cudaFree(c->d_doff);
    cudaFree(c->L);
    cudaFree(c->LT);
    cudaFree(c->DL);
    cudaFree(c->DU);
    delete c;
}

int cov_create(const double *C, const int *bs, int nb, fk_cov **out) {
    if (!C || !bs || !out || nb < 1) return fail(FK_EINVAL, "fk_cov_create: null pointer or nblocks < 1");
    *out = nullptr;
    fk_cov *c = new fk_cov();
    c->nblocks = nb;
    long long tot = 0, el = 0, dl = 0;
    int maxp = 0;
    for (int k = 0; k < nb; ++k) {
        if (bs[k] < 1) {
            delete c;
            return fail(FK_EINVAL, "fk_cov_create: block size < 1");
        }
        if (bs[k] > 46340) {  // n * n must stay within 32-bit element offsets per row product
            delete c;
            return fail(FK_EINVAL, "fk_cov_create: block size > 46340");
        }
        if (tot + bs[k] > (1LL << 30)) {
            delete c;
            return fail(FK_EINVAL, "fk_cov_create: dimension too large");
        }
        c->sizes.push_back(bs[k]);
        c->offs.push_back((int)tot);
        c->loff.push_back(el);
        c->doff.push_back(dl);
        const int np = (bs[k] + PB - 1) / PB;
        tot += bs[k];
        el += (long long)bs[k] * bs[k];
        dl += (long long)np * PB * PB;
        c->maxn = std::max(c->maxn, bs[k]);
        maxp = std::max(maxp, np);
    }
    c->n = (int)tot;
    c->bytes = sizeof(double) * (2 * el + 2 * dl);
    auto cleanup = [&](int st) {
        cov_free(c);
        return st;
    };
    if (cudaMalloc(&c->d_sizes, sizeof(int) * nb) || cudaMalloc(&c->d_offs, sizeof(int) * nb) ||
        cudaMalloc(&c->d_loff, sizeof(long long) * nb) || cudaMalloc(&c->d_doff, sizeof(long long) * nb) ||
        cudaMalloc(&c->L, sizeof(double) * el) || cudaMalloc(&c->LT, sizeof(double) * el) ||
        cudaMalloc(&c->DL, sizeof(double) * dl) || cudaMalloc(&c->DU, sizeof(double) * dl))
        return cleanup(fail(FK_ENOMEM, "fk_cov_create: device allocation failed"));
    int *d_info = nullptr;
    if (cudaMalloc(&d_info, sizeof(int) * nb)) return cleanup(fail(FK_ENOMEM, "fk_cov_create: info"));
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMemcpy(c->d_sizes, c->sizes.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_offs, c->offs.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_loff, c->loff.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->d_doff, c->doff.data(), sizeof(long long) * nb, cudaMemcpyHostToDevice);
    e = e ? e : cudaMemcpy(c->L, C, sizeof(double) * el, cudaMemcpyHostToDevice);
    if (e) {
        cudaFree(d_info);
        return cleanup(cuda_fail(e, "fk_cov_create: copy"));
    }
    k_chol<<<nb, 256>>>(c->d_loff, c->d_sizes, c->L, d_info);
    count_launch();
    e = cudaGetLastError();
    std::vector<int> info(nb, 0);
    e = e ? e : cudaMemcpy(info.data(), d_info, sizeof(int) * nb, cudaMemcpyDeviceToHost);
    cudaFree(d_info);
    if (e) return cleanup(cuda_fail(e, "fk_cov_create: factorisation"));
    for (int k = 0; k < nb; ++k)
        if (info[k])
            return cleanup(fail(FK_EINVAL, "fk_cov_create: block " + std::to_string(k) +
                                               " is not positive definite (pivot " +
                                               std::to_string(info[k] - 1) + ")"));
    k_transpose<<<dim3(nb, 64), 256>>>(c->d_loff, c->d_sizes, c->L, c->LT);
    count_launch();
    e = cudaGetLastError();
    if (!e) {
        k_dinv<<<dim3(nb, maxp, 2), 32>>>(c->d_loff, c->d_doff, c->d_sizes, c->L, c->DL, c->DU);
        count_launch();
        e = cudaGetLastError();
    }
    e = e ? e : cudaDeviceSynchronize();
    if (e) return cleanup(cuda_fail(e, "fk_cov_create: diagonal blocks"));
    *out = c;
    return FK_OK;
}

// Replicas per CTA: as many as keep one CTA's FP64 work (n^2 * RT
// multiply-adds for the two substitutions) within 2^16, so that the chain of
// a block stays short and its replicas spread over many SMs, with the vectors
// of RT replicas within the shared-memory budget.
int pick_rt(int maxn) {
    const long long nn = (long long)maxn * maxn;
    for (int rt : {8, 4, 2})
        if (nn * rt <= (1LL << 16) && (long long)rt * maxn <= SMEM_VEC_DOUBLES) return rt;
    return 1;
}

template <typename TO, int RT>
int chi2_launch(const fk_cov *c, const TO *O, const double *D, int R, double *out, TO *gO, Scratch &scr,
                cudaStream_t s) {
    double *zsq = out;
    if (c->nblocks > 1) FK_CUDA(scr.get(&zsq, (size_t)c->nblocks * R));
    const int ry = (R + RT - 1) / RT;
    constexpr int YMAX = 65535;  // grid height limit: larger R runs in several launches
    double *vg = nullptr;
    size_t smem = (size_t)RT * c->maxn * sizeof(double);
    if ((long long)RT * c->maxn > SMEM_VEC_DOUBLES) {
        FK_CUDA(scr.get(&vg, (size_t)std::min(ry, YMAX) * c->nblocks * RT * c->maxn));
        smem = 0;
    }
    for (int y0 = 0; y0 < ry; y0 += YMAX) {
        const int gy = std::min(YMAX, ry - y0);
        k_chi2_solve<TO, RT><<<dim3(c->nblocks, gy), SOLVE_THREADS, smem, s>>>(cview(c), O, D, R, y0 * RT, zsq,
                                                                               gO, vg);
        count_launch();
        FK_CUDA(cudaGetLastError());
    }
    if (c->nblocks > 1) {
        k_chi2_sum<<<(R + 127) / 128, 128, 0, s>>>(zsq, c->nblocks, R, out);
        count_launch();
        FK_CUDA(cudaGetLastError());
    }
    return FK_OK;
}

template <typename TO>
int chi2_t(const fk_cov *c, const TO *O, const double *D, int R, double *out, TO *gO, cudaStream_t s) {
    Scratch scr(s);
    switch (pick_rt(c->maxn)) {
        case 8: return chi2_launch<TO, 8>(c, O, D, R, out, gO, scr, s);
        case 4: return chi2_launch<TO, 4>(c, O, D, R, out, gO, scr, s);
        case 2: return chi2_launch<TO, 2>(c, O, D, R, out, gO, scr, s);
    }
    return chi2_launch<TO, 1>(c, O, D, R, out, gO, scr, s);
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

int fk_chi2_white(const void *Z, int ldz, const double *Dw, int n, int R, double *chi2, void *gO, int ldg,
                  int io_prec, fk_stream stream) {
    if (!Z || !Dw || !chi2) return fk::fail(FK_EINVAL, "fk_chi2_white: null pointer");
    if (n < 1 || R < 1) return fk::fail(FK_EINVAL, "fk_chi2_white: n < 1 or R < 1");
    if (io_prec < FK_FP64 || io_prec > FK_FP64_TC) return fk::fail(FK_EINVAL, "fk_chi2_white: unknown precision");
    ldz = ldz ? ldz : n;
    ldg = ldg ? ldg : n;
    if (ldz < n || ldg < n) return fk::fail(FK_EINVAL, "fk_chi2_white: ldz or ldg < n");
    const unsigned blocks = (unsigned)((R + 7) / 8);
    cudaStream_t s = (cudaStream_t)stream;
    if (FK_IO64(io_prec))
        fk::k_chi2_white<double><<<blocks, 256, 0, s>>>((const double *)Z, ldz, Dw, n, R, chi2, (double *)gO, ldg);
    else
        fk::k_chi2_white<float><<<blocks, 256, 0, s>>>((const float *)Z, ldz, Dw, n, R, chi2, (float *)gO, ldg);
    fk::count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

int fk_chi2(const fk_cov *cov, const void *O, const double *D, int R, double *chi2, void *gO,
            int io_prec, fk_stream stream) {
    if (!cov || !O || !D || !chi2 || R < 1) return fk::fail(FK_EINVAL, "fk_chi2: null pointer or R < 1");
    if (io_prec < FK_FP64 || io_prec > FK_FP64_TC) return fk::fail(FK_EINVAL, "fk_chi2: unknown precision");
    if (FK_IO64(io_prec))
        return fk::chi2_t<double>(cov, (const double *)O, D, R, chi2, (double *)gO, (cudaStream_t)stream);
    return fk::chi2_t<float>(cov, (const float *)O, D, R, chi2, (float *)gO, (cudaStream_t)stream);
}

}  // extern "C"
