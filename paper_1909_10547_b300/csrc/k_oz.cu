// FP64 results on the tensor cores by exact operand slices (the splitting of
// Ozaki et al.): the FK_FP64_TC mode.
//
// Every FP64 operand row is cut along K into chunks of up to 512 elements;
// within a chunk each value v is written as
//   v = 2^(e - S*B) * sum_{p=0}^{S-1} t_p 2^(B (S-1-p)),   |t_p| <= 64,
// with e the exponent of the chunk's largest |v| plus one (so the scaled value
// is below 2^(S*B - 1)), B = 7 bits per digit and S = 8 digits: every value
// to within 2^-55 of the largest one of its row in the chunk, and every value
// of at least 1/8 of that largest one exactly.  A digit is a small integer,
// exact in BF16.  The 36 most significant digit products (p + q = w <= S - 1)
// run as BF16 MMAs over the chunk; the w + 1 products of one weight w
// accumulate in one accumulator: at most 8 x 512 products of integers of at
// most 2^6 in magnitude, a sum of at most 2^24 in magnitude, so the tensor
// cores' FP32 accumulation of it is exact.  k_oz_combine scales each of the 8
// exact partials of a chunk by its power of two and adds them in FP64, chunks
// in order and weights in order.  Each of the 28 dropped digit products
// (w >= S) is below 2^-56 of the chunk's largest one.
//
// Served products: the dense tables of the paper's Table 3 (O = FK L), DIS
// tables (forward: FK times the gathered PDF; adjoint: gO times the
// transposed table, scattered onto the grid) and hadronic tables (forward:
// the flattened table times the PDF matrix f_a(x_i) f_b(x_j), formed in FP64
// per call; adjoint: W = gO times the transposed flattened table, then the
// product rule on each channel in FP64).  A replica's result does not depend
// on R: the partials are exact and their FP64 sum runs in an order fixed by
// the table.
#include "fk_internal.h"

#include <algorithm>

namespace fk {
namespace {

constexpr int OZ_S = 8;         // digits per value
constexpr int OZ_B = 7;         // bits per digit
constexpr int OZ_CHUNK = 512;   // K per exact FP32 accumulation of one weight
constexpr size_t OZ_PART_BYTES = 1ull << 30;  // partial tiles per launch

// the pairs (p, q) of weight w = p + q, p ascending
int weight_pairs(int w, uint8_t *pa, uint8_t *pb) {
    for (int p = 0; p <= w; ++p) {
        pa[p] = (uint8_t)p;
        pb[p] = (uint8_t)(w - p);
    }
    return w + 1;
}

// grid rows_pad * nchunk (block b: row b / nchunk, chunk b % nchunk), 256
// threads: one row's chunk.  Element (row, k) is
// src[row * ld + k] (trans: src[k * ld + row]); with kmeta, column k reads
// src[row * ld + kmeta[k]] (kmeta[k] < 0: zero).  Rows >= nrows and columns
// >= K (without kmeta) are zero.  out: [S][rows_pad][ktot_pad] digits,
// ex: [rows_pad][nchunk] chunk exponents.
__device__ __forceinline__ long long abs_bits(double v) {
    return __double_as_longlong(v) & 0x7fffffffffffffffLL;  // ordered like |v| for every double
}

// N = round(v 2^(S*B - e)) (ties away from zero), computed on the integer
// pipe from v's bits: v = m 2^(ev - 1075) with the 53-bit significand m.
__device__ __forceinline__ long long scaled_int(double v, int e) {
    const long long bits = __double_as_longlong(v);
    int ev = (int)((bits >> 52) & 0x7ff);
    long long m = bits & ((1LL << 52) - 1);
    if (ev == 0)
        ev = 1;  // subnormal: no implicit bit
    else
        m |= 1LL << 52;
    const int sh = ev - 1075 + OZ_S * OZ_B - e;  // N = m 2^sh, |N| <= 2^(S*B - 1)
    long long N;
    if (sh >= 0)
        N = m << sh;
    else if (sh > -60)
        N = (m + (1LL << (-sh - 1))) >> (-sh);
    else
        N = 0;
    return bits < 0 ? -N : N;
}

__global__ void __launch_bounds__(256) k_oz_slice(const double *__restrict__ src, long long ld, int nrows, long long K,
                                                  const int *__restrict__ kmeta, int trans, int rows_pad,
                                                  int ktot_pad, int kchunk, int nchunk,
                                                  __nv_bfloat16 *__restrict__ out, int *__restrict__ ex) {
    const int row = (int)(blockIdx.x / nchunk), c = (int)(blockIdx.x % nchunk);
    const int k0 = c * kchunk, kn = min(kchunk, ktot_pad - k0);
    constexpr int PER = OZ_CHUNK / 256;
    double v[PER];
    long long mx = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int kk = threadIdx.x + 256 * j;
        v[j] = 0.0;
        if (kk < kn && row < nrows) {
            const long long k = k0 + kk;
            long long col = kmeta ? (long long)__ldg(kmeta + k) : (k < K ? k : -1);
            if (col >= 0 && FK_DBG(trans ? row < ld : col < ld, 30, col))
                v[j] = trans ? src[col * ld + row] : src[(long long)row * ld + col];
        }
        mx = max(mx, abs_bits(v[j]));
    }
    __shared__ long long red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (long long)__shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) mx = max(mx, red[w]);
    // largest |v| below 2^(ilogb + 1): with e = ilogb + 2 the scaled values
    // stay at or below 2^(S*B - 1), so every digit is at most 2^(B-1) = 64
    const int e = mx > 0 ? ilogb(__longlong_as_double(mx)) + 2 : 0;
    if (threadIdx.x == 0) ex[(size_t)row * nchunk + c] = e;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int kk = threadIdx.x + 256 * j;
        if (kk >= kn) continue;
        long long N = scaled_int(v[j], e);
        // balanced base-2^B digits from the top: each digit rounds the
        // remainder (ties up), which then lies in [-2^(sh-1), 2^(sh-1))
#pragma unroll
        for (int p = 0; p < OZ_S; ++p) {
            const int sh = OZ_B * (OZ_S - 1 - p);
            const long long t = sh ? (N + (1LL << (sh - 1))) >> sh : N;
            N -= t * (1LL << sh);
            if (FK_DBG(row < rows_pad && k0 + kk < ktot_pad && t >= -64 && t <= 64, 31, t))
                out[((size_t)p * rows_pad + row) * ktot_pad + k0 + kk] = __float2bfloat16_rn((float)t);
        }
    }
}

// 2^k as a double (k within the normal range; ldexp outside it)
__device__ __forceinline__ double pow2(int k) {
    return (k >= -1022 && k <= 1023) ? __longlong_as_double((long long)(k + 1023) << 52) : ldexp(1.0, k);
}

// O[r][d] (+)= sum_{c in [c0, c0 + nc)} 2^(ea[r][c] + eb[d][c] - 2 S B + B (2S - 2))
//                 * sum_{w < S} 2^(-B w) P[w][c - c0][r][d],
// chunks in order (accumulate: starting from O).  The partials are exact
// integers (at most 2^24): per chunk the weights 0..3 and 4..7 are gathered
// exactly into two integers, hi = sum_{w<4} P_w 2^(B (3 - w)) and
// lo = sum_{w>=4} P_w 2^(B (7 - w)) (below 2^46 each), and each enters the
// FP64 sum through one fused multiply-add by its power of two.
__global__ void k_oz_combine(const float *__restrict__ P, int c0, int nc, int nchunk, int R, int nd,
                             const int *__restrict__ ea, const int *__restrict__ eb, double *__restrict__ O,
                             int ldo, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * nd) return;
    const int r = (int)(idx / nd), d = (int)(idx - (long long)r * nd);
    double s = accumulate ? O[(size_t)r * ldo + d] : 0.0;
    const size_t plane = (size_t)R * nd;
    for (int c = 0; c < nc; ++c) {
        const int base = __ldg(ea + (size_t)r * nchunk + c0 + c) + __ldg(eb + (size_t)d * nchunk + c0 + c) -
                         2 * OZ_S * OZ_B + OZ_B * (2 * OZ_S - 2);
        long long hi = 0, lo = 0;
#pragma unroll
        for (int w = 0; w < OZ_S / 2; ++w) hi = hi * (1 << OZ_B) + __float2ll_rn(P[((size_t)w * nc + c) * plane + idx]);
#pragma unroll
        for (int w = OZ_S / 2; w < OZ_S; ++w)
            lo = lo * (1 << OZ_B) + __float2ll_rn(P[((size_t)w * nc + c) * plane + idx]);
        s = fma((double)hi, pow2(base - OZ_B * (OZ_S / 2 - 1)), s);
        s = fma((double)lo, pow2(base - OZ_B * (OZ_S - 1)), s);
    }
    O[(size_t)r * ldo + d] = s;
}

// DIS adjoint scatter in FP64: gF[r][a_k][xmap[i]] += W[r][k * nx + i]
__global__ void k_oz_dis_scatter(const double *__restrict__ W, int R, int E, int nx, int nxg,
                                 const int *__restrict__ ca, const int *__restrict__ xmap, double *__restrict__ gF) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * E) return;
    const int r = (int)(idx / E), e = (int)(idx - (long long)r * E);
    const int k = e / nx, i = e - k * nx;
    const int a = __ldg(ca + k), m = __ldg(xmap + i);
    if (FK_DBG(a >= 0 && a < NFL && m >= 0 && m < nxg, 32, e)) gF[((size_t)r * NFL + a) * nxg + m] += W[idx];
}

// Hadronic adjoint from W[r][(c, i, j)] = sum_d gO[r][d] FK[d][c][i][j]:
//   gF[r][a][m] (+)= sum_{c: a_c = a} sum_j W[r][(c, i(m), j)] f^r_{b_c}(x_j)
//                  + sum_{c: b_c = a} sum_i W[r][(c, i, i(m))] f^r_{a_c}(x_i)
// with i(m) the table's x index of grid point m (none: 0); one thread per
// (r, a, m), channels in order (FP64).
__global__ void k_oz_had_grad(const double *__restrict__ W, const double *__restrict__ F, int R, TableView tv,
                              int accumulate, double *__restrict__ gF) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)R * NFL * tv.nxg;
    if (idx >= n) return;
    const int m = (int)(idx % tv.nxg);
    const long long ra = idx / tv.nxg;
    const int a = (int)(ra % NFL), r = (int)(ra / NFL);
    const int i0 = __ldg(tv.xinv + m);
    double s = 0.0;
    if (i0 >= 0) {
        const double *f = F + (size_t)r * NFL * tv.nxg;
        const double *w = W + (size_t)r * tv.E;
        const int nx = tv.nx, nx2 = nx * nx;
        for (int c = 0; c < tv.nch; ++c) {
            const int ac = __ldg(tv.ca + c), bc = __ldg(tv.cb + c);
            if (ac == a) {
                const double *wr = w + (size_t)c * nx2 + (size_t)i0 * nx;
                const double *fb = f + (size_t)bc * tv.nxg;
                for (int j = 0; j < nx; ++j) s = fma(wr[j], fb[__ldg(tv.xmap + j)], s);
            }
            if (bc == a) {
                const double *wc = w + (size_t)c * nx2 + i0;
                const double *fa = f + (size_t)ac * tv.nxg;
                for (int i = 0; i < nx; ++i) s = fma(wc[(size_t)i * nx], fa[__ldg(tv.xmap + i)], s);
            }
        }
    }
    gF[idx] = accumulate ? gF[idx] + s : s;
}

int kchunk_of(int ktot_pad) { return std::min(OZ_CHUNK, ktot_pad); }

// Digit slices of the device FP64 matrix (rows nrows over K; trans: stored
// [K][nrows]) into pack pk (allocated here) with exponents *pe.
int oz_pack(fk_table *t, TcPack &pk, int **pe, int *pkchunk, const double *d_src, long long ld, int trans,
            int nrows, long long K, const std::vector<int> &km, cudaStream_t s) {
    pk.n_rows = std::min(256, (nrows + 15) / 16 * 16);
    pk.ntile_n = (nrows + pk.n_rows - 1) / pk.n_rows;
    pk.ktot = (int)((K + 127) / 128 * 128);
    pk.ktot_pad = pk.ktot;
    const int kchunk = kchunk_of(pk.ktot_pad);
    const int nchunk = (pk.ktot_pad + kchunk - 1) / kchunk;
    *pkchunk = kchunk;
    const long long rows = (long long)pk.ntile_n * pk.n_rows;
    const size_t elems = (size_t)OZ_S * rows * pk.ktot_pad;
    if (cudaMalloc(&pk.hi, elems * 2) || cudaMalloc(pe, sizeof(int) * rows * nchunk))
        return fail(FK_ENOMEM, "FP64 tensor-core table slices");
    t->bytes += elems * 2 + sizeof(int) * rows * nchunk;
    if (!km.empty()) {
        std::vector<int> kmp(pk.ktot_pad, -1);
        std::copy(km.begin(), km.end(), kmp.begin());
        if (cudaMalloc(&pk.kmeta, sizeof(int) * kmp.size())) return fail(FK_ENOMEM, "FP64 tensor-core gather map");
        FK_CUDA(cudaMemcpy(pk.kmeta, kmp.data(), sizeof(int) * kmp.size(), cudaMemcpyHostToDevice));
        t->bytes += sizeof(int) * kmp.size();
    }
    if (rows * nchunk > 0x7fffffffLL) return fail(FK_EINVAL, "FP64 tensor-core slicing: table too large");
    k_oz_slice<<<(unsigned)(rows * nchunk), 256, 0, s>>>(d_src, ld, nrows, K, nullptr, trans, (int)rows, pk.ktot_pad,
                                                         kchunk, nchunk, pk.hi, *pe);
    count_launch();
    FK_CUDA(cudaGetLastError());
    int rc = tc_map_bf16(&pk.map_hi, pk.hi, pk.ktot_pad, OZ_S * rows, pk.n_rows);
    if (!rc) rc = tc_map_bf16(&pk.half_hi, pk.hi, pk.ktot_pad, OZ_S * rows, pk.n_rows / 2);
    return rc;
}

// O (+)= A B^T through the slices: A rows from src (R rows, ld, kmeta / K as
// in k_oz_slice), B = pack pk with exponents pe; O [R][nd_out] FP64 (ldo).
int oz_run(const fk_table *t, const TcPack &pk, const int *pe, int kchunk, const double *A, long long lda,
           const int *kmeta, long long K, int R, int nd_out, double *O, int ldo, int accumulate, cudaStream_t s) {
    const int R_pad = (R + 127) / 128 * 128;
    const int nchunk = (pk.ktot_pad + kchunk - 1) / kchunk;
    Scratch scr(s);
    __nv_bfloat16 *Aoz = nullptr;
    int *ea = nullptr;
    FK_CUDA(scr.get(&Aoz, (size_t)OZ_S * R_pad * pk.ktot_pad));
    FK_CUDA(scr.get(&ea, (size_t)R_pad * nchunk));
    if ((long long)R_pad * nchunk > 0x7fffffffLL) return fail(FK_EINVAL, "FP64 tensor-core mode: R x K too large");
    k_oz_slice<<<(unsigned)((long long)R_pad * nchunk), 256, 0, s>>>(A, lda, R, K, kmeta, 0, R_pad, pk.ktot_pad,
                                                                      kchunk, nchunk, Aoz, ea);
    count_launch();
    FK_CUDA(cudaGetLastError());
    CUtensorMap mA;
    int rc = tc_map_bf16(&mA, Aoz, pk.ktot_pad, (long long)OZ_S * R_pad, 128);
    if (rc) return rc;
    // chunks per launch: the 8 weight partials of a chunk within OZ_PART_BYTES
    const size_t per_chunk = (size_t)OZ_S * R * nd_out * sizeof(float);
    const int cb = (int)std::max<size_t>(1, std::min<size_t>(nchunk, OZ_PART_BYTES / std::max<size_t>(per_chunk, 1)));
    float *P = nullptr;
    FK_CUDA(scr.get(&P, (size_t)cb * OZ_S * R * nd_out));
    for (int c0 = 0; c0 < nchunk; c0 += cb) {
        const int nc = std::min(cb, nchunk - c0);
        for (int w = 0; w < OZ_S; ++w) {  // one launch per weight: its w + 1 pairs in one accumulator
            uint8_t pa[OZ_S], pb[OZ_S];
            const int npc = weight_pairs(w, pa, pb);
            rc = tc_slice_pairs(t, pk, mA, R, nd_out, kchunk, c0, nc, 1, npc, pa, pb,
                                P + (size_t)w * nc * R * nd_out, s);
            if (rc) return rc;
        }
        const long long n = (long long)R * nd_out;
        k_oz_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, c0, nc, nchunk, R, nd_out, ea, pe, O, ldo,
                                                                 accumulate || c0 > 0);
        count_launch();
        FK_CUDA(cudaGetLastError());
    }
    return FK_OK;
}

}  // namespace

FK_DBG_READER(dbg_oz)

int oz_build(fk_table *t, const double *host_fk) {
    TcLayout &L = t->tc;
    const long long E = t->E;
    double *d = nullptr;
    cudaStream_t s = nullptr;
    FK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    if (cudaMalloc(&d, sizeof(double) * (size_t)t->ndata * E)) {
        cudaStreamDestroy(s);
        return fail(FK_ENOMEM, "FP64 tensor-core slicing staging");
    }
    int rc = FK_OK;
    cudaError_t e = cudaMemcpyAsync(d, host_fk, sizeof(double) * (size_t)t->ndata * E, cudaMemcpyHostToDevice, s);
    if (e) rc = cuda_fail(e, "FP64 tensor-core table upload");
    std::vector<int> km;
    if (!rc && t->kind == FK_KIND_DIS) {  // forward A operand: F[r][a_k][xmap[i]]
        km.resize(E);
        for (long long k = 0; k < E; ++k) km[k] = t->ca[k / t->nx] * t->nxg + t->xmap[k % t->nx];
    }
    if (!rc) rc = oz_pack(t, L.oz, &L.oz_e, &L.oz_kchunk, d, E, 0, t->ndata, E, km, s);
    if (!rc && t->kind != FK_KIND_DENSE)  // adjoint: rows over the table's columns, K = data points
        rc = oz_pack(t, L.ozT, &L.ozT_e, &L.ozT_kchunk, d, E, 1, (int)E, t->ndata, {}, s);
    if (!rc) {
        e = cudaStreamSynchronize(s);
        if (e) rc = cuda_fail(e, "FP64 tensor-core table slicing");
    }
    cudaFree(d);
    cudaStreamDestroy(s);
    return rc;
}

void oz_free(fk_table *t) {
    TcLayout &L = t->tc;
    for (TcPack *pk : {&L.oz, &L.ozT}) {
        cudaFree(pk->hi);
        cudaFree(pk->kmeta);
        pk->hi = nullptr;
        pk->kmeta = nullptr;
    }
    cudaFree(L.oz_e);
    cudaFree(L.ozT_e);
    L.oz_e = L.ozT_e = nullptr;
}

int oz_dense(const fk_table *t, const double *Lm, int R, double *O, int ldo, cudaStream_t s) {
    const TcLayout &L = t->tc;
    return oz_run(t, L.oz, L.oz_e, L.oz_kchunk, Lm, t->E, nullptr, t->E, R, t->ndata, O, ldo, 0, s);
}

int oz_dis(const fk_table *t, const double *F, int R, double *O, int ldo, cudaStream_t s) {
    const TcLayout &L = t->tc;
    return oz_run(t, L.oz, L.oz_e, L.oz_kchunk, F, (long long)NFL * t->nxg, L.oz.kmeta, t->E, R, t->ndata, O, ldo,
                  0, s);
}

int oz_had(const fk_table *t, const double *F, int R, double *O, int ldo, cudaStream_t s) {
    const TcLayout &L = t->tc;
    Scratch scr(s);
    double *Lm = nullptr;
    FK_CUDA(scr.get(&Lm, (size_t)R * t->E));
    int rc = luminosity_cc(t, F, R, Lm, true, s);
    if (rc) return rc;
    return oz_run(t, L.oz, L.oz_e, L.oz_kchunk, Lm, t->E, nullptr, t->E, R, t->ndata, O, ldo, 0, s);
}

int oz_bwd(const fk_table *t, const double *F, const double *gO, int ldgo, int R, double *gF, int accumulate,
           cudaStream_t s) {
    const TcLayout &L = t->tc;
    const int E = (int)t->E;
    Scratch scr(s);
    double *W = nullptr;
    FK_CUDA(scr.get(&W, (size_t)R * E));
    int rc = oz_run(t, L.ozT, L.ozT_e, L.ozT_kchunk, gO, ldgo, nullptr, t->ndata, R, E, W, E, 0, s);
    if (rc) return rc;
    if (t->kind == FK_KIND_DIS) {
        if (!accumulate) FK_CUDA(cudaMemsetAsync(gF, 0, sizeof(double) * (size_t)R * NFL * t->nxg, s));
        const long long n = (long long)R * E;
        k_oz_dis_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, R, E, t->nx, t->nxg, t->d_ca, t->d_xmap, gF);
    } else {
        const long long n = (long long)R * NFL * t->nxg;
        k_oz_had_grad<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, F, R, view(t), accumulate, gF);
    }
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

}  // namespace fk
