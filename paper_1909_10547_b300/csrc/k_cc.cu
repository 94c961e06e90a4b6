// CUDA-core kernels of the FK convolution in FP64 and FP32.
//
//  * k_stream : one replica (hadronic) or R <= 4 (DIS).  The observable is a dot product of the
//    table row FK[d][.] with the weight vector w[e] (hadronic, Eq. 1:
//    w[(c,i,j)] = f_{a_c}(x_i) f_{b_c}(x_j); DIS: w[(k,i)] = f_{a_k}(x_i)).
//    The table is streamed once with 16-byte loads; each CTA owns an element
//    chunk, keeps its weights in registers and reuses them over DB data points.
//  * k_fac    : hadronic, R >= 2.  Eq. 1 factorised per channel and x_i of
//    its first flavour: a register-blocked product over x_j with the second
//    flavour's PDF, folded into O with the first flavour's PDF; table rows
//    staged by TMA.
//  * k_tile   : DIS, R > 4.  O[d][r] = sum_k FK[d][k] F[r][k] as a tiled
//    product (K = active flavour x point).
//  * k_bwd_*  : the adjoint.  W[e][r] = sum_d FK[d][e] gO[r][d] is formed per
//    tile, then contracted with the PDF of the other flavour of the channel
//    (product rule on each term of Eq. 1).
//
// Reductions across CTAs never use atomics: every CTA writes its partial sums
// to its own slot and a second kernel adds the slots in a fixed order, so the
// result of a (d, r) pair does not depend on R, on the launch shape of other
// replicas or on timing.
#include "fk_internal.h"

#include <algorithm>
#include <mutex>
#include <set>

namespace fk {

__device__ int g_fk_cc_error;  // non-zero after a bounded wait of k_fac ran out

namespace {

template <typename T>
struct V16;
template <>
struct V16<float> {
    using t = float4;
    static constexpr int n = 4;
};
template <>
struct V16<double> {
    using t = double2;
    static constexpr int n = 2;
};

__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2 *p) { return __ldcs(p); }

__device__ __forceinline__ float dotv(float4 x, const float *w, float acc) {
    acc = fmaf(x.x, w[0], acc);
    acc = fmaf(x.y, w[1], acc);
    acc = fmaf(x.z, w[2], acc);
    return fmaf(x.w, w[3], acc);
}
__device__ __forceinline__ double dotv(double2 x, const double *w, double acc) {
    acc = fma(x.x, w[0], acc);
    return fma(x.y, w[1], acc);
}

template <typename T>
struct SmemPdf {
    T f[NFL * MAX_NXG];
    int ca[MAX_CH], cb[MAX_CH], xm[MAX_NX];
};

template <int KIND, typename T>
__device__ __forceinline__ T elem_weight(const SmemPdf<T> &s, long long e, const TableView &tv,
                                         int nx2) {
    if (e >= tv.E) return T(0);
    const int ei = (int)e;
    if (KIND == FK_KIND_HAD) {
        const int c = ei / nx2;
        const int rem = ei - c * nx2;
        const int i = rem / tv.nx;
        const int j = rem - i * tv.nx;
        return s.f[s.ca[c] * tv.nxg + s.xm[i]] * s.f[s.cb[c] * tv.nxg + s.xm[j]];
    } else {
        const int k = ei / tv.nx;
        const int i = ei - k * tv.nx;
        return s.f[s.ca[k] * tv.nxg + s.xm[i]];
    }
}

template <typename T>
struct StreamCfg;
template <>
struct StreamCfg<float> {
    static constexpr int U = 4, DB = 8;
};
template <>
struct StreamCfg<double> {
    static constexpr int U = 8, DB = 16;
};

// grid (nchunk, ceil(ndata/DB), R); part[(chunk * R + r) * ndata + d]
template <int KIND, typename T>
__global__ void __launch_bounds__(256) k_stream(TableView tv, const T *__restrict__ fk,
                                                const T *__restrict__ F, int R,
                                                T *__restrict__ part) {
    using VT = typename V16<T>::t;
    constexpr int V = V16<T>::n;
    constexpr int U = StreamCfg<T>::U, DB = StreamCfg<T>::DB;
    constexpr int CH = 256 * V * U;
    __shared__ SmemPdf<T> s;
    __shared__ T red[DB][256];
    const int r = blockIdx.z;
    if constexpr (KIND != FK_KIND_DENSE) {
        const T *Fr = F + (size_t)r * NFL * tv.nxg;
        for (int k = threadIdx.x; k < NFL * tv.nxg; k += 256) s.f[k] = Fr[k];
        for (int k = threadIdx.x; k < tv.nch; k += 256) {
            s.ca[k] = tv.ca[k];
            if (KIND == FK_KIND_HAD) s.cb[k] = tv.cb[k];
        }
        for (int k = threadIdx.x; k < tv.nx; k += 256) s.xm[k] = tv.xmap[k];
    }
    __syncthreads();

    const int nx2 = tv.nx * tv.nx;
    const long long e0 = (long long)blockIdx.x * CH + threadIdx.x * V;
    T w[U][V];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const long long e = e0 + u * 256 * V + v;
            if constexpr (KIND == FK_KIND_DENSE)  // the PDF matrix row of replica r (F is [R][E])
                w[u][v] = e < tv.E ? __ldg(F + (size_t)r * tv.E + e) : T(0);
            else
                w[u][v] = elem_weight<KIND>(s, e, tv, nx2);
        }

    const int d0 = blockIdx.y * DB;
    T acc[DB];
#pragma unroll
    for (int dd = 0; dd < DB; ++dd) {
        acc[dd] = T(0);
        const int d = d0 + dd;
        if (d < tv.ndata) {
            const T *row = fk + (size_t)d * tv.ldE;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long e = e0 + u * 256 * V;
                if (e < tv.ldE) acc[dd] = dotv(ld_stream(reinterpret_cast<const VT *>(row + e)), w[u], acc[dd]);
            }
        }
    }
#pragma unroll
    for (int dd = 0; dd < DB; ++dd) red[dd][threadIdx.x] = acc[dd];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int dd = warp; dd < DB; dd += 8) {
        T v = T(0);
#pragma unroll
        for (int k = 0; k < 8; ++k) v += red[dd][lane + 32 * k];
#pragma unroll
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        const int d = d0 + dd;
        if (lane == 0 && d < tv.ndata)
            if (FK_DBG(r < R && d < tv.ndata, 1, d)) part[((size_t)blockIdx.x * R + r) * tv.ndata + d] = v;
    }
}

// O[r][d] = sum_k part[(k * R + r) * ndata + d] in a fixed order: k
// ascending when there are few parts; with WIDE_PARTS or more (long rows
// streamed by many chunks, e.g. a dense table with K = 10^7) one warp per
// output, lane l adding parts l, l + 32, ... and a butterfly sum of the lanes,
// so that the loads of all parts are in flight together.  The order depends
// only on nparts, a property of the table.
constexpr int WIDE_PARTS = 64;
template <typename T>
__global__ void k_reduce_parts(const T *__restrict__ part, int nparts, int ndata, int R,
                               T *__restrict__ O, int ldo) {
    const long long n = (long long)R * ndata;
    if (nparts >= WIDE_PARTS) {
        const long long idx = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
        const int lane = threadIdx.x & 31;
        if (idx >= n) return;  // whole warps leave together
        const T *p = part + idx;
        T s = T(0);
        for (int k = lane; k < nparts; k += 32) s += p[(size_t)k * n];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const long long r = idx / ndata, d = idx - r * ndata;
        if (lane == 0 && FK_DBG(r < R && d < ndata && d < ldo, 2, idx)) O[r * ldo + d] = s;
        return;
    }
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const T *p = part + idx;
    T s = T(0);
    for (int k = 0; k < nparts; ++k) s += p[(size_t)k * n];
    const long long r = idx / ndata, d = idx - r * ndata;
    if (FK_DBG(r < R && d < ndata && d < ldo, 2, idx)) O[r * ldo + d] = s;
}

// launch of k_reduce_parts (one thread or one warp per output)
template <typename T>
int reduce_parts(const T *part, int nparts, int ndata, int R, T *O, int ldo, cudaStream_t s) {
    const long long n = (long long)R * ndata;
    const long long threads = nparts >= WIDE_PARTS ? n * 32 : n;
    k_reduce_parts<T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(part, nparts, ndata, R, O, ldo);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// ----------------------------------------------------------------------------
// DIS many-replica tile kernel: O[d][r] = sum_k FK[d][k] F[r][k] over the
// compacted (active flavour, x) index k, a plain product tiled 64 x 64 (data
// points x replicas), the K range split over the grid's z dimension.
// grid (ceil(ndata/64), ceil(R/64), nsplit); part[(split * R + r) * ndata + d]
// ----------------------------------------------------------------------------
template <typename T>
struct TileCfg;
template <>
struct TileCfg<float> {
    static constexpr int KC = 32;
};
template <>
struct TileCfg<double> {
    static constexpr int KC = 16;
};
constexpr int TDT = 64, TRT = 64;

template <typename T>
constexpr size_t tile_smem() {
    return sizeof(T) * (TileCfg<T>::KC * (TDT + 1) + TileCfg<T>::KC * TRT) + sizeof(int) * (MAX_CH + MAX_NX);
}

template <typename T, bool DENSE>
__global__ void __launch_bounds__(256) k_tile(TableView tv, const T *__restrict__ fk,
                                              const T *__restrict__ F, int R, int nsplit,
                                              T *__restrict__ part) {
    constexpr int KC = TileCfg<T>::KC;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Bs = reinterpret_cast<T *>(smem_raw);  // [KC][TRT]
    T *As = Bs + KC * TRT;                    // [KC][TDT + 1]
    int *sfl = reinterpret_cast<int *>(As + KC * (TDT + 1));  // active flavours
    int *sxm = sfl + MAX_CH;

    const int d0 = blockIdx.x * TDT, r0 = blockIdx.y * TRT, sp = blockIdx.z;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int k = threadIdx.x; k < tv.nch; k += 256) sfl[k] = tv.ca[k];
    for (int k = threadIdx.x; k < tv.nx; k += 256) sxm[k] = tv.xmap[k];

    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = T(0);

    const size_t fstride = (size_t)NFL * tv.nxg;
    // this split's range of K, in whole KC chunks
    const long long nk = (tv.E + KC - 1) / KC;
    const long long el_b = nk * sp / nsplit * KC;
    const long long el_e = min(tv.E, nk * (sp + 1) / nsplit * KC);
    __syncthreads();
    for (long long k0 = el_b; k0 < el_e; k0 += KC) {
        for (int idx = threadIdx.x; idx < KC * TDT; idx += 256) {
            const int kk = idx % KC, dd = idx / KC;
            const int d = d0 + dd;
            T v = T(0);
            if (d < tv.ndata && k0 + kk < el_e) v = fk[(size_t)d * tv.ldE + k0 + kk];
            As[kk * (TDT + 1) + dd] = v;
        }
        for (int idx = threadIdx.x; idx < KC * TRT; idx += 256) {
            const int rr = idx % TRT, kk = idx / TRT;
            T v = T(0);
            if (k0 + kk < el_e && r0 + rr < R) {
                if constexpr (DENSE) {  // the PDF matrix, [R][E]
                    v = F[(size_t)(r0 + rr) * tv.E + k0 + kk];
                } else {
                    const int e = (int)(k0 + kk);
                    const int kf = e / tv.nx, i = e - kf * tv.nx;
                    v = F[(size_t)(r0 + rr) * fstride + sfl[kf] * tv.nxg + sxm[i]];
                }
            }
            Bs[kk * TRT + rr] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KC; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) a[p] = As[kk * (TDT + 1) + ty * 4 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Bs[kk * TRT + tx * 4 + q];
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int d = d0 + ty * 4 + p, r = r0 + tx * 4 + q;
            if (d < tv.ndata && r < R) part[((size_t)sp * R + r) * tv.ndata + d] = acc[p][q];
        }
}

// ----------------------------------------------------------------------------
// Factorised many-replica kernel (hadronic, R >= 2).  Eq. 1 per channel c and
// x point x_i of its first flavour:
//   O[d][r] = sum_c sum_i f_{a_c}(x_i)[r] * Y_ci[d][r],
//   Y_ci[d][r] = sum_j FK[d][c][i][j] f_{b_c}(x_j)[r].
// A CTA owns FAC_TDT data points x TRT replicas and the channels of its split.
// Y is a register-blocked product (each thread TM data points x TN replicas,
// K = the nx points x_j).  The FK rows of step (c, i) arrive by one TMA copy
// of a FAC_TDT x W box (W >= nx + the 16-byte alignment remainder), NBUF
// boxes in flight on their mbarriers so that later steps' copies overlap this
// step's products; the two PDF columns of the channel are staged once per
// channel.
// The table is read once per replica tile.
// grid (ceil(ndata / FAC_TDT), ceil(R / TRT), nsplit);
// part[(split * R + r) * ndata + d] as for k_tile.
// ----------------------------------------------------------------------------
constexpr int FAC_TDT = 128;

template <typename T, int TRT>
struct FacCfg {
    static constexpr int TN = sizeof(T) == 4 ? 4 : 2;  // replicas per thread
    static constexpr int RT = TRT / TN;                 // threads along replicas
    static constexpr int DT = 256 / RT;                 // threads along data points
    static constexpr int TM = FAC_TDT / DT;             // data points per thread: td + m * DT
    // table boxes in flight (three measured slower than two for R <= 16:
    // fewer CTAs fit per SM)
    static constexpr int NBUF = 2;
    static_assert(RT * DT == 256 && TM * DT == FAC_TDT, "tile shape");
};

// Box width W of the staged rows: covers nx elements from any start, is a
// multiple of 16 bytes (a TMA box row), and W = 4 (mod 8) so that the rows
// td, td+1, ... a warp reads at one x_j fall in different banks.
__host__ __device__ constexpr int fac_width(int nx, int esz) {
    const int e16 = 16 / esz;
    int w = nx + e16 - 1;
    w = (w + e16 - 1) / e16 * e16;
    while (w % 8 != 4) w += e16;
    return w;
}

// rows of the staged second-flavour PDF column: x points -FAC_PAD .. nx + 2 FAC_PAD
// (zero outside [0, nx)), so that a box column j' reads the PDF of x point
// j' - rem (rem < 16 bytes' worth of elements) without bounds tests
constexpr int FAC_PAD = 4;

template <typename T, int TRT>
size_t fac_smem(int nx) {
    // 1024 for alignment of the TMA destination, the boxes, the two PDF columns
    return 1024 + sizeof(T) * (FacCfg<T, TRT>::NBUF * (size_t)FAC_TDT * fac_width(nx, sizeof(T)) + (size_t)nx * TRT +
                               (size_t)(nx + 3 * FAC_PAD) * TRT);
}

// N consecutive values from shared memory in 16-byte loads
template <typename T, int N>
__device__ __forceinline__ void lds_vec(const T *p, T (&v)[N]) {
    static_assert((N * sizeof(T)) % 16 == 0, "16-byte multiples");
#pragma unroll
    for (int k = 0; k < N * (int)sizeof(T) / 16; ++k) {
        const float4 q = reinterpret_cast<const float4 *>(p)[k];
        memcpy(&v[k * 16 / sizeof(T)], &q, 16);
    }
}

// 2 s per wait; a thread whose wait ran out stops waiting (dead) and raises
// g_fk_cc_error, read by fk_device_status
constexpr unsigned long long FAC_WAIT_NS = 2000000000ull;
__device__ __forceinline__ unsigned long long cc_gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool cc_mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

template <typename T, int TRT>
__global__ void __launch_bounds__(256) k_fac(const __grid_constant__ CUtensorMap map, TableView tv,
                                             const T *__restrict__ F, int R, int nsplit,
                                             T *__restrict__ part) {
    using C = FacCfg<T, TRT>;
    constexpr int TM = C::TM, TN = C::TN, E16 = 16 / (int)sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NB = C::NBUF;
    __shared__ __align__(8) uint64_t bars[NB];
    const int nx = tv.nx, W = fac_width(nx, sizeof(T));
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smem_raw);
    const uint32_t abase = (raw + 1023u) & ~1023u;
    T *As = reinterpret_cast<T *>(smem_raw + (abase - raw));  // [NB][FAC_TDT][W]
    T *Fa = As + NB * FAC_TDT * W;                               // [nx][TRT]
    T *Fb = Fa + nx * TRT;                                       // [nx + 3 FAC_PAD][TRT], row j + FAC_PAD
    const uint32_t box_bytes = (uint32_t)(FAC_TDT * W * sizeof(T));
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);

    const int d0 = blockIdx.x * FAC_TDT, r0 = blockIdx.y * TRT, sp = blockIdx.z;
    const int tr = threadIdx.x % C::RT, td = threadIdx.x / C::RT;
    const int c_b = (int)((long long)tv.nch * sp / nsplit);
    const int c_e = (int)((long long)tv.nch * (sp + 1) / nsplit);
    const int nsteps = (c_e - c_b) * nx;
    const size_t fstride = (size_t)NFL * tv.nxg;

    if (threadIdx.x == 0) {
        for (int b = 0; b < NB; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&map) : "memory");
    }
    __syncthreads();
    // first K element of step s, rounded down to 16 bytes (the box origin)
    auto step_off = [&](int s_) {
        const int c = c_b + s_ / nx, i = s_ - (s_ / nx) * nx;
        return ((long long)c * nx + i) * nx;
    };
    // thread 0: copy the rows of step s into buffer buf
    auto stage = [&](int s_, int buf) {
        const long long off = step_off(s_);
        const int x0 = (int)(off - off % E16);
        const uint32_t bar = bar0 + 8u * buf;
        const uint32_t dst = abase + (uint32_t)buf * box_bytes;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(box_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
            "l"((uint64_t)&map), "r"(bar), "r"(x0), "r"(d0)
            : "memory");
    };

    T acc[TM][TN];
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) acc[m][n] = T(0);

    bool dead = false;
    int issued = 0;  // copies issued by thread 0
    if (threadIdx.x == 0)
        for (; issued < NB - 1 && issued < nsteps; ++issued) stage(issued, issued);
    int cur_c = -1;
    for (int s_ = 0; s_ < nsteps; ++s_) {
        const int buf = s_ % NB;
        const uint32_t par = (uint32_t)(s_ / NB) & 1u;  // phase s / NB of its buffer's barrier
        const int c = c_b + s_ / nx, i = s_ - (s_ / nx) * nx;
        if (c != cur_c) {
            // new channel: its two PDF columns (every thread is past the
            // previous channel's last step: the barrier that ended it)
            const int fa = tv.ca[c], fb = tv.cb[c];
            for (int idx = threadIdx.x; idx < nx * TRT; idx += 256) {
                const int k = idx / TRT, rr = idx - k * TRT;
                const int r = r0 + rr;
                Fa[idx] = r < R ? F[(size_t)r * fstride + fa * tv.nxg + tv.xmap[k]] : T(0);
            }
            for (int idx = threadIdx.x; idx < (nx + 3 * FAC_PAD) * TRT; idx += 256) {
                const int k = idx / TRT - FAC_PAD, rr = idx % TRT;
                const int r = r0 + rr;
                Fb[idx] = (r < R && k >= 0 && k < nx) ? F[(size_t)r * fstride + fb * tv.nxg + tv.xmap[k]] : T(0);
            }
            cur_c = c;
        }
        // step s + NB - 1 streams in while this one computes (its buffer,
        // that of step s - 1, was released by the barrier ending step s - 1)
        if (threadIdx.x == 0 && s_ + NB - 1 < nsteps && !dead) {
            stage(s_ + NB - 1, (s_ + NB - 1) % NB);
            ++issued;
        }
        __syncthreads();  // Fa/Fb written
        // wait for this step's box (phase s/2 of its buffer's barrier)
        if (!dead && !cc_mbar_try(bar0 + 8u * buf, par)) {
            const unsigned long long t0 = cc_gtimer();
            while (!cc_mbar_try(bar0 + 8u * buf, par)) {
                if (cc_gtimer() - t0 > FAC_WAIT_NS) {
                    dead = true;
                    atomicExch(&g_fk_cc_error, 1);
                    break;
                }
            }
        }
        if (!dead) {
            // box column j' holds x point j' - rem; columns outside [rem, rem + nx)
            // meet zero PDF rows.  JV columns per 16-byte load of a row.
            constexpr int JV = 16 / (int)sizeof(T);
            const int rem = (int)(step_off(s_) % E16);
            const int ncol = (rem + nx + JV - 1) / JV * JV;
            const T *A = As + buf * FAC_TDT * W + td * W;  // this step's box
            const T *B = Fb + (FAC_PAD - rem) * TRT + tr * TN;
            T y[TM][TN];
#pragma unroll
            for (int m = 0; m < TM; ++m)
#pragma unroll
                for (int n = 0; n < TN; ++n) y[m][n] = T(0);
            for (int j = 0; j < ncol; j += JV) {
                T a[TM][JV], b[JV][TN];
#pragma unroll
                for (int m = 0; m < TM; ++m) lds_vec<T, JV>(A + m * C::DT * W + j, a[m]);
#pragma unroll
                for (int jj = 0; jj < JV; ++jj) lds_vec<T, TN>(B + (j + jj) * TRT, b[jj]);
#pragma unroll
                for (int jj = 0; jj < JV; ++jj)
#pragma unroll
                    for (int m = 0; m < TM; ++m)
#pragma unroll
                        for (int n = 0; n < TN; ++n) y[m][n] = fma(a[m][jj], b[jj][n], y[m][n]);
            }
            T f[TN];
            lds_vec<T, TN>(Fa + i * TRT + tr * TN, f);
#pragma unroll
            for (int n = 0; n < TN; ++n)
#pragma unroll
                for (int m = 0; m < TM; ++m) acc[m][n] = fma(f[n], y[m][n], acc[m][n]);
        }
        // buffer buf and (at a channel change) Fa/Fb are rewritten next
        __syncthreads();
    }
    if (threadIdx.x == 0 && dead) {
        // let the copies already issued land before the CTA exits
        for (int k = (issued > NB ? issued - NB : 0); k < issued; ++k) {
            const unsigned long long t0 = cc_gtimer();
            while (!cc_mbar_try(bar0 + 8u * (k % NB), (uint32_t)(k / NB) & 1u) && cc_gtimer() - t0 < FAC_WAIT_NS) {
            }
        }
    }
#pragma unroll
    for (int m = 0; m < TM; ++m)
#pragma unroll
        for (int n = 0; n < TN; ++n) {
            const int d = d0 + td + m * C::DT, r = r0 + tr * TN + n;
            if (d < tv.ndata && r < R) part[((size_t)sp * R + r) * tv.ndata + d] = acc[m][n];
        }
}

// ----------------------------------------------------------------------------
// Adjoint.  W[e][r] = sum_d FK[d][e] gO[r][d] over a tile of 128 elements x 64
// replicas, K = data points.
// ----------------------------------------------------------------------------
constexpr int BET = 128, BRT = 64, BKD = 16;

template <typename T>
constexpr size_t bwd_smem() {
    // As [BKD][BET], Gs [BKD][BRT], then Ws [BET][BRT+1] reuses As/Gs, plus
    // Fa, Fb [MAX_NX][BRT]
    size_t ab = sizeof(T) * (BKD * BET + BKD * BRT);
    size_t w = sizeof(T) * BET * (BRT + 1);
    return (ab > w ? ab : w) + sizeof(T) * 2 * MAX_NX * BRT;
}

// Accumulates the W tile for rows [e_b, e_b + rows) of the table, replicas
// [r0, r0 + 64), data points [d_b, d_e), into acc (thread (ty, tx) holds rows
// ty*8.., replicas tx*4..).
template <typename T>
__device__ __forceinline__ void bwd_w_tile(const TableView &tv, const T *__restrict__ fk,
                                           const T *__restrict__ gO, int ldgo, int R, long long e_b,
                                           int rows, int r0, int d_b, int d_e, T *As, T *Gs,
                                           T (&acc)[8][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int dk = d_b; dk < d_e; dk += BKD) {
        for (int idx = threadIdx.x; idx < BKD * BET; idx += 256) {
            const int e = idx % BET, kd = idx / BET;
            const int d = dk + kd;
            T v = T(0);
            if (d < d_e && e < rows) v = fk[(size_t)d * tv.ldE + e_b + e];
            As[kd * BET + e] = v;
        }
        for (int idx = threadIdx.x; idx < BKD * BRT; idx += 256) {
            const int kd = idx % BKD, rr = idx / BKD;
            const int d = dk + kd, r = r0 + rr;
            T v = T(0);
            if (d < d_e && r < R) v = gO[(size_t)r * ldgo + d];
            Gs[kd * BRT + rr] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kd = 0; kd < BKD; ++kd) {
            T a[8], b[4];
#pragma unroll
            for (int p = 0; p < 8; ++p) a[p] = As[kd * BET + ty * 8 + p];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = Gs[kd * BRT + tx * 4 + q];
#pragma unroll
            for (int p = 0; p < 8; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
}

// Hadronic: grid (niblk, ceil(R/64), nch).  Each CTA covers rows i in
// [i0, i0+ib) of channel c (ib*nx <= 128 contiguous elements).
//   U[(c*R + r)*nx + i]              = sum_j W[c,i,j][r] f^r_{b_c}(x_j)
//   Vp[((c*niblk + blk)*R + r)*nx + j] = sum_{i in blk} W[c,i,j][r] f^r_{a_c}(x_i)
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_had(TableView tv, const T *__restrict__ fk,
                                                 const T *__restrict__ F,
                                                 const T *__restrict__ gO, int ldgo, int R,
                                                 int IB, T *__restrict__ U, T *__restrict__ Vp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    size_t ab = sizeof(T) * (BKD * BET + BKD * BRT), w = sizeof(T) * BET * (BRT + 1);
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Gs = As + BKD * BET;
    T *Ws = As;
    T *Fa = reinterpret_cast<T *>(smem_raw + (ab > w ? ab : w));
    T *Fb = Fa + MAX_NX * BRT;
    const int blk = blockIdx.x, r0 = blockIdx.y * BRT, c = blockIdx.z;
    const int niblk = gridDim.x;
    const int i0 = blk * IB;
    const int ib = min(IB, tv.nx - i0);
    const int rows = ib * tv.nx;
    const int nx2 = tv.nx * tv.nx;
    const int fa = tv.ca[c], fb = tv.cb[c];
    const size_t fstride = (size_t)NFL * tv.nxg;
    for (int idx = threadIdx.x; idx < tv.nx * BRT; idx += 256) {
        const int i = idx / BRT, rr = idx - i * BRT;
        const int r = r0 + rr;
        T va = T(0), vb = T(0);
        if (r < R) {
            const int x = tv.xmap[i];
            va = F[(size_t)r * fstride + fa * tv.nxg + x];
            vb = F[(size_t)r * fstride + fb * tv.nxg + x];
        }
        Fa[idx] = va;
        Fb[idx] = vb;
    }
    T acc[8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
    bwd_w_tile<T>(tv, fk, gO, ldgo, R, (long long)c * nx2 + (long long)i0 * tv.nx, rows, r0, 0, tv.ndata,
                  As, Gs, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) Ws[(ty * 8 + p) * (BRT + 1) + tx * 4 + q] = acc[p][q];
    __syncthreads();
    for (int idx = threadIdx.x; idx < ib * BRT; idx += 256) {
        const int il = idx / BRT, rr = idx - il * BRT;
        const int r = r0 + rr;
        T s = T(0);
        for (int j = 0; j < tv.nx; ++j) s = fma(Ws[(il * tv.nx + j) * (BRT + 1) + rr], Fb[j * BRT + rr], s);
        if (r < R) U[((size_t)c * R + r) * tv.nx + i0 + il] = s;
    }
    for (int idx = threadIdx.x; idx < tv.nx * BRT; idx += 256) {
        const int j = idx / BRT, rr = idx - j * BRT;
        const int r = r0 + rr;
        T s = T(0);
        for (int il = 0; il < ib; ++il)
            s = fma(Ws[(il * tv.nx + j) * (BRT + 1) + rr], Fa[(i0 + il) * BRT + rr], s);
        if (r < R) Vp[(((size_t)c * niblk + blk) * R + r) * tv.nx + j] = s;
    }
}

// gF[r][a][m] (+)= sum_{c: ca=a} U[c][r][i(m)] + sum_{c: cb=a} sum_blk Vp[c][blk][r][i(m)]
template <typename T>
__global__ void k_bwd_had_gather(TableView tv, const T *__restrict__ U, const T *__restrict__ Vp,
                                 int R, int niblk, int accumulate, T *__restrict__ gF) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)R * NFL * tv.nxg;
    if (idx >= n) return;
    const int m = (int)(idx % tv.nxg);
    const int a = (int)((idx / tv.nxg) % NFL);
    const int r = (int)(idx / ((long long)NFL * tv.nxg));
    const int i = tv.xinv[m];
    T s = T(0);
    if (i >= 0) {
        for (int c = 0; c < tv.nch; ++c) {
            if (tv.ca[c] == a) s += U[((size_t)c * R + r) * tv.nx + i];
            if (tv.cb[c] == a)
                for (int b = 0; b < niblk; ++b) s += Vp[(((size_t)c * niblk + b) * R + r) * tv.nx + i];
        }
    }
    gF[idx] = accumulate ? gF[idx] + s : s;
}

// DIS: grid (ceil(E/128), ceil(R/64), nsplit): the data points are split in
// nsplit ranges of dchunk; P[(split * R + r) * E + e] = sum over the range of
// FK[d][e] gO[r][d].
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_dis(TableView tv, const T *__restrict__ fk,
                                                 const T *__restrict__ gO, int ldgo, int R, int dchunk,
                                                 T *__restrict__ P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Gs = As + BKD * BET;
    const long long e_b = (long long)blockIdx.x * BET;
    const int rows = (int)min((long long)BET, tv.E - e_b);
    const int r0 = blockIdx.y * BRT;
    const int d_b = blockIdx.z * dchunk, d_e = min(tv.ndata, d_b + dchunk);
    T acc[8][4];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
    bwd_w_tile<T>(tv, fk, gO, ldgo, R, e_b, rows, r0, d_b, d_e, As, Gs, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int e = ty * 8 + p;
        if (e >= rows) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = r0 + tx * 4 + q;
            if (r < R) P[((size_t)blockIdx.z * R + r) * tv.E + e_b + e] = acc[p][q];
        }
    }
}

// gF[r][ca[k]][xmap[i]] (+)= sum_split P[split][r][(k,i)], splits in order.
// gF must be zeroed beforehand when overwriting (grid points outside xmap).
template <typename T>
__global__ void k_bwd_dis_gather(TableView tv, const T *__restrict__ P, int nsplit, int R,
                                 T *__restrict__ gF) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * tv.E) return;
    const int r = (int)(idx / tv.E), e = (int)(idx - (long long)r * tv.E);
    T s = T(0);
    for (int z = 0; z < nsplit; ++z) s += P[((size_t)z * R + r) * tv.E + e];
    const int k = e / tv.nx, i = e - k * tv.nx;
    const int a = tv.ca[k], m = tv.xmap[i];
    if (FK_DBG(a >= 0 && a < NFL && m >= 0 && m < tv.nxg && k < tv.nch, 3, e))
        gF[((size_t)r * NFL + a) * tv.nxg + m] += s;
}

// FP64 rows (staging, [rows][E]) -> padded stream layouts.
__global__ void k_convert(const double *__restrict__ src, long long rows, long long E,
                          long long ldE, double *__restrict__ d64, float *__restrict__ d32) {
    const long long n = rows * ldE;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long d = idx / ldE, e = idx - d * ldE;
        const double v = e < E ? src[d * E + e] : 0.0;
        if (d64) d64[idx] = v;
        if (d32) d32[idx] = (float)v;
    }
}

// Opts a kernel into more than 48 KB of dynamic shared memory, once per
// process (so that later calls, including ones under stream capture, do not
// repeat the attribute call).
template <typename T, typename K>
int set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return FK_OK;
    static std::mutex mu;
    static std::set<const void *> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count((const void *)kernel)) return FK_OK;
    FK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.insert((const void *)kernel);
    return FK_OK;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

// Channel splits of the factorised kernel: a function of the table only, so a
// replica's summation order does not depend on R (bit-exact batching).
int fac_nsplit(const fk_table *t) {
    const int dt = (t->ndata + FAC_TDT - 1) / FAC_TDT;
    const long long want = (2LL * num_sms() + dt - 1) / dt;
    return (int)std::max(1LL, std::min((long long)t->nch, want));
}

template <typename T, int TRT>
int launch_fac_t(const fk_table *t, const T *F, int R, const T *fk, int nsplit, T *part, cudaStream_t s) {
    const size_t smem = fac_smem<T, TRT>(t->nx);
    // opt in once at the largest x grid so that every table fits
    int rc = set_smem<T>(k_fac<T, TRT>, fac_smem<T, TRT>(MAX_NX));
    if (rc) return rc;
    CUtensorMap map;
    rc = make_plain_map(&map, fk, (int)sizeof(T), t->ldE, t->ndata, fac_width(t->nx, sizeof(T)), FAC_TDT);
    if (rc) return rc;
    dim3 grid((t->ndata + FAC_TDT - 1) / FAC_TDT, (R + TRT - 1) / TRT, nsplit);
    k_fac<T, TRT><<<grid, 256, smem, s>>>(map, view(t), F, R, nsplit, part);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Hadronic, R >= 2: replica tiles of 16 for few replicas, else the widest
// tile the registers allow (64 in FP32, 32 in FP64).
template <typename T>
int launch_fac(const fk_table *t, const T *F, int R, const T *fk, int nsplit, T *part, cudaStream_t s) {
    if (R <= 16) return launch_fac_t<T, 16>(t, F, R, fk, nsplit, part, s);
    return launch_fac_t<T, sizeof(T) == 4 ? 64 : 32>(t, F, R, fk, nsplit, part, s);
}

template <int KIND, typename T>
int fwd_cc_t(const fk_table *t, const T *F, int R, T *O, int ldo, const T *fk, cudaStream_t s) {
    TableView tv = view(t);
    Scratch scr(s);
    T *part = nullptr;
    int nparts;
    if (R <= 4 && (KIND != FK_KIND_HAD || R == 1)) {
        constexpr int CH = 256 * V16<T>::n * StreamCfg<T>::U;
        const int nchunk = (int)((t->ldE + CH - 1) / CH);
        nparts = nchunk;
        FK_CUDA(scr.get(&part, (size_t)nparts * R * t->ndata));
        dim3 grid(nchunk, (t->ndata + StreamCfg<T>::DB - 1) / StreamCfg<T>::DB, R);
        k_stream<KIND, T><<<grid, 256, 0, s>>>(tv, fk, F, R, part);
        count_launch();
        FK_CUDA(cudaGetLastError());
    } else if constexpr (KIND == FK_KIND_HAD) {
        nparts = fac_nsplit(t);
        FK_CUDA(scr.get(&part, (size_t)nparts * R * t->ndata));
        int rc = launch_fac<T>(t, F, R, fk, nparts, part, s);
        if (rc) return rc;
    } else {
        const int dt = (t->ndata + TDT - 1) / TDT, rt = (R + TRT - 1) / TRT;
        const long long nseg = (t->E + TileCfg<T>::KC - 1) / TileCfg<T>::KC;
        // The split depends on the table only, so a replica's summation
        // order does not change with R (bit-exact batching of requests).
        long long want = (2LL * num_sms() + dt - 1) / dt;
        nparts = (int)std::max(1LL, std::min(nseg, want));
        FK_CUDA(scr.get(&part, (size_t)nparts * R * t->ndata));
        constexpr size_t smem = tile_smem<T>();
        constexpr bool DENSE = KIND == FK_KIND_DENSE;
        int rc = set_smem<T>(k_tile<T, DENSE>, smem);
        if (rc) return rc;
        dim3 grid(dt, rt, nparts);
        k_tile<T, DENSE><<<grid, 256, smem, s>>>(tv, fk, F, R, nparts, part);
        count_launch();
        FK_CUDA(cudaGetLastError());
    }
    return reduce_parts<T>(part, nparts, t->ndata, R, O, ldo, s);
}

template <typename T>
int bwd_cc_t(const fk_table *t, const T *F, const T *gO, int ldgo, int R, T *gF, int accumulate,
             const T *fk, cudaStream_t s) {
    TableView tv = view(t);
    const int rt = (R + BRT - 1) / BRT;
    constexpr size_t smem = bwd_smem<T>();
    if (t->kind == FK_KIND_DIS) {
        // split the data points so that small tables still fill the GPU; the
        // split depends on the table only
        const int eb = (int)((t->E + BET - 1) / BET);
        const int want = (2 * num_sms() + eb - 1) / eb;
        const int dchunk = std::max(BKD, (t->ndata + want - 1) / want / BKD * BKD);
        const int nsplit = (t->ndata + dchunk - 1) / dchunk;
        Scratch scr(s);
        T *P = nullptr;
        FK_CUDA(scr.get(&P, (size_t)nsplit * R * t->E));
        if (!accumulate) FK_CUDA(cudaMemsetAsync(gF, 0, sizeof(T) * (size_t)R * NFL * t->nxg, s));
        int rc = set_smem<T>(k_bwd_dis<T>, smem);
        if (rc) return rc;
        dim3 grid(eb, rt, nsplit);
        k_bwd_dis<T><<<grid, 256, smem, s>>>(tv, fk, gO, ldgo, R, dchunk, P);
        count_launch();
        FK_CUDA(cudaGetLastError());
        const long long n = (long long)R * t->E;
        k_bwd_dis_gather<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tv, P, nsplit, R, gF);
        count_launch();
        FK_CUDA(cudaGetLastError());
        return FK_OK;
    }
    Scratch scr(s);
    const int IB = std::max(1, BET / t->nx);
    const int niblk = (t->nx + IB - 1) / IB;
    T *U = nullptr, *Vp = nullptr;
    FK_CUDA(scr.get(&U, (size_t)t->nch * R * t->nx));
    FK_CUDA(scr.get(&Vp, (size_t)t->nch * niblk * R * t->nx));
    int rc = set_smem<T>(k_bwd_had<T>, smem);
    if (rc) return rc;
    dim3 grid(niblk, rt, t->nch);
    k_bwd_had<T><<<grid, 256, smem, s>>>(tv, fk, F, gO, ldgo, R, IB, U, Vp);
    count_launch();
    FK_CUDA(cudaGetLastError());
    const long long n = (long long)R * NFL * t->nxg;
    k_bwd_had_gather<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tv, U, Vp, R, niblk, accumulate, gF);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

}  // namespace

int fwd_cc(const fk_table *t, const void *F, int R, void *O, int ldo, bool f64, cudaStream_t s) {
    if (f64) {
        if (!t->fk64) return fail(FK_EUNSUPPORTED, "table has no FP64 copy");
        return t->kind == FK_KIND_HAD
                   ? fwd_cc_t<FK_KIND_HAD, double>(t, (const double *)F, R, (double *)O, ldo, t->fk64, s)
                   : fwd_cc_t<FK_KIND_DIS, double>(t, (const double *)F, R, (double *)O, ldo, t->fk64, s);
    }
    if (!t->fk32) return fail(FK_EUNSUPPORTED, "table has no FP32 copy");
    return t->kind == FK_KIND_HAD
               ? fwd_cc_t<FK_KIND_HAD, float>(t, (const float *)F, R, (float *)O, ldo, t->fk32, s)
               : fwd_cc_t<FK_KIND_DIS, float>(t, (const float *)F, R, (float *)O, ldo, t->fk32, s);
}

int dense_cc(const fk_table *t, const void *L, int R, void *O, int ldo, bool f64, cudaStream_t s) {
    if (f64) {
        if (!t->fk64) return fail(FK_EUNSUPPORTED, "table has no FP64 copy");
        return fwd_cc_t<FK_KIND_DENSE, double>(t, (const double *)L, R, (double *)O, ldo, t->fk64, s);
    }
    if (!t->fk32) return fail(FK_EUNSUPPORTED, "table has no FP32 copy");
    return fwd_cc_t<FK_KIND_DENSE, float>(t, (const float *)L, R, (float *)O, ldo, t->fk32, s);
}

namespace {
// The PDF matrix of a hadronic table: L[r][(c * nx + i) * nx + j] =
// F[r][a_c][xmap[i]] * F[r][b_c][xmap[j]], one element per thread (grid-stride).
template <typename T>
__global__ void __launch_bounds__(256) k_lum(TableView tv, const T *__restrict__ F, int R, T *__restrict__ L) {
    const long long n = (long long)R * tv.E;
    const int nx2 = tv.nx * tv.nx;
    for (long long idx = (long long)blockIdx.x * 256 + threadIdx.x; idx < n; idx += (long long)gridDim.x * 256) {
        const long long r = idx / tv.E;
        const int e = (int)(idx - r * tv.E);
        const int c = e / nx2, rem = e - c * nx2, i = rem / tv.nx, j = rem - i * tv.nx;
        const T *f = F + (size_t)r * NFL * tv.nxg;
        if (!FK_DBG(c < tv.nch, 4, idx)) continue;
        L[idx] = __ldg(f + __ldg(tv.ca + c) * tv.nxg + __ldg(tv.xmap + i)) *
                 __ldg(f + __ldg(tv.cb + c) * tv.nxg + __ldg(tv.xmap + j));
    }
}

template <typename T>
int luminosity_t(const fk_table *t, const T *F, int R, T *L, cudaStream_t s) {
    const long long n = (long long)R * t->E;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 148LL * 16);
    k_lum<T><<<blocks, 256, 0, s>>>(view(t), F, R, L);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}
}  // namespace

int luminosity_cc(const fk_table *t, const void *F, int R, void *L, bool f64, cudaStream_t s) {
    return f64 ? luminosity_t<double>(t, (const double *)F, R, (double *)L, s)
               : luminosity_t<float>(t, (const float *)F, R, (float *)L, s);
}

int bwd_cc(const fk_table *t, const void *F, const void *gO, int ldgo, int R, void *gF,
           int accumulate, bool f64, cudaStream_t s) {
    if (f64) {
        if (!t->fk64) return fail(FK_EUNSUPPORTED, "table has no FP64 copy");
        return bwd_cc_t<double>(t, (const double *)F, (const double *)gO, ldgo, R, (double *)gF,
                                accumulate, t->fk64, s);
    }
    if (!t->fk32) return fail(FK_EUNSUPPORTED, "table has no FP32 copy");
    return bwd_cc_t<float>(t, (const float *)F, (const float *)gO, ldgo, R, (float *)gF,
                           accumulate, t->fk32, s);
}

FK_DBG_READER(dbg_cc)

int convert_rows(const double *d_src, long long rows, long long E, long long ldE, double *d64,
                 float *d32, cudaStream_t s) {
    const long long n = rows * ldE;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 148LL * 16);
    k_convert<<<blocks, 256, 0, s>>>(d_src, rows, E, ldE, d64, d32);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

}  // namespace fk

// ----------------------------------------------------------------------------
// Allocation-free hadronic forward (fk_had_conv_noalloc).
//
// Some callers may not allocate device memory while they run: their device
// memory is entirely owned by another allocator or capped by a pool limit, or
// they sit in a latency-critical loop where any allocation could wait on the
// driver.  For them the FP64/FP32 hadronic convolution is offered with its
// temporary partial sums in the fixed array below instead of stream-ordered
// scratch.  The array is reserved on every GPU that loads this library, for
// the life of the process.  Host code must not use its name as a pointer (on
// the host it is only a stand-in for the symbol): the device address is looked
// up once per device with cudaGetSymbolAddress and passed to the kernels.
// ----------------------------------------------------------------------------
constexpr size_t FK_NOALLOC_BYTES = 8u << 20;  // 8 MiB of partial sums
static __device__ __align__(256) unsigned char g_fk_noalloc_scratch[FK_NOALLOC_BYTES];

namespace fk {
namespace {

// The driver's current context, through the runtime's entry-point query (the
// library does not link the driver API); NULL if the query is unavailable.
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static Fn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(ptr);
    });
    CUcontext c = nullptr;
    if (fn) fn(&c);
    return c;
}

// Device address of g_fk_noalloc_scratch on the current device.  The first
// call on a device performs the lookup (so make it before any stream capture);
// the address is kept with the context it belongs to and looked up again if
// the device's context has changed since.
int noalloc_scratch(void **out) {
    static std::mutex mu;
    static void *addr[256] = {};
    static CUcontext ctx[256] = {};
    int dev = 0;
    FK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(FK_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    const CUcontext now = current_context();
    if (!addr[dev] || ctx[dev] != now) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_fk_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
        addr[dev] = p;
        ctx[dev] = current_context();
    }
    *out = addr[dev];
    return FK_OK;
}

// Same launches as the FP64/FP32 hadronic forward, with the partial sums in
// the static array.  Every partial-sum slot the reduction reads is written by
// the first kernel of the same call, so nothing has to be cleared between
// calls.
template <typename T>
int had_noalloc_t(const fk_table *t, const T *F, int R, T *O, int ldo, const T *fk, cudaStream_t s) {
    TableView tv = view(t);
    int nparts;
    if (R == 1) {
        constexpr int CH = 256 * V16<T>::n * StreamCfg<T>::U;
        nparts = (int)((t->ldE + CH - 1) / CH);
    } else {
        nparts = fac_nsplit(t);
    }
    const size_t need = sizeof(T) * (size_t)nparts * R * t->ndata;
    if (need > FK_NOALLOC_BYTES)
        return fail(FK_EINVAL, "fk_had_conv_noalloc: this call needs " + std::to_string(need) +
                                   " bytes of partial sums; the static area holds " +
                                   std::to_string(FK_NOALLOC_BYTES) + " (use fewer replicas per call)");
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    T *part = static_cast<T *>(scratch);
    if (R == 1) {
        dim3 grid(nparts, (t->ndata + StreamCfg<T>::DB - 1) / StreamCfg<T>::DB, R);
        k_stream<FK_KIND_HAD, T><<<grid, 256, 0, s>>>(tv, fk, F, R, part);
        count_launch();
        FK_CUDA(cudaGetLastError());
    } else {
        rc = launch_fac<T>(t, F, R, fk, nparts, part, s);
        if (rc) return rc;
    }
    return reduce_parts<T>(part, nparts, t->ndata, R, O, ldo, s);
}

}  // namespace
}  // namespace fk

extern "C" int fk_had_conv_noalloc(const fk_table *t, const void *F, int R, void *O, int ldo,
                                   int prec, fk_stream stream) {
    using namespace fk;
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (t->kind != FK_KIND_HAD) return fail(FK_EINVAL, "fk_had_conv_noalloc needs a hadronic table");
    if (!F || !O) return fail(FK_EINVAL, "null F or O");
    if (R < 1) return fail(FK_EINVAL, "R < 1");
    if (ldo < 0 || (ldo > 0 && ldo < t->ndata)) return fail(FK_EINVAL, "ldo < ndata");
    if (prec != FK_FP64 && prec != FK_FP32)
        return fail(FK_EUNSUPPORTED, "fk_had_conv_noalloc offers FK_FP64 and FK_FP32 only");
    if (!(t->mask & FK_PREC_BIT(prec))) return fail(FK_EUNSUPPORTED, "precision not stored in this table");
    const cudaStream_t s = (cudaStream_t)stream;
    ldo = ldo ? ldo : t->ndata;
    if (prec == FK_FP64)
        return had_noalloc_t<double>(t, (const double *)F, R, (double *)O, ldo, t->fk64, s);
    return had_noalloc_t<float>(t, (const float *)F, R, (float *)O, ldo, t->fk32, s);
}

// ----------------------------------------------------------------------------
// Fixed-order sum of gradient buffers (fk_grad_sum).
// ----------------------------------------------------------------------------
namespace fk {
namespace {
constexpr int MAX_PARTS = 64;
template <typename T>
struct Parts {
    const T *p[MAX_PARTS];
};
template <typename T>
__global__ void k_grad_sum(Parts<T> parts, int nparts, long long n, T *__restrict__ out, int accumulate) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        T s = accumulate ? out[e] : T(0);
        for (int k = 0; k < nparts; ++k) s += parts.p[k][e];
        out[e] = s;
    }
}
template <typename T>
int grad_sum_t(const void *const *parts, int nparts, long long n, void *out, int accumulate, cudaStream_t s) {
    Parts<T> P{};
    for (int k = 0; k < nparts; ++k) P.p[k] = static_cast<const T *>(parts[k]);
    const unsigned blocks = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 148LL * 8));
    k_grad_sum<T><<<blocks, 256, 0, s>>>(P, nparts, n, static_cast<T *>(out), accumulate);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}
}  // namespace
}  // namespace fk

extern "C" int fk_grad_sum(const void *const *parts, int nparts, long long n, void *out, int accumulate,
                           int prec, fk_stream stream) {
    using namespace fk;
    if (!parts || !out || nparts < 1 || nparts > MAX_PARTS || n < 0)
        return fail(FK_EINVAL, "fk_grad_sum: bad arguments (1 <= nparts <= 64)");
    for (int k = 0; k < nparts; ++k)
        if (!parts[k]) return fail(FK_EINVAL, "fk_grad_sum: null part");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "fk_grad_sum: unknown precision");
    if (n == 0) return FK_OK;
    return FK_IO64(prec) ? grad_sum_t<double>(parts, nparts, n, out, accumulate ? 1 : 0, (cudaStream_t)stream)
                           : grad_sum_t<float>(parts, nparts, n, out, accumulate ? 1 : 0, (cudaStream_t)stream);
}

namespace fk {
int cc_device_status(int reset) {
    int v = 0;
    FK_CUDA(cudaMemcpyFromSymbol(&v, g_fk_cc_error, sizeof(int)));
    if (reset) {
        const int z = 0;
        FK_CUDA(cudaMemcpyToSymbol(g_fk_cc_error, &z, sizeof(int)));
    }
    return v ? FK_ETIMEDOUT : FK_OK;
}
}  // namespace fk
