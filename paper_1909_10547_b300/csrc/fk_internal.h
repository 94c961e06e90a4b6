// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the driver is reached through cudart)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fk.h"

namespace fk {

constexpr int NFL = 14;
constexpr int MAX_NX = 64;        // x points per table (stream kernels keep F in smem)
constexpr int MAX_NXG = 64;       // points of the PDF grid
constexpr int MAX_CH = NFL * NFL; // ordered flavour pairs

// Thread-local error detail; returns the status for `return fail(...)`.
int fail(int status, const std::string &msg);
// Counts kernel launches (fk_kernel_launches); call once per <<<>>> launch.
void count_launch(int n = 1);
int cuda_fail(cudaError_t e, const char *what);
#define FK_CUDA(call)                                        \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::fk::cuda_fail(e_, #call); \
    } while (0)

// Debug builds (-DFK_DEBUG, libfk_debug.so): index checks in the kernels
// raise a device word holding the first failed check's code and index, and
// skip the access, instead of touching memory out of range; per-call scratch
// buffers carry guard bytes that are checked when the call's scratch is
// released.  Release builds compile every check away.  Each translation unit
// has its own word (static), read by its dbg_* function.
#ifdef FK_DEBUG
static __device__ unsigned long long g_fk_dbg;
__device__ __forceinline__ bool fk_dbg_ok(bool cond, int code, long long idx) {
    if (!cond)
        atomicCAS(&g_fk_dbg, 0ull,
                  ((unsigned long long)code << 40) | ((unsigned long long)idx & ((1ull << 40) - 1)));
    return cond;
}
#define FK_DBG(cond, code, idx) fk_dbg_ok((cond), (code), (long long)(idx))
constexpr size_t FK_GUARD_BYTES = 256;
constexpr unsigned char FK_GUARD_BYTE = 0xA5;
static __global__ void k_guard_check(const unsigned char *g) {
    for (unsigned i = threadIdx.x; i < FK_GUARD_BYTES; i += blockDim.x)
        if (g[i] != FK_GUARD_BYTE) {
            fk_dbg_ok(false, 90, i);
            break;
        }
}
#define FK_DBG_READER(fn)                                                                    \
    int fn(int reset, unsigned long long *w) {                                               \
        FK_CUDA(cudaMemcpyFromSymbol(w, g_fk_dbg, sizeof(*w)));                              \
        if (reset) {                                                                         \
            const unsigned long long z = 0;                                                  \
            FK_CUDA(cudaMemcpyToSymbol(g_fk_dbg, &z, sizeof(z)));                            \
        }                                                                                    \
        return FK_OK;                                                                        \
    }
#else
#define FK_DBG(cond, code, idx) true
#define FK_DBG_READER(fn)                                                                    \
    int fn(int, unsigned long long *w) {                                                     \
        *w = 0;                                                                              \
        return FK_OK;                                                                        \
    }
#endif

// Stream-ordered scratch memory for one call (cudaMallocAsync/cudaFreeAsync).
struct Scratch {
    cudaStream_t stream;
    std::vector<void *> ptrs;
#ifdef FK_DEBUG
    std::vector<unsigned char *> guards;
#endif
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch() {
#ifdef FK_DEBUG
        for (unsigned char *g : guards) k_guard_check<<<1, 256, 0, stream>>>(g);
#endif
        for (void *p : ptrs) cudaFreeAsync(p, stream);
    }
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        void *q = nullptr;
#ifdef FK_DEBUG
        const size_t used = (count * sizeof(T) + 15) / 16 * 16;
        cudaError_t e = cudaMallocAsync(&q, used + FK_GUARD_BYTES + 256, stream);
        if (e == cudaSuccess) {
            ptrs.push_back(q);
            unsigned char *g = static_cast<unsigned char *>(q) + used;
            guards.push_back(g);
            e = cudaMemsetAsync(g, FK_GUARD_BYTE, FK_GUARD_BYTES, stream);
        }
#else
        cudaError_t e = cudaMallocAsync(&q, count * sizeof(T) + 256, stream);
        if (e == cudaSuccess) ptrs.push_back(q);
#endif
        *p = reinterpret_cast<T *>(q);
        return e;
    }
};

// Channel groups of a hadronic table for the tensor-core path (k_tc.cu):
// group g collects the channels (a_g, b) of one first flavour a_g.  Along the
// contraction axis K the groups are concatenated, each padded to a multiple of
// 16 elements; inside a group, K runs over (channel, x_j).
struct TcGroups {
    int ngroups;
    int flav[NFL];    // a_g
    int nch[NFL];     // channels in group g
    int ch0[NFL];     // first entry of group g in chan[]
    int kbeg[NFL];    // K range [kbeg, kend) of group g
    int kend[NFL];
    int chan[MAX_CH]; // channel ids ordered by group
};

// One packing of a hadronic table as the B operand of the MMA: one tile of
// n_rows rows per G data points, K-major with row length ktot_pad.
//  - forward packing: groups by the first flavour a_c; row n = i * G + d % G
//    holds x_i, K runs over (channel, x_j);
//  - transposed packing (adjoint): groups by the second flavour b_c; row
//    n = j * G + d % G holds x_j, K runs over (channel, x_i).
struct TcPack {
    TcGroups grp{};
    int n_rows = 0;     // B rows per tile (MMA N)
    int ntile_n = 0;    // B tiles
    int ktot = 0;       // used K (sum of padded group lengths)
    int ktot_pad = 0;   // row length: whole pipeline stages (a multiple of 64 or 128)
    __nv_bfloat16 *hi = nullptr;  // BF16 / hi part
    __nv_bfloat16 *lo = nullptr;  // lo part (BF16X3)
    float *f32 = nullptr;         // TF32 operand (FP32 bits, rounded)
    // A-operand gather maps (device): kmeta[k] = offset o * nx_grid + xmap[j]
    // of the PDF value f_o(x_j) in one replica's F row for K column k (o the
    // channel's other flavour), or -1 for padding; mmeta[g * nx + i] = offset
    // of f_{a_g}(x_i), the forward epilogue multiplier
    int *kmeta = nullptr;
    int *mmeta = nullptr;
    CUtensorMap map_hi;   // (the type is 128-byte aligned)
    CUtensorMap map_lo;
    CUtensorMap map_f32;
    // the same tensors with boxes of n_rows / 2 rows: each CTA of a pair
    // running 2-SM MMAs loads one half of every B tile
    CUtensorMap half_hi, half_lo, half_f32;
    // hi+lo on single CTAs: boxes of 64-byte rows (64-byte swizzle); nar
    // tells whether they were built
    CUtensorMap nar_hi, nar_lo;
    bool nar = false;
};

struct TcLayout {
    int G = 0;          // data points per tile (4, 5, 6, 7, 8, 12 or 16; G * nx <= 256)
    int ntile_n = 0;    // ceil(ndata / G)
    int n_rows = 0;     // MMA N = G * nx rounded up to 16
    TcPack fwd, bwd;
    int8_t *gmap = nullptr;  // device [2][14]: group of flavour a in fwd / bwd packing, or -1
    // FP64 on the tensor cores (k_oz.cu): the table as exact BF16 digit
    // slices, rows [ndata] over K (oz) and, for the adjoints, rows over K
    // = ndata (ozT: DIS [(k, i)][d], hadronic [(c, i, j)][d]); hi holds the
    // S slices stacked [S][ntile_n * n_rows][ktot_pad], oz_e the exponent
    // of each (row, K chunk)
    TcPack oz, ozT;
    int *oz_e = nullptr, *ozT_e = nullptr;
    int oz_kchunk = 0, ozT_kchunk = 0;
    // The paper's dense formulation of the hadronic forward (Sec. 3, Table
    // 3) with the PDF matrix formed in shared memory: the table flattened to
    // [ndata][(c, i, j)], j padded to lum_nxp (a power of two, 16 to 64,
    // zeros past nx); lum_mmeta[a * nx + x] = a * nx_grid + xmap[x], the F offsets of
    // the builders' transposed PDF rows.  lum_on: the forward uses it.
    TcPack lum;
    int lum_nxp = 0;
    int *lum_mmeta = nullptr;
    bool lum_on = false;
};

}  // namespace fk

// Device-resident table.  Stream layouts keep the caller's element order
// (channel, x_i, x_j) per data point, each row padded to ldE elements.  A
// dense table (the paper's Table 3 product) holds [ndata][E = K] with
// nch = nx = nxg = 0.
struct fk_table {
    int kind = 0;
    int ndata = 0, nch = 0, nx = 0, nxg = 0;
    long long E = 0;    // elements per data point
    long long ldE = 0;  // padded row length
    unsigned mask = 0;
    int device = 0;
    std::vector<int> ca, cb, xmap;  // host copies (DIS: ca = active flavours)
    int *d_ca = nullptr, *d_cb = nullptr, *d_xmap = nullptr;
    int *d_xinv = nullptr;          // [nxg] local x index of a grid point, or -1
    double *fk64 = nullptr;         // [ndata][ldE]
    float *fk32 = nullptr;          // [ndata][ldE]
    // tensor-core layouts (hadronic): packed B operand tiles
    fk::TcLayout tc;
    size_t bytes = 0;
};

// Plain view passed to kernels by value.
struct TableView {
    int ndata, nch, nx, nxg;
    long long E, ldE;
    const int *ca, *cb, *xmap, *xinv;
};

inline TableView view(const fk_table *t) {
    return TableView{t->ndata, t->nch, t->nx, t->nxg, t->E, t->ldE,
                     t->d_ca, t->d_cb, t->d_xmap, t->d_xinv};
}

namespace fk {
// CUDA-core paths (k_cc.cu)
int fwd_cc(const fk_table *t, const void *F, int R, void *O, int ldo, bool f64, cudaStream_t s);
// dense tables (the paper's Table 3 product) and the PDF matrix of a hadronic table
int dense_cc(const fk_table *t, const void *L, int R, void *O, int ldo, bool f64, cudaStream_t s);
int luminosity_cc(const fk_table *t, const void *F, int R, void *L, bool f64, cudaStream_t s);
int bwd_cc(const fk_table *t, const void *F, const void *gO, int ldgo, int R, void *gF,
           int accumulate, bool f64, cudaStream_t s);
// tensor-core path (k_tc.cu)
// form: 0 (automatic), FK_TABLE_FACTORED or FK_TABLE_LUMI
int tc_build(fk_table *t, const double *host_fk, unsigned form);
int fwd_tc(const fk_table *t, const float *F, int R, float *O, int ldo, int prec, cudaStream_t s);
int tc_build_dense(fk_table *t, const double *host_fk);
int dense_tc(const fk_table *t, const float *L, int R, float *O, int ldo, int prec, cudaStream_t s);
// DIS tables on the tensor cores: the forward is the plain product
// FK[d][(k,i)] F[r][(a_k, x_i)], the adjoint the product of gO with FK^T
int tc_build_dis(fk_table *t, const double *host_fk);
int dis_tc(const fk_table *t, const float *F, int R, float *O, int ldo, int prec, cudaStream_t s);
int dis_bwd_tc(const fk_table *t, const float *gO, int ldgo, int R, float *gF, int accumulate, int prec,
               cudaStream_t s);
int bwd_tc(const fk_table *t, const float *F, const float *gO, int ldgo, int R, float *gF,
           int accumulate, int prec, cudaStream_t s);
// saved forward products (hadronic tables, factorised form): the forward also
// writes its products Y_g (saved_elems floats), the adjoint forms its first
// term from them
size_t saved_elems(const fk_table *t, int R);
int fwd_tc_save(const fk_table *t, const float *F, int R, float *O, int ldo, float *Y, int prec, cudaStream_t s);
int bwd_tc_saved(const fk_table *t, const float *F, const float *gO, int ldgo, int R, const float *Y, float *gF,
                 int accumulate, int prec, cudaStream_t s);
void tc_free(fk_table *t);
// operand-slice products (k_tc.cu) and FP64 on the tensor cores (k_oz.cu)
int tc_map_bf16(CUtensorMap *m, const void *ptr, long long cols, long long rows, int box_rows);
int tc_slice_pairs(const fk_table *t, const TcPack &pk, const CUtensorMap &mA, int R, int nd_out, int kchunk,
                   int c0, int nsplit, int npair, int npc, const uint8_t *pa, const uint8_t *pb, float *P,
                   cudaStream_t s);
int oz_build(fk_table *t, const double *host_fk);
void oz_free(fk_table *t);
int oz_dense(const fk_table *t, const double *L, int R, double *O, int ldo, cudaStream_t s);
int oz_dis(const fk_table *t, const double *F, int R, double *O, int ldo, cudaStream_t s);
int oz_had(const fk_table *t, const double *F, int R, double *O, int ldo, cudaStream_t s);
int oz_bwd(const fk_table *t, const double *F, const double *gO, int ldgo, int R, double *gF, int accumulate,
           cudaStream_t s);
// FK_ETIMEDOUT if a kernel's bounded wait ran out since the last reset
// (device_status: tensor-core kernels; cc_device_status: CUDA-core kernels)
int device_status(int reset);
int cc_device_status(int reset);
// 2-D tensor map over a row-major [rows][cols] array of esz-byte (4 or 8)
// floating-point elements, boxes of box_cols x box_rows, no swizzle,
// zero-filled outside the array (k_tc.cu)
int make_plain_map(CUtensorMap *m, const void *ptr, int esz, long long cols, long long rows, int box_cols,
                   int box_rows);
// debug-build check words of each translation unit (0 when clean or in a
// release build): code << 40 | index of the first failed check
int dbg_cc(int reset, unsigned long long *w);
int dbg_tc(int reset, unsigned long long *w);
int dbg_chi2(int reset, unsigned long long *w);
int dbg_oz(int reset, unsigned long long *w);
int dbg_api(int reset, unsigned long long *w);
// conversion helpers (k_cc.cu)
int convert_rows(const double *d_src, long long rows, long long E, long long ldE, double *d64,
                 float *d32, cudaStream_t s);
}  // namespace fk
