// C ABI of the FK convolution library: errors, tables, convolution dispatch.
#include "fk_internal.h"

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <set>
#include <utility>

namespace fk {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int fail(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? FK_ENOMEM : FK_ECUDA;
}

namespace {

constexpr unsigned ALL_PRECS = FK_PREC_BIT(FK_FP64) | FK_PREC_BIT(FK_FP32) | FK_PREC_BIT(FK_BF16) |
                               FK_PREC_BIT(FK_BF16X3) | FK_PREC_BIT(FK_TF32) | FK_PREC_BIT(FK_FP64_TC);
constexpr unsigned TC_PRECS = FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_BF16X3) | FK_PREC_BIT(FK_TF32);

void keep_pool() {
    // Keep freed stream-ordered scratch in the device pool instead of
    // returning it to the driver after every synchronisation.  Reuse across
    // streams only through event dependencies: with opportunistic reuse and
    // internal dependencies on, after a fit step had spread its scratch over
    // 80 streams every later allocation cost about 0.3 ms of host time
    // (a one-request convolution 0.14 -> 0.47 ms, growing with further steps);
    // with both off it stays at 0.14 ms.
    static bool done = false;
    if (done) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        int off = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowOpportunistic, &off);
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &off);
    }
    done = true;
}

void table_free(fk_table *t) {
    if (!t) return;
    cudaFree(t->d_ca);
    cudaFree(t->d_cb);
    cudaFree(t->d_xmap);
    cudaFree(t->d_xinv);
    cudaFree(t->fk64);
    cudaFree(t->fk32);
    tc_free(t);
    oz_free(t);
    delete t;
}

template <typename T>
int upload(T **d, const std::vector<T> &h, size_t *bytes) {
    if (h.empty()) return FK_OK;
    if (cudaMalloc(d, sizeof(T) * h.size())) return fail(FK_ENOMEM, "table index arrays");
    FK_CUDA(cudaMemcpy(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    *bytes += sizeof(T) * h.size();
    return FK_OK;
}

// Copies the host FP64 rows [ndata][E] into the table's FP64 / FP32 stream
// layouts (rows padded to ldE), staged through a bounded device buffer.
int upload_rows(fk_table *t, const double *fk) {
    int rc = FK_OK;
    const size_t rowsz = (size_t)t->ldE * t->ndata;
    const bool need64 = t->mask & FK_PREC_BIT(FK_FP64);
    const bool need32 = t->mask & FK_PREC_BIT(FK_FP32);
    if ((need64 && cudaMalloc(&t->fk64, sizeof(double) * rowsz)) ||
        (need32 && cudaMalloc(&t->fk32, sizeof(float) * rowsz))) {
        return fail(FK_ENOMEM, "table storage");
    }
    t->bytes += (need64 ? sizeof(double) * rowsz : 0) + (need32 ? sizeof(float) * rowsz : 0);
    if (need64 || need32) {
        // stage the host rows through a bounded device buffer
        const long long rows_per = std::max(1LL, (64LL << 20) / (t->E * 8));
        double *stage = nullptr;
        cudaStream_t st = nullptr;
        if (cudaMalloc(&stage, sizeof(double) * t->E * std::min<long long>(rows_per, t->ndata)) ||
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) {
            cudaFree(stage);
            return fail(FK_ENOMEM, "table staging buffer");
        }
        for (long long d0 = 0; d0 < t->ndata && rc == FK_OK; d0 += rows_per) {
            const long long nr = std::min<long long>(rows_per, t->ndata - d0);
            cudaError_t e = cudaMemcpyAsync(stage, fk + d0 * t->E, sizeof(double) * nr * t->E,
                                            cudaMemcpyHostToDevice, st);
            if (e) {
                rc = cuda_fail(e, "table upload");
                break;
            }
            rc = convert_rows(stage, nr, t->E, t->ldE, t->fk64 ? t->fk64 + d0 * t->ldE : nullptr,
                              t->fk32 ? t->fk32 + d0 * t->ldE : nullptr, st);
            if (!rc) {
                e = cudaStreamSynchronize(st);
                if (e) rc = cuda_fail(e, "table conversion");
            }
        }
        cudaStreamDestroy(st);
        cudaFree(stage);
    }
    return rc;
}

int table_create(int kind, const double *fk, int ndata, const int *ca, const int *cb, int nch,
                 int nx, const int *xmap, int nxg, unsigned mask, fk_table **out) {
    if (!out) return fail(FK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!fk || !ca || (kind == FK_KIND_HAD && !cb)) return fail(FK_EINVAL, "null table or channel array");
    if (ndata < 1) return fail(FK_EINVAL, "ndata < 1");
    if (nx < 1 || nx > MAX_NX) return fail(FK_EINVAL, "nx must be in 1..64");
    if (nxg < nx || nxg > MAX_NXG) return fail(FK_EINVAL, "nx_grid must be in nx..64");
    // the forward-formulation flags apply to hadronic tables only, one at a time
    const unsigned form = mask & (FK_TABLE_FACTORED | FK_TABLE_LUMI);
    mask &= ~(FK_TABLE_FACTORED | FK_TABLE_LUMI);
    if (form && (kind != FK_KIND_HAD || form == (FK_TABLE_FACTORED | FK_TABLE_LUMI)))
        return fail(FK_EINVAL, "FK_TABLE_FACTORED / FK_TABLE_LUMI: one of them, hadronic tables only");
    if (!mask || (mask & ~ALL_PRECS)) return fail(FK_EINVAL, "bad precision mask");
    const int maxch = kind == FK_KIND_HAD ? MAX_CH : NFL;
    if (nch < 1 || nch > maxch) return fail(FK_EINVAL, "channel count out of range");
    std::set<std::pair<int, int>> seen;
    for (int c = 0; c < nch; ++c) {
        const int a = ca[c], b = kind == FK_KIND_HAD ? cb[c] : 0;
        if (a < 0 || a >= NFL || b < 0 || b >= NFL) return fail(FK_EINVAL, "flavour index out of 0..13");
        if (!seen.insert({a, b}).second) return fail(FK_EINVAL, "duplicate channel or flavour");
    }
    std::vector<int> xm(nx), xinv(nxg, -1);
    for (int i = 0; i < nx; ++i) {
        xm[i] = xmap ? xmap[i] : i;
        if (xm[i] < 0 || xm[i] >= nxg) return fail(FK_EINVAL, "xmap entry out of range");
        if (xinv[xm[i]] >= 0) return fail(FK_EINVAL, "xmap entries must be distinct");
        xinv[xm[i]] = i;
    }

    keep_pool();
    fk_table *t = new fk_table();
    t->kind = kind;
    t->ndata = ndata;
    t->nch = nch;
    t->nx = nx;
    t->nxg = nxg;
    t->E = kind == FK_KIND_HAD ? (long long)nch * nx * nx : (long long)nch * nx;
    t->ldE = (t->E + 31) / 32 * 32;
    t->mask = mask;
    cudaGetDevice(&t->device);
    t->ca.assign(ca, ca + nch);
    if (kind == FK_KIND_HAD) t->cb.assign(cb, cb + nch);
    t->xmap = xm;
    int rc = FK_OK;
    if ((rc = upload(&t->d_ca, t->ca, &t->bytes)) || (rc = upload(&t->d_cb, t->cb, &t->bytes)) ||
        (rc = upload(&t->d_xmap, t->xmap, &t->bytes)) || (rc = upload(&t->d_xinv, xinv, &t->bytes))) {
        table_free(t);
        return rc;
    }
    if ((rc = upload_rows(t, fk))) {
        table_free(t);
        return rc;
    }
    if (mask & TC_PRECS) {
        rc = kind == FK_KIND_HAD ? tc_build(t, fk, form) : tc_build_dis(t, fk);
        if (rc) {
            table_free(t);
            return rc;
        }
    }
    if (mask & FK_PREC_BIT(FK_FP64_TC)) {
        rc = oz_build(t, fk);
        if (rc) {
            table_free(t);
            return rc;
        }
    }
    *out = t;
    return FK_OK;
}

int dense_create(const double *fk, int ndata, long long K, unsigned mask, fk_table **out) {
    if (!out) return fail(FK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!fk) return fail(FK_EINVAL, "null table");
    if (ndata < 1) return fail(FK_EINVAL, "ndata < 1");
    if (K < 1 || K > (1LL << 30)) return fail(FK_EINVAL, "K must be in 1..2^30");
    if (!mask || (mask & ~ALL_PRECS)) return fail(FK_EINVAL, "bad precision mask");
    keep_pool();
    fk_table *t = new fk_table();
    t->kind = FK_KIND_DENSE;
    t->ndata = ndata;
    t->E = K;
    t->ldE = (K + 31) / 32 * 32;
    t->mask = mask;
    cudaGetDevice(&t->device);
    int rc = upload_rows(t, fk);
    if (!rc && (mask & TC_PRECS)) rc = tc_build_dense(t, fk);
    if (!rc && (mask & FK_PREC_BIT(FK_FP64_TC))) rc = oz_build(t, fk);
    if (rc) {
        table_free(t);
        return rc;
    }
    *out = t;
    return FK_OK;
}

int check_conv(const fk_table *t, int kind, const void *F, int R, const void *O, int ldo, int prec) {
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (t->kind != kind) return fail(FK_EINVAL, "wrong table kind for this call");
    if (!F || !O) return fail(FK_EINVAL, "null F or O");
    if (R < 1) return fail(FK_EINVAL, "R < 1");
    if (ldo < 0 || (ldo > 0 && ldo < t->ndata)) return fail(FK_EINVAL, "ldo < ndata");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "unknown precision");
    if (!(t->mask & FK_PREC_BIT(prec)))
        return fail(FK_EUNSUPPORTED, "precision not stored in this table");
    return FK_OK;
}

// The saved-product calls: a hadronic table in the factorised form, a
// tensor-core mode it stores, and (when given) a buffer of at least
// saved_elems floats, 4-byte aligned.
int check_saved(const fk_table *t, int R, int prec, const void *saved, size_t saved_bytes, bool need_buf) {
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (t->kind != FK_KIND_HAD) return fail(FK_EINVAL, "saved products need a hadronic table");
    if (R < 1) return fail(FK_EINVAL, "R < 1");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "unknown precision");
    if (prec != FK_BF16 && prec != FK_BF16X3 && prec != FK_TF32)
        return fail(FK_EUNSUPPORTED, "saved products only in the tensor-core modes BF16, BF16 hi+lo and TF32");
    if (!(t->mask & FK_PREC_BIT(prec))) return fail(FK_EUNSUPPORTED, "precision not stored in this table");
    if (t->tc.lum_on) return fail(FK_EUNSUPPORTED, "saved products need the factorised form");
    if (!need_buf) return FK_OK;
    if (!saved) return fail(FK_EINVAL, "null saved buffer");
    if ((uintptr_t)saved % 4) return fail(FK_EINVAL, "saved buffer not 4-byte aligned");
    const size_t need = saved_elems(t, R) * sizeof(float);
    if (saved_bytes < need) {
        char msg[96];
        snprintf(msg, sizeof msg, "saved buffer too small: %zu bytes, %zu needed", saved_bytes, need);
        return fail(FK_EINVAL, msg);
    }
    return FK_OK;
}

#ifdef FK_DEBUG
// Writes buf[idx] through a debug check: with idx out of range the check
// records it and the write is skipped.  Launched only in debug builds.
__global__ void k_dbg_selftest(int *buf, int n, int idx) {
    if (FK_DBG(idx >= 0 && idx < n, 99, idx)) buf[idx] = 1;
}
#endif

}  // namespace

FK_DBG_READER(dbg_api)

}  // namespace fk

using namespace fk;

extern "C" {

const char *fk_strerror(int s) {
    switch (s) {
        case FK_OK: return "ok";
        case FK_EINVAL: return "invalid argument";
        case FK_ENOMEM: return "out of memory";
        case FK_EBUDGET: return "request exceeds the memory budget";
        case FK_EPENDING: return "request pending";
        case FK_ETIMEDOUT: return "timed out";
        case FK_ECUDA: return "CUDA error";
        case FK_ENOTFOUND: return "not found";
        case FK_EUNSUPPORTED: return "unsupported precision or table kind";
        case FK_ECANCELED: return "request cancelled";
        default: return "unknown status";
    }
}

const char *fk_last_error_message(void) { return g_last_error.c_str(); }

int fk_version(void) { return 100; }

uint64_t fk_kernel_launches(void) { return g_launches.load(); }

int fk_debug_status(int reset, int *code, long long *index) {
#ifdef FK_DEBUG
    int (*readers[])(int, unsigned long long *) = {dbg_api, dbg_cc, dbg_tc, dbg_chi2, dbg_oz};
    unsigned long long first = 0;
    for (auto rd : readers) {
        unsigned long long w = 0;
        const int rc = rd(reset, &w);
        if (rc) return rc;
        if (!first) first = w;
    }
    if (code) *code = (int)(first >> 40);
    if (index) *index = (long long)(first & ((1ull << 40) - 1));
    return FK_OK;
#else
    (void)reset;
    if (code) *code = 0;
    if (index) *index = 0;
    return fail(FK_EUNSUPPORTED, "fk_debug_status: not a debug build (libfk_debug.so)");
#endif
}

int fk_debug_selftest(void) {
#ifdef FK_DEBUG
    int *buf = nullptr;
    FK_CUDA(cudaMalloc(&buf, 4 * sizeof(int)));
    unsigned long long w = 0;
    int rc = dbg_api(1, &w);
    if (!rc) {
        k_dbg_selftest<<<1, 1>>>(buf, 4, 4);  // index 4 of 4: the check must catch it
        count_launch();
        const cudaError_t e = cudaDeviceSynchronize();
        if (e) rc = cuda_fail(e, "fk_debug_selftest");
    }
    if (!rc) rc = dbg_api(1, &w);
    cudaFree(buf);
    if (rc) return rc;
    if ((w >> 40) != 99 || (w & ((1ull << 40) - 1)) != 4)
        return fail(FK_ECUDA, "fk_debug_selftest: the failed check was not reported");
    return FK_OK;
#else
    return fail(FK_EUNSUPPORTED, "fk_debug_selftest: not a debug build (libfk_debug.so)");
#endif
}

int fk_device_status(int reset) {
    const int a = device_status(reset);
    const int b = cc_device_status(reset);
    return a != FK_OK ? a : b;
}

int fk_table_create_dis(const double *fk, int ndata, const int *flav, int nflav, int nx,
                        const int *xmap, int nx_grid, unsigned prec_mask, fk_table **out) {
    return table_create(FK_KIND_DIS, fk, ndata, flav, nullptr, nflav, nx, xmap, nx_grid, prec_mask, out);
}

int fk_table_create_had(const double *fk, int ndata, const int *ca, const int *cb, int nc, int nx,
                        const int *xmap, int nx_grid, unsigned prec_mask, fk_table **out) {
    return table_create(FK_KIND_HAD, fk, ndata, ca, cb, nc, nx, xmap, nx_grid, prec_mask, out);
}

int fk_table_destroy(fk_table *t) {
    table_free(t);
    return FK_OK;
}

int fk_table_info(const fk_table *t, int *kind, int *ndata, int *nchannels, int *nx, int *nx_grid,
                  unsigned *prec_mask, size_t *device_bytes) {
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (kind) *kind = t->kind;
    if (ndata) *ndata = t->ndata;
    if (nchannels) *nchannels = t->nch;
    if (nx) *nx = t->nx;
    if (nx_grid) *nx_grid = t->nxg;
    if (prec_mask) *prec_mask = t->mask | (t->tc.lum_on ? FK_TABLE_LUMI : 0u);
    if (device_bytes) *device_bytes = t->bytes;
    return FK_OK;
}

int fk_dis_conv(const fk_table *t, const void *F, int R, void *O, int ldo, int prec,
                fk_stream stream) {
    int rc = check_conv(t, FK_KIND_DIS, F, R, O, ldo, prec);
    if (rc) return rc;
    ldo = ldo ? ldo : t->ndata;
    if (prec == FK_FP64 || prec == FK_FP32)
        return fwd_cc(t, F, R, O, ldo, prec == FK_FP64, (cudaStream_t)stream);
    if (prec == FK_FP64_TC) return oz_dis(t, (const double *)F, R, (double *)O, ldo, (cudaStream_t)stream);
    return dis_tc(t, (const float *)F, R, (float *)O, ldo, prec, (cudaStream_t)stream);
}

int fk_had_conv(const fk_table *t, const void *F, int R, void *O, int ldo, int prec,
                fk_stream stream) {
    int rc = check_conv(t, FK_KIND_HAD, F, R, O, ldo, prec);
    if (rc) return rc;
    ldo = ldo ? ldo : t->ndata;
    if (prec == FK_FP64 || prec == FK_FP32)
        return fwd_cc(t, F, R, O, ldo, prec == FK_FP64, (cudaStream_t)stream);
    if (prec == FK_FP64_TC) return oz_had(t, (const double *)F, R, (double *)O, ldo, (cudaStream_t)stream);
    return fwd_tc(t, (const float *)F, R, (float *)O, ldo, prec, (cudaStream_t)stream);
}

int fk_table_create_dense(const double *fk, int ndata, long long K, unsigned prec_mask, fk_table **out) {
    return dense_create(fk, ndata, K, prec_mask, out);
}

int fk_dense_conv(const fk_table *t, const void *L, int R, void *O, int ldo, int prec, fk_stream stream) {
    int rc = check_conv(t, FK_KIND_DENSE, L, R, O, ldo, prec);
    if (rc) return rc;
    ldo = ldo ? ldo : t->ndata;
    if (prec == FK_FP64 || prec == FK_FP32)
        return dense_cc(t, L, R, O, ldo, prec == FK_FP64, (cudaStream_t)stream);
    if (prec == FK_FP64_TC) return oz_dense(t, (const double *)L, R, (double *)O, ldo, (cudaStream_t)stream);
    return dense_tc(t, (const float *)L, R, (float *)O, ldo, prec, (cudaStream_t)stream);
}

int fk_luminosity(const fk_table *t, const void *F, int R, void *L, int prec, fk_stream stream) {
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (t->kind != FK_KIND_HAD) return fail(FK_EINVAL, "the PDF matrix needs a hadronic table");
    if (!F || !L) return fail(FK_EINVAL, "null F or L");
    if (R < 1) return fail(FK_EINVAL, "R < 1");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "unknown precision");
    return luminosity_cc(t, F, R, L, FK_IO64(prec), (cudaStream_t)stream);
}

int fk_saved_size(const fk_table *t, int R, int prec, size_t *bytes) {
    if (!bytes) return fail(FK_EINVAL, "null bytes");
    *bytes = 0;
    const int rc = check_saved(t, R, prec, nullptr, 0, false);
    if (rc) return rc;
    *bytes = saved_elems(t, R) * sizeof(float);
    return FK_OK;
}

int fk_had_conv_save(const fk_table *t, const void *F, int R, void *O, int ldo, void *saved, size_t saved_bytes,
                     int prec, fk_stream stream) {
    int rc = check_conv(t, FK_KIND_HAD, F, R, O, ldo, prec);
    if (!rc) rc = check_saved(t, R, prec, saved, saved_bytes, true);
    if (rc) return rc;
    ldo = ldo ? ldo : t->ndata;
    return fwd_tc_save(t, (const float *)F, R, (float *)O, ldo, (float *)saved, prec, (cudaStream_t)stream);
}

int fk_conv_backward_saved(const fk_table *t, const void *F, const void *gO, int ldgo, int R, const void *saved,
                           size_t saved_bytes, void *gF, int accumulate, int prec, fk_stream stream) {
    int rc = check_saved(t, R, prec, saved, saved_bytes, true);
    if (rc) return rc;
    if (!F || !gO || !gF) return fail(FK_EINVAL, "null F, gO or gF");
    if (ldgo < 0 || (ldgo > 0 && ldgo < t->ndata)) return fail(FK_EINVAL, "ldgo < ndata");
    ldgo = ldgo ? ldgo : t->ndata;
    return bwd_tc_saved(t, (const float *)F, (const float *)gO, ldgo, R, (const float *)saved, (float *)gF,
                        accumulate ? 1 : 0, prec, (cudaStream_t)stream);
}

int fk_conv_backward(const fk_table *t, const void *F, const void *gO, int ldgo, int R, void *gF,
                     int accumulate, int prec, fk_stream stream) {
    if (!t) return fail(FK_EINVAL, "table is NULL");
    if (t->kind == FK_KIND_DENSE) return fail(FK_EUNSUPPORTED, "no adjoint for dense tables");
    if (!gO || !gF || (t->kind == FK_KIND_HAD && !F)) return fail(FK_EINVAL, "null F, gO or gF");
    if (R < 1) return fail(FK_EINVAL, "R < 1");
    if (ldgo < 0 || (ldgo > 0 && ldgo < t->ndata)) return fail(FK_EINVAL, "ldgo < ndata");
    if (prec < FK_FP64 || prec > FK_FP64_TC) return fail(FK_EINVAL, "unknown precision");
    if (!(t->mask & FK_PREC_BIT(prec))) return fail(FK_EUNSUPPORTED, "precision not stored in this table");
    const bool f64 = prec == FK_FP64;
    ldgo = ldgo ? ldgo : t->ndata;
    if (prec == FK_FP64_TC)
        return oz_bwd(t, (const double *)F, (const double *)gO, ldgo, R, (double *)gF, accumulate ? 1 : 0,
                      (cudaStream_t)stream);
    if (prec != FK_FP64 && prec != FK_FP32) {  // tensor-core modes
        if (t->kind == FK_KIND_DIS)
            return dis_bwd_tc(t, (const float *)gO, ldgo, R, (float *)gF, accumulate ? 1 : 0, prec,
                              (cudaStream_t)stream);
        return bwd_tc(t, (const float *)F, (const float *)gO, ldgo, R, (float *)gF, accumulate ? 1 : 0,
                      prec, (cudaStream_t)stream);
    }
    return bwd_cc(t, F, gO, ldgo, R, gF, accumulate ? 1 : 0, f64, (cudaStream_t)stream);
}

}  // extern "C"
