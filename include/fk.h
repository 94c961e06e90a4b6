/*
 * fk.h -- C ABI of the B300 FK-table convolution library (libfk.so).
 *
 * The library evaluates the observables of a PDF fit from precomputed Fast
 * Kernel (FK) tables, as in Sec. 3 of arXiv:1909.10547 ("Towards hardware
 * acceleration for parton densities estimation"):
 *
 *   hadronic (Eq. 1):  O[r][d] = sum_c sum_i sum_j FK[d][c][i][j] f^r_{a_c}(x_i) f^r_{b_c}(x_j)
 *   DIS:               O[r][d] = sum_k sum_i     FK[d][k][i]    f^r_{a_k}(x_i)
 *
 * for R PDF replicas r at once (Sec. 3: fitting all replicas simultaneously on
 * the accelerator), together with the gradient of the observables with
 * respect to the PDF (the custom operator's gradient, Sec. 3 and Table 1), the
 * chi^2 of the fit with an FP64 Cholesky-factorised covariance, and a
 * continuously batched serving loop over device-resident tables.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status (FK_OK = 0 or an FK_E* code) and
 *    never throws.  fk_last_error_message() gives a human-readable detail for
 *    the calling thread's last failure.
 *  - Flavours are the 14 evolution-basis flavours, indexed 0..13.
 *  - PDF replicas F are laid out [R][14][nx_grid], row-major, where nx_grid is
 *    the size of the x grid the PDFs are sampled on.  A table is defined on nx
 *    of those points; xmap[i] (strictly increasing is not required, but the
 *    entries must be distinct) gives the grid index of the table's x_i.
 *  - Observables O are laid out [R][ndata]; gradients gF like F.
 *  - "Device" pointers are CUDA global-memory pointers on the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every buffer it
 *    passes; the library owns tables, covariances and servers, which live until
 *    the matching *_destroy call.
 *  - Asynchronous calls (fk_*_conv, fk_conv_backward, fk_chi2) enqueue work on
 *    `stream` (a cudaStream_t; NULL means the legacy default stream) and return
 *    before it completes.  Input buffers must stay valid, and outputs must not
 *    be read, until the stream has reached that point.  Temporary device
 *    memory comes from CUDA's stream-ordered allocator on the same stream.
 *    The first table created configures the device's default memory pool:
 *    freed memory stays in the pool (release threshold at its maximum), and
 *    a block freed on one stream is reused on another only once its free is
 *    known complete through event dependencies (opportunistic reuse and
 *    internal dependencies off), so that after work spread over many
 *    streams an allocation costs no more host time than before.
 *  - Argument errors are detected on the host before anything is enqueued:
 *    such a call returns FK_EINVAL and enqueues nothing.
 */
#ifndef FK_H
#define FK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fk_table fk_table;
typedef struct fk_cov fk_cov;
typedef struct fk_server fk_server;
typedef void *fk_stream; /* cudaStream_t */

/* Status codes. */
enum {
    FK_OK = 0,
    FK_EINVAL = 1,      /* bad argument (shape, pointer, precision, index) */
    FK_ENOMEM = 2,      /* device or host allocation failed */
    FK_EBUDGET = 3,     /* request can never fit the server's memory budget */
    FK_EPENDING = 4,    /* served request not finished yet */
    FK_ETIMEDOUT = 5,   /* a bounded wait ran out */
    FK_ECUDA = 6,       /* a CUDA runtime call or kernel launch failed */
    FK_ENOTFOUND = 7,   /* unknown ticket or table id */
    FK_EUNSUPPORTED = 8, /* precision not stored in this table, or not offered */
    FK_ECANCELED = 9    /* served request cancelled (or its server destroyed first) */
};

/* Arithmetic modes.  FP64 and FP32 read and write buffers of that type.  The
 * reduced modes read FP32 F and write FP32 O; the table's stored copy and the
 * packed PDF operand are rounded to the mode's type, products go through the
 * tensor cores and accumulate in FP32.  BF16X3 splits each operand into
 * hi = bf16(v), lo = bf16(v - hi) and sums hi*hi + hi*lo + lo*hi.
 * FP64_TC reads and writes FP64 buffers and gives FP64 results on the tensor
 * cores: every FP64 operand is split, per row and per K chunk of up to 512
 * elements, into 8 exact BF16 digits of 7 bits (each value held to 2^-55 of
 * the largest of its row in the chunk); the 36 most significant digit
 * products run as BF16 MMAs whose FP32 sums are exact, and are scaled and
 * added in FP64 in a fixed order (the slicing of Ozaki et al.).  It is
 * offered for dense tables (fk_dense_conv), DIS tables (forward and adjoint)
 * and hadronic tables (forward through the PDF matrix of the paper's Table 3,
 * adjoint through W = gO FK); the table stores the digit slices (16 bytes
 * per element, twice for DIS and hadronic tables: one copy per product). */
enum {
    FK_FP64 = 0,
    FK_FP32 = 1,
    FK_BF16 = 2,
    FK_BF16X3 = 3,
    FK_TF32 = 4,
    FK_FP64_TC = 5
};
#define FK_PREC_BIT(p) (1u << (p))
/* Forward formulation of a hadronic table in the reduced modes (BF16,
 * BF16X3, TF32), fixed when the table is created so that a replica's result
 * never depends on R:
 *  - factorised: the tensor cores contract (channel, x_j) for each first
 *    flavour a and the epilogue applies f_a(x_i) and sums over x_i;
 *  - dense: the paper's formulation (Sec. 3, Table 3), the table flattened
 *    to [ndata][(c, i, j)] times the PDF matrix
 *    L[r][(c, i, j)] = f_{a_c}(x_i) f_{b_c}(x_j), with L formed stage by stage
 *    in shared memory (never in device memory) and K split into fixed runs
 *    of 1536 columns whose partial results are added in a fixed order.  The
 *    table then also stores the flattened packing.
 * The factorised form is the default; FK_TABLE_LUMI in the prec_mask of
 * fk_table_create_had selects the dense form (forming the PDF matrix costs
 * the SM more issue slots per stage than the MMAs take, so it is slower on
 * the tables measured), FK_TABLE_FACTORED states the default explicitly;
 * fk_table_info reports FK_TABLE_LUMI in the mask when the dense form is
 * used.  The adjoint is factorised in either case. */
#define FK_TABLE_FACTORED (1u << 16)
#define FK_TABLE_LUMI (1u << 17)
/* Modes whose buffers are double: FK_FP64 and FK_FP64_TC. */
#define FK_IO64(p) ((p) == FK_FP64 || (p) == FK_FP64_TC)

/* Table kinds reported by fk_table_info. */
enum { FK_KIND_DIS = 0, FK_KIND_HAD = 1, FK_KIND_DENSE = 2 };

/* ---------------------------------------------------------------- errors */

/* Static description of a status code. */
const char *fk_strerror(int status);
/* Detail of the calling thread's most recent failure ("" if none). */
const char *fk_last_error_message(void);
/* Library ABI version (major * 100 + minor). */
int fk_version(void);
/* Number of CUDA kernels this library has launched in this process so far
 * (all threads, all devices); for accounting in benchmarks. */
uint64_t fk_kernel_launches(void);
/* Device-side health of the current device: every wait inside the library's
 * pipelined kernels (tensor-core convolution and adjoint, factorised CUDA-core
 * convolution: waits on a copy, an MMA or another warp) is bounded in time; if
 * one ran out, the kernel stopped early, left its outputs incomplete and
 * raised a flag.  Returns FK_ETIMEDOUT if the flag is set, else FK_OK; clears
 * it if reset != 0.  Synchronises with the device (a blocking copy). */
int fk_device_status(int reset);
/* Check of that mechanism: launches one thread that waits, through the same
 * bounded wait the tensor-core kernels use but with a limit of limit_us
 * microseconds (1 .. 1000000), on a barrier nothing arrives on; the wait runs
 * out, the kernel returns and raises the flag.  Synchronises with the device.
 * Returns FK_OK if the flag was raised (and clears it; a flag set before the
 * call is cleared too), FK_ECUDA otherwise.  The device stays usable. */
int fk_wait_selftest(int limit_us);

/*
 * Debug builds.  libfk_debug.so (python -m paper_1909_10547_b300.build
 * --debug; loaded by the Python binding when FK_DEBUG=1) compiles index
 * checks into the kernels: a check that fails records its code and the
 * offending index in a device word and skips the access instead of touching
 * memory out of range, and every per-call scratch buffer carries guard bytes
 * that are verified when the call's scratch is released (code 90).
 * fk_debug_status reads the first failed check since the last reset (code 0:
 * none) and clears it if reset != 0; fk_debug_selftest launches one check
 * that must fail (index 4 of a 4-element buffer, code 99) and verifies it is
 * reported.  Both return FK_EUNSUPPORTED in a release build.  They have no
 * counterpart in the paper.
 */
int fk_debug_status(int reset, int *code, long long *index);
int fk_debug_selftest(void);

/* ---------------------------------------------------------------- tables */

/*
 * DIS FK table: fk is HOST memory, [ndata][nflav][nx] FP64, holding the
 * slices of the nflav active flavours flav[0..nflav) (each in 0..13,
 * distinct).  xmap (host, [nx], may be NULL for the identity with
 * nx_grid == nx) maps x_i to the PDF grid of size nx_grid.  prec_mask is an OR
 * of FK_PREC_BIT(p) for each precision to keep on the device.  The data are
 * copied; the caller may free its arrays on return.
 * Errors: FK_EINVAL (sizes <= 0, nx_grid < nx, flavour or xmap out of range,
 * empty mask), FK_ENOMEM, FK_ECUDA.
 */
int fk_table_create_dis(const double *fk, int ndata, const int *flav, int nflav, int nx,
                        const int *xmap, int nx_grid, unsigned prec_mask, fk_table **out);

/*
 * Hadronic FK table (Eq. 1): fk is HOST memory, [ndata][nc][nx][nx] FP64, one
 * nx*nx block per active channel c coupling flavour ca[c] at x_i (first x
 * index) with flavour cb[c] at x_j (second x index).  Channels are ordered
 * pairs and must be distinct; (a, a) is allowed.  prec_mask may also hold
 * one of FK_TABLE_FACTORED / FK_TABLE_LUMI (both: FK_EINVAL).  Other
 * arguments as for fk_table_create_dis.
 */
int fk_table_create_had(const double *fk, int ndata, const int *ca, const int *cb, int nc,
                        int nx, const int *xmap, int nx_grid, unsigned prec_mask,
                        fk_table **out);

/* Frees the table's device memory.  NULL is accepted. */
int fk_table_destroy(fk_table *t);

/* Shape and resident size of a table.  Any output pointer may be NULL.
 * prec_mask holds the stored precisions, plus FK_TABLE_LUMI when the
 * reduced-mode forward of a hadronic table uses the dense form. */
int fk_table_info(const fk_table *t, int *kind, int *ndata, int *nchannels, int *nx,
                  int *nx_grid, unsigned *prec_mask, size_t *device_bytes);

/* ---------------------------------------------------------- convolution */

/*
 * DIS observables of table t (kind DIS) for R >= 1 replicas.  FP64 and FP32
 * run on the CUDA cores; the reduced modes run the plain product
 * O[r][d] = sum_{(k,i)} FK[d][(k,i)] F[r][flav[k]][xmap[i]] on the tensor
 * cores (M = replicas, N = data points, K = active flavours x points, never
 * split, so a replica's result does not depend on R).
 * F: DEVICE [R][14][nx_grid] (double for FK_FP64, float otherwise).
 * O: DEVICE, same type, replica r's ndata values at O + r * ldo (ldo = 0
 *    means ldo = ndata, i.e. a dense [R][ndata] array); overwritten.  A
 *    larger ldo lets several tables write into one [R][sum ndata] vector.
 * Errors: FK_EINVAL (wrong kind, R < 1, NULL pointer, 0 < ldo < ndata),
 * FK_EUNSUPPORTED (precision not in the table's mask), FK_ENOMEM, FK_ECUDA.
 */
int fk_dis_conv(const fk_table *t, const void *F, int R, void *O, int ldo, int prec,
                fk_stream stream);

/* Hadronic observables (Eq. 1) of table t (kind HAD); arguments as above. */
int fk_had_conv(const fk_table *t, const void *F, int R, void *O, int ldo, int prec,
                fk_stream stream);

/* -------------------------------------- dense product (Sec. 3, Table 3) */

/*
 * The dense formulation the paper times in Sec. 3 (Table 3): an FK table
 * flattened to [ndata][K] times a "PDF matrix" with K rows per replica,
 *   O[r][d] = sum_k fk[d][k] * L[r][k].
 * With L from fk_luminosity this is Eq. 1 again; any K and any L are accepted.
 *
 * fk: HOST [ndata][K] doubles, copied into device memory the table owns, in
 * the precisions of prec_mask (FP64, FP32, BF16, BF16 hi+lo, TF32).
 * fk_table_info reports kind FK_KIND_DENSE, nchannels = nx = nx_grid = 0.
 * Errors: FK_EINVAL (NULL, ndata < 1, K < 1 or K > 2^30, bad mask),
 * FK_ENOMEM, FK_ECUDA.
 */
int fk_table_create_dense(const double *fk, int ndata, long long K, unsigned prec_mask,
                          fk_table **out);

/*
 * O = FK L for a dense table t.  L: DEVICE [R][K], replica-major (double for
 * FK_FP64, float otherwise; the reduced modes round it to the mode, as F in
 * fk_had_conv).  O: DEVICE, as in fk_had_conv (ldo = 0: [R][ndata]),
 * overwritten.  FP64 and FP32 run on the CUDA cores, BF16 / BF16 hi+lo / TF32
 * on the tensor cores with FP32 accumulation.  Asynchronous on stream.  The
 * summation order depends on R (the streaming kernel serves R <= 4, and the
 * tensor-core modes split K when the tiles leave SMs idle), so unlike
 * fk_had_conv a replica's last bits may differ between calls with different R.
 * Errors: as fk_had_conv (a table of another kind: FK_EINVAL).
 */
int fk_dense_conv(const fk_table *t, const void *L, int R, void *O, int ldo, int prec,
                  fk_stream stream);

/*
 * The PDF matrix of hadronic table t for fk_dense_conv (the luminosity the
 * paper forms before its Table 3 product):
 *   L[r][(c * nx + i) * nx + j] = F[r][ca[c]][xmap[i]] * F[r][cb[c]][xmap[j]],
 * K = nc * nx * nx.  F: DEVICE [R][14][nx_grid]; L: DEVICE [R][K], written;
 * both double for FK_FP64 and float for every other prec.  Asynchronous.
 * Errors: FK_EINVAL (not a hadronic table, NULL pointer, R < 1, unknown
 * prec), FK_ECUDA.
 */
int fk_luminosity(const fk_table *t, const void *F, int R, void *L, int prec, fk_stream stream);

/*
 * fk_had_conv for FK_FP64 and FK_FP32 without any device allocation.  The
 * paper has no counterpart to this entry point: it exists for callers that
 * may not allocate device memory while they run (for example an application
 * whose GPU memory is entirely owned by its own allocator or capped by a pool
 * limit, or a latency-critical loop in which an allocation could wait on the
 * driver).  Arguments, layouts and results are those of fk_had_conv.
 *  - Temporary partial sums go to one static device array of 8 MiB that every
 *    GPU loading this library reserves until the process exits.  A call whose
 *    partial sums do not fit (roughly ndata * ceil(E / 4096) values for R = 1,
 *    R * ndata * min(nc, ~300 / ceil(ndata / 128)) values otherwise, of 8 or
 *    4 bytes; E = nc * nx * nx) returns FK_EINVAL and says how many bytes it
 *    needed; split the replicas over several calls.
 *  - The first call on each device looks up the array's device address (a
 *    one-time set-up); make that first call before any stream capture.
 *  - All calls share the array and nothing is carried from one call to the
 *    next; calls whose work overlaps on the GPU (for example on two streams
 *    with no ordering between them) race on it and give wrong results, so
 *    order them on one stream or with events.
 * Errors: FK_EINVAL (as fk_had_conv, or scratch too small), FK_EUNSUPPORTED
 * (reduced modes, or precision not stored), FK_ECUDA.
 */
int fk_had_conv_noalloc(const fk_table *t, const void *F, int R, void *O, int ldo, int prec,
                        fk_stream stream);

/*
 * Adjoint of the convolution (the gradient of Sec. 3 / Table 1):
 *   gF[r][a][xmap[i]] (+)= sum_d gO[r][d] * dO[r][d] / df^r_a(x_i)
 * for either table kind.  F: DEVICE [R][14][nx_grid]; gO: DEVICE, replica
 * r's ndata values at gO + r * ldgo (ldgo = 0 means ndata); gF: DEVICE
 * [R][14][nx_grid]; all of the mode's I/O type (double for FK_FP64, float
 * otherwise).  accumulate = 0 overwrites all of gF (grid points the table does
 * not use are set to 0); accumulate = 1 adds into gF, so the gradients of
 * several tables sharing one grid can be summed in call order.  F is not read
 * for DIS tables (may be NULL).  The reduced modes run on the tensor cores
 * with the forward's operand rounding.  Hadronic tables: the products of the
 * table with the PDF of one flavour go through the MMA in the mode's type with
 * FP32 accumulation, and gO and the remaining PDF factor are applied in FP32.
 * DIS tables: the product gO FK (K = data points) goes through the MMA with gO
 * rounded to the mode, then is scattered onto the grid.  Dense tables have no
 * adjoint here (FK_EUNSUPPORTED).
 */
int fk_conv_backward(const fk_table *t, const void *F, const void *gO, int ldgo, int R,
                     void *gF, int accumulate, int prec, fk_stream stream);

/*
 * Saved forward products, for a fit step that runs the forward and then the
 * adjoint of the same replicas (Sec. 2: each step of the gradient descent
 * evaluates the observables, the chi^2 and its gradient).  With the channels
 * of a hadronic table grouped by their first flavour a_g, the tensor-core
 * forward forms, per group g, data point d and x point i,
 *   Y_g[r][d][i] = sum_{c in g, j} FK[d][c][i][j] f^r_{b_c}(x_j)
 * and reduces it with f^r_{a_g}(x_i) into O (Eq. 1).  The adjoint's
 * derivative with respect to f^r_{a_g}(x_i) is sum_d gO[r][d] Y_g[r][d][i]:
 * the same products, contracted with gO instead.  fk_had_conv_save keeps
 * them, and fk_conv_backward_saved forms that term from them instead of a
 * second tensor-core pass over the table; the other term (derivative with
 * respect to the second flavour) is computed as in fk_conv_backward.
 * Hadronic tables in the factorised form (not FK_TABLE_LUMI) and the modes
 * FK_BF16, FK_BF16X3, FK_TF32 only.
 *
 * fk_saved_size: *bytes = the size of the buffer the two calls need for
 * table t, R replicas and prec (4 * ceil(ndata / G) * groups * G * nx *
 * ceil(R / 128) * 128, G the table's data points per tile; about
 * 4 * ndata * groups * nx * R).  *bytes = 0 on error.
 * fk_had_conv_save: fk_had_conv (same arguments, O bit for bit the same) that
 * also writes the products to saved (DEVICE, 4-byte aligned, saved_bytes at
 * least fk_saved_size; the layout is the library's own, and the part of it
 * that belongs to padding replicas past R is left unwritten).
 * fk_conv_backward_saved: fk_conv_backward (same arguments, gF bit for bit
 * the same) for a saved buffer written by fk_had_conv_save with the same
 * table, F, R and prec, ordered before this call (same stream or an event).
 * Nothing checks that: products of another F give that F's first term.
 * Errors: FK_EINVAL (as fk_had_conv / fk_conv_backward, NULL or misaligned
 * saved, saved_bytes too small: the message gives the size needed),
 * FK_EUNSUPPORTED (another mode, a mode not stored, a dense-form table),
 * FK_ENOMEM, FK_ECUDA.
 */
int fk_saved_size(const fk_table *t, int R, int prec, size_t *bytes);
int fk_had_conv_save(const fk_table *t, const void *F, int R, void *O, int ldo, void *saved,
                     size_t saved_bytes, int prec, fk_stream stream);
int fk_conv_backward_saved(const fk_table *t, const void *F, const void *gO, int ldgo, int R,
                           const void *saved, size_t saved_bytes, void *gF, int accumulate, int prec,
                           fk_stream stream);

/*
 * Sum of gradient buffers, for adjoints computed concurrently (on several
 * streams, each into its own buffer) that must be combined in a fixed order:
 *   out[e] (+)= parts[0][e] + parts[1][e] + ... + parts[nparts-1][e]
 * parts: HOST array of nparts (1..64) DEVICE pointers to n elements each;
 * out: DEVICE, n elements; element type double for FK_FP64, float otherwise.
 * The sum runs in the listed order, so the result does not depend on timing.
 */
int fk_grad_sum(const void *const *parts, int nparts, long long n, void *out, int accumulate,
                int prec, fk_stream stream);

/* ---------------------------------------------------------------- chi^2 */

/*
 * Block-diagonal experimental covariance, one dense SPD block per dataset.
 * C_blocks: HOST FP64, the blocks one after another, each row-major
 * [n_k][n_k]; block_sizes: HOST [nblocks], each 1 .. 46340, their sum at most
 * 2^30.  The blocks are copied to the device and factorised there in FP64
 * (C_k = L_k L_k^T); the 32 x 32 diagonal blocks of L_k (and of L_k^T read
 * backwards) are inverted for the blocked substitutions of fk_chi2.  The call
 * synchronises with the device.  Errors: FK_EINVAL (sizes, or a block that is
 * not positive definite: a non-positive pivot), FK_ENOMEM, FK_ECUDA.
 */
int fk_cov_create(const double *C_blocks, const int *block_sizes, int nblocks, fk_cov **out);
int fk_cov_destroy(fk_cov *cov);
/* Total dimension sum_k n_k (0 for NULL). */
int fk_cov_size(const fk_cov *cov);

/*
 * chi^2 per replica: chi2[r] = (O_r - D)^T C^{-1} (O_r - D), evaluated in
 * FP64 as |z|^2 blockwise, z the solution of L z = O_r - D by blocked forward
 * substitution (panels of 32 rows).  If gO is not NULL it receives
 * d chi2[r] / d O_r = 2 C^{-1} (O_r - D) = 2 w, w the solution of L^T w = z
 * by blocked back substitution.  One kernel launch per call (two when the
 * covariance has several blocks: their chi^2 are then added in block order);
 * a replica's results do not depend on R or on the other replicas.
 * O: DEVICE [R][n] and gO: DEVICE [R][n] or NULL, both double if io_prec is
 * FK_FP64 and float for any other mode (so the observables and gradient of a
 * reduced-precision fit need no conversion; the arithmetic is FP64 either
 * way).  D: DEVICE [n] double; chi2: DEVICE [R] double (n = fk_cov_size).
 * Errors: FK_EINVAL, FK_ENOMEM, FK_ECUDA.
 */
int fk_chi2(const fk_cov *cov, const void *O, const double *D, int R, double *chi2, void *gO,
            int io_prec, fk_stream stream);

/*
 * chi^2 of whitened observables.  With C = L L^T, chi2 = (O - D)^T C^{-1}
 * (O - D) = |L^{-1} O - L^{-1} D|^2, and L^{-1} O is the convolution of the
 * tables multiplied by L^{-1} (the whitened tables, formed once when a fit is
 * set up, since the covariance does not change during it).  Given Z = L^{-1} O
 * and Dw = L^{-1} D:
 *   chi2[r] = sum_i (Z[r][i] - Dw[i])^2,  gO[r][i] = 2 (Z[r][i] - Dw[i]) = d chi2[r] / d Z[r][i],
 * which the adjoint of the whitened tables turns into d chi2 / dF.  No
 * triangular solve is left in the step.  FP64 arithmetic; each sum runs in an
 * order that depends on n only.  Z: DEVICE, replica r's n values at
 * Z + r * ldz (ldz = 0: n); gO: DEVICE at gO + r * ldg (ldg = 0: n) or NULL;
 * both double if io_prec is FK_FP64 and float otherwise.  Dw: DEVICE [n]
 * double; chi2: DEVICE [R] double.  Asynchronous.  Errors: FK_EINVAL (NULL
 * pointer, n < 1, R < 1, ldz or ldg < n, unknown precision), FK_ECUDA.
 */
int fk_chi2_white(const void *Z, int ldz, const double *Dw, int n, int R, double *chi2, void *gO, int ldg,
                  int io_prec, fk_stream stream);

/* ----------------------------------------------------- gradient descent */

/*
 * PDF parametrisation for the fit, which minimises chi^2 by gradient descent
 * over the parameters of the PDFs (Sec. 2; the paper's parametrisation is a
 * neural network, the analytic form below stands in for it).  Per replica r
 * and flavour a:
 *   f^r_a(x) = exp(t[r][a][0] + t[r][a][1] ln x + t[r][a][2] ln(1 - x)),
 * i.e. A x^alpha (1 - x)^beta with t = (ln A, alpha, beta).
 * theta: DEVICE [R][14][3]; x_grid: DEVICE [nx_grid] double, 0 < x < 1;
 * F: DEVICE [R][14][nx_grid].  theta and F are double for FK_FP64 and float
 * for any other mode; the exponent is evaluated in that type.
 * Errors: FK_EINVAL.
 */
int fk_pdf_eval(const void *theta, int R, const double *x_grid, int nx_grid, void *F, int prec,
                fk_stream stream);

/*
 * Chain rule through fk_pdf_eval:
 *   gtheta[r][a][k] = sum_m gF[r][a][m] * dF[r][a][m] / dtheta[r][a][k],
 * dF/dt0 = F, dF/dt1 = F ln x_m, dF/dt2 = F ln(1 - x_m), with F the output of
 * fk_pdf_eval for the same theta.  F, gF: DEVICE [R][14][nx_grid]; gtheta:
 * DEVICE [R][14][3]; types as for fk_pdf_eval.  The sum over the grid runs in
 * a fixed order.  Errors: FK_EINVAL.
 */
int fk_pdf_grad(const void *F, const void *gF, int R, const double *x_grid, int nx_grid, void *gtheta,
                int prec, fk_stream stream);

/*
 * One Adam step (Kingma and Ba) on n parameters, step number t >= 1:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 * p, g, m, v: DEVICE, n elements of the mode's type (m and v start at 0 and
 * are updated in place).  Errors: FK_EINVAL.
 */
int fk_adam_step(void *p, const void *g, void *m, void *v, long long n, int t, double lr, double b1,
                 double b2, double eps, int prec, fk_stream stream);

/* ------------------------------------------------------------ measurement */

/*
 * Arithmetic-rate probe (no counterpart in the paper: it measures the FP32 and
 * FP64 multiply-add rates of the CUDA cores that the library's CUDA-core
 * kernels are compared against).  Launches `blocks` CTAs of 256 threads; each
 * thread runs 8 independent chains of `iters` fused multiply-adds in the
 * precision prec (FK_FP32 or FK_FP64), i.e. 2 * 8 * iters * 256 * blocks
 * flops.  sink: DEVICE, `blocks` elements of that type, never written in
 * practice (it keeps the chains from being optimised away).  Asynchronous on
 * stream.  Errors: FK_EINVAL, FK_ECUDA.
 */
int fk_fma_probe(int prec, int blocks, int iters, void *sink, fk_stream stream);

/*
 * Tensor-core issue probe: one CTA issues `iters` BF16 tcgen05.mma
 * instructions of M = 128, N = n, K = 16 back to back (shared-memory operands
 * of zeros (fill = 0) or of finite values of varying sign, exponent and
 * mantissa (fill = 1), one TMEM accumulator) and writes the SM cycles from
 * the first issue to the completion of the last to cycles[0] (DEVICE, one
 * unsigned long long; 0 if the bounded wait ran out).  Used to measure the
 * cycles one instruction takes as a function of N.  Asynchronous on stream.
 * Errors: FK_EINVAL (n not a multiple of 16 in 16..256, iters outside
 * 1..2^24, fill not 0 or 1, cycles NULL), FK_ECUDA.
 */
int fk_mma_probe(int n, int iters, int fill, unsigned long long *cycles, fk_stream stream);

/* -------------------------------------------------------------- serving */

/*
 * A server owns a scheduler thread and its own CUDA streams.  Tables added to
 * it stay resident on the device.  Requests (table, PDF replicas, precision)
 * are admitted while the device memory they need fits in hbm_budget_bytes
 * (counting the resident tables) and fewer than max_inflight are running;
 * requests on the same table and precision that are waiting together are
 * coalesced along the replica axis into one launch.  Each result equals the
 * same request run alone (bit for bit in FK_FP64 and FK_FP32 modes).
 */
int fk_serve_create(size_t hbm_budget_bytes, int max_inflight, fk_server **out);
/* Registers table t (the server does not take ownership; keep t alive until
 * fk_serve_destroy).  FK_EBUDGET if the table alone exceeds the budget,
 * FK_EUNSUPPORTED for a dense table. */
int fk_serve_add_table(fk_server *s, fk_table *t, int *table_id);
/*
 * Queues a request.  F_host: HOST [R][14][nx_grid] of the mode's I/O type; it
 * is copied before the call returns.  *ticket identifies the request.
 * FK_EBUDGET if the request could never fit the budget, FK_ENOTFOUND for an
 * unknown table id, FK_EUNSUPPORTED for a precision the table lacks.
 */
int fk_serve_submit(fk_server *s, int table_id, const void *F_host, int R, int prec,
                    uint64_t *ticket);
/*
 * Non-blocking.  If the request is done, copies its O ([R][ndata], I/O type)
 * to O_host, sets *done = 1, forgets the ticket and returns the request's
 * status; otherwise sets *done = 0 and returns FK_EPENDING.
 */
int fk_serve_poll(fk_server *s, uint64_t ticket, void *O_host, int *done);
/* As fk_serve_poll, but waits up to timeout_ms; FK_EPENDING if the request
 * has not finished by then (the ticket stays valid).  A request that finished
 * with a failure returns that failure's status (FK_ETIMEDOUT: its completion
 * was lost, see below). */
int fk_serve_wait(fk_server *s, uint64_t ticket, void *O_host, int timeout_ms);
/*
 * Counters since creation: completed requests, sum of ndata*R over them,
 * device launches, peak bytes in use (tables + in-flight requests), queue
 * depth now.  Any pointer may be NULL.
 */
int fk_serve_stats(const fk_server *s, uint64_t *completed, uint64_t *datapoint_replicas,
                   uint64_t *launches, size_t *peak_bytes, int *queued);
/*
 * Cancels a request: one not started yet is removed from the queue; one
 * running finishes but its result is discarded.  Either way its poll/wait
 * then returns FK_ECANCELED (a request already finished keeps its result).
 * FK_ENOTFOUND for an unknown ticket.
 */
int fk_serve_cancel(fk_server *s, uint64_t ticket);

/*
 * Failure detection.  Every failure of a served request ends in its own
 * status at poll/wait, and nothing waits forever:
 *  - a failed pinned staging allocation: fk_serve_submit returns FK_ENOMEM;
 *  - a failed device allocation for a batch: its requests end FK_ENOMEM;
 *  - a failed convolution launch: its requests end FK_ECUDA;
 *  - a lost completion message (the batch's work finished but the host was
 *    never told): once the batch's work has finished and 200 ms have passed,
 *    its requests end FK_ETIMEDOUT and its budget is returned;
 *  - fk_serve_destroy with requests queued: they end FK_ECANCELED.
 * fk_serve_inject arms `count` occurrences of one host-side fault, so that
 * these paths can be tested without any fault on the GPU: FK_FAULT_PINNED
 * (the next submits' pinned allocation fails), FK_FAULT_DEVICE (the next
 * batches' device allocation fails), FK_FAULT_LAUNCH (the next batches'
 * convolution launch fails), FK_FAULT_DROP (the next batches' completion
 * message is lost).  The environment variable FK_FAULT="kind:count,..."
 * (kinds pinned, device, launch, drop) arms the same at fk_serve_create.
 * The paper has no counterpart (it describes no serving).
 */
enum { FK_FAULT_PINNED = 1, FK_FAULT_DEVICE = 2, FK_FAULT_LAUNCH = 3, FK_FAULT_DROP = 4 };
int fk_serve_inject(fk_server *s, int fault, int count);

/* Stops the scheduler: requests still queued end FK_ECANCELED, the ones in
 * flight finish; frees the requests and the server. */
int fk_serve_destroy(fk_server *s);

#ifdef __cplusplus
}
#endif
#endif /* FK_H */
