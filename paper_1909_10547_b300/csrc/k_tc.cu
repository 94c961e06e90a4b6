// Many-replica hadronic convolution on the 5th-generation tensor cores
// (tcgen05, sm_103a), with TMA operand staging and TMEM accumulators.
//
// Eq. 1 per data point d and replica r, with the channels grouped by their
// first flavour a (group g, channels (a_g, b)):
//
//   O[r][d] = sum_g sum_i f^r_{a_g}(x_i) * Y_g[r][(i, d)],
//   Y_g[r][(i, d)] = sum_{(c, j) in g} F_g[r][(c, j)] * FK[d][c][i][j],
//   F_g[r][(c, j)] = f^r_{b_c}(x_j).
//
// Y_g is a dense product (M = replicas, N = (x_i, data point) rows of one
// tile, K = the group's (channel, x_j) pairs) and runs on the tensor cores;
// the Hadamard product with f^r_{a_g}(x_i) and the sum over i and g are fused
// into the epilogue, which reads Y_g straight out of TMEM.  Each thread of the
// epilogue owns one replica (one TMEM lane), so the reduction over (g, i) is a
// fixed-order register accumulation with no atomics.
//
// Roles per CTA (192 threads, persistent over tiles):
//   warp 0 lane 0 : TMA producer (A = packed PDF operand, B = packed table)
//   warp 1 lane 0 : MMA issuer; warp 1 also allocates / frees TMEM
//   warps 2..5    : epilogue, TMEM lane quarter (warp % 4)
// Pipelines: an S-stage shared-memory ring (full/empty mbarriers) and two
// 256-column TMEM accumulators (acc_full/acc_empty), so the epilogue of
// group g overlaps the MMAs of group g+1.  Every wait is bounded by the
// global timer; on time-out the CTA sets an error word, stops issuing work,
// lets its copies land, frees TMEM and returns.
#include "fk_internal.h"

#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>

namespace fk {

__device__ int g_fk_device_error;  // non-zero after a bounded wait ran out

namespace {

constexpr int TC_M = 128;   // replicas per tile (MMA M)
constexpr int TC_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr int KPAD = 16;    // K padding of each group (a multiple of both K steps)
constexpr int PW_SLACK = 2; // stages of slack for a producer-side accumulator wait

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// As mbar_try, but the thread may stay suspended in the barrier unit for up
// to `ns` nanoseconds until the phase completes: a waiting thread issues no
// instructions, so it takes no issue slots from the producer and MMA threads
// that share its scheduler.
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
constexpr uint32_t SLEEP_NS = 100000;  // suspend-time hint per poll
// Waits for the phase of the given parity.  Gives up after WAIT_NS and raises
// the device error word; `dead` latches per thread, so after one time-out a
// role stops waiting at once and the CTA drains within a few time-outs
// instead of waiting on every remaining barrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, bool &dead,
                                          uint64_t limit_ns = WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    if (dead) return false;
    const uint64_t t0 = gtimer();
    while (!mbar_try_sleep(bar, parity, SLEEP_NS)) {
        if (gtimer() - t0 > limit_ns) {
            dead = true;
            atomicExch(&g_fk_device_error, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// As tma_load_2d for a CTA pair running 2-SM MMAs: the copy lands in this
// CTA's shared memory and completes its bytes on the mbarrier at `bar`, a
// shared::cluster address that may be in the peer CTA.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                                 int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// shared::cluster address of this CTA's shared-memory address `addr` in CTA `rank`
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
// arrive on an mbarrier given by its shared::cluster address (any CTA of the cluster)
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Every thread of both CTAs of the cluster; orders mbarrier initialisation
// and shared-memory use across the pair.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128 B,
// 8-row groups 1024 B apart (SBO), descriptor version 1.
__host__ __device__ constexpr uint64_t sw128_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4)  // start address, 16-byte units
           | (uint64_t)1 << 16                  // LBO (unused for swizzled K-major)
           | (uint64_t)(1024 >> 4) << 32        // SBO
           | (uint64_t)1 << 46                  // version
           | (uint64_t)2 << 61;                 // SWIZZLE_128B
}
// The same for rows of 64 B (64-byte swizzle, 8-row groups 512 B apart).
__host__ __device__ constexpr uint64_t sw64_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4)  // start address, 16-byte units
           | (uint64_t)1 << 16                  // LBO (unused for swizzled K-major)
           | (uint64_t)(512 >> 4) << 32         // SBO
           | (uint64_t)1 << 46                  // version
           | (uint64_t)4 << 61;                 // SWIZZLE_64B
}
// The same descriptor in two words: desc_lo (start address and LBO) varies
// per operand and K step, DESC_HI (SBO, version, swizzle) is shared.
constexpr uint32_t DESC_HI = (uint32_t)(sw128_desc(0) >> 32);
constexpr uint32_t DESC_HI64 = (uint32_t)(sw64_desc(0) >> 32);
__host__ __device__ constexpr uint32_t desc_lo(uint32_t addr) { return (uint32_t)sw128_desc(addr); }
template <bool NW = false>
__host__ __device__ constexpr uint64_t desc64(uint32_t lo) {
    return ((uint64_t)(NW ? DESC_HI64 : DESC_HI) << 32) | lo;
}
static_assert(desc64(desc_lo(0x2A7C0u)) == sw128_desc(0x2A7C0u), "descriptor split");
static_assert(desc64<true>(desc_lo(0x2A7C0u)) == sw64_desc(0x2A7C0u), "descriptor split (64-byte rows)");
static_assert(desc_lo(0x2A7C0u) + 0x403u == desc_lo(0x2A7C0u + 0x4030u), "a K-step offset adds to the address field");
// D[tmem] (+)= A * B^T for one K step.  CG = 1: M = 128 rows of this CTA.
// CG = 2 (issued by the even CTA of a pair): M = 256, rows 0..127 from the even
// CTA's A and rows 128..255 from the odd CTA's A at the same shared-memory
// offset; the B rows (the N axis) are split in halves the same way; each CTA's
// TMEM receives the D rows of its own A rows over all N columns.
template <int PREC, int CG>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accum) {
    if (PREC == FK_TF32) {
        if (CG == 2)
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                "l"(a), "l"(b), "r"(idesc), "r"(accum)
                : "memory");
        else
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                "l"(a), "l"(b), "r"(idesc), "r"(accum)
                : "memory");
    } else {
        if (CG == 2)
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                "l"(a), "l"(b), "r"(idesc), "r"(accum)
                : "memory");
        else
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
                "l"(a), "l"(b), "r"(idesc), "r"(accum)
                : "memory");
    }
}
// Arrives on the mbarrier (of this CTA) once every MMA issued so far by this
// thread has completed.
template <int CG>
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    if (CG == 2)
        asm volatile(
            "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
    else
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
            : "memory");
}
// As mma_commit<2>, arriving on the mbarrier at this offset in both CTAs of the pair.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(bar), "h"((uint16_t)0x3)
        : "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t slot) {
    if (CG == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(slot) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(slot) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}
template <int CG>
__device__ __forceinline__ void tmem_free(uint32_t tmem) {
    if (CG == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}
// 64 consecutive accumulator columns of this warp's 32 TMEM lanes (one
// column per register), waited for inside the same statement so that no use
// of v can be scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
          "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
          "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr)
        : "memory");
}

// TF32 operand value: FP32 rounded to the nearest TF32, ties away from zero
__device__ __forceinline__ float tf32_rna(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

// ------------------------------------------------------------ kernel ----
// NW (narrow rows): 64-byte swizzled rows instead of 128-byte ones, so a
// stage spans half the K and half the bytes and twice as many stages fit
// (used for hi+lo on single CTAs, whose 96 KB stages otherwise allow only two).
template <int PREC, bool NW = false>
struct Tr {
    static constexpr bool X3 = PREC == FK_BF16X3;
    static constexpr int ESZ = PREC == FK_TF32 ? 4 : 2;
    static constexpr int ROWB = NW ? 64 : 128;  // bytes per swizzled row
    static constexpr int KC = ROWB / ESZ;       // K elements per swizzled row
    static constexpr int KSTEP = 32 / ESZ;      // K per MMA instruction
    static constexpr int NOPS = X3 ? 2 : 1;     // operand copies (hi, lo)
    // swizzle atoms per stage along K: two for the single-copy modes (8 MMAs
    // between stage barriers), one for hi+lo (already 12 MMAs, 6 with NW)
    static constexpr int ATOMS = X3 ? 1 : 2;
    static constexpr int KCS = KC * ATOMS;      // K elements per stage
    static constexpr uint32_t FMT = PREC == FK_TF32 ? 2u : 1u;  // TF32 : BF16
};
// Pipeline depth: a CTA of a pair holds half of each B tile, so its stages
// are smaller and more of them fit; narrow rows halve a stage again.
template <int PREC, int CL, bool NW = false>
__host__ __device__ constexpr int tc_stages() {
    return NW ? 4 : CL == 2 ? 3 : 2;
}

// Epilogue modes of the tensor-core kernel.
//  FWD: O[r][d]   = sum_g sum_i f^r_{a_g}(x_i) Y_g[r][(i, d)]
//  ADJ: P[t][g][i][r] = sum_{d in tile t} gO[r][d] Y_g[r][(i, d)]
// (with the transposed packing, i stands for x_j and g for the second flavour)
// MODE_DENSE: the plain product of the paper's Table 3 (one group spanning K,
// the accumulator columns are the tile's data points, stored as they are)
// MODE_LUMI: the same product for a hadronic table flattened to
// [ndata][(c, i, j)], with the A operand, the PDF matrix
// L[r][(c, i, j)] = f^r_{a_c}(x_i) f^r_{b_c}(x_j), formed stage by stage in
// shared memory by eight builder warps instead of loaded
enum { MODE_FWD = 0, MODE_ADJ = 1, MODE_DENSE = 2, MODE_LUMI = 3 };
// builder warps of MODE_LUMI (two per A row: each forms half of a stage's columns)
constexpr int LB_WARPS = 8;
template <int MODE>
__host__ __device__ constexpr int tc_threads() {
    return MODE == MODE_LUMI ? TC_THREADS + 32 * LB_WARPS : TC_THREADS;
}
// K columns per split of a MODE_LUMI product: a table property, so a
// replica's result does not depend on R
constexpr int LUMI_KSPLIT = 1536;

struct TcParams {
    int ntiles, nrt, nchunks, n_rows, ngroups, nx, ndata, R, R_pad, ldo;
    int nbl;  // log2 of the TMEM accumulator buffers (2 of 256 columns or 4 of 128)
    int kbeg[NFL], kend[NFL];
    uint32_t pwait;   // bit g: the producer makes group g's accumulator wait (tc_pwait)
    const float *Fm;  // forward: [ngroups][nx][R_pad] epilogue multipliers f^r_{a_g}(x_i)
    float *O;         // forward: observables, row stride ldo
    const float *gO;  // adjoint: weights gO[r * ldo + d]
    float *P;         // adjoint: partial sums [ntile_n][ngroups][nx][R_pad]
    float *Y;         // forward, optional: the products Y_g saved as [ntile_n][ngroups][nrt][G * nx][128]
    int narrow;       // host side: the launch runs hi+lo single CTAs on 64-byte rows
    // K split (dense products with fewer tiles than SMs): work item w covers
    // data tile nt and K split sp, ntile_n data tiles; split sp starts at K
    // element sp * kspl and writes its partial tile at O + sp * ostride
    int ntile_n, nsplit, kspl;
    long long ostride;
    // operand slices (FP64 on the tensor cores): work items also run over
    // npair (A slice, B slice) pairs; pair u reads A rows from
    // pa[u] * a_rows and B rows from pb[u] * b_rows and writes its partial
    // tiles at O + (u * nsplit + sp) * ostride.  npair = 1, pa = pb = 0 for
    // every other product.
    int npair, a_rows, b_rows;
    uint8_t pa[64], pb[64];
    int kbase;  // K element where split 0 starts
    // npc > 1: a work item accumulates npc operand pairs in one accumulator;
    // its stages run pair j = q / spc over the split's K (stage q % spc), and
    // pair u of the launch stands for pairs pa/pb[u * npc + j]
    int npc, spc;
    // MODE_LUMI: FT[(a * nx + x) * R_pad + r] = f^r_a(x_x) for the builders;
    // lfl[c] = a_c, lfl[MAX_CH + c] = b_c, the flavours of the table's lnc
    // channels (in the parameters: the builders' addresses need no load from
    // memory); K columns are (c, i, j) with j padded to lnxp (a power of two,
    // 16 to 64) and read as zero from j = nx
    const float *FT;
    uint8_t lfl[2 * MAX_CH];
    int lnc, lnxp;
};


template <int PREC, int CL, bool NW = false>
size_t tc_smem_bytes(int n_rows) {
    using T = Tr<PREC, NW>;
    const size_t stage = (size_t)T::NOPS * T::ATOMS * (TC_M * T::ROWB + (size_t)(n_rows / CL) * T::ROWB);
    return 1024 + tc_stages<PREC, CL, NW>() * stage + 512;
}

// One work item is a (replica tile, data tile) pair of the product
// Y_g = A_g B_g^T (A: packed PDFs, B: packed table), reduced by the epilogue.
//  CL = 1: one CTA per tile, 128 x n_rows MMAs.
//  CL = 2: a cluster of two CTAs owns replica tiles 2u and 2u+1 of one data
//  tile and runs 256 x n_rows MMAs on both SMs' tensor cores: each CTA loads
//  its own 128 A rows and one half of the B rows, so every SM takes in half of
//  the table tile.  The even CTA issues the MMAs; the copies of both CTAs
//  complete on its `full` barriers, its commits release `empty` and signal
//  `accf` in both CTAs, and both CTAs' epilogues release its `acce`.
template <int PREC, int G, int MODE, int CL, bool NW = false>
__global__ void __launch_bounds__(tc_threads<MODE>(), 1)
    k_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapA2,
         const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapB2,
         TcParams p) {
    static_assert(!NW || (CL == 1 && MODE != MODE_LUMI), "narrow rows: single CTAs, copied A operand");
    using T = Tr<PREC, NW>;
    constexpr int S = tc_stages<PREC, CL, NW>();
    const uint32_t rank = CL == 2 ? cluster_rank() : 0u;
    const bool leader = rank == 0;
    // work items: tiles (CL = 1) or pairs of replica tiles (CL = 2)
    const int w_first = CL == 2 ? (int)cluster_id() : (int)blockIdx.x;
    const int w_step = CL == 2 ? (int)cluster_count() : (int)gridDim.x;
    const int w_count = p.ntiles / CL;
    auto tile_of = [&](int w, int &rt, int &nt, int &sp, int &pr) {
        if (CL == 2) {
            const int half = p.nrt / 2;
            nt = w / half;
            rt = 2 * (w % half) + (int)rank;
        } else {
            rt = w % p.nrt;
            nt = w / p.nrt;
        }
        sp = nt / p.ntile_n;
        nt -= sp * p.ntile_n;
        pr = sp / p.nsplit;
        sp -= pr * p.nsplit;
    };
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const int b_rows = p.n_rows / CL;  // B rows held by this CTA
    const uint32_t a_bytes = TC_M * T::ROWB, b_bytes = (uint32_t)b_rows * T::ROWB;
    const uint32_t stage_bytes = T::NOPS * T::ATOMS * (a_bytes + b_bytes);
    // a stage: the A atoms, then the B atoms (then the lo copies for hi+lo)
    const uint32_t offB = T::ATOMS * a_bytes, offA2 = T::ATOMS * (a_bytes + b_bytes), offB2 = offA2 + offB;
    const uint32_t bar0 = base + S * stage_bytes;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (S + s); };
    auto accf = [&](int b) { return bar0 + 8u * (2 * S + b); };
    auto acce = [&](int b) { return bar0 + 8u * (2 * S + 4 + b); };
    const uint32_t drain = bar0 + 8u * (2 * S + 8);  // all MMAs of this CTA done
    uint8_t *gen = smem_raw + (bar0 - raw) + 8 * (2 * S + 9);
    // group bounds in shared memory (the 256 bytes after the barrier block):
    // sk[g] = kbeg, sk[NFL + g] = kend, sk[2 * NFL + h] = K of the first
    // group at or after h whose accumulator the MMA thread waits for (or
    // INT_MAX); read by the producer and the MMA thread instead of indexing
    // the kernel parameters at run time
    int *sk = reinterpret_cast<int *>(smem_raw + (bar0 - raw) + 256);
    // accumulator buffers: NB = 1 << nbl of bcols TMEM columns each; use u of
    // the accumulator is buffer u & NBM, phase u >> nbl of its barriers
    const int nbl = p.nbl, NB = 1 << nbl, NBM = NB - 1;
    const uint32_t bcols = 512u >> nbl;
    volatile uint32_t *tmem_slot = reinterpret_cast<volatile uint32_t *>(gen);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool dead = false;  // this thread's waits have timed out once
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            // MODE_LUMI: the builder warps of every CTA of the pair arrive too
            mbar_init(full(s), MODE == MODE_LUMI ? 1 + LB_WARPS * CL : 1);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < 4; ++b) {
            mbar_init(accf(b), 1);
            mbar_init(acce(b), 4 * CL);  // the epilogue warps of every CTA of the pair
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        prefetch_map(&mapA);
        prefetch_map(&mapB);
        if (T::X3) {
            prefetch_map(&mapA2);
            prefetch_map(&mapB2);
        }
    }
    if (threadIdx.x <= NFL) {
        const int h = threadIdx.x;
        if (h < p.ngroups) {
            sk[h] = p.kbeg[h];
            sk[NFL + h] = p.kend[h];
        }
        const uint32_t mwait = ~p.pwait & ((1u << p.ngroups) - 1u);
        const uint32_t m = h < p.ngroups ? mwait >> h : 0u;
        sk[2 * NFL + h] = m ? p.kbeg[h + __ffs(m) - 1] : 0x7fffffff;
    }
    if (warp == 1) tmem_alloc<CL>(smem_u32((const void *)tmem_slot));
    tc_fence_before();
    if (CL == 2)
        cluster_sync();  // the peer's barriers exist before any copy or arrive targets them
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // Launched as a programmatic dependent of the previous kernel in the
    // stream (the operand packing): the set-up above ran while that kernel
    // finished; nothing it writes is read, and nothing is written, before
    // this wait for its completion.
    asm volatile("griddepcontrol.wait;" ::: "memory");

    // groups whose accumulator hand-off the producer takes (tc_pwait)
    const uint32_t pwait = p.pwait;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int it = 0, pgc = 0;  // pgc: accumulator uses (groups) reached so far
        bool ok = true;
        for (int w = w_first; w < w_count && ok; w += w_step) {
            int rt, nt, sp, pr;
            tile_of(w, rt, nt, sp, pr);
            const int koff = p.kbase + sp * p.kspl;  // the split's first K element
            int pg = 0;  // next group whose first stage is still to be loaded
            for (int q = 0; q < p.nchunks; ++q, ++it) {
                // the operand pair and K stage of this stage (one pair unless npc > 1)
                const int j = p.npc > 1 ? q / p.spc : 0;
                const int qk = q - j * (p.npc > 1 ? p.spc : 0);
                const int u = p.npc > 1 ? pr * p.npc + j : pr;
                const int brow = p.pb[u] * p.b_rows + nt * p.n_rows + (int)rank * b_rows;
                const int arow = p.pa[u] * p.a_rows + rt * TC_M;
                const int s = it % S;
                if (leader) {
                    // the accumulator of every group starting in this stage
                    // must be free before the MMAs can read the stage
                    while (pg < p.ngroups && sk[pg] < (q + 1) * T::KCS) {
                        if (((pwait >> pg) & 1u) && !mbar_wait(acce(pgc & NBM), ((pgc >> nbl) & 1) ^ 1, dead)) {
                            ok = false;
                            break;
                        }
                        ++pg;
                        ++pgc;
                    }
                    if (!ok) break;
                }
                if (!mbar_wait(empty(s), ((it / S) & 1) ^ 1, dead)) {
                    ok = false;
                    break;
                }
                const uint32_t st = base + s * stage_bytes;
                // MODE_LUMI: only the B tiles are copied (the builders form A)
                constexpr bool LOAD_A = MODE != MODE_LUMI;
                const uint32_t tx = LOAD_A ? stage_bytes : T::NOPS * T::ATOMS * b_bytes;
                if (CL == 2) {
                    const uint32_t fb = mapa(full(s), 0);
                    if (leader) mbar_expect_tx(full(s), 2 * tx);
#pragma unroll
                    for (int a = 0; a < T::ATOMS; ++a) {
                        const int x = koff + qk * T::KCS + a * T::KC;
                        if (LOAD_A) tma_load_2d_pair(st + a * a_bytes, &mapA, fb, x, arow);
                        tma_load_2d_pair(st + offB + a * b_bytes, &mapB, fb, x, brow);
                        if (T::X3) {
                            if (LOAD_A) tma_load_2d_pair(st + offA2 + a * a_bytes, &mapA2, fb, x, arow);
                            tma_load_2d_pair(st + offB2 + a * b_bytes, &mapB2, fb, x, brow);
                        }
                    }
                } else {
                    mbar_expect_tx(full(s), tx);
#pragma unroll
                    for (int a = 0; a < T::ATOMS; ++a) {
                        const int x = koff + qk * T::KCS + a * T::KC;
                        if (LOAD_A) tma_load_2d(st + a * a_bytes, &mapA, full(s), x, arow);
                        tma_load_2d(st + offB + a * b_bytes, &mapB, full(s), x, brow);
                        if (T::X3) {
                            if (LOAD_A) tma_load_2d(st + offA2 + a * a_bytes, &mapA2, full(s), x, arow);
                            tma_load_2d(st + offB2 + a * b_bytes, &mapB2, full(s), x, brow);
                        }
                    }
                }
            }
        }
        if (ok && CL == 2) {
            // the last stages are released by commits of the peer's MMA
            // issuer: take them before the CTA may exit
            for (int j = it > S ? it - S : 0; j < it; ++j)
                if (!mbar_wait(empty(j % S), (j / S) & 1, dead)) break;
        }
        if (!ok) {
            if (leader) {
                // let the copies already issued land before the CTA exits
                // (for a pair this includes the odd CTA's halves)
                for (int k = 1; k <= S && it - k >= 0; ++k) {
                    const int j = it - k;
                    const uint64_t t0 = gtimer();
                    while (!mbar_try(full(j % S), (j / S) & 1) && gtimer() - t0 < WAIT_NS) {
                    }
                }
            } else {
                // the odd CTA's copies complete on the even CTA's barriers:
                // give them a bounded time to land
                const uint64_t t0 = gtimer();
                while (gtimer() - t0 < 1000000ull) {
                }
            }
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ------------------------------------------------ MMA issuer
        // The tensor pipe is fed best by straight-line MMA issue: the K steps
        // of a stage are unrolled, and a stage in which no group needs the
        // MMA thread to wait for the epilogue runs a loop without any wait
        // code; only stages where such a (short) group starts take the loop
        // with the wait.
        const uint32_t idesc = (1u << 4) | (T::FMT << 7) | (T::FMT << 10) |
                               ((uint32_t)(p.n_rows >> 3) << 17) | ((uint32_t)((CL * TC_M) >> 4) << 24);
        constexpr int SLOW_UNROLL = T::X3 ? 1 : T::KCS / T::KSTEP;
        // K index where the first MMA-waited group at or after group h starts
        auto next_wait_k = [&](int h) -> int { return sk[2 * NFL + h]; };
        // The issue loop does little besides issuing: the stage's descriptors
        // are built once per stage and a K step only adds its offset to the
        // start-address field (16-byte units; shared-memory addresses stay
        // below 256 KB, so the 14-bit field never carries), and the
        // accumulator address changes only when a group ends.
        const uint32_t bstep = b_bytes >> 4;           // one B atom, descriptor units
        constexpr uint32_t ASTEP = (TC_M * T::ROWB) >> 4;  // one A atom
        const int ng = p.ngroups;
        const int klast = sk[NFL + ng - 1];  // K after the last group
        int it = 0, gc = 0;
        bool ok = true;
        for (int w = w_first; w < w_count && ok; w += w_step) {
            // the current group's K range lives in registers; the parameter
            // arrays are read only when a group ends
            int g = 0, kb = sk[0], ke = sk[NFL];
            int kw = next_wait_k(0);
            uint32_t d = tmem + (uint32_t)(gc & NBM) * bcols;
            for (int q = 0; q < p.nchunks && ok; ++q, ++it) {
                const int s = it % S;
                if (!mbar_wait(full(s), (it / S) & 1, dead)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = base + s * stage_bytes;
                const uint32_t a0 = desc_lo(st), b0 = desc_lo(st + offB);
                const uint32_t a20 = T::X3 ? desc_lo(st + offA2) : 0u, b20 = T::X3 ? desc_lo(st + offB2) : 0u;
                if (kw >= (q + 1) * T::KCS) {
                    // no group of this stage needs the MMA thread to wait
#pragma unroll
                    for (int ks = 0; ks < T::KCS / T::KSTEP; ++ks) {
                        const int k = q * T::KCS + ks * T::KSTEP;
                        if (k >= klast) break;  // K padding after the last group
                        // K step ks: atom ks / (KC / KSTEP), 32 bytes (2 descriptor units) per step within it
                        const uint32_t atom = (uint32_t)(ks / (T::KC / T::KSTEP));
                        const uint32_t off = (uint32_t)(ks % (T::KC / T::KSTEP)) * 2u;
                        const uint32_t ao = atom * ASTEP + off, bo = atom * bstep + off;
                        mma<PREC, CL>(d, desc64<NW>(a0 + ao), desc64<NW>(b0 + bo), idesc, k != kb);
                        if (T::X3) {
                            mma<PREC, CL>(d, desc64<NW>(a0 + ao), desc64<NW>(b20 + bo), idesc, 1);
                            mma<PREC, CL>(d, desc64<NW>(a20 + ao), desc64<NW>(b0 + bo), idesc, 1);
                        }
                        if (k + T::KSTEP == ke) {
                            if (CL == 2)
                                mma_commit_pair(accf(gc & NBM));
                            else
                                mma_commit<1>(accf(gc & NBM));
                            ++gc;
                            ++g;
                            d = tmem + (uint32_t)(gc & NBM) * bcols;
                            if (g < ng) {
                                kb = sk[g];
                                ke = sk[NFL + g];
                            }
                        }
                    }
                } else {
                    // a group whose accumulator the MMA thread waits for
                    // starts in this stage: the same pass with the wait at
                    // that group's first K step (k == kw); unrolled except
                    // for hi+lo, whose three MMAs per step make it large
#pragma unroll SLOW_UNROLL
                    for (int ks = 0; ks < T::KCS / T::KSTEP; ++ks) {
                        const int k = q * T::KCS + ks * T::KSTEP;
                        if (k >= klast) break;  // K padding after the last group
                        if (k == kw) {  // first K step of a group the MMA thread waits for
                            if (!mbar_wait(acce(gc & NBM), ((gc >> nbl) & 1) ^ 1, dead)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            kw = next_wait_k(g + 1);
                        }
                        // K step ks: atom ks / (KC / KSTEP), 32 bytes (2 descriptor units) per step within it
                        const uint32_t atom = (uint32_t)(ks / (T::KC / T::KSTEP));
                        const uint32_t off = (uint32_t)(ks % (T::KC / T::KSTEP)) * 2u;
                        const uint32_t ao = atom * ASTEP + off, bo = atom * bstep + off;
                        mma<PREC, CL>(d, desc64<NW>(a0 + ao), desc64<NW>(b0 + bo), idesc, k != kb);
                        if (T::X3) {
                            mma<PREC, CL>(d, desc64<NW>(a0 + ao), desc64<NW>(b20 + bo), idesc, 1);
                            mma<PREC, CL>(d, desc64<NW>(a20 + ao), desc64<NW>(b0 + bo), idesc, 1);
                        }
                        if (k + T::KSTEP == ke) {
                            if (CL == 2)
                                mma_commit_pair(accf(gc & NBM));
                            else
                                mma_commit<1>(accf(gc & NBM));
                            ++gc;
                            ++g;
                            d = tmem + (uint32_t)(gc & NBM) * bcols;
                            if (g < ng) {
                                kb = sk[g];
                                ke = sk[NFL + g];
                            }
                        }
                    }
                }
                if (CL == 2)
                    mma_commit_pair(empty(s));
                else
                    mma_commit<1>(empty(s));
            }
        }
        // TMEM is freed only after every MMA issued here has completed
        mma_commit<CL>(drain);
        const uint64_t t0 = gtimer();
        while (!mbar_try_sleep(drain, 0, SLEEP_NS)) {
            if (gtimer() - t0 > WAIT_NS) {
                atomicExch(&g_fk_device_error, 1);
                break;
            }
        }
    } else if (warp >= 2 && warp < 6) {
        // ------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int rl = quarter * 32 + lane;
        const uint32_t acce0 = CL == 2 ? mapa(acce(0), 0) : acce(0);
        int gc = 0;
        bool ok = true;
        for (int w = w_first; w < w_count && ok; w += w_step) {
            int rt, nt, sp, pr;
            tile_of(w, rt, nt, sp, pr);
            const int r = rt * TC_M + rl;
            float acc[G];
#pragma unroll
            for (int u = 0; u < G; ++u) acc[u] = 0.f;
            // adjoint: this replica's weights for the tile's G data points
            if (MODE == MODE_ADJ) {
#pragma unroll
                for (int dl = 0; dl < G; ++dl) {
                    const int dd = nt * G + dl;
                    acc[dl] = (r < p.R && dd < p.ndata) ? __ldg(p.gO + (size_t)r * p.ldo + dd) : 0.f;
                }
            }
            const int ncols = G * p.nx;      // accumulator columns in use: column i * G + dl
            constexpr int MI = 255 / G + 1;  // x points a 256-column accumulator can hold
            for (int g = 0; g < p.ngroups; ++g, ++gc) {
                const int b = gc & NBM;
                // the multipliers f^r_{a_g}(x_i) do not depend on the MMA:
                // fetch them all before waiting so their latency overlaps it
                float m[MODE == MODE_FWD ? MI : 1];
                if (MODE == MODE_FWD) {
                    const float *fm = p.Fm + (size_t)g * p.nx * p.R_pad + r;
#pragma unroll
                    for (int i = 0; i < MI; ++i) m[i] = i < p.nx ? __ldg(fm + (size_t)i * p.R_pad) : 0.f;
                }
                // one lane waits, the warp follows (tcgen05.ld is warp-collective)
                int got = 1;
                if (lane == 0) got = mbar_wait(accf(b), (gc >> nbl) & 1, dead);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * bcols;
                // adjoint: per x point, the sum over the tile's data points
                float ps[MODE == MODE_ADJ ? MI : 1];
                if (MODE == MODE_ADJ) {
#pragma unroll
                    for (int i = 0; i < MI; ++i) ps[i] = 0.f;
                }
                if constexpr (MODE == MODE_DENSE || MODE == MODE_LUMI) {
                    // column col of the accumulator is data point nt * n_rows + col
                    const int dbase = nt * p.n_rows;
#pragma unroll 1
                    for (int c = 0; c < 4; ++c) {  // rolled: one 64-register buffer
                        if (c * 64 < p.n_rows) {
                            uint32_t v[64];
                            tmem_ld64(taddr + (uint32_t)(c * 64), v);
                            if (r < p.R) {
                                float *orow = p.O + ((long long)pr * p.nsplit + sp) * p.ostride + (size_t)r * p.ldo +
                                              dbase + c * 64;
#pragma unroll
                                for (int k = 0; k < 64; ++k)
                                    if (dbase + c * 64 + k < p.ndata) orow[k] = __uint_as_float(v[k]);
                            }
                        }
                    }
                }
                // 64 columns per TMEM round trip; the column -> (x point,
                // data point) split is fixed at compile time; columns of x
                // points >= nx (never written by the MMA) are skipped
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (MODE != MODE_DENSE && MODE != MODE_LUMI && c * 64 < ncols) {
                        uint32_t v[64];
                        tmem_ld64(taddr + (uint32_t)(c * 64), v);
                        // forward with saved products: the raw columns, one
                        // 128-byte line per warp and column, columns of a
                        // replica tile 512 bytes apart (immediate offsets);
                        // padding replicas (r >= R) store nothing
                        if (MODE == MODE_FWD && p.Y && r < p.R && FK_DBG(nt < p.ntile_n && rt < p.nrt, 15, nt)) {
                            float *y = p.Y + ((((size_t)nt * p.ngroups + g) * p.nrt + rt) * ncols + c * 64) * TC_M + rl;
#pragma unroll
                            for (int k = 0; k < 64; ++k)
                                if (c * 64 + k < ncols) y[k * TC_M] = __uint_as_float(v[k]);
                        }
#pragma unroll
                        for (int k = 0; k < 64; ++k) {
                            const int col = c * 64 + k, i = col / G, dl = col % G;
                            if (i < p.nx) {
                                if (MODE == MODE_FWD)
                                    acc[dl] = fmaf(m[i], __uint_as_float(v[k]), acc[dl]);
                                else
                                    ps[i] = fmaf(acc[dl], __uint_as_float(v[k]), ps[i]);
                            }
                        }
                    }
                }
                if (MODE == MODE_ADJ && r < p.R) {  // padding replicas: never gathered
                    float *pg = p.P + (((size_t)nt * p.ngroups + g) * p.nx) * p.R_pad + r;
                    if (FK_DBG(nt < p.ntile_n && r < p.R_pad, 14, nt)) {
#pragma unroll
                        for (int i = 0; i < MI; ++i)
                            if (i < p.nx) pg[(size_t)i * p.R_pad] = ps[i];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (CL == 2)
                        mbar_arrive_cluster(acce0 + 8u * b);
                    else
                        mbar_arrive(acce(b));
                }
            }
            if (!ok) break;
            if (MODE == MODE_FWD && r < p.R) {
#pragma unroll
                for (int dl = 0; dl < G; ++dl) {
                    const int dd = nt * G + dl;
                    if (dd < p.ndata) p.O[(size_t)r * p.ldo + dd] = acc[dl];
                }
            }
        }
    }
    if (MODE == MODE_LUMI && warp >= 6) {
        // ------------------------------------------------ PDF matrix builders
        // K runs over rows (c, i) of lnxp columns j (a power of two, at least
        // 16, zero from j = nx), so a stage holds KCS / lnxp whole rows.
        // Thread (m, h) forms A row m, columns j in [h, h + 1) * lnxp / 2 of
        // every row of every stage: it keeps its f^r_{b_c}(x_j) in registers
        // for the whole channel (reloaded when the channel changes) and loads
        // one f^r_{a_c}(x_i) per row.  Values are rounded to the mode as the
        // packing kernels round and written 16 bytes at a time at their place
        // in the 128-byte swizzled K-major layout of the MMA descriptors.
        const int bt = threadIdx.x - TC_THREADS;
        const int m = bt & (TC_M - 1), h = bt >> 7;
        const uint32_t m128 = (uint32_t)m * 128u, m7 = (uint32_t)(m & 7);
        constexpr int CW = T::ESZ == 4 ? 4 : 8;  // columns per 16-byte chunk (8 chunks per atom row)
        constexpr int JH_MAX = 32;               // columns per thread and row (lnxp <= 64)
        const int jh = p.lnxp >> 1;
        const int rows_s = T::KCS / p.lnxp;      // rows per stage
        constexpr int RS_MAX = T::KCS / 16;      // rows per stage at most (lnxp >= 16)
        float fbr[JH_MAX];
#pragma unroll
        for (int u = 0; u < JH_MAX; ++u) fbr[u] = 0.f;
        int cur_c = -1;  // channel whose f_b values fbr holds
        int it = 0;
        bool ok = true;
        for (int w = w_first; w < w_count && ok; w += w_step) {
            int rt, nt, sp, pr;
            tile_of(w, rt, nt, sp, pr);
            const int koff = p.kbase + sp * p.kspl;
            const float *FTr = p.FT + (size_t)rt * TC_M + m;
            for (int q = 0; q < p.nchunks; ++q, ++it) {
                const int s = it % S;
                int got = 1;
                if (lane == 0) got = mbar_wait(empty(s), ((it / S) & 1) ^ 1, dead);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                const uint32_t st = base + s * stage_bytes;
                const int row0 = (koff + q * T::KCS) / p.lnxp;
                // the f_a values of all the stage's rows are loaded first, so
                // their latencies overlap
                float fav[RS_MAX];
                {
                    int c = row0 / p.nx, i = row0 - (row0 / p.nx) * p.nx;
#pragma unroll
                    for (int ir = 0; ir < RS_MAX; ++ir) {
                        fav[ir] = (ir < rows_s && c < p.lnc) ? __ldg(FTr + (size_t)(p.lfl[c] * p.nx + i) * p.R_pad)
                                                             : 0.f;
                        if (++i == p.nx) {
                            i = 0;
                            ++c;
                        }
                    }
                }
                int c = row0 / p.nx, i = row0 - (row0 / p.nx) * p.nx;
#pragma unroll 1
                for (int ir = 0; ir < rows_s; ++ir) {
                    // this row's f_a, then the queue moves up one (constant indices)
                    const float fa = fav[0];
#pragma unroll
                    for (int k = 0; k + 1 < RS_MAX; ++k) fav[k] = fav[k + 1];
                    if (c < p.lnc && c != cur_c) {
                        const float *fb = FTr + (size_t)(p.lfl[MAX_CH + c] * p.nx + h * jh) * p.R_pad;
#pragma unroll
                        for (int u = 0; u < JH_MAX; ++u)
                            fbr[u] = (u < jh && h * jh + u < p.nx) ? __ldg(fb + (size_t)u * p.R_pad) : 0.f;
                        cur_c = c;
                    }
                    // 16-byte chunks of this row owned by this thread: cs0, cs0 + 1, ...
                    const int cs0 = (ir * p.lnxp + h * jh) / CW;
#pragma unroll
                    for (int cc = 0; cc < JH_MAX / CW; ++cc) {
                        if (cc * CW < jh) {
                            const int cs = cs0 + cc;
                            const uint32_t addr = st + (uint32_t)(cs >> 3) * a_bytes + m128 +
                                                  ((uint32_t)((cs & 7) ^ m7) << 4);
                            if (T::ESZ == 4) {
                                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr),
                                             "r"(__float_as_uint(tf32_rna(fa * fbr[cc * CW]))),
                                             "r"(__float_as_uint(tf32_rna(fa * fbr[cc * CW + 1]))),
                                             "r"(__float_as_uint(tf32_rna(fa * fbr[cc * CW + 2]))),
                                             "r"(__float_as_uint(tf32_rna(fa * fbr[cc * CW + CW - 1])))
                                             : "memory");
                            } else {
                                // two values per conversion; lo = bf16(v - hi) from the same pair
                                uint32_t hw[4], lw[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const float v0 = fa * fbr[cc * CW + 2 * u], v1 = fa * fbr[cc * CW + 2 * u + 1];
                                    const __nv_bfloat162 hp = __floats2bfloat162_rn(v0, v1);
                                    hw[u] = *reinterpret_cast<const uint32_t *>(&hp);
                                    if (T::X3) {
                                        const __nv_bfloat162 lp =
                                            __floats2bfloat162_rn(v0 - __low2float(hp), v1 - __high2float(hp));
                                        lw[u] = *reinterpret_cast<const uint32_t *>(&lp);
                                    }
                                }
                                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(hw[0]),
                                             "r"(hw[1]), "r"(hw[2]), "r"(hw[3])
                                             : "memory");
                                if (T::X3)
                                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr + offA2),
                                                 "r"(lw[0]), "r"(lw[1]), "r"(lw[2]), "r"(lw[3])
                                                 : "memory");
                            }
                        }
                    }
                    if (++i == p.nx) {
                        i = 0;
                        ++c;
                    }
                }
                // the generic-proxy stores must be visible to the MMAs (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    if (CL == 2)
                        mbar_arrive_cluster(mapa(full(s), 0));
                    else
                        mbar_arrive(full(s));
                }
            }
        }
    }
    tc_fence_before();
    if (CL == 2)
        cluster_sync();  // no MMA, commit, copy or arrive of the pair still targets this CTA
    else
        __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_free<CL>(tmem);
}

// ------------------------------------------------------------ packing ----

template <int PREC>
__device__ __forceinline__ void store_op(long long idx, float v, __nv_bfloat16 *hi,
                                         __nv_bfloat16 *lo, float *f32) {
    if (PREC == FK_TF32) {
        f32[idx] = tf32_rna(v);
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[idx] = h;
        if (PREC == FK_BF16X3) lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// group of K index k (groups are contiguous and sorted); -1 past the last
__device__ __forceinline__ int group_of(const TcGroups &gr, int k) {
    for (int g = 0; g < gr.ngroups; ++g)
        if (k < gr.kend[g]) return g;
    return -1;
}

// stores 8 consecutive operand values at element index at (a multiple of 8)
template <int PREC>
__device__ __forceinline__ void store8(size_t at, const float (&v)[8], __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                                       float *f32) {
    if (PREC == FK_TF32) {
        float4 a, b;
        a.x = tf32_rna(v[0]);
        a.y = tf32_rna(v[1]);
        a.z = tf32_rna(v[2]);
        a.w = tf32_rna(v[3]);
        b.x = tf32_rna(v[4]);
        b.y = tf32_rna(v[5]);
        b.z = tf32_rna(v[6]);
        b.w = tf32_rna(v[7]);
        reinterpret_cast<float4 *>(f32 + at)[0] = a;
        reinterpret_cast<float4 *>(f32 + at)[1] = b;
    } else {
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            h[u] = __float2bfloat16_rn(v[u]);
            l[u] = __float2bfloat16_rn(v[u] - __bfloat162float(h[u]));
        }
        *reinterpret_cast<uint4 *>(hi + at) = *reinterpret_cast<const uint4 *>(h);
        if (PREC == FK_BF16X3) *reinterpret_cast<uint4 *>(lo + at) = *reinterpret_cast<const uint4 *>(l);
    }
}

// One A operand packing to fill: its column map, padded width, column chunks
// of 2048 (nk) and destination copies.
struct PackDst {
    const int *kmeta;
    int ktot_pad, nk;
    __nv_bfloat16 *hi, *lo;
    float *f32;
};

// A operand A[r][k] = f^r_{o_c}(x_j) for k = (channel c of its group, j), where
// o_c is the channel's other flavour (b_c for the forward packing, a_c for the
// transposed one), gathered through kmeta.  One launch fills one packing
// (d1.nk = 0) or two (the adjoint's forward and transposed packings):
// grid (d0.nk + d1.nk, min(R_pad, 65535)), column chunk blockIdx.x of d0, or
// blockIdx.x - d0.nk of d1; rows r strided by the grid height: 8 consecutive K
// columns per thread, one 16-byte store per operand copy (ktot_pad is a
// multiple of 64).
template <int PREC>
__global__ void __launch_bounds__(256) k_pack_pdf(const PackDst d0, const PackDst d1,
                                                  const float *__restrict__ F, int frow, int R, int R_pad) {
    // the tensor-core kernel that follows may start its set-up now (it waits
    // for this grid's completion before reading what it writes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const bool second = (int)blockIdx.x >= d0.nk;
    const int *kmeta = second ? d1.kmeta : d0.kmeta;
    const int ktot_pad = second ? d1.ktot_pad : d0.ktot_pad;
    __nv_bfloat16 *hi = second ? d1.hi : d0.hi, *lo = second ? d1.lo : d0.lo;
    float *f32 = second ? d1.f32 : d0.f32;
    const int k0 = (((int)blockIdx.x - (second ? d0.nk : 0)) * 256 + threadIdx.x) * 8;
    if (k0 >= ktot_pad) return;
    int o[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) o[u] = __ldg(kmeta + k0 + u);
    for (int r = blockIdx.y; r < R_pad; r += gridDim.y) {
        const float *Fr = F + (size_t)r * frow;
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            v[u] = (r < R && o[u] >= 0 && FK_DBG(o[u] < frow, 10, o[u])) ? __ldg(Fr + o[u]) : 0.f;
        if (FK_DBG(r < R_pad && k0 + 8 <= ktot_pad, 11, k0)) store8<PREC>((size_t)r * ktot_pad + k0, v, hi, lo, f32);
    }
}

// The forward's two packings in one launch: blocks [0, nk * ny) pack the A
// operand as k_pack_pdf does (column chunk blockIdx.x % nk, rows from
// blockIdx.x / nk strided by ny), the blocks after them the epilogue
// multipliers Fm[m][r] as k_pack_fm does (m = b % nm, replicas
// (b / nm) * 256 + thread).
template <int PREC>
__global__ void __launch_bounds__(256) k_pack_fwd(const int *__restrict__ kmeta, int ktot_pad,
                                                  const float *__restrict__ F, int frow, int R, int R_pad,
                                                  __nv_bfloat16 *hi, __nv_bfloat16 *lo, float *f32, int nk, int ny,
                                                  const int *__restrict__ mmeta, int nm, float *__restrict__ Fm) {
    // the tensor-core kernel that follows may start its set-up now (it waits
    // for this grid's completion before reading what it writes)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int b = blockIdx.x;
    if (b < nk * ny) {
        const int k0 = ((b % nk) * 256 + threadIdx.x) * 8;
        if (k0 >= ktot_pad) return;
        int o[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) o[u] = __ldg(kmeta + k0 + u);
        for (int r = b / nk; r < R_pad; r += ny) {
            const float *Fr = F + (size_t)r * frow;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = (r < R && o[u] >= 0 && FK_DBG(o[u] < frow, 10, o[u])) ? __ldg(Fr + o[u]) : 0.f;
            if (FK_DBG(k0 + 8 <= ktot_pad, 11, k0)) store8<PREC>((size_t)r * ktot_pad + k0, v, hi, lo, f32);
        }
    } else {
        const int e = b - nk * ny, m = e % nm;
        const int r = (e / nm) * 256 + threadIdx.x;
        if (r >= R_pad) return;
        const int o = __ldg(mmeta + m);
        Fm[(size_t)m * R_pad + r] = r < R ? __ldg(F + (size_t)r * frow + o) : 0.f;
    }
}

// Forward epilogue multipliers Fm[m][r] = f^r(mmeta[m]), m = g * nx + i (the
// value f^r_{a_g}(x_i)); zero for padding replicas.  Grid (nm, ceil(R_pad / 256)).
__global__ void __launch_bounds__(256) k_pack_fm(const int *__restrict__ mmeta, const float *__restrict__ F,
                                                 int frow, int R, int R_pad, float *__restrict__ Fm) {
    const int m = blockIdx.x;
    const int r = blockIdx.y * 256 + threadIdx.x;
    if (r >= R_pad) return;
    const int o = __ldg(mmeta + m);
    Fm[(size_t)m * R_pad + r] = r < R ? __ldg(F + (size_t)r * frow + o) : 0.f;
}

// B operand from the FP64 table [ndata][nc][nx][nx]: row nt * n_rows + u * G + dl
// holds data point d = nt * G + dl at the row's x point u; column k = (channel
// of its group, x point v).  Forward packing: (u, v) = (i, j); transposed
// packing (trans = 1): (u, v) = (j, i).
template <int PREC>
__global__ void k_pack_table(const TcGroups gr, const double *__restrict__ fk, int ndata, int nc,
                             int nx, int G, int n_rows, int ntile_n, int ktot_pad, int trans,
                             __nv_bfloat16 *hi, __nv_bfloat16 *lo, float *f32) {
    const long long n = (long long)ntile_n * n_rows * ktot_pad;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long row = idx / ktot_pad;
        const int k = (int)(idx % ktot_pad);
        const int nt = (int)(row / n_rows), nr = (int)(row % n_rows);
        const int i = nr / G, dl = nr % G;
        const int d = nt * G + dl;
        float v = 0.f;
        const int g = group_of(gr, k);
        if (i < nx && d < ndata && g >= 0) {
            const int q = (k - gr.kbeg[g]) / nx, j = (k - gr.kbeg[g]) % nx;
            if (q < gr.nch[g]) {
                const int c = gr.chan[gr.ch0[g] + q];
                const int xi = trans ? j : i, xj = trans ? i : j;
                v = (float)fk[(((size_t)d * nc + c) * nx + xi) * nx + xj];
            }
        }
        store_op<PREC>(idx, v, hi, lo, f32);
    }
}

// B operand of a dense table from its FP64 rows [ndata][K]: row d of the
// packing (tile d / n_rows) holds data point d; columns k >= K and rows
// d >= ndata are zero.
template <int PREC>
__global__ void k_pack_dense(const double *__restrict__ fk, int ndata, long long K, long long rows,
                             int ktot_pad, __nv_bfloat16 *hi, __nv_bfloat16 *lo, float *f32) {
    const long long n = rows * ktot_pad;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long d = idx / ktot_pad, k = idx % ktot_pad;
        const float v = (d < ndata && k < K) ? (float)fk[d * K + k] : 0.f;
        store_op<PREC>(idx, v, hi, lo, f32);
    }
}

// B operand of the dense formulation of a hadronic table from its FP64
// table [ndata][nc][nx][nx]: row d holds data point d, column
// k = (c * nx + i) * nxp + j holds FK[d][c][i][j] for j < nx and zero for the
// padding j >= nx, columns past nc * nx * nxp and rows past ndata are zero.
template <int PREC>
__global__ void k_pack_lum(const double *__restrict__ fk, int ndata, int nc, int nx, int nxp, long long rows,
                           int ktot_pad, __nv_bfloat16 *hi, __nv_bfloat16 *lo, float *f32) {
    const long long n = rows * ktot_pad;
    const int nxnxp = nx * nxp;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long d = idx / ktot_pad;
        const int k = (int)(idx % ktot_pad);
        const int c = k / nxnxp, rem = k % nxnxp, i = rem / nxp, j = rem % nxp;
        const float v = (d < ndata && c < nc && j < nx) ? (float)fk[((d * nc + c) * nx + i) * nx + j] : 0.f;
        store_op<PREC>(idx, v, hi, lo, f32);
    }
}

// Adjoint term 1 from the forward's saved products:
//   P1[t][g][i][r] = sum_dl gO[r][t * G + dl] * Y[t][g][rt][i * G + dl][r % 128],
// each sum a chain of fused multiply-adds over dl = 0 .. G-1 starting from 0,
// the order in which the adjoint epilogue forms it from the accumulator, so
// P1 is the one the tensor-core pass over the forward packing would write.
// The forward stores no products for padding replicas (r >= R): their
// threads read replica R - 1's (written, finite) with weights 0 and write
// nothing (the gather reads replicas below R only).
// Grid (R_pad / 128 * ADJ_XS, ngroups, ntile): replicas across threads
// (coalesced loads of Y and stores of P1), the x points split over ADJ_XS
// blocks, the tile's G weights in registers, the loads of UI x points in
// flight together.
constexpr int ADJ_XS = 2;
template <int G>
__global__ void __launch_bounds__(128) k_adj_saved(const float *__restrict__ Y, const float *__restrict__ gO,
                                                   int ldgo, int ndata, int nx, int ngroups, int R, int R_pad,
                                                   float *__restrict__ P1) {
    constexpr int UI = G <= 8 ? 4 : 2;
    const int rt = blockIdx.x / ADJ_XS, xs = blockIdx.x % ADJ_XS, r = rt * TC_M + threadIdx.x;
    const int g = blockIdx.y, t = blockIdx.z;
    const int ibeg = xs * nx / ADJ_XS, iend = (xs + 1) * nx / ADJ_XS;
    float w[G];
#pragma unroll
    for (int dl = 0; dl < G; ++dl) {
        const int dd = t * G + dl;
        w[dl] = (r < R && dd < ndata) ? __ldg(gO + (size_t)r * ldgo + dd) : 0.f;
    }
    const size_t tg = (size_t)t * ngroups + g;
    const int lane_src = r < R ? (int)threadIdx.x : R - 1 - rt * TC_M;
    const float *y = Y + ((tg * (gridDim.x / ADJ_XS) + rt) * G * nx) * TC_M + lane_src;
    float *o = P1 + tg * nx * R_pad + r;
    for (int i0 = ibeg; i0 < iend; i0 += UI) {
        // x points past the block's range re-read its last one (every load
        // unconditional, so all UI * G are issued before the first multiply-add)
        float v[UI][G];
#pragma unroll
        for (int u = 0; u < UI; ++u) {
            const float *yu = y + (size_t)min(i0 + u, iend - 1) * G * TC_M;
#pragma unroll
            for (int dl = 0; dl < G; ++dl) v[u][dl] = __ldg(yu + dl * TC_M);
        }
#pragma unroll
        for (int u = 0; u < UI; ++u) {
            float ps = 0.f;
#pragma unroll
            for (int dl = 0; dl < G; ++dl) ps = fmaf(w[dl], v[u][dl], ps);
            if (i0 + u < iend && r < R) o[(size_t)(i0 + u) * R_pad] = ps;
        }
    }
}

// Adjoint gather: gF[r][a][m] (+)= sum_t P1[t][g1(a)][i(m)][r] + sum_t P2[t][g2(a)][i(m)][r]
// with i(m) the table's x index of grid point m, g1/g2 the groups of flavour a
// in the forward and transposed packings (-1: none).  Grid (ceil(R / 128),
// nxg, 14): one (a, m) per block row, replicas across threads.  Each sum over
// tiles runs as four interleaved partial sums (t mod 4) added in a fixed
// order, so the loads of four tiles are in flight at once.
__global__ void __launch_bounds__(128) k_adj_gather(const float *__restrict__ P1, const float *__restrict__ P2,
                                                    int ntile, int ng1, int ng2, const int8_t *__restrict__ g1,
                                                    const int8_t *__restrict__ g2, const int *__restrict__ xinv,
                                                    int nx, int nxg, int R, int R_pad, int accumulate,
                                                    float *__restrict__ gF) {
    const int r = blockIdx.x * 128 + threadIdx.x;
    const int m = blockIdx.y, a = blockIdx.z;
    if (r >= R) return;
    const int i = __ldg(xinv + m);
    float s = 0.f;
    if (i >= 0) {
        const int ga[2] = {__ldg(g1 + a), __ldg(g2 + a)};
        const int ng[2] = {ng1, ng2};
        const float *P[2] = {P1, P2};
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            if (ga[pass] < 0) continue;
            // element (t, g, i, r) at ((t * ng + g) * nx + i) * R_pad + r
            const size_t step = (size_t)ng[pass] * nx * R_pad;
            const float *p = P[pass] + ((size_t)ga[pass] * nx + i) * R_pad + r;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int t = 0;
            for (; t + 4 <= ntile; t += 4) {
                s0 += __ldg(p + (size_t)t * step);
                s1 += __ldg(p + (size_t)(t + 1) * step);
                s2 += __ldg(p + (size_t)(t + 2) * step);
                s3 += __ldg(p + (size_t)(t + 3) * step);
            }
            for (; t < ntile; ++t) s0 += __ldg(p + (size_t)t * step);
            s += (s0 + s1) + (s2 + s3);
        }
    }
    const size_t o = ((size_t)r * NFL + a) * nxg + m;
    if (FK_DBG(i < nx, 12, i)) gF[o] = accumulate ? gF[o] + s : s;
}

// ------------------------------------------------------------ host ----
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// 2-D K-major operand [rows][cols] with 128-byte swizzled boxes of
// (128 B) x box_rows.
// rowb: bytes per box row and swizzle span, 128 (default) or 64
int make_map(CUtensorMap *m, const void *ptr, int esz, long long cols, long long rows, int box_rows,
             int rowb = 128) {
    auto fn = encoder();
    if (!fn) return fail(FK_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
    const cuuint32_t box[2] = {(cuuint32_t)(rowb / esz), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    rowb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FK_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return FK_OK;
}

// Dynamic shared memory of a tensor-core launch: at least half of an SM's,
// so that one CTA runs per SM.  Each CTA allocates all 512 TMEM columns; a
// second CTA on the same SM would wait in its allocation for the first to
// finish, and with CTA pairs such waits could form a cycle.
size_t one_per_sm(size_t need) {
    static size_t floor_bytes = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        floor_bytes = per_sm > 0 ? (size_t)per_sm / 2 + 1024 : 0;
    });
    return std::max(need, floor_bytes);
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

template <typename K>
int opt_in_smem(K kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<const void *> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count((const void *)kernel)) return FK_OK;
    FK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    // run with the largest shared-memory carveout: the SM then keeps room
    // beside the tensor-core CTA for the small CUDA-core kernels (chi^2,
    // packing, DIS) of concurrent streams
    FK_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    done.insert((const void *)kernel);
    return FK_OK;
}

// Largest number of co-resident 2-CTA clusters of this kernel (cached per
// kernel and shared-memory size); 0 if the query fails.
template <typename K>
int max_clusters(K kernel, size_t smem, int threads) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> known;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair((const void *)kernel, smem);
    auto it = known.find(key);
    if (it != known.end()) return it->second;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * 74, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    known[key] = n;
    return n;
}

// The B operand maps of one packing for precision PREC: full tiles (first,
// second operand copy) and half tiles for the CTA-pair launch.
struct BMaps {
    const CUtensorMap *b, *b2, *h, *h2;
    const CUtensorMap *n = nullptr, *n2 = nullptr;  // hi+lo, 64-byte rows (or NULL)
};
template <int PREC>
BMaps b_maps(const TcPack &pk) {
    if (PREC == FK_TF32) return {&pk.map_f32, &pk.map_f32, &pk.half_f32, &pk.half_f32};
    if (PREC == FK_BF16X3)
        return {&pk.map_hi, &pk.map_lo, &pk.half_hi, &pk.half_lo, pk.nar ? &pk.nar_hi : nullptr,
                pk.nar ? &pk.nar_lo : nullptr};
    return {&pk.map_hi, &pk.map_hi, &pk.half_hi, &pk.half_hi};
}

// The hi+lo B maps of 64-byte rows for a packing that stores both copies.
int make_narrow_maps(TcPack &pk, long long rows) {
    if (!pk.hi || !pk.lo) return FK_OK;
    int rc = make_map(&pk.nar_hi, pk.hi, 2, pk.ktot_pad, rows, pk.n_rows, 64);
    if (!rc) rc = make_map(&pk.nar_lo, pk.lo, 2, pk.ktot_pad, rows, pk.n_rows, 64);
    pk.nar = rc == FK_OK;
    return rc;
}

// Accumulator hand-off.  Use u of the NB-buffered accumulator (one use per
// channel group, counted across the CTA's tiles) may start once the epilogue
// has released use u - NB, the same buffer.  For group g that wait is made by
// the (even CTA's) producer before it loads the stage holding the group's
// first K step: the MMAs reach that stage only through its full barrier, so
// they are ordered after the release, and the MMA thread itself does not wait
// on the epilogue.  The producer runs S stages ahead of the MMAs, so it takes
// the wait only where use u - NB ends at least S + PW_SLACK stages before that
// stage (in this tile or an earlier one): then the release is due and the
// wait costs nothing, and use u - NB needs no stage the producer has yet to
// load.  For groups that follow closer behind (short groups), the MMA thread
// waits at the group's first K step, with the stage already loaded.  Returns
// the mask of producer-side groups; it depends only on the table's packing
// and the pipeline shape, so it is computed here once per launch.
uint32_t tc_pwait(const TcParams &p, int S, int KCS) {
    const int NB = 1 << p.nbl;
    uint32_t pwait = 0;
    for (int g = 0; g < p.ngroups; ++g) {
        int u2 = g - NB, back = 0;  // group of use u - NB, tiles back
        while (u2 < 0) {
            u2 += p.ngroups;
            ++back;
        }
        const int e2 = (p.kend[u2] + KCS - 1) / KCS - back * p.nchunks;  // stage after its last
        if (p.kbeg[g] / KCS - S - e2 >= PW_SLACK) pwait |= 1u << g;
    }
    return pwait;
}

// CTA pairs (256-row MMAs on two SMs) whenever the replica tiles pair up
// and the channel groups span two stages or more on average.  A pair halves
// the B bytes each SM loads but adds cross-SM hand-offs per stage and per
// group; with groups of about one stage (config-2 shaped tables) single CTAs
// measured faster (BF16 forward 30.8 against 34.9 us), with long groups or one
// group pairs win (stress table BF16 1081 against 1030 TFLOP/s, the Table 3
// product 381 against 416 us).  nchunks counts stages of 128-byte rows.
bool use_pairs(const TcParams &p) {
    const bool long_groups = p.ngroups == 1 || p.nchunks >= 2 * p.ngroups;
    return p.nrt % 2 == 0 && long_groups;
}

template <int PREC, int G, int MODE>
int launch_tc(const fk_table *t, const CUtensorMap &mA, const CUtensorMap &mA2, const BMaps &mb,
              const TcParams &p0, cudaStream_t s, const CUtensorMap *nA = nullptr) {
    TcParams p = p0;
    if (!p.narrow && use_pairs(p)) {
        p.pwait = tc_pwait(p, tc_stages<PREC, 2>(), Tr<PREC>::KCS);
        auto kern = k_tc<PREC, G, MODE, 2>;
        const size_t smem = one_per_sm(tc_smem_bytes<PREC, 2>(p.n_rows));
        // opt in once at the largest tile (n_rows = 256) so that every table fits
        int rc = opt_in_smem(kern, tc_smem_bytes<PREC, 2>(256));
        if (rc) return rc;
        const int nc = std::min(p.ntiles / 2, max_clusters(kern, smem, tc_threads<MODE>()));
        if (nc > 0) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[2];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[1].val.programmaticStreamSerializationAllowed = 1;
            cfg.gridDim = dim3(2 * nc, 1, 1);
            cfg.blockDim = dim3(tc_threads<MODE>(), 1, 1);
            cfg.dynamicSmemBytes = smem;
            cfg.stream = s;
            cfg.attrs = attr;
            cfg.numAttrs = 2;
            FK_CUDA(cudaLaunchKernelEx(&cfg, kern, mA, mA2, *mb.h, *mb.h2, p));
            count_launch();
            return FK_OK;
        }
    }
    const int grid = std::min(p.ntiles, sm_count());
    if constexpr (PREC == FK_BF16X3 && MODE != MODE_LUMI) {
        // hi+lo on single CTAs: 64-byte rows, four stages of half the K (the
        // 96 KB stages of 128-byte rows leave room for two); the same MMAs in
        // the same order, so the same results
        if (p.narrow && nA && mb.n) {
            constexpr int NK = Tr<PREC>::KCS / Tr<PREC, true>::KCS;  // narrow stages per wide one
            p.nchunks *= NK;
            p.spc *= NK;
            p.pwait = tc_pwait(p, tc_stages<PREC, 1, true>(), Tr<PREC, true>::KCS);
            auto kern = k_tc<PREC, G, MODE, 1, true>;
            int rc = opt_in_smem(kern, tc_smem_bytes<PREC, 1, true>(256));
            if (rc) return rc;
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.gridDim = dim3(grid, 1, 1);
            cfg.blockDim = dim3(tc_threads<MODE>(), 1, 1);
            cfg.dynamicSmemBytes = one_per_sm(tc_smem_bytes<PREC, 1, true>(p.n_rows));
            cfg.stream = s;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            FK_CUDA(cudaLaunchKernelEx(&cfg, kern, nA[0], nA[1], *mb.n, *mb.n2, p));
            count_launch();
            return FK_OK;
        }
    }
    p.pwait = tc_pwait(p, tc_stages<PREC, 1>(), Tr<PREC>::KCS);
    auto kern = k_tc<PREC, G, MODE, 1>;
    int rc = opt_in_smem(kern, tc_smem_bytes<PREC, 1>(256));
    if (rc) return rc;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(tc_threads<MODE>(), 1, 1);
    cfg.dynamicSmemBytes = one_per_sm(tc_smem_bytes<PREC, 1>(p.n_rows));
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    FK_CUDA(cudaLaunchKernelEx(&cfg, kern, mA, mA2, *mb.b, *mb.b2, p));
    count_launch();
    return FK_OK;
}

template <int PREC, int MODE>
int launch_tc_g(const fk_table *t, const CUtensorMap &mA, const CUtensorMap &mA2, const TcPack &pk,
                const TcParams &p, cudaStream_t s, const CUtensorMap *nA = nullptr) {
    const BMaps mb = b_maps<PREC>(pk);
    switch (t->tc.G) {
        case 4: return launch_tc<PREC, 4, MODE>(t, mA, mA2, mb, p, s, nA);
        case 5: return launch_tc<PREC, 5, MODE>(t, mA, mA2, mb, p, s, nA);
        case 6: return launch_tc<PREC, 6, MODE>(t, mA, mA2, mb, p, s, nA);
        case 7: return launch_tc<PREC, 7, MODE>(t, mA, mA2, mb, p, s, nA);
        case 8: return launch_tc<PREC, 8, MODE>(t, mA, mA2, mb, p, s, nA);
        case 12: return launch_tc<PREC, 12, MODE>(t, mA, mA2, mb, p, s, nA);
        case 16: return launch_tc<PREC, 16, MODE>(t, mA, mA2, mb, p, s, nA);
    }
    return fail(FK_EINVAL, "bad tile height");
}

// k_pack_pdf over one packing (d1.nk = 0) or two, in one launch.
template <int PREC>
cudaError_t launch_pack(const PackDst &d0, const PackDst &d1, const float *F, int frow, int R, int R_pad,
                        cudaStream_t s) {
    k_pack_pdf<PREC><<<dim3((unsigned)(d0.nk + d1.nk), (unsigned)std::min(R_pad, 65535)), 256, 0, s>>>(
        d0, d1, F, frow, R, R_pad);
    count_launch();
    return cudaGetLastError();
}

// Packs the A operand (and, if Fm is not NULL, the forward multipliers) for one
// packing of the table, builds its tensor maps and fills the common params.
// With defer (and no Fm) the A packing is described in *defer instead of
// launched: the caller launches it, possibly together with another.
template <int PREC>
int prepare(const fk_table *t, const TcPack &pk, const float *F, int R, Scratch &scr, float *Fm,
            cudaStream_t s, CUtensorMap &mA, CUtensorMap &mA2, TcParams &p, int frow_in = -1,
            PackDst *defer = nullptr, CUtensorMap *nar = nullptr) {
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    __nv_bfloat16 *hi = nullptr, *lo = nullptr;
    float *f32 = nullptr;
    const size_t nA = (size_t)R_pad * pk.ktot_pad;
    if (PREC == FK_TF32) {
        FK_CUDA(scr.get(&f32, nA));
    } else {
        FK_CUDA(scr.get(&hi, nA));
        if (PREC == FK_BF16X3) FK_CUDA(scr.get(&lo, nA));
    }
    // A rows: the PDF grid of a replica, or a dense table's PDF matrix row
    // (or, when given, rows of frow_in elements: the adjoint's gO)
    const int frow = frow_in >= 0 ? frow_in : t->kind == FK_KIND_DENSE ? (int)t->E : NFL * t->nxg;
    if (Fm) {
        // the forward: A operand and epilogue multipliers in one launch
        const int nk = (pk.ktot_pad + 2047) / 2048, ny = std::min(R_pad, 4096);
        const int nm = pk.grp.ngroups * t->nx;
        const long long blocks = (long long)nk * ny + (long long)nm * ((R_pad + 255) / 256);
        k_pack_fwd<PREC><<<(unsigned)blocks, 256, 0, s>>>(pk.kmeta, pk.ktot_pad, F, frow, R, R_pad, hi, lo, f32, nk,
                                                          ny, pk.mmeta, nm, Fm);
        count_launch();
        FK_CUDA(cudaGetLastError());
    } else {
        const PackDst d{pk.kmeta, pk.ktot_pad, (pk.ktot_pad + 2047) / 2048, hi, lo, f32};
        if (defer) {
            *defer = d;  // the caller launches it, with another packing
        } else {
            FK_CUDA(launch_pack<PREC>(d, PackDst{}, F, frow, R, R_pad, s));
        }
    }
    p = TcParams{};
    p.npair = 1;  // pa = pb = 0: one operand pair
    p.nrt = R_pad / TC_M;
    p.ntiles = pk.ntile_n * p.nrt;
    p.ntile_n = pk.ntile_n;
    p.nsplit = 1;
    p.nchunks = pk.ktot_pad / Tr<PREC>::KCS;
    p.n_rows = pk.n_rows;
    // narrow tiles (G * nx <= 128, i.e. nx <= 8) keep four accumulators of 128
    // TMEM columns in flight instead of two of 256, so the short channel
    // groups of such tables wait less on the epilogue
    p.nbl = pk.n_rows <= 128 ? 2 : 1;
    p.ngroups = pk.grp.ngroups;
    p.nx = t->nx;
    p.ndata = t->ndata;
    p.R = R;
    p.R_pad = R_pad;
    for (int g = 0; g < pk.grp.ngroups; ++g) {
        p.kbeg[g] = pk.grp.kbeg[g];
        p.kend[g] = pk.grp.kend[g];
    }
    // the A maps of the launch shape: 64-byte rows (nar[0], nar[1]) for hi+lo
    // on single CTAs when the packing has its narrow B maps, else 128-byte rows
    const int esz = Tr<PREC>::ESZ;
    p.narrow = PREC == FK_BF16X3 && nar && pk.nar && !use_pairs(p);
    int rc;
    if (p.narrow) {
        rc = make_map(&nar[0], hi, esz, pk.ktot_pad, R_pad, TC_M, 64);
        if (!rc) rc = make_map(&nar[1], lo, esz, pk.ktot_pad, R_pad, TC_M, 64);
    } else {
        rc = make_map(&mA, PREC == FK_TF32 ? (const void *)f32 : (const void *)hi, esz, pk.ktot_pad, R_pad, TC_M);
        if (!rc && PREC == FK_BF16X3) rc = make_map(&mA2, lo, esz, pk.ktot_pad, R_pad, TC_M);
        if (PREC != FK_BF16X3) mA2 = mA;
    }
    return rc;
}

// O[r][d] = sum over splits sp (in order) of part[sp][r][d]
__global__ void __launch_bounds__(256) k_dense_sum(const float *__restrict__ part, int nsplit, int ndata,
                                                   int R, float *__restrict__ O, int ldo) {
    const long long idx = (long long)blockIdx.x * 256 + threadIdx.x;
    const long long n = (long long)R * ndata;
    if (idx >= n) return;
    float v = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) v += part[(size_t)sp * n + idx];
    const long long r = idx / ndata, d = idx - r * ndata;
    O[r * ldo + d] = v;
}

template <int PREC>
int lum_tc_t(const fk_table *t, const float *F, int R, float *O, int ldo, cudaStream_t s);

// Y (optional): the products Y_g are also written there, as
// [ntile_n][ngroups][G * nx][R_pad] floats (saved_elems)
template <int PREC>
int fwd_tc_t(const fk_table *t, const float *F, int R, float *O, int ldo, cudaStream_t s, float *Y = nullptr) {
    const TcLayout &L = t->tc;
    if (L.lum_on) return lum_tc_t<PREC>(t, F, R, O, ldo, s);
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    Scratch scr(s);
    float *Fm = nullptr;
    FK_CUDA(scr.get(&Fm, (size_t)L.fwd.grp.ngroups * t->nx * R_pad));
    CUtensorMap mA, mA2, nA[2];
    TcParams p;
    int rc = prepare<PREC>(t, L.fwd, F, R, scr, Fm, s, mA, mA2, p, -1, nullptr, nA);
    if (rc) return rc;
    p.ldo = ldo;
    p.Fm = Fm;
    p.O = O;
    p.Y = Y;
    return launch_tc_g<PREC, MODE_FWD>(t, mA, mA2, L.fwd, p, s, nA);
}

// Dense product (Table 3): the A operand is the caller's PDF matrix, the B
// operand the packed table, one group over K; the epilogue stores the tile.
// When the (replica, data) tiles leave SMs idle, K is split into runs of at
// least 8 stages, each run a work item writing a partial tile; k_dense_sum
// adds the partials in split order.  The split count minimises waves x (stages
// per item + a fixed cost per item), one CTA per SM, plus the partials' cost
// per extra split; ties keep fewer splits.  It depends on R (through the tile
// count), so in these modes a replica's last bits can differ between calls
// with different R.

template <int PREC>
int dense_tc_t(const fk_table *t, const float *Lm, int R, float *O, int ldo, cudaStream_t s) {
    Scratch scr(s);
    CUtensorMap mA, mA2;
    TcParams p;
    int rc = prepare<PREC>(t, t->tc.fwd, Lm, R, scr, nullptr, s, mA, mA2, p);
    if (rc) return rc;
    const int stages = p.nchunks, items = p.ntiles, sms = sm_count();
    int nsplit = 1;
    constexpr int ITEM_COST = 4;  // stages' worth of pipeline fill and epilogue per work item
    // each extra split writes and re-reads R x ndata partials: two stages' worth per 128 x 256 tile of them
    const double split_cost = 2.0 * R * t->ndata / (TC_M * 256.0);
    double best = (double)((items + sms - 1) / sms) * (stages + ITEM_COST);
    for (int ns = 2; ns <= std::min(stages / 8, 2 * sms); ++ns) {
        const double cost =
            (double)((items * ns + sms - 1) / sms) * ((stages + ns - 1) / ns + ITEM_COST) + split_cost * (ns - 1);
        if (cost < best) {
            best = cost;
            nsplit = ns;
        }
    }
    const int cps = (stages + nsplit - 1) / nsplit;  // stages per split
    nsplit = (stages + cps - 1) / cps;
    p.nchunks = cps;
    p.kbeg[0] = 0;
    p.kend[0] = cps * Tr<PREC>::KCS;  // past K the operands read as zero (TMA fill)
    p.kspl = cps * Tr<PREC>::KCS;
    p.nsplit = nsplit;
    p.ntiles = items * nsplit;
    float *part = nullptr;
    if (nsplit > 1) {
        FK_CUDA(scr.get(&part, (size_t)nsplit * R * t->ndata));
        p.O = part;
        p.ldo = t->ndata;
        p.ostride = (long long)R * t->ndata;
    } else {
        p.O = O;
        p.ldo = ldo;
    }
    rc = launch_tc<PREC, 16, MODE_DENSE>(t, mA, mA2, b_maps<PREC>(t->tc.fwd), p, s);
    if (rc || nsplit == 1) return rc;
    const long long n = (long long)R * t->ndata;
    k_dense_sum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, nsplit, t->ndata, R, O, ldo);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Forward in the dense formulation (MODE_LUMI): the builders' transposed
// PDF rows FT[(a * nx + x) * R_pad + r] = f^r_a(x_x) (k_pack_fm through
// lum_mmeta), one k_tc launch over (replica tile, data tile, K split) work
// items with K split into fixed runs of LUMI_KSPLIT columns, and the
// partial tiles added in split order (k_dense_sum) when there are several.
template <int PREC>
int lum_tc_t(const fk_table *t, const float *F, int R, float *O, int ldo, cudaStream_t s) {
    const TcLayout &L = t->tc;
    const TcPack &pk = L.lum;
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    Scratch scr(s);
    float *FT = nullptr;
    FK_CUDA(scr.get(&FT, (size_t)NFL * t->nx * R_pad));
    k_pack_fm<<<dim3((unsigned)(NFL * t->nx), (unsigned)((R_pad + 255) / 256)), 256, 0, s>>>(
        L.lum_mmeta, F, NFL * t->nxg, R, R_pad, FT);
    count_launch();
    FK_CUDA(cudaGetLastError());
    TcParams p{};
    p.npair = 1;  // pa = pb = 0
    p.nrt = R_pad / TC_M;
    p.ntile_n = pk.ntile_n;
    p.n_rows = pk.n_rows;
    p.nbl = pk.n_rows <= 128 ? 2 : 1;
    p.ngroups = 1;
    p.nx = t->nx;
    p.ndata = t->ndata;
    p.R = R;
    p.R_pad = R_pad;
    const int stages = pk.ktot_pad / Tr<PREC>::KCS;
    const int cps = std::min(stages, LUMI_KSPLIT / Tr<PREC>::KCS);  // stages per split
    const int nsplit = (stages + cps - 1) / cps;
    p.nchunks = cps;
    p.kbeg[0] = 0;
    p.kend[0] = cps * Tr<PREC>::KCS;  // past K both operands read as zero
    p.kspl = cps * Tr<PREC>::KCS;
    p.nsplit = nsplit;
    p.ntiles = p.nrt * pk.ntile_n * nsplit;
    p.FT = FT;
    for (int c = 0; c < t->nch; ++c) {
        p.lfl[c] = (uint8_t)t->ca[c];
        p.lfl[MAX_CH + c] = (uint8_t)t->cb[c];
    }
    p.lnc = t->nch;
    p.lnxp = L.lum_nxp;
    float *part = nullptr;
    if (nsplit > 1) {
        FK_CUDA(scr.get(&part, (size_t)nsplit * R * t->ndata));
        p.O = part;
        p.ldo = t->ndata;
        p.ostride = (long long)R * t->ndata;
    } else {
        p.O = O;
        p.ldo = ldo;
    }
    const BMaps mb = b_maps<PREC>(pk);
    // the A maps are not read in this mode (the builders form A)
    int rc = launch_tc<PREC, 16, MODE_LUMI>(t, *mb.b, *mb.b, mb, p, s);
    if (rc || nsplit == 1) return rc;
    const long long n = (long long)R * t->ndata;
    k_dense_sum<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, nsplit, t->ndata, R, O, ldo);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Adjoint: term 1 (derivative with respect to the first flavour of each
// channel) from the forward packing, term 2 (second flavour) from the
// transposed packing, both as per-tile partial sums, then one fixed-order
// gather into gF.  Both A operands are packed by one launch.
template <int PREC>
int bwd_tc_t(const fk_table *t, const float *F, const float *gO, int ldgo, int R, float *gF,
             int accumulate, cudaStream_t s) {
    const TcLayout &L = t->tc;
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    Scratch scr(s);
    float *P1 = nullptr, *P2 = nullptr;
    FK_CUDA(scr.get(&P1, (size_t)L.ntile_n * L.fwd.grp.ngroups * t->nx * R_pad));
    FK_CUDA(scr.get(&P2, (size_t)L.ntile_n * L.bwd.grp.ngroups * t->nx * R_pad));
    const TcPack *packs[2] = {&L.fwd, &L.bwd};
    float *parts[2] = {P1, P2};
    CUtensorMap mA[2], mA2[2], nA[2][2];
    TcParams p[2];
    PackDst pd[2];
    for (int k = 0; k < 2; ++k) {
        const int rc = prepare<PREC>(t, *packs[k], F, R, scr, nullptr, s, mA[k], mA2[k], p[k], -1, &pd[k], nA[k]);
        if (rc) return rc;
    }
    FK_CUDA(launch_pack<PREC>(pd[0], pd[1], F, NFL * t->nxg, R, R_pad, s));
    for (int k = 0; k < 2; ++k) {
        p[k].ldo = ldgo;
        p[k].gO = gO;
        p[k].P = parts[k];
        const int rc = launch_tc_g<PREC, MODE_ADJ>(t, mA[k], mA2[k], *packs[k], p[k], s, nA[k]);
        if (rc) return rc;
    }
    k_adj_gather<<<dim3((unsigned)((R + 127) / 128), (unsigned)t->nxg, NFL), 128, 0, s>>>(
        P1, P2, L.ntile_n, L.fwd.grp.ngroups, L.bwd.grp.ngroups, L.gmap, L.gmap + NFL, t->d_xinv, t->nx,
        t->nxg, R, R_pad, accumulate, gF);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Adjoint with the forward's saved products Y: term 1 is contracted from Y
// (k_adj_saved, the partial sums the forward-packing pass would write), term 2
// is the tensor-core pass over the transposed packing as above, then the same
// gather.
template <int PREC>
int bwd_tc_saved_t(const fk_table *t, const float *F, const float *gO, int ldgo, int R, const float *Y,
                   float *gF, int accumulate, cudaStream_t s) {
    const TcLayout &L = t->tc;
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    Scratch scr(s);
    float *P1 = nullptr, *P2 = nullptr;
    FK_CUDA(scr.get(&P1, (size_t)L.ntile_n * L.fwd.grp.ngroups * t->nx * R_pad));
    FK_CUDA(scr.get(&P2, (size_t)L.ntile_n * L.bwd.grp.ngroups * t->nx * R_pad));
    const dim3 grid((unsigned)(R_pad / TC_M * ADJ_XS), (unsigned)L.fwd.grp.ngroups, (unsigned)L.ntile_n);
    const int ng = L.fwd.grp.ngroups, nd = t->ndata, nx = t->nx;
    switch (L.G) {
        case 4: k_adj_saved<4><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 5: k_adj_saved<5><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 6: k_adj_saved<6><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 7: k_adj_saved<7><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 8: k_adj_saved<8><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 12: k_adj_saved<12><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        case 16: k_adj_saved<16><<<grid, 128, 0, s>>>(Y, gO, ldgo, nd, nx, ng, R, R_pad, P1); break;
        default: return fail(FK_EINVAL, "unexpected data points per tile");
    }
    count_launch();
    FK_CUDA(cudaGetLastError());
    CUtensorMap mA, mA2, nA[2];
    TcParams p;
    int rc = prepare<PREC>(t, L.bwd, F, R, scr, nullptr, s, mA, mA2, p, -1, nullptr, nA);
    if (rc) return rc;
    p.ldo = ldgo;
    p.gO = gO;
    p.P = P2;
    rc = launch_tc_g<PREC, MODE_ADJ>(t, mA, mA2, L.bwd, p, s, nA);
    if (rc) return rc;
    k_adj_gather<<<dim3((unsigned)((R + 127) / 128), (unsigned)t->nxg, NFL), 128, 0, s>>>(
        P1, P2, L.ntile_n, L.fwd.grp.ngroups, L.bwd.grp.ngroups, L.gmap, L.gmap + NFL, t->d_xinv, t->nx,
        t->nxg, R, R_pad, accumulate, gF);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

template <int PREC>
int pack_table(fk_table *t, TcPack &pk, int trans, const double *d_fk, cudaStream_t s) {
    const TcLayout &L = t->tc;
    const long long n = (long long)L.ntile_n * L.n_rows * pk.ktot_pad;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 148LL * 32);
    k_pack_table<PREC><<<blocks, 256, 0, s>>>(pk.grp, d_fk, t->ndata, t->nch, t->nx, L.G, L.n_rows,
                                              L.ntile_n, pk.ktot_pad, trans, pk.hi, pk.lo, pk.f32);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Channel groups keyed by `key` (the first flavour for the forward packing,
// the second for the transposed one), each padded to KPAD along K.
void make_groups(const fk_table *t, const std::vector<int> &key, TcPack &pk) {
    TcGroups &gr = pk.grp;
    gr.ngroups = 0;
    int k = 0, pos = 0;
    for (int a = 0; a < NFL; ++a) {
        int n = 0;
        for (int c = 0; c < t->nch; ++c)
            if (key[c] == a) {
                if (!n) {
                    gr.flav[gr.ngroups] = a;
                    gr.ch0[gr.ngroups] = pos;
                    gr.kbeg[gr.ngroups] = k;
                }
                gr.chan[pos++] = c;
                ++n;
            }
        if (n) {
            gr.nch[gr.ngroups] = n;
            k += (n * t->nx + KPAD - 1) / KPAD * KPAD;
            gr.kend[gr.ngroups] = k;
            ++gr.ngroups;
        }
    }
    pk.ktot = k;
    // whole pipeline stages: 128 K elements for BF16 and TF32 (two swizzle
    // atoms per stage), 64 when the table holds only the hi+lo operands
    const int kal = (t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_TF32))) ? 128 : 64;
    pk.ktot_pad = (k + kal - 1) / kal * kal;
}

}  // namespace

int tc_build(fk_table *t, const double *host_fk, unsigned form) {
    TcLayout &L = t->tc;
    make_groups(t, t->ca, L.fwd);
    make_groups(t, t->cb, L.bwd);
    // data points per tile: the largest G of the compiled set with G * nx <=
    // 256 (MMA N and one TMEM accumulator): wider MMAs do more work per
    // instruction issued
    L.G = 4;
    for (int g : {16, 12, 8, 7, 6, 5, 4})
        if (g * t->nx <= 256) {
            L.G = g;
            break;
        }
    L.n_rows = (L.G * t->nx + 15) / 16 * 16;
    L.ntile_n = (t->ndata + L.G - 1) / L.G;
    L.fwd.n_rows = L.bwd.n_rows = L.n_rows;
    L.fwd.ntile_n = L.bwd.ntile_n = L.ntile_n;
    const bool want_hi = t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_BF16X3));
    const bool want_lo = t->mask & FK_PREC_BIT(FK_BF16X3);
    const bool want_f32 = t->mask & FK_PREC_BIT(FK_TF32);
    // gather maps of the A operand and of the forward multipliers, and the
    // adjoint gather's flavour -> group maps
    {
        const std::vector<int> *other[2] = {&t->cb, &t->ca};
        TcPack *packs[2] = {&L.fwd, &L.bwd};
        for (int w = 0; w < 2; ++w) {
            TcPack &pk = *packs[w];
            std::vector<int> km(pk.ktot_pad, -1), mm((size_t)pk.grp.ngroups * t->nx);
            for (int g = 0; g < pk.grp.ngroups; ++g) {
                for (int q = 0; q < pk.grp.nch[g]; ++q) {
                    const int c = pk.grp.chan[pk.grp.ch0[g] + q];
                    for (int j = 0; j < t->nx; ++j)
                        km[pk.grp.kbeg[g] + q * t->nx + j] = (*other[w])[c] * t->nxg + t->xmap[j];
                }
                for (int i = 0; i < t->nx; ++i) mm[(size_t)g * t->nx + i] = pk.grp.flav[g] * t->nxg + t->xmap[i];
            }
            if (cudaMalloc(&pk.kmeta, km.size() * sizeof(int)) || cudaMalloc(&pk.mmeta, mm.size() * sizeof(int)))
                return fail(FK_ENOMEM, "tensor-core gather maps");
            FK_CUDA(cudaMemcpy(pk.kmeta, km.data(), km.size() * sizeof(int), cudaMemcpyHostToDevice));
            FK_CUDA(cudaMemcpy(pk.mmeta, mm.data(), mm.size() * sizeof(int), cudaMemcpyHostToDevice));
            t->bytes += (km.size() + mm.size()) * sizeof(int);
        }
        int8_t hmap[2 * NFL];
        for (int a = 0; a < 2 * NFL; ++a) hmap[a] = -1;
        for (int g = 0; g < L.fwd.grp.ngroups; ++g) hmap[L.fwd.grp.flav[g]] = (int8_t)g;
        for (int g = 0; g < L.bwd.grp.ngroups; ++g) hmap[NFL + L.bwd.grp.flav[g]] = (int8_t)g;
        if (cudaMalloc(&L.gmap, sizeof(hmap))) return fail(FK_ENOMEM, "tensor-core gather maps");
        FK_CUDA(cudaMemcpy(L.gmap, hmap, sizeof(hmap), cudaMemcpyHostToDevice));
    }
    for (TcPack *pk : {&L.fwd, &L.bwd}) {
        const size_t elems = (size_t)L.ntile_n * L.n_rows * pk->ktot_pad;
        if ((want_hi && cudaMalloc(&pk->hi, elems * 2)) || (want_lo && cudaMalloc(&pk->lo, elems * 2)) ||
            (want_f32 && cudaMalloc(&pk->f32, elems * 4)))
            return fail(FK_ENOMEM, "tensor-core table storage");
        t->bytes += elems * (2 * want_hi + 2 * want_lo + 4 * want_f32);
    }

    // The paper's dense formulation with the PDF matrix formed on the chip
    // (MODE_LUMI) for the forward, on request (FK_TABLE_LUMI).  It is not
    // chosen by default: forming the operand takes 16K FP32 products,
    // conversions and 32 KB of shared-memory stores per 1.3k-cycle MMA stage
    // on the SM's issue slots, and the builders stay about four times behind
    // the tensor cores (config 2, BF16: 87 us against 31 us factorised).  A
    // table property: a replica's result does not depend on R.
    L.lum_nxp = 16;
    while (L.lum_nxp < t->nx) L.lum_nxp *= 2;
    const long long Kl = (long long)t->nch * t->nx * L.lum_nxp;
    L.lum_on = form == FK_TABLE_LUMI;
    if (L.lum_on) {
        TcPack &pk = L.lum;
        pk.n_rows = std::min(256, (t->ndata + 15) / 16 * 16);
        pk.ntile_n = (t->ndata + pk.n_rows - 1) / pk.n_rows;
        pk.grp = TcGroups{};
        pk.grp.ngroups = 1;
        pk.grp.kbeg[0] = 0;
        pk.grp.kend[0] = (int)((Kl + KPAD - 1) / KPAD * KPAD);
        pk.ktot = pk.grp.kend[0];
        const int kal = (t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_TF32))) ? 128 : 64;
        pk.ktot_pad = (pk.ktot + kal - 1) / kal * kal;
        const size_t elems = (size_t)pk.ntile_n * pk.n_rows * pk.ktot_pad;
        if ((want_hi && cudaMalloc(&pk.hi, elems * 2)) || (want_lo && cudaMalloc(&pk.lo, elems * 2)) ||
            (want_f32 && cudaMalloc(&pk.f32, elems * 4)))
            return fail(FK_ENOMEM, "tensor-core table storage");
        t->bytes += elems * (2 * want_hi + 2 * want_lo + 4 * want_f32);
        std::vector<int> mm((size_t)NFL * t->nx);
        for (int a = 0; a < NFL; ++a)
            for (int x = 0; x < t->nx; ++x) mm[(size_t)a * t->nx + x] = a * t->nxg + t->xmap[x];
        if (cudaMalloc(&L.lum_mmeta, mm.size() * sizeof(int))) return fail(FK_ENOMEM, "tensor-core gather maps");
        FK_CUDA(cudaMemcpy(L.lum_mmeta, mm.data(), mm.size() * sizeof(int), cudaMemcpyHostToDevice));
        t->bytes += mm.size() * sizeof(int);
    }

    // full FP64 copy on the device for the packing kernels, then freed
    double *owned = nullptr;
    cudaStream_t s = nullptr;
    FK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int rc = FK_OK;
    const size_t src_elems = (size_t)t->ndata * t->E;
    if (cudaMalloc(&owned, src_elems * 8)) {
        cudaStreamDestroy(s);
        return fail(FK_ENOMEM, "tensor-core packing staging");
    }
    cudaError_t e = cudaMemcpyAsync(owned, host_fk, src_elems * 8, cudaMemcpyHostToDevice, s);
    if (e) rc = cuda_fail(e, "tensor-core table upload");
    for (int tr = 0; tr < 2 && !rc; ++tr) {
        TcPack &pk = tr ? L.bwd : L.fwd;
        if (!rc && want_f32) rc = pack_table<FK_TF32>(t, pk, tr, owned, s);
        if (!rc && want_lo) rc = pack_table<FK_BF16X3>(t, pk, tr, owned, s);
        else if (!rc && want_hi) rc = pack_table<FK_BF16>(t, pk, tr, owned, s);
    }
    if (!rc && L.lum_on) {
        const TcPack &pk = L.lum;
        const long long rows = (long long)pk.ntile_n * pk.n_rows;
        const unsigned blocks = (unsigned)std::min<long long>((rows * pk.ktot_pad + 255) / 256, 148LL * 32);
        if (want_f32)
            k_pack_lum<FK_TF32><<<blocks, 256, 0, s>>>(owned, t->ndata, t->nch, t->nx, L.lum_nxp, rows, pk.ktot_pad,
                                                      pk.hi, pk.lo, pk.f32);
        if (want_lo)
            k_pack_lum<FK_BF16X3><<<blocks, 256, 0, s>>>(owned, t->ndata, t->nch, t->nx, L.lum_nxp, rows,
                                                        pk.ktot_pad, pk.hi, pk.lo, pk.f32);
        else if (want_hi)
            k_pack_lum<FK_BF16><<<blocks, 256, 0, s>>>(owned, t->ndata, t->nch, t->nx, L.lum_nxp, rows, pk.ktot_pad,
                                                      pk.hi, pk.lo, pk.f32);
        count_launch();
        e = cudaGetLastError();
        if (e) rc = cuda_fail(e, "tensor-core table packing");
    }
    if (!rc) {
        e = cudaStreamSynchronize(s);
        if (e) rc = cuda_fail(e, "tensor-core table packing");
    }
    cudaFree(owned);
    cudaStreamDestroy(s);
    if (rc) return rc;
    const long long rows = (long long)L.ntile_n * L.n_rows;
    for (TcPack *pk : {&L.fwd, &L.bwd}) {
        if (want_hi && (rc = make_map(&pk->map_hi, pk->hi, 2, pk->ktot_pad, rows, L.n_rows))) return rc;
        if (want_lo && (rc = make_map(&pk->map_lo, pk->lo, 2, pk->ktot_pad, rows, L.n_rows))) return rc;
        if (want_f32 && (rc = make_map(&pk->map_f32, pk->f32, 4, pk->ktot_pad, rows, L.n_rows))) return rc;
        const int h = L.n_rows / 2;  // a multiple of 8 rows: whole 1024-byte swizzle atoms
        if (want_hi && (rc = make_map(&pk->half_hi, pk->hi, 2, pk->ktot_pad, rows, h))) return rc;
        if (want_lo && (rc = make_map(&pk->half_lo, pk->lo, 2, pk->ktot_pad, rows, h))) return rc;
        if (want_f32 && (rc = make_map(&pk->half_f32, pk->f32, 4, pk->ktot_pad, rows, h))) return rc;
        if (want_lo && (rc = make_narrow_maps(*pk, rows))) return rc;
    }
    if (L.lum_on) {
        TcPack &pk = L.lum;
        const long long lrows = (long long)pk.ntile_n * pk.n_rows;
        const int h = pk.n_rows / 2;
        if (want_hi && ((rc = make_map(&pk.map_hi, pk.hi, 2, pk.ktot_pad, lrows, pk.n_rows)) ||
                        (rc = make_map(&pk.half_hi, pk.hi, 2, pk.ktot_pad, lrows, h))))
            return rc;
        if (want_lo && ((rc = make_map(&pk.map_lo, pk.lo, 2, pk.ktot_pad, lrows, pk.n_rows)) ||
                        (rc = make_map(&pk.half_lo, pk.lo, 2, pk.ktot_pad, lrows, h))))
            return rc;
        if (want_f32 && ((rc = make_map(&pk.map_f32, pk.f32, 4, pk.ktot_pad, lrows, pk.n_rows)) ||
                         (rc = make_map(&pk.half_f32, pk.f32, 4, pk.ktot_pad, lrows, h))))
            return rc;
    }
    return FK_OK;
}

namespace {

// Plain products on the tensor cores (the dense tables of the paper's Table
// 3 and the DIS tables): the B operand is a row-major FP64 matrix [nrows][K]
// packed into tiles of n_rows = min(256, nrows rounded up to 16) rows, one
// group spanning K; the A operand is gathered through km (K entries; -1 for
// none), from a dense table's PDF matrix, a DIS replica's PDF grid or gO.
int plain_layout(fk_table *t, TcPack &pk, int nrows, long long K, const std::vector<int> &km_in) {
    pk.n_rows = std::min(256, (nrows + 15) / 16 * 16);
    pk.ntile_n = (nrows + pk.n_rows - 1) / pk.n_rows;
    pk.grp = TcGroups{};
    pk.grp.ngroups = 1;
    pk.grp.kbeg[0] = 0;
    pk.grp.kend[0] = (int)((K + KPAD - 1) / KPAD * KPAD);
    pk.ktot = pk.grp.kend[0];
    const int kal = (t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_TF32))) ? 128 : 64;
    pk.ktot_pad = (pk.ktot + kal - 1) / kal * kal;
    std::vector<int> km(pk.ktot_pad, -1);
    for (long long k = 0; k < K; ++k) km[k] = km_in.empty() ? (int)k : km_in[k];
    if (cudaMalloc(&pk.kmeta, km.size() * sizeof(int))) return fail(FK_ENOMEM, "tensor-core gather map");
    FK_CUDA(cudaMemcpy(pk.kmeta, km.data(), km.size() * sizeof(int), cudaMemcpyHostToDevice));
    t->bytes += km.size() * sizeof(int);
    const bool want_hi = t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_BF16X3));
    const bool want_lo = t->mask & FK_PREC_BIT(FK_BF16X3);
    const bool want_f32 = t->mask & FK_PREC_BIT(FK_TF32);
    const size_t elems = (size_t)pk.ntile_n * pk.n_rows * pk.ktot_pad;
    if ((want_hi && cudaMalloc(&pk.hi, elems * 2)) || (want_lo && cudaMalloc(&pk.lo, elems * 2)) ||
        (want_f32 && cudaMalloc(&pk.f32, elems * 4)))
        return fail(FK_ENOMEM, "tensor-core table storage");
    t->bytes += elems * (2 * want_hi + 2 * want_lo + 4 * want_f32);
    return FK_OK;
}

template <int PREC>
int pack_plain(const TcPack &pk, const double *d_src, int nrows, long long K, cudaStream_t s) {
    const long long rows = (long long)pk.ntile_n * pk.n_rows;
    const unsigned blocks = (unsigned)std::min<long long>((rows * pk.ktot_pad + 255) / 256, 148LL * 32);
    k_pack_dense<PREC><<<blocks, 256, 0, s>>>(d_src, nrows, K, rows, pk.ktot_pad, pk.hi, pk.lo, pk.f32);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

// Copies the host FP64 matrix [nrows][K] to the device, packs it in every
// tensor-core precision of the table's mask and builds the tensor maps.
int plain_fill(fk_table *t, TcPack &pk, const double *host, int nrows, long long K) {
    const bool want_hi = t->mask & (FK_PREC_BIT(FK_BF16) | FK_PREC_BIT(FK_BF16X3));
    const bool want_lo = t->mask & FK_PREC_BIT(FK_BF16X3);
    const bool want_f32 = t->mask & FK_PREC_BIT(FK_TF32);
    double *owned = nullptr;
    cudaStream_t s = nullptr;
    FK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const size_t src = (size_t)nrows * K;
    if (cudaMalloc(&owned, src * 8)) {
        cudaStreamDestroy(s);
        return fail(FK_ENOMEM, "tensor-core packing staging");
    }
    int rc = FK_OK;
    cudaError_t e = cudaMemcpyAsync(owned, host, src * 8, cudaMemcpyHostToDevice, s);
    if (e) rc = cuda_fail(e, "table upload for packing");
    if (!rc && want_f32) rc = pack_plain<FK_TF32>(pk, owned, nrows, K, s);
    if (!rc && want_lo) rc = pack_plain<FK_BF16X3>(pk, owned, nrows, K, s);
    else if (!rc && want_hi) rc = pack_plain<FK_BF16>(pk, owned, nrows, K, s);
    if (!rc) {
        e = cudaStreamSynchronize(s);
        if (e) rc = cuda_fail(e, "table packing");
    }
    cudaFree(owned);
    cudaStreamDestroy(s);
    if (rc) return rc;
    const long long rows = (long long)pk.ntile_n * pk.n_rows;
    const int h = pk.n_rows / 2;  // a multiple of 8 rows
    if (want_hi && ((rc = make_map(&pk.map_hi, pk.hi, 2, pk.ktot_pad, rows, pk.n_rows)) ||
                    (rc = make_map(&pk.half_hi, pk.hi, 2, pk.ktot_pad, rows, h))))
        return rc;
    if (want_lo && ((rc = make_map(&pk.map_lo, pk.lo, 2, pk.ktot_pad, rows, pk.n_rows)) ||
                    (rc = make_map(&pk.half_lo, pk.lo, 2, pk.ktot_pad, rows, h))))
        return rc;
    if (want_f32 && ((rc = make_map(&pk.map_f32, pk.f32, 4, pk.ktot_pad, rows, pk.n_rows)) ||
                     (rc = make_map(&pk.half_f32, pk.f32, 4, pk.ktot_pad, rows, h))))
        return rc;
    if (want_lo && (rc = make_narrow_maps(pk, rows))) return rc;
    return FK_OK;
}

}  // namespace

// Dense table (the paper's Table 3 product): the table [ndata][K] is the B
// operand, the A operand the caller's PDF matrix through the identity map.
int tc_build_dense(fk_table *t, const double *host_fk) {
    TcLayout &L = t->tc;
    L.G = 16;  // not used by the dense epilogue
    int rc = plain_layout(t, L.fwd, t->ndata, t->E, {});
    if (rc) return rc;
    L.n_rows = L.fwd.n_rows;
    L.ntile_n = L.fwd.ntile_n;
    return plain_fill(t, L.fwd, host_fk, t->ndata, t->E);
}

// DIS table: forward packing = the compacted table [ndata][(k, i)] with the A
// operand gathered from F[r][a_k][xmap[i]]; adjoint packing = its transpose
// [(k, i)][ndata] with the A operand gO[r][d].
int tc_build_dis(fk_table *t, const double *host_fk) {
    TcLayout &L = t->tc;
    L.G = 16;
    const int E = (int)t->E;
    std::vector<int> km(E);
    for (int e = 0; e < E; ++e) km[e] = t->ca[e / t->nx] * t->nxg + t->xmap[e % t->nx];
    int rc = plain_layout(t, L.fwd, t->ndata, E, km);
    if (!rc) rc = plain_fill(t, L.fwd, host_fk, t->ndata, E);
    if (rc) return rc;
    std::vector<double> tr((size_t)E * t->ndata);
    for (int d = 0; d < t->ndata; ++d)
        for (int e = 0; e < E; ++e) tr[(size_t)e * t->ndata + d] = host_fk[(size_t)d * E + e];
    rc = plain_layout(t, L.bwd, E, t->ndata, {});
    if (!rc) rc = plain_fill(t, L.bwd, tr.data(), E, t->ndata);
    L.n_rows = L.fwd.n_rows;
    L.ntile_n = L.fwd.ntile_n;
    return rc;
}

namespace {

// DIS adjoint scatter: gF[r][a_k][xmap[i]] (+)= P[r][k * nx + i]; the grid
// points and flavours the table does not use are left alone (zeroed by the
// caller when overwriting).
__global__ void k_dis_scatter(const float *__restrict__ P, int R, int E, int nx, int nxg,
                              const int *__restrict__ ca, const int *__restrict__ xmap, float *__restrict__ gF) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * E) return;
    const int r = (int)(idx / E), e = (int)(idx - (long long)r * E);
    const int k = e / nx, i = e - k * nx;
    const int a = __ldg(ca + k), m = __ldg(xmap + i);
    if (FK_DBG(a >= 0 && a < NFL && m >= 0 && m < nxg, 13, e)) gF[((size_t)r * NFL + a) * nxg + m] += P[idx];
}

template <int PREC>
int dis_tc_t(const fk_table *t, const float *F, int R, float *O, int ldo, cudaStream_t s) {
    Scratch scr(s);
    CUtensorMap mA, mA2, nA[2];
    TcParams p;
    int rc = prepare<PREC>(t, t->tc.fwd, F, R, scr, nullptr, s, mA, mA2, p, -1, nullptr, nA);
    if (rc) return rc;
    // K (active flavours x points, at most 14 x 64) is never split: a
    // replica's result does not depend on R
    p.O = O;
    p.ldo = ldo;
    return launch_tc<PREC, 16, MODE_DENSE>(t, mA, mA2, b_maps<PREC>(t->tc.fwd), p, s, nA);
}

template <int PREC>
int dis_bwd_tc_t(const fk_table *t, const float *gO, int ldgo, int R, float *gF, int accumulate,
                 cudaStream_t s) {
    Scratch scr(s);
    CUtensorMap mA, mA2, nA[2];
    TcParams p;
    int rc = prepare<PREC>(t, t->tc.bwd, gO, R, scr, nullptr, s, mA, mA2, p, ldgo, nullptr, nA);
    if (rc) return rc;
    const int E = (int)t->E;
    float *P = nullptr;
    FK_CUDA(scr.get(&P, (size_t)R * E));
    p.ndata = E;  // the product's rows are the table's (flavour, x) columns
    p.O = P;
    p.ldo = E;
    rc = launch_tc<PREC, 16, MODE_DENSE>(t, mA, mA2, b_maps<PREC>(t->tc.bwd), p, s, nA);
    if (rc) return rc;
    if (!accumulate) FK_CUDA(cudaMemsetAsync(gF, 0, sizeof(float) * (size_t)R * NFL * t->nxg, s));
    const long long n = (long long)R * E;
    k_dis_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, R, E, t->nx, t->nxg, t->d_ca, t->d_xmap, gF);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

}  // namespace

int dis_tc(const fk_table *t, const float *F, int R, float *O, int ldo, int prec, cudaStream_t s) {
    switch (prec) {
        case FK_BF16: return dis_tc_t<FK_BF16>(t, F, R, O, ldo, s);
        case FK_BF16X3: return dis_tc_t<FK_BF16X3>(t, F, R, O, ldo, s);
        case FK_TF32: return dis_tc_t<FK_TF32>(t, F, R, O, ldo, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

int dis_bwd_tc(const fk_table *t, const float *gO, int ldgo, int R, float *gF, int accumulate, int prec,
               cudaStream_t s) {
    switch (prec) {
        case FK_BF16: return dis_bwd_tc_t<FK_BF16>(t, gO, ldgo, R, gF, accumulate, s);
        case FK_BF16X3: return dis_bwd_tc_t<FK_BF16X3>(t, gO, ldgo, R, gF, accumulate, s);
        case FK_TF32: return dis_bwd_tc_t<FK_TF32>(t, gO, ldgo, R, gF, accumulate, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

int dense_tc(const fk_table *t, const float *Lm, int R, float *O, int ldo, int prec, cudaStream_t s) {
    switch (prec) {
        case FK_BF16: return dense_tc_t<FK_BF16>(t, Lm, R, O, ldo, s);
        case FK_BF16X3: return dense_tc_t<FK_BF16X3>(t, Lm, R, O, ldo, s);
        case FK_TF32: return dense_tc_t<FK_TF32>(t, Lm, R, O, ldo, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

int fwd_tc(const fk_table *t, const float *F, int R, float *O, int ldo, int prec, cudaStream_t s) {
    if (t->kind != FK_KIND_HAD) return fail(FK_EUNSUPPORTED, "tensor-core modes need a hadronic table");
    switch (prec) {
        case FK_BF16: return fwd_tc_t<FK_BF16>(t, F, R, O, ldo, s);
        case FK_BF16X3: return fwd_tc_t<FK_BF16X3>(t, F, R, O, ldo, s);
        case FK_TF32: return fwd_tc_t<FK_TF32>(t, F, R, O, ldo, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

int bwd_tc(const fk_table *t, const float *F, const float *gO, int ldgo, int R, float *gF, int accumulate,
           int prec, cudaStream_t s) {
    if (t->kind != FK_KIND_HAD) return fail(FK_EUNSUPPORTED, "tensor-core modes need a hadronic table");
    switch (prec) {
        case FK_BF16: return bwd_tc_t<FK_BF16>(t, F, gO, ldgo, R, gF, accumulate, s);
        case FK_BF16X3: return bwd_tc_t<FK_BF16X3>(t, F, gO, ldgo, R, gF, accumulate, s);
        case FK_TF32: return bwd_tc_t<FK_TF32>(t, F, gO, ldgo, R, gF, accumulate, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

size_t saved_elems(const fk_table *t, int R) {
    const TcLayout &L = t->tc;
    const size_t R_pad = (size_t)(R + TC_M - 1) / TC_M * TC_M;
    return (size_t)L.ntile_n * L.fwd.grp.ngroups * L.G * t->nx * R_pad;
}

int fwd_tc_save(const fk_table *t, const float *F, int R, float *O, int ldo, float *Y, int prec, cudaStream_t s) {
    switch (prec) {
        case FK_BF16: return fwd_tc_t<FK_BF16>(t, F, R, O, ldo, s, Y);
        case FK_BF16X3: return fwd_tc_t<FK_BF16X3>(t, F, R, O, ldo, s, Y);
        case FK_TF32: return fwd_tc_t<FK_TF32>(t, F, R, O, ldo, s, Y);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

int bwd_tc_saved(const fk_table *t, const float *F, const float *gO, int ldgo, int R, const float *Y, float *gF,
                 int accumulate, int prec, cudaStream_t s) {
    switch (prec) {
        case FK_BF16: return bwd_tc_saved_t<FK_BF16>(t, F, gO, ldgo, R, Y, gF, accumulate, s);
        case FK_BF16X3: return bwd_tc_saved_t<FK_BF16X3>(t, F, gO, ldgo, R, Y, gF, accumulate, s);
        case FK_TF32: return bwd_tc_saved_t<FK_TF32>(t, F, gO, ldgo, R, Y, gF, accumulate, s);
    }
    return fail(FK_EINVAL, "not a tensor-core precision");
}

void tc_free(fk_table *t) {
    for (fk::TcPack *pk : {&t->tc.fwd, &t->tc.bwd}) {
        cudaFree(pk->hi);
        cudaFree(pk->lo);
        cudaFree(pk->f32);
        cudaFree(pk->kmeta);
        cudaFree(pk->mmeta);
        pk->hi = pk->lo = nullptr;
        pk->f32 = nullptr;
        pk->kmeta = pk->mmeta = nullptr;
    }
    cudaFree(t->tc.gmap);
    t->tc.gmap = nullptr;
    fk::TcPack &lum = t->tc.lum;
    cudaFree(lum.hi);
    cudaFree(lum.lo);
    cudaFree(lum.f32);
    lum.hi = lum.lo = nullptr;
    lum.f32 = nullptr;
    cudaFree(t->tc.lum_mmeta);
    t->tc.lum_mmeta = nullptr;
}

namespace {
// Tensor-core issue probe (fk_mma_probe): one CTA, one thread issues `iters`
// BF16 tcgen05.mma instructions of 128 x n x 16 back to back from a 128-byte
// swizzled operand pair in shared memory (zeros, or with fill = 1 finite
// values of varying sign, exponent and mantissa) into one TMEM accumulator,
// commits them to an mbarrier and waits (bounded); the clock64 interval from
// the first issue to the commit's arrival, in SM cycles, goes to cycles[0].
__global__ void __launch_bounds__(64, 1) k_mma_probe(int n, int iters, int fill, unsigned long long *cycles) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t a_bytes = TC_M * 128, b_bytes = (uint32_t)n * 128;
    const uint32_t bar = base + a_bytes + b_bytes;
    volatile uint32_t *slot = reinterpret_cast<volatile uint32_t *>(smem_raw + (bar - raw) + 16);
    const int warp = threadIdx.x >> 5;
    for (uint32_t o = threadIdx.x * 16u; o < a_bytes + b_bytes; o += 64u * 16u) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // two BF16 values per word: |v| in [2^-4, 2^4), both signs
            const uint32_t h = (o + 4u * u) * 2654435761u;
            const uint32_t v0 = ((h >> 31) << 15) | ((123u + ((h >> 8) & 7u)) << 7) | (h & 0x7Fu);
            const uint32_t v1 = (((h >> 30) & 1u) << 15) | ((123u + ((h >> 12) & 7u)) << 7) | ((h >> 16) & 0x7Fu);
            w[u] = fill ? (v0 | (v1 << 16)) : 0u;
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(base + o), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                     "r"(w[3])
                     : "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc<1>(smem_u32((const void *)slot));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    if (threadIdx.x == 32) {
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
        const uint32_t a0 = desc_lo(base), b0 = desc_lo(base + a_bytes);
        bool dead = false;
        const unsigned long long t0 = clock64();
        for (int i = 0; i < iters; ++i) {
            const uint32_t off = (uint32_t)(i & 3) * 2u;  // the four K steps of the swizzle atom
            mma<FK_BF16, 1>(tmem, desc64(a0 + off), desc64(b0 + off), idesc, 1);
        }
        mma_commit<1>(bar);
        mbar_wait(bar, 0, dead);
        cycles[0] = dead ? 0ull : clock64() - t0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_free<1>(tmem);
}

// One thread waits on an mbarrier that expects one arrival nobody makes: the
// bounded wait gives up after limit_ns and raises the device error word.
__global__ void k_wait_selftest(uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool dead = false;
    mbar_wait(b, 0, dead, limit_ns);
}
}  // namespace

int mma_probe(int n, int iters, int fill, unsigned long long *cycles, cudaStream_t s) {
    const size_t smem = 1024 + (size_t)TC_M * 128 + (size_t)n * 128 + 256;
    FK_CUDA(cudaFuncSetAttribute(k_mma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_per_sm(smem)));
    k_mma_probe<<<1, 64, one_per_sm(smem), s>>>(n, iters, fill, cycles);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}

int make_plain_map(CUtensorMap *m, const void *ptr, int esz, long long cols, long long rows, int box_cols,
                   int box_rows) {
    auto fn = encoder();
    if (!fn) return fail(FK_ECUDA, "cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, esz == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(FK_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return FK_OK;
}

FK_DBG_READER(dbg_tc)

int device_status(int reset) {
    int v = 0;
    FK_CUDA(cudaMemcpyFromSymbol(&v, g_fk_device_error, sizeof(int)));
    if (reset) {
        const int z = 0;
        FK_CUDA(cudaMemcpyToSymbol(g_fk_device_error, &z, sizeof(int)));
    }
    return v ? FK_ETIMEDOUT : FK_OK;
}

}  // namespace fk

int fk_mma_probe(int n, int iters, int fill, unsigned long long *cycles, fk_stream stream) {
    using namespace fk;
    if (n < 16 || n > 256 || n % 16 || iters < 1 || iters > (1 << 24) || (fill != 0 && fill != 1) || !cycles)
        return fail(FK_EINVAL,
                    "fk_mma_probe: n a multiple of 16 in 16..256, iters in 1..2^24, fill 0 or 1, cycles not NULL");
    return mma_probe(n, iters, fill, cycles, (cudaStream_t)stream);
}

int fk_wait_selftest(int limit_us) {
    using namespace fk;
    if (limit_us < 1 || limit_us > 1000000) return fail(FK_EINVAL, "fk_wait_selftest: limit_us in 1 .. 1000000");
    int rc = device_status(1);  // start from a clear flag
    if (rc != FK_OK && rc != FK_ETIMEDOUT) return rc;
    k_wait_selftest<<<1, 1>>>((uint64_t)limit_us * 1000ull);
    count_launch();
    FK_CUDA(cudaGetLastError());
    FK_CUDA(cudaDeviceSynchronize());
    rc = device_status(1);
    if (rc == FK_ETIMEDOUT) return FK_OK;
    if (rc != FK_OK) return rc;
    return fail(FK_ECUDA, "fk_wait_selftest: the bounded wait did not report");
}

// ---------------------------------------------- operand slices (k_oz.cu) ----
namespace fk {

int tc_map_bf16(CUtensorMap *m, const void *ptr, long long cols, long long rows, int box_rows) {
    return make_map(m, ptr, 2, cols, rows, box_rows);
}

// The BF16 products of npair groups of npc (A slice, B slice) pairs over K
// chunks c0 .. c0 + nsplit - 1 of kchunk elements (a multiple of 128): A map
// over [S * R_pad][ktot_pad] (slice p's rows start at p * R_pad), B the pack's
// stacked slices (q * ntile_n * n_rows); group u sums its pairs
// (pa, pb)[u * npc + j] in one accumulator, and its partial tile for chunk
// c0 + sp lands at P + (u * nsplit + sp) * R * nd_out, [R][nd_out].  The last
// chunk may run past the operands' K, which the tensor maps read as zeros.
int tc_slice_pairs(const fk_table *t, const TcPack &pk, const CUtensorMap &mA, int R, int nd_out, int kchunk,
                   int c0, int nsplit, int npair, int npc, const uint8_t *pa, const uint8_t *pb, float *P,
                   cudaStream_t s) {
    if (npair < 1 || npc < 1 || npair * npc > 64 || kchunk % Tr<FK_BF16>::KCS)
        return fail(FK_EINVAL, "tc_slice_pairs: bad pair count or chunk");
    const int R_pad = (R + TC_M - 1) / TC_M * TC_M;
    TcParams p{};
    p.nrt = R_pad / TC_M;
    p.ntile_n = pk.ntile_n;
    p.n_rows = pk.n_rows;
    p.nbl = pk.n_rows <= 128 ? 2 : 1;
    p.ngroups = 1;
    p.kbeg[0] = 0;
    p.kspl = kchunk;
    p.kbase = c0 * kchunk;
    p.spc = kchunk / Tr<FK_BF16>::KCS;
    p.npc = npc;
    p.nchunks = npc * p.spc;  // stages per work item: npc pairs over one chunk
    p.kend[0] = npc * kchunk;
    p.nsplit = nsplit;
    p.npair = npair;
    for (int u = 0; u < npair * npc; ++u) {
        p.pa[u] = pa[u];
        p.pb[u] = pb[u];
    }
    p.a_rows = R_pad;
    p.b_rows = pk.ntile_n * pk.n_rows;
    p.ndata = nd_out;
    p.R = R;
    p.R_pad = R_pad;
    p.O = P;
    p.ldo = nd_out;
    p.ostride = (long long)R * nd_out;
    p.ntiles = p.nrt * p.ntile_n * nsplit * npair;
    return launch_tc<FK_BF16, 16, MODE_DENSE>(t, mA, mA, b_maps<FK_BF16>(pk), p, s);
}

}  // namespace fk
