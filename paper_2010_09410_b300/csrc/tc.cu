// tc.cu -- the tensor-core form of BlindRotate.
//
// One BlindRotate step over a tile of 128 gates is a dense contraction of the gadget
// digits D (|d| <= Bg/2 <= 32) by the negacyclic Toeplitz matrices of the key
// polynomials q = BSK_i[r][c] (T[n][k] = q[n-k] for n >= k, -q[n-k+N] otherwise):
//   Y[g][c][n] = sum_{r < 2l} sum_{k < N} D_g[r][k] * T_{r,c}[n][k]   (mod 2^32).
// It runs on the sm_103a tensor cores (tcgen05.mma kind::f16, fp16 operands, fp32
// accumulators in TMEM).  fp16 holds small integers exactly: the (combined) digits and
// the signed byte planes of the key, q = sum_p 2^{8p} q_p with q_p in [-128, 128).  Each
// accumulation covers the l rows of one polynomial of the TRLWE and is read out of TMEM,
// rounded to int32 and recombined mod 2^32 as sum_p 2^{8p} Y_p.
//
// Karatsuba terms.  A negacyclic matrix of size N has the block form [[A, -B], [B, A]]
// with Toeplitz halves A, B, so y = T x is y0 = P1 - P3, y1 = P1 + P2 with the three
// half-size products P1 = (A+B) x0, P2 = A (x1 - x0), P3 = B (x0 + x1).  A Toeplitz
// product splits the same way ([[T00, T01], [T10, T00]]: P = T00 (x0 + x1),
// y0 = P + (T01 - T00) x1, y1 = P + (T10 - T00) x0).  After L levels a step is 3^L
// Toeplitz products of size s = N / 2^L, each with a signed combination of digit blocks
// (|x| <= 32 * 2^L), a key generator that is a signed sum of shifted key segments, and
// signed output blocks; the host builds this plan (build_plan).  An accumulation over l
// rows sums l*s terms below 32 * 2^L * 128, at most l*N*32*128 <= 2^24, so it stays
// exact; a job's 2l rows go in one pass when the digit jobs' bound allows it (see
// ONE_PASS_LIMIT).
//
// The Toeplitz operand is never materialised.  Row n' of a size-s Toeplitz matrix with
// generator t (T[n'][k'] = t[n'-k']) is the window r_vec[s-1-n'+k'] of
// r_vec[x] = t[s-1-x] (x < 2s-1, zero beyond).  Shared memory holds "units": unit u is
// the 16 bytes r_vec[u .. u+7] of one byte plane (fp16).  For an output block n' in
// [c0-NB+1, c0] (column idx = c0 - n') and digits k' in [k0, k0+KS), element (idx, k')
// is r_vec[P0 + idx + k'] with P0 = s-1-c0, i.e. element t of unit (P0 + k0) + idx +
// (k' - k0 - t).  A K-major, no-swizzle UMMA descriptor reads row idx's 8-element
// core-matrix row at base + 16*idx and the next 8 k's at +128 B, so LBO = SBO = 128 B
// walk the windows directly.  The units of every step, term, key polynomial and plane
// are expanded once when the keys are loaded (k_tc_windows), so a key (B) stage is four
// contiguous bulk copies, like the digit (A) stage.
//
// Digits of term j are written per 128-gate tile in the A-operand layout:
// [tile][term j][row r < 2l][stage < s/KS] blocks of 32 KB, each [mg < 16][kb < 16]
// [m8 < 8][8 fp16] for gate m = 8 mg + m8 and digit index k' = stage*KS + 8 kb + e.
// The accumulators live gate-fastest within tiles ([tile][c][word][128 gates]) while the
// BlindRotate runs, so the read-out warps' L2 reductions and the digit jobs' loads are
// whole 128-byte lines; the gate path's key switch reads them in that layout, other
// callers get [G][2][N] from a re-layout launch.
// One launch of k_tc_blind_rotate runs all n steps.  Every wait polls a bounded number
// of times; on time-out the block records TFHE_ETIMEOUT in the context's error word and
// winds down.
//
// SM pairs (optional): a cluster of two CTAs multiplies a 256-gate tile pair with
// cta_group::2 MMAs of M = 256; each CTA stages its own tile's digits and half of the key
// window columns.  CTA 0 fetches the jobs, mirrors them into CTA 1's job ring and issues
// the MMAs; CTA 1's MMA warp forwards "stage full" to CTA 0; commits arrive on both CTAs'
// barriers.
#include <algorithm>
#include <map>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"

namespace {

constexpr int TILE_M = 128;  // gates per tile (TMEM lanes)
constexpr int NB = 128;      // output columns per tile and MMA N
constexpr int KS = 128;      // digits (K) per pipeline stage
constexpr int PLANES = 4;    // byte planes of the key
constexpr int STAGES = 3;
constexpr int A_STAGE_BYTES = TILE_M * KS * 2;            // 32 KB
constexpr int B_UNITS = NB + KS;                          // units per plane and stage
constexpr int B_PLANE_BYTES = B_UNITS * 16;               // 4 KB
constexpr int B_STAGE_BYTES = PLANES * B_PLANE_BYTES;     // 16 KB
// SM-pair form: each CTA of the pair stages half of the B columns of a column block
constexpr int PB_COLS = NB / 2;
constexpr int PB_UNITS = PB_COLS + KS;                     // units per plane and stage
constexpr int PB_PLANE_BYTES = PB_UNITS * 16;              // 3 KB
constexpr int PB_STAGE_BYTES = PLANES * PB_PLANE_BYTES;    // 12 KB
__host__ __device__ constexpr int b_plane_bytes(bool pair) { return pair ? PB_PLANE_BYTES : B_PLANE_BYTES; }
__host__ __device__ constexpr int b_stage_bytes(bool pair) { return pair ? PB_STAGE_BYTES : B_STAGE_BYTES; }
// stages + digit staging (one accumulator polynomial of 8 gates, rows padded by 12 words)
__host__ __device__ constexpr int smem_bytes(int N, bool pair) {
    return STAGES * (A_STAGE_BYTES + b_stage_bytes(pair)) + 8 * (N + 12) * 4;
}
constexpr long long WAIT_CYCLES = 4000000000LL;           // ~2 s at 2 GHz

// ---- PTX wrappers ----------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// try_wait with cluster-scope acquire: for barriers that the peer CTA of a pair arrives
// on, so that the peer's writes before its arrival are visible after the wait.
__device__ __forceinline__ bool mbar_test_cl(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// ---- thread-block-cluster (SM pair) wrappers ----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// shared::cluster address of this CTA's variable `p` in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_addr(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr)
                 : "memory");
}
__device__ __forceinline__ void st_remote_u32(uint32_t caddr, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(caddr), "r"(v) : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// Bounded wait for the phase with the given parity to complete.  Returns false (and
// raises the block's abort flag and the error word) on time-out or when another role
// has already aborted.  CL: cluster-scope acquire (barriers the peer CTA arrives on).
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort,
                                          int *err) {
    const long long t0 = clock64();
    while (!(CL ? mbar_test_cl(bar, parity) : mbar_test(bar, parity))) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            atomicCAS(err, 0, TFHE_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// mbar_wait for a whole warp: lane 0 polls, the others sleep in the shuffle, so 32 threads
// do not compete for issue slots with the MMA and copy threads while they wait.
template <bool CL = false>
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, uint32_t parity, volatile int *abort,
                                               int *err) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait<CL>(bar, parity, abort, err);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    return ok && (CL ? mbar_test_cl(bar, parity) : mbar_test(bar, parity));
}

// Bounded wait that ignores the abort flag: used to let this block's own asynchronous
// work (copies, MMAs) finish before it exits.
__device__ __forceinline__ void mbar_wait_settle(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity) && clock64() - t0 < WAIT_CYCLES) {
    }
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// UMMA shared-memory descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout SWIZZLE_NONE
}

// Instruction descriptor, kind::f16: D f32, A and B f16 (format 0), both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// A-operand collector buffer: the MMAs of one K-step multiply the same digit block A by
// the four key planes, so the first of them reads A from shared memory into the
// collector (fill), the next two reuse it (use) and the last reuses and releases it
// (lastuse).  COLL: 0 fill, 1 use, 2 lastuse.  Cuts the A reads from shared memory 4x.
template <int COLL>
__device__ __forceinline__ void mma_f16_coll(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc) {
    if constexpr (COLL == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, 1, 1;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc));
    else if constexpr (COLL == 1)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, 1, 1;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::use [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.eq.u32 p, 1, 1;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}" ::"r"(
                d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc));
}

// Pair form: one thread of the even CTA issues an M = 256 MMA whose A rows 0-127 and
// B columns 0 .. N/2-1 come from its own shared memory and A rows 128-255 and B columns
// N/2 .. N-1 from the odd CTA's (same offsets); rows 0-127 of D go to the even CTA's
// TMEM, rows 128-255 to the odd CTA's.
__device__ __forceinline__ void mma_f16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// arrive on `bar` (same offset) in both CTAs of the pair once the issued MMAs are done
__device__ __forceinline__ void mma_commit_pair_both(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
        "[%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

// arrive on `bar` in the issuing CTA only
__device__ __forceinline__ void mma_commit_pair_own(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// fp16 bit pattern of a small integer |x| <= 2048 (exact).
__device__ __forceinline__ uint32_t f16_bits(int x) {
    return __half_as_ushort(__int2half_rn(x));
}

// signed byte planes: q = sum_p 2^{8p} q_p (mod 2^32), q_p in [-128, 128)
__device__ __forceinline__ void byte_planes(uint32_t q, int (&pl)[PLANES]) {
#pragma unroll
    for (int p = 0; p < PLANES; p++) {
        const int d = (int)(int8_t)(q & 0xFF);
        pl[p] = d;
        q = (q - (uint32_t)d) >> 8;
    }
}

// ---------------------------------------------------------------------------
// Karatsuba term plan
// ---------------------------------------------------------------------------

constexpr int MAX_TERMS = 27;  // 3^L, L <= 3
constexpr int MAX_BLK = 8;     // 2^L blocks of size s per polynomial

// Digit combination of each term (weight of input block b) and the sign with which its
// product enters output block b, per level, in build_plan's term order; the host checks
// its plan against these tables.  Compile-time weights let the digit jobs add only the
// blocks a term uses and recombine the term products without a table lookup.
__host__ __device__ constexpr int in_coef_tab(int L, int j, int b) {
    constexpr int t0[1][1] = {{1}};
    constexpr int t1[3][2] = {{1, 0}, {-1, 1}, {1, 1}};
    constexpr int t2[9][4] = {{1, 1, 0, 0},   {0, 1, 0, 0},  {1, 0, 0, 0},
                              {-1, -1, 1, 1}, {0, -1, 0, 1}, {-1, 0, 1, 0},
                              {1, 1, 1, 1},   {0, 1, 0, 1},  {1, 0, 1, 0}};
    constexpr int t3[27][8] = {
        {1, 1, 1, 1, 0, 0, 0, 0},     {0, 1, 0, 1, 0, 0, 0, 0},     {1, 0, 1, 0, 0, 0, 0, 0},
        {0, 0, 1, 1, 0, 0, 0, 0},     {0, 0, 0, 1, 0, 0, 0, 0},     {0, 0, 1, 0, 0, 0, 0, 0},
        {1, 1, 0, 0, 0, 0, 0, 0},     {0, 1, 0, 0, 0, 0, 0, 0},     {1, 0, 0, 0, 0, 0, 0, 0},
        {-1, -1, -1, -1, 1, 1, 1, 1}, {0, -1, 0, -1, 0, 1, 0, 1},   {-1, 0, -1, 0, 1, 0, 1, 0},
        {0, 0, -1, -1, 0, 0, 1, 1},   {0, 0, 0, -1, 0, 0, 0, 1},    {0, 0, -1, 0, 0, 0, 1, 0},
        {-1, -1, 0, 0, 1, 1, 0, 0},   {0, -1, 0, 0, 0, 1, 0, 0},    {-1, 0, 0, 0, 1, 0, 0, 0},
        {1, 1, 1, 1, 1, 1, 1, 1},     {0, 1, 0, 1, 0, 1, 0, 1},     {1, 0, 1, 0, 1, 0, 1, 0},
        {0, 0, 1, 1, 0, 0, 1, 1},     {0, 0, 0, 1, 0, 0, 0, 1},     {0, 0, 1, 0, 0, 0, 1, 0},
        {1, 1, 0, 0, 1, 1, 0, 0},     {0, 1, 0, 0, 0, 1, 0, 0},     {1, 0, 0, 0, 1, 0, 0, 0}};
    return L == 0 ? t0[j][b] : (L == 1 ? t1[j][b] : (L == 2 ? t2[j][b] : t3[j][b]));
}
__host__ __device__ constexpr int out_coef_tab(int L, int j, int b) {
    constexpr int t0[1][1] = {{1}};
    constexpr int t1[3][2] = {{1, 1}, {0, 1}, {-1, 0}};
    constexpr int t2[9][4] = {{1, 1, 1, 1},   {1, 0, 1, 0},  {0, 1, 0, 1},
                              {0, 0, 1, 1},   {0, 0, 1, 0},  {0, 0, 0, 1},
                              {-1, -1, 0, 0}, {-1, 0, 0, 0}, {0, -1, 0, 0}};
    constexpr int t3[27][8] = {
        {1, 1, 1, 1, 1, 1, 1, 1},     {1, 0, 1, 0, 1, 0, 1, 0},     {0, 1, 0, 1, 0, 1, 0, 1},
        {1, 1, 0, 0, 1, 1, 0, 0},     {1, 0, 0, 0, 1, 0, 0, 0},     {0, 1, 0, 0, 0, 1, 0, 0},
        {0, 0, 1, 1, 0, 0, 1, 1},     {0, 0, 1, 0, 0, 0, 1, 0},     {0, 0, 0, 1, 0, 0, 0, 1},
        {0, 0, 0, 0, 1, 1, 1, 1},     {0, 0, 0, 0, 1, 0, 1, 0},     {0, 0, 0, 0, 0, 1, 0, 1},
        {0, 0, 0, 0, 1, 1, 0, 0},     {0, 0, 0, 0, 1, 0, 0, 0},     {0, 0, 0, 0, 0, 1, 0, 0},
        {0, 0, 0, 0, 0, 0, 1, 1},     {0, 0, 0, 0, 0, 0, 1, 0},     {0, 0, 0, 0, 0, 0, 0, 1},
        {-1, -1, -1, -1, 0, 0, 0, 0}, {-1, 0, -1, 0, 0, 0, 0, 0},   {0, -1, 0, -1, 0, 0, 0, 0},
        {-1, -1, 0, 0, 0, 0, 0, 0},   {-1, 0, 0, 0, 0, 0, 0, 0},    {0, -1, 0, 0, 0, 0, 0, 0},
        {0, 0, -1, -1, 0, 0, 0, 0},   {0, 0, -1, 0, 0, 0, 0, 0},    {0, 0, 0, -1, 0, 0, 0, 0}};
    return L == 0 ? t0[j][b] : (L == 1 ? t1[j][b] : (L == 2 ? t2[j][b] : t3[j][b]));
}

// Packed fp16 pairs of small integers: sums and differences stay exact while every value
// stays within |x| <= 2048 (11-bit significand); the digits and their Karatsuba
// combinations are at most 2^L * Bg/2 <= 256 in magnitude.
__device__ __forceinline__ uint32_t hadd2(uint32_t x, uint32_t y) {
    uint32_t r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
    return r;
}
__device__ __forceinline__ uint32_t hsub2(uint32_t x, uint32_t y) {
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
    return r;
}
__device__ __forceinline__ uint32_t habs2(uint32_t x) { return x & 0x7FFF7FFFu; }
// sum of the two halves of a packed pair of integers in [0, 512): 1536 + x has the fp16
// pattern 0x6600 + x
__device__ __forceinline__ int fold_f16_sums(uint32_t x) {
    const uint32_t v = hadd2(x, 0x66006600u);
    return (int)(v & 0xFFFFu) + (int)(v >> 16) - 2 * 0x6600;
}

// Gadget digits of two offset values as one packed fp16 pair: the Bgbit-wide fields at bit
// `sh` (raw in [0, Bg)) are placed under the fp16 pattern 0x6600 (the value 1536 + raw:
// exponent 10 gives unit spacing on [1024, 2048)), and one packed subtraction of
// dsub = 1536 + Bg/2 in both halves leaves raw - Bg/2, the signed digit.  Bg <= 512.
__device__ __forceinline__ uint32_t digit_pair(uint32_t u0, uint32_t u1, int sh, uint32_t fmask,
                                               uint32_t dsub) {
    const uint32_t t = __byte_perm(u0 >> sh, u1 >> sh, 0x5410);  // low halves of both
    return hsub2((t & fmask) | 0x66006600u, dsub);
}

// The 3^L Karatsuba digit combinations of 8 positions, v[b][w] the packed digits of
// positions 2w, 2w+1 in size-s block b of the polynomial, built as the plan's tree
// (negacyclic split: x0, x1 - x0, x0 + x1; then per Toeplitz split: x0 + x1, x1, x0)
// instead of one dense sum per term: 23 additions per position at L = 3 instead of 80.
// emit(j, x) receives term j (a std::integral_constant, build_plan's order) and its 4
// packed words.
__host__ __device__ constexpr int pow3(int k) { return k == 0 ? 1 : 3 * pow3(k - 1); }
__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x / 2); }
constexpr int DW = 4;  // packed words per thread and block (8 positions)

template <int M, int J0, typename F>
__device__ __forceinline__ void kara_split(const uint32_t (&v)[M][DW], F &emit) {
    if constexpr (M == 1) {
        emit(std::integral_constant<int, J0>(), v[0]);
    } else {
        constexpr int H = M / 2, SUB = pow3(ilog2c(H));
        uint32_t sa[H][DW], s1[H][DW], s0[H][DW];
#pragma unroll
        for (int h = 0; h < H; h++)
#pragma unroll
            for (int w = 0; w < DW; w++) {
                sa[h][w] = hadd2(v[h][w], v[H + h][w]);
                s1[h][w] = v[H + h][w];
                s0[h][w] = v[h][w];
            }
        kara_split<H, J0>(sa, emit);
        kara_split<H, J0 + SUB>(s1, emit);
        kara_split<H, J0 + 2 * SUB>(s0, emit);
    }
}

template <int M, typename F>
__device__ __forceinline__ void kara_terms(const uint32_t (&v)[M][DW], F &emit) {
    if constexpr (M == 1) {
        emit(std::integral_constant<int, 0>(), v[0]);
    } else {
        constexpr int H = M / 2, SUB = pow3(ilog2c(H));
        uint32_t p1[H][DW], p2[H][DW], p3[H][DW];
#pragma unroll
        for (int h = 0; h < H; h++)
#pragma unroll
            for (int w = 0; w < DW; w++) {
                p1[h][w] = v[h][w];
                p2[h][w] = hsub2(v[H + h][w], v[h][w]);
                p3[h][w] = hadd2(v[h][w], v[H + h][w]);
            }
        kara_split<H, 0>(p1, emit);
        kara_split<H, SUB>(p2, emit);
        kara_split<H, 2 * SUB>(p3, emit);
    }
}

// Stores term j's 8 combinations of one thread (16 bytes) into the A-operand layout: the
// digit blocks of the terms of one (tile, row, stage) are consecutive, so term j's unit is
// j blocks after term 0's (a constant offset).
// The stores carry an L2 evict-last policy: a digit block waits in L2 for its product
// jobs while the windows and accumulators stream past it (78 GB of DRAM traffic per
// 4096-gate launch instead of 96 GB with plain stores).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
struct DigitStore {
    uint4 *p;      // the thread's unit in term 0's block
    uint64_t pol;  // L2 evict-last policy
#ifdef TFHE_BOUNDS_CHECK
    size_t left;   // units of the digit buffer from p on
    int *err;
#endif
    template <int j>
    __device__ __forceinline__ void operator()(std::integral_constant<int, j>, const uint32_t (&x)[DW]) const {
#ifdef TFHE_BOUNDS_CHECK
        if (!tfhe_in_bounds((size_t)j * (A_STAGE_BYTES / 16), left, err)) return;
#endif
        asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p + (size_t)j * (A_STAGE_BYTES / 16)),
                     "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "l"(pol)
                     : "memory");
    }
};

// u[e] = (X^rot p - p)[k0 + e] + off for the 8 positions k0 .. k0+7 (k0 a multiple of 8)
// of the row p of one gate in shared memory: X^rot p at k is p[k - rk] for k >= rk and
// -p[k - rk + N] below it, all negated once more when rot >= N (rneg all ones).  The row
// holds -p[0..7] after its N words, so that positions crossing the wrap read the right
// sign without a branch.  plain (CMUX mode, the row holds d1 - d0): u = p + off.
__device__ __forceinline__ void rotated_diff8(const uint32_t *row, int N, int k0, int rk, uint32_t rneg,
                                              uint32_t off, bool plain, uint32_t (&u)[8]) {
    const uint4 o0 = *(const uint4 *)(row + k0), o1 = *(const uint4 *)(row + k0 + 4);
    const uint32_t own[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
    if (plain) {
#pragma unroll
        for (int e = 0; e < 8; e++) u[e] = own[e] + off;
        return;
    }
    int src = k0 - rk;
    uint32_t sg = rneg;
    if (src < 0) {
        src += N;
        sg = ~rneg;
    }
    const uint32_t base = off - sg;  // (v ^ sg) - sg is v or -v
#pragma unroll
    for (int e = 0; e < 8; e++) u[e] = (row[src + e] ^ sg) + base - own[e];
}

// The same tree as coefficients (weight of input block b in term j), checked against
// in_coef_tab at compile time.
__host__ __device__ constexpr int tree_split_coef(int M, int j, int b) {
    if (M == 1) return b == 0 ? 1 : 0;
    const int H = M / 2, SUB = pow3(ilog2c(H));
    const int child = j / SUB, c = tree_split_coef(H, j % SUB, b % H), hi = b / H;
    return child == 0 ? c : (child == 1 ? (hi ? c : 0) : (hi ? 0 : c));
}
__host__ __device__ constexpr int tree_coef(int L, int j, int b) {
    if (L == 0) return b == 0 ? 1 : 0;
    const int M = 1 << L, H = M / 2, SUB = pow3(L - 1);
    const int child = j / SUB, c = tree_split_coef(H, j % SUB, b % H), hi = b / H;
    return child == 0 ? (hi ? 0 : c) : (child == 1 ? (hi ? c : -c) : c);
}
__host__ __device__ constexpr bool tree_matches_tables() {
    for (int L = 0; L <= 3; L++)
        for (int j = 0; j < pow3(L); j++)
            for (int b = 0; b < (1 << L); b++)
                if (tree_coef(L, j, b) != in_coef_tab(L, j, b)) return false;
    return true;
}
static_assert(tree_matches_tables(), "Karatsuba tree and term table disagree");

struct KTerm {
    int n_in, in_blk[MAX_BLK], in_sgn[MAX_BLK];      // digit combination: sum sgn * block (size s)
    int n_out, out_blk[MAX_BLK], out_sgn[MAX_BLK];   // output blocks (size s) receiving sgn * P
    int n_key, key_off[MAX_BLK], key_coef[MAX_BLK];  // generator t_j[d] = sum coef * t[d + off]
    int in_coef[MAX_BLK];                            // the digit combination as block weights
    int out_coef[MAX_BLK];                           // the output signs as block weights
};

// Negacyclic generator of the key polynomial q: t[e] = q[e] (e >= 0), -q[e+N] (e < 0).
__device__ __forceinline__ uint32_t neg_gen(const uint32_t *__restrict__ q, int N, int e) {
    return e >= 0 ? __ldg(q + e) : 0u - __ldg(q + e + N);
}

// Window units of term T for every (key, row, column) polynomial:
// win[((poly * nterms + j) * 4 + p) * 2s + u] holds byte plane p of r_vec_j[u .. u+7].
// blockIdx.x = key polynomial (keys of ppk polynomials: BSK_i, or CMUX selectors that lie
// key_stride polynomials apart), blockIdx.y = term.
__global__ void k_tc_windows(const uint32_t *__restrict__ polys, int N, int s, int nterms,
                             const KTerm *__restrict__ terms, uint4 *__restrict__ win, int ppk,
                             int64_t key_stride) {
    const size_t poly = blockIdx.x;
    const int j = blockIdx.y;
    const uint32_t *q = polys + ((int64_t)(poly / ppk) * key_stride + poly % ppk) * N;
    const KTerm T = terms[j];
    for (int u = threadIdx.x; u < 2 * s; u += blockDim.x) {
        uint32_t w[PLANES][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            uint32_t val[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int x = u + e + h;
                uint32_t v = 0;
                if (x < 2 * s - 1) {
                    const int d = s - 1 - x;
                    for (int m = 0; m < T.n_key; m++)
                        v += (uint32_t)T.key_coef[m] * neg_gen(q, N, d + T.key_off[m]);
                }
                val[h] = v;
            }
            int pl0[PLANES], pl1[PLANES];
            byte_planes(val[0], pl0);
            byte_planes(val[1], pl1);
#pragma unroll
            for (int p = 0; p < PLANES; p++) w[p][e / 2] = f16_bits(pl0[p]) | (f16_bits(pl1[p]) << 16);
        }
#pragma unroll
        for (int p = 0; p < PLANES; p++)
            win[((poly * nterms + j) * PLANES + p) * 2 * s + u] =
                make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
}

// The tensor-core path keeps its accumulators gate-fastest within 128-gate tiles:
// word k of polynomial c of gate g = 128 t + m sits at acc_t[((t * 2 + c) * N + k) * 128 + m],
// so a warp's 32 gates touch one 128-byte line per word.  The step-0 digit jobs write
// ACC(0) = X^{-b~} (0, v), v_j = mu: coefficient j of X^{-b~} v is +mu when
// (j + b~) mod 2N < N; gates >= G (padding of the last tile) start at zero.
static_assert(TILE_M == TFHE_TC_TILE, "tile size shared with the key switch");

// acc[g][c][k] = acc_t word (g, c, k): 32 x 32 blocks through shared memory.
// grid (N / 32, 4 * tiles, 2), block (32, 8).
__global__ void k_tc_untile_acc(int N, int G, const uint32_t *__restrict__ acc_t,
                                uint32_t *__restrict__ acc) {
    __shared__ uint32_t t[32][33];
    const int k0 = blockIdx.x * 32, g0 = blockIdx.y * 32, c = blockIdx.z;
    const int tile = g0 / TILE_M, m0 = g0 % TILE_M;
    const uint32_t *src = acc_t + ((size_t)(tile * 2 + c) * N + k0) * TILE_M + m0;
#pragma unroll
    for (int i = 0; i < 32; i += 8)
        t[threadIdx.y + i][threadIdx.x] = src[(size_t)(threadIdx.y + i) * TILE_M + threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int g = g0 + threadIdx.y + i;
        if (g < G) acc[((size_t)g * 2 + c) * N + k0 + threadIdx.x] = t[threadIdx.x][threadIdx.y + i];
    }
}

// CMUX mode: out + x ox + y oy (+ c N + k) = acc_t word (tile, c, k, m) for the tile's
// CMUX x = (tile % tpg) * 128 + m of group y = tile / tpg.  grid (N / 32, 4 * tiles, 2).
__global__ void k_tc_untile_cmux(int N, int tpg, int nx, int64_t count, int64_t ox, int64_t oy,
                                 const uint32_t *__restrict__ acc_t, uint32_t *__restrict__ out) {
    __shared__ uint32_t t[32][33];
    const int k0 = blockIdx.x * 32, g0 = blockIdx.y * 32, c = blockIdx.z;
    const int tile = g0 / TILE_M, m0 = g0 % TILE_M;
    const uint32_t *src = acc_t + ((size_t)(tile * 2 + c) * N + k0) * TILE_M + m0;
#pragma unroll
    for (int i = 0; i < 32; i += 8)
        t[threadIdx.y + i][threadIdx.x] = src[(size_t)(threadIdx.y + i) * TILE_M + threadIdx.x];
    __syncthreads();
    const int y = tile / tpg;
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
        const int x = (tile % tpg) * TILE_M + m0 + threadIdx.y + i;
        if (x < nx && (int64_t)y * nx + x < count)
            out[x * ox + y * oy + (int64_t)c * N + k0 + threadIdx.x] = t[threadIdx.x][threadIdx.y + i];
    }
}

// ---------------------------------------------------------------------------
// Persistent BlindRotate: all n steps in one launch, one block per SM.
//
// Jobs: D(i, gt, part) writes the digits (all terms) of gates 8*part .. 8*part+7 of gate
// tile gt for step i (16 parts per tile) from ACC(i), the accumulator before step i;
// E(i, gt, j, c, b) is the tensor-core product P_j of term j for column block b of output
// polynomial c, added with its signs into every output block of ACC that it enters (the
// Karatsuba recombination) by reductions at L2, so the products of one tile and step run
// in any order (integer addition mod 2^32 commutes).  Two job streams, each taken in
// order from its own global counter: digit jobs (step, tile, part) by the digit warps of
// any block, product jobs (step, tile, term, polynomial, block) by the loaders.  With
// D(i) < E(i) < D(i+1) a job only waits for jobs earlier in that order, each stream is
// handed out in order, and no role holds anything a later job needs, so the schedule
// cannot deadlock:
//   stages of E(i, gt, ...), and its additions into ACC, wait for done_D[gt] >= 16 (i+1)
//   (every digit job of the step has read ACC(i));
//   D(i, gt, .) waits for done_E[gt] >= E_per_tile * i (ACC(i) is complete).
// Every wait is bounded.
//
// Warp roles (512 threads): warps 0-7 read TMEM out (warp w owns lanes 32(w%4)..+31 and
// columns 64(w/4)..+63 of the block), warp 8 owns TMEM and one lane issues the MMAs,
// warp 12 fetches jobs and streams stages with cp.async.bulk, warps 9-11 and 13-15
// compute digits.  The four planes of TMEM are handed back one by one after each K-pass's
// read-out, so the next pass's MMAs on plane p start as soon as plane p has been read;
// the passes of a job accumulate in registers and the product is added once.
// ---------------------------------------------------------------------------
constexpr int P_THREADS = 512;
constexpr int EPI_WARPS = 8;                 // read-out warps: 2 per TMEM lane quarter
constexpr int EPI_THREADS = EPI_WARPS * 32;
// A warp issues on SM sub-partition (warp index mod 4).  The MMA-issuing warp shares its
// sub-partition only with the loader and two read-out warps; the ALU-heavy digit warps
// (9-11, 13-15) sit two each on the other three.  16 warps of 128 registers fill the
// register file.
constexpr int MMA_WARP = 8;                  // TMEM owner + MMA issue
constexpr int LOAD_WARP = 12;                // job fetch + stage loads
__device__ __forceinline__ int digit_warp_index(int warp) { return warp < LOAD_WARP ? warp - 9 : warp - 10; }
constexpr int DG_THREADS = 192;              // digit warps 9-11 and 13-15
__device__ __forceinline__ void dg_sync() { asm volatile("bar.sync 2, %0;" ::"n"(DG_THREADS) : "memory"); }
constexpr int EPI_COLS = NB / 2;             // columns per read-out warp
// read-out conversion constants: 1.5*2^23 and its bit pattern; the initial sum cancels the
// bit-pattern offset added by both K-halves of all four planes (mod 2^32)
constexpr float RO_MAGIC = 12582912.0f;
constexpr uint32_t RO_MAGIC_BITS = 0x4B400000u;
constexpr float RO_FAST_LIMIT = 4194304.0f;  // 2^22
constexpr int RO_COLS = 32;                   // columns per TMEM load slice
// bit-pattern offset that one K-pass adds over the four planes (mod 2^32)
constexpr uint32_t RO_MAGIC_PER_PASS =
    RO_MAGIC_BITS + (RO_MAGIC_BITS << 8) + (RO_MAGIC_BITS << 16) + (RO_MAGIC_BITS << 24);
// A product job accumulates its whole K (2l rows of s digits) in one TMEM pass when every
// gate g of the tile has sum_k |x_gk| <= 2^17 for the job's term: each partial sum is then
// at most 128 * 2^17 = 2^24 in magnitude (|key byte| <= 128), so fp32 stays exact.  The
// digit jobs check a bound of it (the sum over the term's input blocks of sum |digit|);
// a (tile, step) where the bound fails is marked and its products take two passes of l
// rows each, for which the worst case l * s * (32 * 2^L) * 128 <= 2^24.
constexpr int ONE_PASS_LIMIT = 1 << 17;  // default and largest allowed limit
constexpr int JQ = 8;       // job ring depth
// Fewest product jobs per step of a tile chunk, in waves of the SMs: 32 tiles at
// Karatsuba level 2 (36 jobs per tile and step) make two chunks of 16 on 148 SMs.  Smaller
// chunks were slower on B300 (3.2 waves: +17 %), as were uneven ones.
constexpr double CHUNK_WAVES = 3.8;
constexpr int DPARTS = 16;  // digit parts per gate tile (8 gates each)

enum { JOB_STOP = 0, JOB_D = 1, JOB_E = 2, JOB_NOP = 3 };

// packed job-table entry: kind (2 bits) | gt (12) | term (5) | c (1) | sub (4)
__host__ __device__ constexpr uint32_t pack_job(int kind, int gt, int j, int c, int sub) {
    return (uint32_t)kind | ((uint32_t)gt << 2) | ((uint32_t)j << 14) | ((uint32_t)c << 19) |
           ((uint32_t)sub << 20);
}

struct Job {
    int kind, i, gt, j, c, sub;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// gpu-scope release increment of a progress counter (pairs with ld_acquire)
__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// relaxed reduction at L2: the read-out adds term products into the accumulators
__device__ __forceinline__ void red_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool wait_count(const uint32_t *p, uint32_t target, volatile int *abort,
                                           int *err) {
    const long long t0 = clock64();
    while (ld_acquire(p) < target) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            atomicCAS(err, 0, TFHE_ETIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

struct BrArgs {
    int N, l, Bgbit, G, n, n1;
    int s, nterms;              // term size N / 2^L and count 3^L
    int tiles, cbs;             // gate tiles, column blocks per term output (2 * s / NB)
    int tiles_pad;              // tiles rounded up to the pair size (pair form) or tiles
    int one_pass_limit;         // largest per-gate sum of |digit| accumulated in one pass
    int e_per_tile;             // product jobs per tile and step
    int step_len;               // entries of the per-step product-job table
    long long total_e, total_d;
    // Tiles are processed in nchunks chunks of job-table units (tiles, or tile pairs) of
    // nearly equal size (the first units % nchunks chunks hold one unit more): both job
    // streams run all steps of one chunk before the next, so a step's digit blocks and
    // accumulators of the chunk stay in L2.  units: table units in all.
    int units, nchunks;
    const uint32_t *table;      // per-step job table
    const KTerm *terms;
    const uint32_t *bar;        // [G][n+1] ModSwitched combinations (written at step 0 when fused)
    // fused gate combination: when `in` is set, the step-0 digit jobs form bar[g] =
    // ModSwitch(combination of in[idx[g][0]], in[idx[g][1]] for gate type types[g]) into
    // bar_w (which `bar` aliases); a bad type or index gives a zero row and TFHE_EINVAL
    const uint32_t *in;
    int64_t num_in;
    const uint8_t *types;
    const int32_t *idx;
    uint32_t *bar_w;
    int ms_shift;               // ModSwitch shift 32 - log2(2N)
    // CMUX mode (one step): tile gt holds CMUXes x = (gt % tpg) * 128 + lane of group
    // y = gt / tpg, whose selector's windows are key y; ACC(0) = d0 and the digits are
    // those of d1 - d0 (no rotation); CMUX (x, y) reads d1/d0 + x dx + y dy (words)
    int cmux, tpg;
    const uint32_t *cm_d1, *cm_d0;
    int64_t cm_dx, cm_dy;
    int cm_nx;
    int64_t cm_count;
    uint32_t *acc;              // [tiles_pad][2][N][128] (gate-fastest within a tile)
    uint4 *digits;              // [tiles][2l][s/KS][nterms] x 32 KB
    const uint4 *win;           // [n][2l][2][nterms][4][2s] units
    uint32_t *sync;             // [0] product-job counter, [1] digit-job counter,
                                // then per padded tile: done_D, done_E, two_pass (the last
                                // step + 1 whose products need two passes)
    int *err;
    // extents of the digit, accumulator, window and combination buffers, for the debug
    // build's index checks (TFHE_BOUNDS_CHECK)
    size_t digits_units, acc_words, win_units, bar_words;
};

// Chunk of stream entry `job` when `units` units are split into `nchunks` chunks of
// nearly equal size (the first units % nchunks one larger) and each unit contributes
// per_unit entries per chunk pass: the chunk's first unit u0, its size uc, and the
// entry's offset rem within the chunk.
__device__ __forceinline__ void chunk_of(long long job, int units, int nchunks, long long per_unit,
                                         int *u0, int *uc, long long *rem) {
    const int base = units / nchunks, extra = units % nchunks;
    const long long big = (long long)extra * (base + 1) * per_unit;  // entries of the larger chunks
    int c;
    if (job < big) {
        c = (int)(job / ((base + 1) * per_unit));
        *rem = job - (long long)c * (base + 1) * per_unit;
    } else {
        c = extra + (int)((job - big) / (base * per_unit));
        *rem = job - big - (long long)(c - extra) * base * per_unit;
    }
    *u0 = c * base + min(c, extra);
    *uc = base + (c < extra ? 1 : 0);
}

__device__ __forceinline__ Job decode_e(const BrArgs &a, int job) {
    Job J{JOB_STOP, 0, 0, 0, 0, 0};
    if (job < 0) return J;
    // the table lists every unit's e_per_tile entries in unit order
    int u0, uc;
    long long rem;
    chunk_of(job, a.units, a.nchunks, (long long)a.n * a.e_per_tile, &u0, &uc, &rem);
    const int len_c = uc * a.e_per_tile;
    const uint32_t e = __ldg(a.table + (long long)u0 * a.e_per_tile + rem % len_c);
    J.kind = JOB_E;
    J.i = (int)(rem / len_c);
    J.gt = (int)((e >> 2) & 0xFFF);
    J.j = (int)((e >> 14) & 0x1F);
    J.c = (int)((e >> 19) & 1);
    J.sub = (int)((e >> 20) & 0xF);
    return J;
}

// TMEM passes of product job J (1 or 2): 2 when the digit jobs of its tile (both tiles of
// a pair) marked its step.  Waits (acquire) for those digit jobs first.
template <bool PAIR>
__device__ __forceinline__ int passes_for(const BrArgs &a, const Job &J, const uint32_t *done_D,
                                          const uint32_t *two_pass) {
    int passes = 1;
    for (int u = 0; u < (PAIR ? 2 : 1); u++) {
        const int gt = PAIR ? 2 * J.gt + u : J.gt;
        if (gt >= a.tiles) continue;
        const long long t0 = clock64();
        while (ld_acquire(&done_D[gt]) < (uint32_t)(DPARTS * (J.i + 1)) && clock64() - t0 < WAIT_CYCLES) {
        }
        if (*(volatile const uint32_t *)&two_pass[gt] == (uint32_t)(J.i + 1)) passes = 2;
    }
    return passes;
}

template <int L, bool PAIR>
__global__ void __launch_bounds__(P_THREADS, 1) k_tc_blind_rotate(BrArgs a) {
    constexpr int NBLK = 1 << L;                      // size-s blocks per polynomial
    constexpr int NT = L == 0 ? 1 : (L == 1 ? 3 : (L == 2 ? 9 : 27));  // terms
    constexpr int BPL = b_plane_bytes(PAIR), BST = b_stage_bytes(PAIR);
    extern __shared__ __align__(128) uint8_t smem[];  // no swizzle: 16-byte alignment suffices
    uint8_t *a_st = smem;
    uint8_t *b_st = smem + STAGES * A_STAGE_BYTES;
    uint32_t *d_rows = (uint32_t *)(b_st + STAGES * BST);  // [8][N + 12]
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], pfull[STAGES];
    __shared__ __align__(8) uint64_t acc_full[PLANES], acc_empty[PLANES], drain;
    __shared__ __align__(8) uint64_t job_full[JQ], job_empty[JQ];
    __shared__ int jobs[JQ];
    __shared__ int job_passes[JQ];  // set by the loader before the job's first stage is full
    // one-SM form: the MMA thread hands the job's pass count to the read-out (ro_passes,
    // published by an arrival on passes_ready), so the read-out needs no global round trip
    __shared__ int ro_passes[JQ];
    __shared__ __align__(8) uint64_t passes_ready[JQ];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int8_t out_tab[NT][NBLK];  // out_coef_tab of this level

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // pair form: CTA 0 of the cluster fetches the product jobs and issues the MMAs
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const int N = a.N, l = a.l, s = a.s;
    const int kstages = s / KS;
    const int half_stages = l * kstages;
    const int total_stages = 2 * half_stages;
    const int bpp = s / NB;  // column blocks per term output polynomial
    uint32_t *e_counter = a.sync;
    uint32_t *d_counter = a.sync + 1;
    uint32_t *done_D = a.sync + 2;
    uint32_t *done_E = a.sync + 2 + a.tiles_pad;
    uint32_t *two_pass = a.sync + 2 + 2 * a.tiles_pad;

    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
            mbar_init(&pfull[q], 1);  // pair form: the odd CTA's stage q is full
        }
        for (int p = 0; p < PLANES; p++) mbar_init(&acc_full[p], 1);
        // one arrival per read-out warp (of both CTAs in the pair form)
        for (int p = 0; p < PLANES; p++) mbar_init(&acc_empty[p], (PAIR ? 2 : 1) * EPI_WARPS);
        mbar_init(&drain, 1);
        for (int q = 0; q < JQ; q++) {
            mbar_init(&job_full[q], 1);
            // MMA lane, read-out leader; pair form also the odd CTA's loader, stage
            // forwarder and read-out leader
            mbar_init(&job_empty[q], PAIR ? 5 : 2);
            mbar_init(&passes_ready[q], 1);
        }
        abort_flag = 0;
#pragma unroll
        for (int j = 0; j < NT; j++)
#pragma unroll
            for (int b = 0; b < NBLK; b++) out_tab[j][b] = (int8_t)out_coef_tab(L, j, b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMA_WARP) {
        if constexpr (PAIR) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(512));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(512));
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync_all();  // both CTAs' barriers exist before any remote use
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;
    int *err = a.err;

    if (warp == LOAD_WARP) {
        // ---- job fetch + stage loads ----
        if (lane == 0) {
            // CTA 0 hands out job q+1 while it streams job q's stages (one job ahead),
            // so the fetch latency hides behind the stage ring.
            auto publish = [&](int qq) -> int {  // -2: aborted
                const int sl = qq % JQ;
                if (qq >= JQ && !mbar_wait<PAIR>(&job_empty[sl], ((qq / JQ) - 1) & 1, abort, err))
                    return -2;
                const unsigned jn = atomicAdd(e_counter, 1u);
                const int jb = (long long)jn < a.total_e ? (int)jn : -1;
                jobs[sl] = jb;
                if constexpr (PAIR) {  // the odd CTA takes the same job
                    st_remote_u32(cluster_addr(&jobs[sl], 1), (uint32_t)jb);
                    mbar_arrive_remote(cluster_addr(&job_full[sl], 1));
                }
                mbar_arrive(&job_full[sl]);
                return jb;
            };
            int t_global = 0, issued = 0;
            int next = rank == 0 ? publish(0) : 0;
            const int fetch_at = total_stages > 1 ? 1 : 0;
            for (int q = 0;; q++) {
                const int slot = q % JQ;
                int job;
                if (rank == 0) {
                    job = next;
                    if (job == -2) break;
                } else {
                    if (!mbar_wait<true>(&job_full[slot], (q / JQ) & 1, abort, err)) break;
                    job = jobs[slot];
                    mbar_arrive_remote(cluster_addr(&job_empty[slot], 0));
                }
                if (job < 0) break;
                const Job J = decode_e(a, job);
                const int gt = PAIR ? 2 * J.gt + (int)rank : J.gt;  // this CTA's gate tile
                const int bcol = J.sub % bpp;
                // first window unit of this CTA's B columns (the odd CTA of a pair holds
                // columns PB_COLS .. NB-1 of the block)
                const int P0 = s - NB - bcol * NB + (PAIR ? PB_COLS * (int)rank : 0);
                if (gt < a.tiles && !wait_count(&done_D[gt], (uint32_t)(DPARTS * (J.i + 1)), abort, err))
                    break;
                if (rank == 0) job_passes[slot] = passes_for<PAIR>(a, J, done_D, two_pass);
                asm volatile("fence.proxy.async.global;" ::: "memory");
                bool ok = true;
                for (int ts = 0; ts < total_stages; ts++, t_global++) {
                    const int st = t_global % STAGES;
                    if (rank == 0 && ts == fetch_at) next = publish(q + 1);
                    if (t_global >= STAGES &&
                        !mbar_wait(&empty[st], ((t_global / STAGES) - 1) & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    const int r = ts / kstages, ks = ts % kstages;
                    const size_t blk = (((size_t)gt * 2 * l + r) * kstages + ks) * a.nterms + J.j;
                    size_t a_src = blk * (A_STAGE_BYTES / 16);
                    if (!tfhe_in_bounds(a_src + A_STAGE_BYTES / 16 - 1, a.digits_units, a.err)) a_src = 0;
                    mbar_arrive_tx(&full[st], A_STAGE_BYTES + BST);
                    bulk_g2s(a_st + st * A_STAGE_BYTES, a.digits + a_src, A_STAGE_BYTES, &full[st]);
                    const size_t poly = ((size_t)(a.cmux ? gt / a.tpg : J.i) * 2 * l + r) * 2 + J.c;
                    size_t w_src = ((poly * a.nterms + J.j) * PLANES) * 2 * s + (P0 + ks * KS);
                    if (!tfhe_in_bounds(w_src + (size_t)(PLANES - 1) * 2 * s + BPL / 16 - 1, a.win_units, a.err))
                        w_src = 0;
                    const uint4 *wsrc = a.win + w_src;
#pragma unroll
                    for (int p = 0; p < PLANES; p++)
                        bulk_g2s(b_st + st * BST + p * BPL, wsrc + (size_t)p * 2 * s, BPL, &full[st]);
                    issued = t_global + 1;
                }
                if (!ok) break;
            }
            for (int t = issued - STAGES; t < issued; t++)
                if (t >= 0) mbar_wait_settle(&full[t % STAGES], (t / STAGES) & 1);
        }
    } else if (warp == MMA_WARP) {
        if (lane == 0 && rank == 0) {
            // ---- MMA issue (pair form: M = 256 over both CTAs' stages) ----
            constexpr uint32_t idesc = make_idesc(PAIR ? 2 * TILE_M : TILE_M, NB);
            int t_global = 0, khalf = 0;
            bool ok = true;
            for (int q = 0; ok; q++) {
                const int slot = q % JQ;
                if (!mbar_wait(&job_full[slot], (q / JQ) & 1, abort, err)) break;
                const int job = jobs[slot];
                if (job < 0) {
                    mbar_arrive(&job_empty[slot]);
                    break;
                }
                int pass_stages = total_stages;  // stages per TMEM pass, decided per job
                for (int ts = 0; ts < total_stages && ok; ts++, t_global++) {
                    const int st = t_global % STAGES;
                    if (!mbar_wait(&full[st], (t_global / STAGES) & 1, abort, err) ||
                        (PAIR && !mbar_wait<true>(&pfull[st], (t_global / STAGES) & 1, abort, err))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (ts == 0) {
                        if (job_passes[slot] == 2) pass_stages = half_stages;
                        if constexpr (!PAIR) {
                            ro_passes[slot] = job_passes[slot];
                            mbar_arrive(&passes_ready[slot]);
                        }
                        mbar_arrive(&job_empty[slot]);  // the slot is read
                    }
                    // descriptors of the stage; K-steps and planes add their byte offset / 16
                    // to the start-address field (shared addresses < 256 KB: no carry)
                    const uint64_t a_desc = make_desc(smem_u32(a_st + st * A_STAGE_BYTES), 128, 2048);
                    const uint64_t b_desc = make_desc(smem_u32(b_st + st * BST), 128, 128);
                    const bool first = ts % pass_stages == 0, last = (ts + 1) % pass_stages == 0;
                    if (first || last) {
                        // first and last stage of a pass go plane by plane: in the first,
                        // plane p starts once its previous contents have been read out; in the
                        // last, plane p is committed on its own (acc_full[p]), so its read-out
                        // (and the next job's MMAs on it) overlap the later planes' MMAs
#pragma unroll
                        for (int p = 0; p < PLANES; p++) {
                            if (first && khalf > 0 &&
                                !mbar_wait<PAIR>(&acc_empty[p], (khalf - 1) & 1, abort, err)) {
                                ok = false;
                                break;
                            }
                            if (first) tc_fence_after();
#pragma unroll
                            for (int kk = 0; kk < KS / 16; kk++) {
                                const uint64_t ad = a_desc + (uint64_t)(kk * 256 / 16);
                                const uint64_t bd = b_desc + (uint64_t)((p * BPL + kk * 256) / 16);
                                const uint32_t accum = (first && kk == 0) ? 0u : 1u;
                                if constexpr (PAIR)
                                    mma_f16_pair(tmem + p * NB, ad, bd, idesc, accum);
                                else
                                    mma_f16(tmem + p * NB, ad, bd, idesc, accum);
                            }
                            if (last) {
                                if constexpr (PAIR) mma_commit_pair_both(&acc_full[p]);
                                else mma_commit(&acc_full[p]);
                            }
                        }
                        if (!ok) break;
                    } else {
#pragma unroll
                        for (int kk = 0; kk < KS / 16; kk++) {
                            const uint64_t ad = a_desc + (uint64_t)(kk * 256 / 16);
                            if constexpr (PAIR) {
#pragma unroll
                                for (int p = 0; p < PLANES; p++) {
                                    const uint64_t bd = b_desc + (uint64_t)((p * BPL + kk * 256) / 16);
                                    mma_f16_pair(tmem + p * NB, ad, bd, idesc, 1u);
                                }
                            } else {
                                static_assert(PLANES == 4, "collector sequence assumes 4 planes");
                                const uint64_t bd = b_desc + (uint64_t)(kk * 256 / 16);
                                mma_f16_coll<0>(tmem, ad, bd, idesc);
                                mma_f16_coll<1>(tmem + NB, ad, bd + BPL / 16, idesc);
                                mma_f16_coll<1>(tmem + 2 * NB, ad, bd + 2 * BPL / 16, idesc);
                                mma_f16_coll<2>(tmem + 3 * NB, ad, bd + 3 * BPL / 16, idesc);
                            }
                        }
                    }
                    if constexpr (PAIR) mma_commit_pair_both(&empty[st]);
                    else mma_commit(&empty[st]);
                    if (last) khalf++;
                }
            }
            if constexpr (PAIR) mma_commit_pair_own(&drain);
            else mma_commit(&drain);
            mbar_wait_settle(&drain, 0);
        } else if (PAIR && lane == 0) {
            // ---- odd CTA of a pair: tell the MMA issuer when each of its stages is full ----
            int t_global = 0;
            bool ok = true;
            for (int q = 0; ok; q++) {
                const int slot = q % JQ;
                if (!mbar_wait<true>(&job_full[slot], (q / JQ) & 1, abort, err)) break;
                const int job = jobs[slot];
                mbar_arrive_remote(cluster_addr(&job_empty[slot], 0));
                if (job < 0) break;
                for (int ts = 0; ts < total_stages; ts++, t_global++) {
                    const int st = t_global % STAGES;
                    if (!mbar_wait(&full[st], (t_global / STAGES) & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_remote(cluster_addr(&pfull[st], 0));
                }
            }
        }
    } else if (warp < EPI_WARPS) {
        // ---- TMEM read-out: thread = TMEM lane = gate of the tile; this warp's 64 columns
        const int tid = threadIdx.x;
        __shared__ int epi_passes;
        const int lane_q = warp & 3, colh = warp >> 2;
        const uint32_t lane_base = tmem + (((uint32_t)(lane_q * 32)) << 16) + colh * EPI_COLS;
        const int gl = lane_q * 32 + lane;  // gate within the tile
        int khalf = 0;
        for (int q = 0;; q++) {
            const int slot = q % JQ;
            if (!mbar_wait_warp<PAIR>(&job_full[slot], (q / JQ) & 1, abort, err)) break;
            const int job = jobs[slot];
            auto release_slot = [&]() {  // every read-out thread has read the slot
                if (tid == 0) {
                    if (rank == 0) mbar_arrive(&job_empty[slot]);
                    else mbar_arrive_remote(cluster_addr(&job_empty[slot], 0));
                }
            };
            if constexpr (PAIR) {
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
                release_slot();
            }
            if (job < 0) {
                if constexpr (!PAIR) release_slot();
                break;
            }
            const Job J = decode_e(a, job);
            const int gt = PAIR ? 2 * J.gt + (int)rank : J.gt;  // this CTA's gate tile
            const int bcol = J.sub % bpp;
            int passes;
            if constexpr (PAIR) {
                if (tid == 0) epi_passes = passes_for<PAIR>(a, J, done_D, two_pass);
                asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
                passes = epi_passes;
            } else {
                // The leader's acquire orders this job's additions into ACC after the digit
                // jobs of its step (the readers of ACC(i)); taken now, it overlaps the
                // read-out of the planes (the barrier before the additions publishes it).
                if (tid == 0 && gt < a.tiles) wait_count(&done_D[gt], (uint32_t)(DPARTS * (J.i + 1)), abort, err);
                if (!mbar_wait_warp<false>(&passes_ready[slot], (q / JQ) & 1, abort, err)) break;
                passes = ro_passes[slot];
            }
            uint32_t sum[EPI_COLS];
            const uint32_t sum_init = 0u - (uint32_t)passes * RO_MAGIC_PER_PASS;
#pragma unroll
            for (int e = 0; e < EPI_COLS; e++) sum[e] = sum_init;
            bool ok = true;
            for (int h = 0; h < passes && ok; h++, khalf++) {
#pragma unroll
                for (int p = 0; p < PLANES; p++) {
                    // plane p of this pass is complete once its own commit has arrived
                    if (!mbar_wait_warp<PAIR>(&acc_full[p], khalf & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // exact fp32 -> int: for |x| < 2^22 the sum x + 1.5*2^23 is exact and its
                    // bit pattern is RO_MAGIC_BITS + x; the constant is removed once through
                    // the initial value of sum.  A slice holding a larger |x| (possible, never
                    // typical) takes the rounding conversion instead, so the result stays
                    // exact either way.  Slices of RO_COLS columns bound the live registers.
#pragma unroll
                    for (int c0 = 0; c0 < EPI_COLS; c0 += RO_COLS) {
                        uint32_t v[RO_COLS];
#pragma unroll
                        for (int jc = 0; jc < RO_COLS / 16; jc++)
                            tmem_ld16(lane_base + p * NB + c0 + jc * 16, v + jc * 16);
                        tmem_wait_ld();
                        float m = 0.f;
#pragma unroll
                        for (int e = 0; e < RO_COLS; e++) m = fmaxf(m, fabsf(__uint_as_float(v[e])));
                        if (m < RO_FAST_LIMIT) {
#pragma unroll
                            for (int e = 0; e < RO_COLS; e++)
                                sum[c0 + e] += __float_as_uint(__uint_as_float(v[e]) + RO_MAGIC) << (8 * p);
                        } else {
#pragma unroll
                            for (int e = 0; e < RO_COLS; e++)
                                sum[c0 + e] +=
                                    ((uint32_t)__float2int_rn(__uint_as_float(v[e])) + RO_MAGIC_BITS) << (8 * p);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        if (rank == 0) mbar_arrive(&acc_empty[p]);
                        else mbar_arrive_remote(cluster_addr(&acc_empty[p], 0));
                    }
                }
            }
            if (!ok) break;
            // accumulator update: column idx of the block is word n' = c0 - idx of P_j,
            // added with sign out_tab[j][b] into output block b.  The leader's acquire
            // orders these additions after this step's digit jobs of the tile (the
            // readers of ACC(i)).
            if (PAIR && tid == 0 && gt < a.tiles)
                wait_count(&done_D[gt], (uint32_t)(DPARTS * (J.i + 1)), abort, err);
            asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
            if constexpr (!PAIR) release_slot();
            if (*abort) break;
            if (gt * TILE_M + gl < a.G) {
                // this warp's columns idx = 64 colh + e map to words c0 - idx, i.e. the
                // 64 words starting at bcol*NB + 64 (1 - colh), in reverse order; in the
                // tiled accumulator each word of the warp's 32 gates is one 128-byte line
                const int w0 = bcol * NB + EPI_COLS * (1 - colh);
#pragma unroll 1
                for (int b = 0; b < NBLK; b++) {
                    const int sg = out_tab[J.j][b];
                    if (!sg) continue;
                    const size_t col0 = ((size_t)(gt * 2 + J.c) * N + (size_t)b * s + w0) * TILE_M + gl;
                    uint32_t *col = a.acc + col0;
                    if (sg > 0) {
#pragma unroll
                        for (int q = 0; q < EPI_COLS; q++)
                            if (tfhe_in_bounds(col0 + (size_t)q * TILE_M, a.acc_words, a.err))
                                red_add_u32(col + (size_t)q * TILE_M, sum[EPI_COLS - 1 - q]);
                    } else {
#pragma unroll
                        for (int q = 0; q < EPI_COLS; q++)
                            if (tfhe_in_bounds(col0 + (size_t)q * TILE_M, a.acc_words, a.err))
                                red_add_u32(col + (size_t)q * TILE_M, 0u - sum[EPI_COLS - 1 - q]);
                    }
                }
            }
            // publish: the barrier orders every read-out thread's stores before the
            // leader's release (cumulative), so one fenced increment suffices
            asm volatile("bar.sync 1, %0;" ::"n"(EPI_THREADS) : "memory");
            if (tid == 0 && gt < a.tiles) red_release_add(&done_E[gt], 1u);
        }
    } else {
        // ---- warps 9-11 and 13-15: digit jobs ----
        const int tid = digit_warp_index(warp) * 32 + lane;
        const uint32_t off = gadget_offset(l, a.Bgbit);
        // One-pass check (see ONE_PASS_LIMIT): sum |x| over a term's K is bounded by the
        // sum, over the term's input blocks, of sum |digit| per block (triangle
        // inequality), so the digit jobs keep one counter per block.  Levels 0-2 hold a
        // thread's rotated differences over the l digits; level 3 recomputes them per digit
        // (registers).
        constexpr bool HOLD = NBLK <= 4;
        const int Bgbit = a.Bgbit;
        const uint32_t fmask = ((1u << Bgbit) - 1u) * 0x10001u;
        const uint32_t dsub = f16_bits(1536 + (1 << (Bgbit - 1))) * 0x10001u;
        const uint64_t pol = l2_evict_last_policy();
        __shared__ int d_job;
        __shared__ int d_abs[8 * NBLK];  // per gate of the part and input block
        for (;;) {
            if (tid == 0) {
                const unsigned jn = atomicAdd(d_counter, 1u);
                d_job = (long long)jn < a.total_d ? (int)jn : -1;
            }
            dg_sync();
            const int job = d_job;
            dg_sync();
            if (job < 0 || *abort) break;
            int i, gt, mg;
            {
                // chunks of the digit stream follow those of the product stream (the pair
                // form runs one chunk: all tiles)
                int t0, tiles_c;
                long long rem;
                chunk_of(job, a.tiles, PAIR ? 1 : a.nchunks, (long long)a.n * DPARTS, &t0, &tiles_c, &rem);
                i = (int)(rem / (tiles_c * DPARTS));
                const int r = (int)(rem % (tiles_c * DPARTS));
                const int paired = PAIR ? (a.tiles / 2) * 2 * DPARTS : 0;
                if (r < paired) {  // pair form: the two tiles of a pair alternate parts
                    gt = 2 * (r / (2 * DPARTS)) + (r & 1);
                    mg = (r % (2 * DPARTS)) >> 1;
                } else {
                    gt = t0 + (paired / DPARTS) + (r - paired) / DPARTS;
                    mg = (r - paired) % DPARTS;
                }
            }
            if (tid == 0) wait_count(&done_E[gt], (uint32_t)(a.e_per_tile * i), abort, err);
            dg_sync();
            if (*abort) break;
            if (i > 0 && !a.cmux) {
                // Every product job of the tile's step i-1 has copied its digit stages, so
                // the part's digit lines of that step are dead until this job rewrites
                // them: drop them from L2 without writing them back (2 KB per block: the
                // part's 8 gates of each 32 KB stage block, 16 lines of 128 bytes).
                const int nblk = NT * 2 * l * kstages;
                for (int q = tid; q < nblk * 16; q += DG_THREADS) {
                    const uint4 *ln = a.digits + (size_t)(gt * nblk + q / 16) * (A_STAGE_BYTES / 16) +
                                      (size_t)mg * 128 + (q % 16) * 8;
#ifdef TFHE_BOUNDS_CHECK
                    if (!tfhe_in_bounds((size_t)(ln - a.digits) + 7, a.digits_units, a.err)) continue;
#endif
                    asm volatile("discard.global.L2 [%0], 128;" ::"l"(ln) : "memory");
                }
            }
            // One accumulator polynomial of the part's 8 gates at a time: the rows are copied
            // into shared memory, then each work unit (stage kc, position group kb, gate
            // m8 = tid & 7) digitises positions kp = kc*KS + 8 kb .. + 7 of every size-s
            // block of gate m8, so 8 consecutive threads write 128 contiguous bytes of the
            // A-operand layout (stage kc, row r, term j).  X^{a} p at k is p[k - a] (sign by
            // wrap).  Row pitch N + 12: room for the negated first 8 words, and 8 rows on
            // distinct bank quads.
            const int pitch = N + 12;
            __shared__ uint32_t bbar_s[8];  // b~ of the part's gates (step 0)
            // ModSwitched coefficient k of gate g's combination (fused form; 0 for a bad
            // gate type or index)
            auto ms_coef = [&](int64_t g, int k) -> uint32_t {
                if (!gate_ok(a.types, a.idx, a.num_in, g)) return 0u;
                uint32_t kappa, s1, s2;
                gate_coeffs(a.types[g], kappa, s1, s2);
                uint32_t x = s1 * __ldg(a.in + (int64_t)a.idx[2 * g] * a.n1 + k) +
                             s2 * __ldg(a.in + (int64_t)a.idx[2 * g + 1] * a.n1 + k);
                if (k == a.n1 - 1) x += kappa;
                return (x + (1u << (a.ms_shift - 1))) >> a.ms_shift;
            };
            if (i == 0 && !a.cmux) {
                // step 0: the part's ModSwitched combinations (fused form) and b~
                const int n1 = a.n1;
                if (a.in) {
                    for (int e = tid; e < 8 * n1; e += DG_THREADS) {
                        const int m = e / n1, k = e - m * n1;
                        const int64_t g = (int64_t)gt * TILE_M + mg * 8 + m;
                        if (g >= a.G) continue;
                        if (k == 0 && !gate_ok(a.types, a.idx, a.num_in, g)) atomicCAS(err, 0, TFHE_EINVAL);
                        if (tfhe_in_bounds((size_t)g * n1 + k, a.bar_words, a.err)) a.bar_w[g * n1 + k] = ms_coef(g, k);
                    }
                    dg_sync();
                }
                if (tid < 8) {
                    const int g = gt * TILE_M + mg * 8 + tid;
                    bbar_s[tid] = g < a.G && tfhe_in_bounds((size_t)g * n1 + n1 - 1, a.bar_words, a.err)
                                      ? __ldcg(a.bar + (size_t)g * n1 + n1 - 1) % (uint32_t)(2 * N) : 0u;
                }
                dg_sync();
            }
            // the thread's gate: every work unit of the thread has gate m8 (DG_THREADS and
            // the unit strides are multiples of 8); a' written at step 0 of this launch when
            // fused: coherent load
            const int m8 = tid & 7;
            const int g8 = gt * TILE_M + mg * 8 + m8;
            const int rot = g8 < a.G && !a.cmux && tfhe_in_bounds((size_t)g8 * a.n1 + i, a.bar_words, a.err)
                                ? (int)(__ldcg(a.bar + (size_t)g8 * a.n1 + i) % (uint32_t)(2 * N)) : 0;
            for (int v = tid; v < 8 * NBLK; v += DG_THREADS) d_abs[v] = 0;
            int asum[NBLK];
#pragma unroll
            for (int b = 0; b < NBLK; b++) asum[b] = 0;
            const int rk = rot >= N ? rot - N : rot;      // X^rot = (-1)^{rot >= N} X^rk
            const uint32_t rneg = rot >= N ? 0xFFFFFFFFu : 0u;
            const uint32_t *row = d_rows + m8 * pitch;
            for (int c = 0; c < 2; c++) {
                dg_sync();  // previous polynomial consumed
                {
                    // item (k, h): word k for gates 4h .. 4h+3 of the part, 16 bytes of the
                    // tiled accumulator; the rows of two gate halves land on disjoint banks.
                    // Words 0..7 are also written negated after the row's N words.
                    // Step 0 writes ACC(0) instead of reading it.
                    uint32_t *accp = a.acc + (size_t)(gt * 2 + c) * N * TILE_M + mg * 8;
                    const size_t acc0 = (size_t)(gt * 2 + c) * N * TILE_M + mg * 8;
                    auto acc_ok = [&](int k, int h) {
                        return tfhe_in_bounds(acc0 + (size_t)k * TILE_M + 4 * h + 3, a.acc_words, a.err);
                    };
                    auto put = [&](int it, const uint4 &o) {
                        const int k = it >> 1, h = it & 1;
                        uint32_t *rr = d_rows + 4 * h * pitch + k;
                        rr[0] = o.x;
                        rr[pitch] = o.y;
                        rr[2 * pitch] = o.z;
                        rr[3 * pitch] = o.w;
                        if (k < 8) {
                            rr[N] = 0u - o.x;
                            rr[pitch + N] = 0u - o.y;
                            rr[2 * pitch + N] = 0u - o.z;
                            rr[3 * pitch + N] = 0u - o.w;
                        }
                    };
                    if (a.cmux || i == 0) {
#pragma unroll 4
                        for (int it = tid; it < 2 * N; it += DG_THREADS) {
                            const int k = it >> 1, h = it & 1;
                            uint4 o;
                            if (a.cmux) {
                                // ACC(0) = d0; the shared rows take d1 - d0
                                uint32_t v0[4], v1[4];
#pragma unroll
                                for (int q = 0; q < 4; q++) {
                                    const int x = (gt % a.tpg) * TILE_M + mg * 8 + 4 * h + q, y = gt / a.tpg;
                                    const bool ok = x < a.cm_nx && (int64_t)y * a.cm_nx + x < a.cm_count;
                                    const int64_t o_ = (int64_t)x * a.cm_dx + (int64_t)y * a.cm_dy + (int64_t)c * N + k;
                                    v0[q] = ok ? __ldg(a.cm_d0 + o_) : 0u;
                                    v1[q] = ok ? __ldg(a.cm_d1 + o_) - v0[q] : 0u;
                                }
                                if (acc_ok(k, h))
                                    __stcg((uint4 *)(accp + (size_t)k * TILE_M) + h, make_uint4(v0[0], v0[1], v0[2], v0[3]));
                                o = make_uint4(v1[0], v1[1], v1[2], v1[3]);
                            } else {
                                uint32_t v[4] = {0u, 0u, 0u, 0u};
                                if (c == 1) {
#pragma unroll
                                    for (int q = 0; q < 4; q++) {
                                        const int g = gt * TILE_M + mg * 8 + 4 * h + q;
                                        const uint32_t mu = 1u << 29;
                                        if (g < a.G) v[q] = ((uint32_t)k + bbar_s[4 * h + q]) % (uint32_t)(2 * N) < (uint32_t)N ? mu : 0u - mu;
                                    }
                                }
                                o = make_uint4(v[0], v[1], v[2], v[3]);
                                if (acc_ok(k, h)) __stcg((uint4 *)(accp + (size_t)k * TILE_M) + h, o);
                            }
                            put(it, o);
                        }
                    } else {
                        // 8 loads in flight per thread before their shared-memory stores
                        for (int it0 = tid; it0 < 2 * N; it0 += 8 * DG_THREADS) {
                            uint4 ov[8];
#pragma unroll
                            for (int q = 0; q < 8; q++) {
                                const int it = it0 + q * DG_THREADS;
                                if (it < 2 * N)
                                    ov[q] = acc_ok(it >> 1, it & 1)
                                                ? __ldcg((const uint4 *)(accp + (size_t)(it >> 1) * TILE_M) + (it & 1))
                                                : make_uint4(0u, 0u, 0u, 0u);
                            }
#pragma unroll
                            for (int q = 0; q < 8; q++)
                                if (it0 + q * DG_THREADS < 2 * N) put(it0 + q * DG_THREADS, ov[q]);
                        }
                    }
                }
                dg_sync();
                // Work units: spans (stage kc, position group kb, gate m8) of 8 positions with
                // all l digits (levels 0-2: the rotated differences are computed once per span),
                // or one digit of a span (level 3: registers).  Consecutive threads take
                // consecutive gates of a span group: 8 threads write 128 contiguous bytes.
                const int spans = 128 * kstages;
                const int units = HOLD ? spans : spans * l;
                const size_t jd_stride = (size_t)kstages * NT * (A_STAGE_BYTES / 16);
                // packed sums of |digit| per block, folded into asum every 3 digits (each half
                // then holds at most 3 * 4 * Bg/2 <= 384: exact, and below 512)
                uint32_t ah[NBLK];
#pragma unroll
                for (int b = 0; b < NBLK; b++) ah[b] = 0u;
                int nacc = 0;
                for (int v = tid; v < units; v += DG_THREADS) {
                    const int sp = v % spans;
                    const int jd0 = HOLD ? 0 : v / spans, jd1 = HOLD ? l : jd0 + 1;
                    const int kc = sp >> 7, kb = (sp >> 3) & 15;
                    const int kp = kc * KS + kb * 8;
                    // the unit's 16 bytes in the block of term 0, row c*l + jd, stage kc: the
                    // blocks of a tile are ordered [2l rows][stages][terms]
                    uint4 *dst0 = a.digits + (((size_t)gt * 2 * l + c * l) * kstages + kc) * NT * (A_STAGE_BYTES / 16) +
                                  ((size_t)mg * 16 + kb) * 8 + m8;
                    uint32_t uh[HOLD ? NBLK : 1][8];
                    if constexpr (HOLD) {
#pragma unroll
                        for (int b = 0; b < NBLK; b++) rotated_diff8(row, N, b * s + kp, rk, rneg, off, a.cmux, uh[b]);
                    }
                    for (int jd = jd0; jd < jd1; jd++) {
                        const int sh = 32 - (jd + 1) * Bgbit;
                        uint32_t dg[NBLK][DW];
#pragma unroll
                        for (int b = 0; b < NBLK; b++) {
                            uint32_t u[8];
                            if constexpr (HOLD) {
#pragma unroll
                                for (int e = 0; e < 8; e++) u[e] = uh[b][e];
                            } else {
                                rotated_diff8(row, N, b * s + kp, rk, rneg, off, a.cmux, u);
                            }
#pragma unroll
                            for (int w = 0; w < DW; w++) {
                                dg[b][w] = digit_pair(u[2 * w], u[2 * w + 1], sh, fmask, dsub);
                                ah[b] = hadd2(ah[b], habs2(dg[b][w]));
                            }
                        }
                        uint4 *dst = dst0 + (size_t)jd * jd_stride;
#ifdef TFHE_BOUNDS_CHECK
                        const size_t used = (size_t)(dst - a.digits);
                        DigitStore emit{dst, pol, used < a.digits_units ? a.digits_units - used : 0, a.err};
#else
                        DigitStore emit{dst, pol};
#endif
                        kara_terms<NBLK>(dg, emit);
                        if (++nacc == 3) {
#pragma unroll
                            for (int b = 0; b < NBLK; b++) {
                                asum[b] += fold_f16_sums(ah[b]);
                                ah[b] = 0u;
                            }
                            nacc = 0;
                        }
                    }
                }
                if (nacc > 0) {
#pragma unroll
                    for (int b = 0; b < NBLK; b++) asum[b] += fold_f16_sums(ah[b]);
                }
            }
            // one-pass check: reduce the block sums over the threads of each gate, then mark
            // the step if some gate exceeds the bound for some term (read by the product
            // jobs)
#pragma unroll
            for (int b = 0; b < NBLK; b++) {
                int v = asum[b];
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
                if (lane < 8) atomicAdd(&d_abs[lane * NBLK + b], v);
            }
            dg_sync();
            for (int t = tid; t < 8 * NT; t += DG_THREADS) {
                const int gq = t / NT, jt = t % NT;
                int v = 0;
#pragma unroll
                for (int j = 0; j < NT; j++) {  // compile-time coefficients, selected by jt
                    if (j != jt) continue;
#pragma unroll
                    for (int b = 0; b < NBLK; b++)
                        if (in_coef_tab(L, j, b) != 0) v += d_abs[gq * NBLK + b];
                }
                if (v > a.one_pass_limit) atomicMax(&two_pass[gt], (uint32_t)(i + 1));
            }
            dg_sync();
            if (tid == 0) red_release_add(&done_D[gt], 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    // pair form: neither CTA leaves while the other may still touch its shared memory
    // or TMEM (the even CTA has drained its MMAs before reaching this point)
    if constexpr (PAIR) cluster_sync_all();
    if (warp == MMA_WARP) {
        tc_fence_after();
        if constexpr (PAIR)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

// Terms of the L-level split (see the top of this file), in a deterministic order.
static void build_plan(int N, int L, std::vector<KTerm> &terms) {
    terms.clear();
    auto mk = [](int nin, const int *ib, const int *is, int nout, const int *ob, const int *os,
                 int nk, const int *ko, const int *kc) {
        KTerm t{};
        t.n_in = nin;
        t.n_out = nout;
        t.n_key = nk;
        for (int m = 0; m < nin; m++) { t.in_blk[m] = ib[m]; t.in_sgn[m] = is[m]; }
        for (int m = 0; m < nout; m++) { t.out_blk[m] = ob[m]; t.out_sgn[m] = os[m]; }
        for (int m = 0; m < nk; m++) { t.key_off[m] = ko[m]; t.key_coef[m] = kc[m]; }
        return t;
    };
    if (L == 0) {
        const int b0[1] = {0}, p1[1] = {1}, k0[1] = {0};
        terms.push_back(mk(1, b0, p1, 1, b0, p1, 1, k0, p1));
    }
    // level 1: negacyclic split, s = N/2.  A: t[d], B: t[d + s].
    const int s1 = N / 2;
    if (L >= 1) {
        const int in1[1] = {0}, in1s[1] = {1};
        const int out1[2] = {0, 1}, out1s[2] = {1, 1};
        const int k1[2] = {0, s1}, k1c[2] = {1, 1};
        terms.push_back(mk(1, in1, in1s, 2, out1, out1s, 2, k1, k1c));          // P1 = (A+B) x0
        const int in2[2] = {1, 0}, in2s[2] = {1, -1};
        const int out2[1] = {1}, out2s[1] = {1};
        const int k2[1] = {0}, k2c[1] = {1};
        terms.push_back(mk(2, in2, in2s, 1, out2, out2s, 1, k2, k2c));          // P2 = A (x1 - x0)
        const int in3[2] = {0, 1}, in3s[2] = {1, 1};
        const int out3[1] = {0}, out3s[1] = {-1};
        const int k3[1] = {s1}, k3c[1] = {1};
        terms.push_back(mk(2, in3, in3s, 1, out3, out3s, 1, k3, k3c));          // P3 = B (x0 + x1)
    }
    for (int lev = 2; lev <= L; lev++) {
        const int h = N >> lev;  // new block size
        std::vector<KTerm> next;
        for (const KTerm &P : terms) {
            KTerm a{}, q0{}, q1{};
            // inputs: x0 = first halves (2b), x1 = second halves (2b+1)
            for (int m = 0; m < P.n_in; m++) {
                a.in_blk[a.n_in] = 2 * P.in_blk[m]; a.in_sgn[a.n_in++] = P.in_sgn[m];
                a.in_blk[a.n_in] = 2 * P.in_blk[m] + 1; a.in_sgn[a.n_in++] = P.in_sgn[m];
                q0.in_blk[q0.n_in] = 2 * P.in_blk[m] + 1; q0.in_sgn[q0.n_in++] = P.in_sgn[m];
                q1.in_blk[q1.n_in] = 2 * P.in_blk[m]; q1.in_sgn[q1.n_in++] = P.in_sgn[m];
            }
            // outputs: y0 = P + Q0 (blocks 2b), y1 = P + Q1 (blocks 2b+1)
            for (int m = 0; m < P.n_out; m++) {
                a.out_blk[a.n_out] = 2 * P.out_blk[m]; a.out_sgn[a.n_out++] = P.out_sgn[m];
                a.out_blk[a.n_out] = 2 * P.out_blk[m] + 1; a.out_sgn[a.n_out++] = P.out_sgn[m];
                q0.out_blk[q0.n_out] = 2 * P.out_blk[m]; q0.out_sgn[q0.n_out++] = P.out_sgn[m];
                q1.out_blk[q1.n_out] = 2 * P.out_blk[m] + 1; q1.out_sgn[q1.n_out++] = P.out_sgn[m];
            }
            // keys: T00 = t[d], T01 = t[d - h], T10 = t[d + h]
            for (int m = 0; m < P.n_key; m++) {
                a.key_off[a.n_key] = P.key_off[m]; a.key_coef[a.n_key++] = P.key_coef[m];
                q0.key_off[q0.n_key] = P.key_off[m] - h; q0.key_coef[q0.n_key++] = P.key_coef[m];
                q1.key_off[q1.n_key] = P.key_off[m] + h; q1.key_coef[q1.n_key++] = P.key_coef[m];
            }
            for (int m = 0; m < P.n_key; m++) {
                q0.key_off[q0.n_key] = P.key_off[m]; q0.key_coef[q0.n_key++] = -P.key_coef[m];
                q1.key_off[q1.n_key] = P.key_off[m]; q1.key_coef[q1.n_key++] = -P.key_coef[m];
            }
            next.push_back(a);
            next.push_back(q0);
            next.push_back(q1);
        }
        terms.swap(next);
    }
    for (KTerm &t : terms) {
        for (int b = 0; b < MAX_BLK; b++) t.in_coef[b] = t.out_coef[b] = 0;
        for (int m = 0; m < t.n_in; m++) t.in_coef[t.in_blk[m]] += t.in_sgn[m];
        for (int m = 0; m < t.n_out; m++) t.out_coef[t.out_blk[m]] += t.out_sgn[m];
    }
    // the kernels' compile-time tables must agree (a term enters each output block once)
    for (size_t j = 0; j < terms.size(); j++)
        for (int b = 0; b < MAX_BLK; b++) {
            const bool in_range = b < (1 << L);
            if (terms[j].in_coef[b] != (in_range ? in_coef_tab(L, (int)j, b) : 0) ||
                terms[j].out_coef[b] != (in_range ? out_coef_tab(L, (int)j, b) : 0)) {
                terms.clear();
                return;
            }
        }
}

struct TcWorkspace {
    // per Karatsuba level: term plan and key windows (several levels can be resident, so
    // a plan can run each batch width at the level that suits it)
    struct Level {
        std::vector<KTerm> terms;
        KTerm *d_terms = nullptr;
        uint4 *win = nullptr;      // window units for every step
        size_t win_cap = 0;        // bytes
        bool ready = false;        // windows expanded for the current keys
    };
    Level lv[4];
    uint4 *digits = nullptr;
    size_t digits_cap = 0;     // bytes
    uint32_t *sync = nullptr;  // job counter and per-tile progress counters
    size_t sync_cap = 0;       // words
    uint32_t *acc_t = nullptr; // accumulators, gate-fastest within 128-gate tiles
    size_t acc_t_cap = 0;      // bytes
    uint4 *cm_win = nullptr;   // windows of the CMUX selectors of one call
    size_t cm_win_cap = 0;     // bytes
    struct JobTable {
        uint32_t *d = nullptr;  // per-step product-job table
        int len = 0;            // entries
    };
    std::map<int, JobTable> tables;  // by (level, pair form, gate tiles); kept: captured
                                     // graphs use them
    int sms = 0;
    int max_pairs[4] = {-1, -1, -1, -1};  // co-resident SM pairs of the pair kernel, per level
    int want_level = -1;       // requested Karatsuba levels (-1: default)
    int want_variant = -1;     // TFHE_TC_SINGLE_SM, TFHE_TC_SM_PAIR, -1: default
    int one_pass_limit = ONE_PASS_LIMIT;
};

int tfhe_tc_supported(const tfhe_ctx *ctx) {
    const tfhe_params &p = ctx->p;
    return p.N >= 256 && p.N <= 1024 && p.N % NB == 0 && p.N % KS == 0 && p.Bgbit <= 6 &&
           (int64_t)p.l * p.N * 32 * 128 <= (1 << 24);
}

// Measured on B300 at N = 1024 (4096-gate level): level 2 fastest; smaller N keeps
// blocks of at least 256 columns.
static int default_level(const tfhe_params &p) { return p.N >= 1024 ? 2 : (p.N >= 512 ? 1 : 0); }

// One SM per tile unless the pair form was asked for (measured slower on B300: the
// coupled SMs wait for each other more than the halved key staging saves).
static bool use_pair(tfhe_ctx *ctx) {
    return ctx->tc && ctx->tc->want_variant == TFHE_TC_SM_PAIR;
}

static bool level_ok(const tfhe_params &p, int L) {
    if (L < 0 || L > 3) return false;
    const int s = p.N >> L;
    return s >= NB && s % NB == 0 && s % KS == 0;
}

void tfhe_tc_free(tfhe_ctx *ctx) {
    if (!ctx->tc) return;
    TcWorkspace *w = ctx->tc;
    for (auto &L : w->lv) {
        if (L.d_terms) cudaFree(L.d_terms);
        if (L.win) cudaFree(L.win);
    }
    if (w->digits) cudaFree(w->digits);
    if (w->sync) cudaFree(w->sync);
    if (w->acc_t) cudaFree(w->acc_t);
    if (w->cm_win) cudaFree(w->cm_win);
    for (auto &t : w->tables) cudaFree(t.second.d);
    delete w;
    ctx->tc = nullptr;
}

static int grow_dev(tfhe_ctx *ctx, void **ptr, size_t *cap, size_t need, const char *what) {
    return tfhe_grow(ctx, ptr, cap, need, what);
}

// The term plan of `level` on the device (built once; the CMUX form needs it without keys).
static int ensure_plan(tfhe_ctx *ctx, int level, cudaStream_t st) {
    TcWorkspace::Level &V = ctx->tc->lv[level];
    if (!V.terms.empty() && V.d_terms) return TFHE_OK;
    if (ctx->capturing)
        return tfhe_set_error(ctx, TFHE_EINVAL, "tensor-core plan: cannot build while recording");
    build_plan(ctx->p.N, level, V.terms);
    if (V.terms.empty())
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "Karatsuba plan differs from the kernels' table");
    if (!V.d_terms && cudaMalloc(&V.d_terms, sizeof(KTerm) * MAX_TERMS) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core term plan");
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(V.d_terms, V.terms.data(), sizeof(KTerm) * V.terms.size(),
                                       cudaMemcpyHostToDevice, st));
    return TFHE_OK;
}

// (Re)build the term plan of `level` and expand the windows of the whole BSK for it.
static int prepare_windows(tfhe_ctx *ctx, int level, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    TcWorkspace::Level &V = ctx->tc->lv[level];
    if (ctx->capturing)
        return tfhe_set_error(ctx, TFHE_EINVAL, "tensor-core windows: cannot rebuild while recording");
    int rc = ensure_plan(ctx, level, st);
    if (rc != TFHE_OK) return rc;
    const int T = (int)V.terms.size();
    const int s = p.N >> level;
    const size_t npoly = (size_t)p.n * 2 * p.l * 2;
    const size_t bytes = npoly * T * PLANES * 2 * (size_t)s * sizeof(uint4);
    rc = grow_dev(ctx, (void **)&V.win, &V.win_cap, bytes, "tensor-core key windows");
    if (rc != TFHE_OK) return rc;
    k_tc_windows<<<dim3((unsigned)npoly, T), 256, 0, st>>>(ctx->bsk_raw, p.N, s, T, V.d_terms,
                                                          V.win, 1, 1);
    rc = tfhe_check_launch(ctx, "tc_windows");
    if (rc != TFHE_OK) return rc;
    V.ready = true;
    return TFHE_OK;
}

static int resolve_level(tfhe_ctx *ctx, int level) {
    return level >= 0 ? level
                      : (ctx->tc && ctx->tc->want_level >= 0 ? ctx->tc->want_level : default_level(ctx->p));
}

// Windows of `level` (-1: the context's level) expanded for the loaded keys.
int tfhe_tc_ensure_level(tfhe_ctx *ctx, int level, cudaStream_t st) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    level = resolve_level(ctx, level);
    if (!level_ok(ctx->p, level))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "Karatsuba level not supported for this N");
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    if (!ctx->has_keys || ctx->tc->lv[level].ready) return TFHE_OK;
    return prepare_windows(ctx, level, st);
}

// New keys: re-expand every level in use (and the context's level).
int tfhe_tc_prepare_keys(tfhe_ctx *ctx, const uint32_t *, cudaStream_t st) {
    if (!tfhe_tc_supported(ctx)) return TFHE_OK;
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    const int L0 = resolve_level(ctx, -1);
    for (int L = 0; L < 4; L++) {
        TcWorkspace::Level &V = ctx->tc->lv[L];
        if (V.ready || L == L0) {
            V.ready = false;
            const int rc = prepare_windows(ctx, L, st);
            if (rc != TFHE_OK) return rc;
        }
    }
    return TFHE_OK;
}

// Free the key windows of levels outside `mask` (bit L = level L) except the context's
// level; they are expanded again if a later call needs them.
void tfhe_tc_keep_levels(tfhe_ctx *ctx, unsigned mask) {
    if (!ctx->tc) return;
    const int L0 = resolve_level(ctx, -1);
    for (int L = 0; L < 4; L++) {
        TcWorkspace::Level &V = ctx->tc->lv[L];
        if (L == L0 || (mask >> L) & 1 || !V.win) continue;
        cudaFree(V.win);
        V.win = nullptr;
        V.win_cap = 0;
        V.ready = false;
        ctx->mem_gen++;
    }
}

int tfhe_tc_set_level(tfhe_ctx *ctx, int level) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    if (level < 0) level = default_level(ctx->p);
    if (!level_ok(ctx->p, level))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "Karatsuba level not supported for this N");
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    ctx->tc->want_level = level;
    return tfhe_tc_ensure_level(ctx, level, 0);
}

int tfhe_tc_level(tfhe_ctx *ctx) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    return resolve_level(ctx, -1);
}

// Per-step job table for `tiles` gate tiles (see the kernel comment for the order).
static int prepare_table(tfhe_ctx *ctx, int level, int tiles, bool pair,
                         const TcWorkspace::JobTable **out) {
    TcWorkspace *w = ctx->tc;
    const std::vector<KTerm> &terms = w->lv[level].terms;
    const int key = ((level * 2 + (pair ? 1 : 0)) << 16) | tiles;
    auto it = w->tables.find(key);
    if (it != w->tables.end()) {
        *out = &it->second;
        return TFHE_OK;
    }
    if (ctx->capturing)
        return tfhe_set_error(ctx, TFHE_EINVAL, "tensor-core job table missing while recording a graph");
    const int s = ctx->p.N >> level;
    const int bpp = s / NB;
    // entries name the gate tile, or in the pair form the tile pair (tiles 2u, 2u+1); the
    // terms write disjoint buffers, so a tile's products of one step are independent
    const int units = pair ? (tiles + 1) / 2 : tiles;
    std::vector<uint32_t> tab;
    for (int gt = 0; gt < units; gt++)
        for (int j = 0; j < (int)terms.size(); j++)
            for (int c = 0; c < 2; c++)
                for (int b = 0; b < bpp; b++) tab.push_back(pack_job(JOB_E, gt, j, c, b));
    TcWorkspace::JobTable t;
    if (cudaMalloc(&t.d, tab.size() * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core job table");
    if (cudaMemcpy(t.d, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(t.d);
        return tfhe_set_error(ctx, TFHE_ECUDA, "tensor-core job table upload");
    }
    t.len = (int)tab.size();
    *out = &(w->tables[key] = t);
    return TFHE_OK;
}

// Buffers and job table of a G-gate BlindRotate, sized before the first launch (and
// before a graph that contains it is recorded).
static int reserve_tc(tfhe_ctx *ctx, int G, int level, const TcWorkspace::JobTable **table) {
    const tfhe_params &p = ctx->p;
    TcWorkspace *w = ctx->tc;
    const bool pair = use_pair(ctx);
    const int tiles = (G + TILE_M - 1) / TILE_M;
    const int tiles_pad = pair ? (tiles + 1) / 2 * 2 : tiles;
    const int T = (int)w->lv[level].terms.size();
    const int s = p.N >> level;
    const uint4 *old_digits = w->digits;
    int rc = grow_dev(ctx, (void **)&w->digits, &w->digits_cap,
                      (size_t)tiles_pad * T * 2 * p.l * s * TILE_M * 2, "tensor-core digit buffer");
    if (rc != TFHE_OK) return rc;
    // the odd tile that pads a pair is never written: keep its digits zero
    if (w->digits != old_digits) TFHE_CUDA_TRY(ctx, cudaMemset(w->digits, 0, w->digits_cap));
    rc = grow_dev(ctx, (void **)&w->sync, &w->sync_cap, (2 + 3 * (size_t)tiles_pad) * 4,
                  "tensor-core progress counters");
    if (rc != TFHE_OK) return rc;
    rc = grow_dev(ctx, (void **)&w->acc_t, &w->acc_t_cap, (size_t)tiles_pad * 2 * p.N * TILE_M * 4,
                  "tensor-core accumulators");
    if (rc != TFHE_OK) return rc;
    const TcWorkspace::JobTable *t = nullptr;
    rc = prepare_table(ctx, level, tiles, pair, &t);
    if (rc == TFHE_OK && table) *table = t;
    return rc;
}

int tfhe_tc_reserve(tfhe_ctx *ctx, int gates, int level) {
    if (gates <= 0 || !tfhe_tc_supported(ctx) || !ctx->has_keys) return TFHE_OK;
    int rc = tfhe_tc_ensure_level(ctx, level, 0);  // nothing to size before the keys are loaded
    if (rc != TFHE_OK) return rc;
    return reserve_tc(ctx, gates, resolve_level(ctx, level), nullptr);
}

// Arguments of a `steps`-step persistent launch over the tiles of G rows (gates or
// CMUXes), with the buffers and job table sized for it; the caller sets the mode fields.
static int persistent_args(tfhe_ctx *ctx, int G, int steps, int level, const uint4 *win,
                           size_t win_bytes, BrArgs &args) {
    const tfhe_params &p = ctx->p;
    TcWorkspace *w = ctx->tc;
    const TcWorkspace::Level &V = w->lv[level];
    const int tiles = (G + TILE_M - 1) / TILE_M;
    const int T = (int)V.terms.size();
    const int s = p.N >> level;
    const TcWorkspace::JobTable *table = nullptr;
    int rc = reserve_tc(ctx, G, level, &table);
    if (rc != TFHE_OK) return rc;
    if (!w->sms) {
        int sms = 0;
        TFHE_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        w->sms = sms;
    }
    const bool pair = use_pair(ctx);
    args = BrArgs{};
    args.N = p.N;
    args.l = p.l;
    args.Bgbit = p.Bgbit;
    args.G = G;
    args.n = steps;
    args.n1 = p.n + 1;
    args.s = s;
    args.nterms = T;
    args.tiles = tiles;
    args.tiles_pad = pair ? (tiles + 1) / 2 * 2 : tiles;
    args.one_pass_limit = w->one_pass_limit;
    args.cbs = 2 * (s / NB);
    args.e_per_tile = T * 2 * (s / NB);
    args.step_len = table->len;
    args.total_e = (long long)steps * table->len;
    args.total_d = (long long)steps * tiles * DPARTS;
    // as many equal chunks as keep at least CHUNK_WAVES waves of product jobs per step in
    // each (one SM per tile); the pair form keeps all tiles in one chunk
    args.units = pair ? (tiles + 1) / 2 : tiles;
    {
        const int min_units = (int)ceil(CHUNK_WAVES * w->sms / args.e_per_tile);
        args.nchunks = pair ? 1 : std::max(1, args.units / std::max(1, min_units));
    }
    args.table = table->d;
    args.terms = V.d_terms;
    args.ms_shift = 32 - (ctx->logN + 1);
    args.acc = w->acc_t;
    args.digits = w->digits;
    args.digits_units = w->digits_cap / 16;
    args.acc_words = w->acc_t_cap / 4;
    args.win_units = win_bytes / 16;
    args.bar_words = (size_t)G * (p.n + 1);
    args.win = win;
    args.sync = w->sync;
    args.err = ctx->d_err;
    return TFHE_OK;
}

// Launch the persistent kernel of `level` with `args` (one block per SM, or SM pairs).
static int launch_persistent(tfhe_ctx *ctx, const BrArgs &args, int level, cudaStream_t st) {
    TcWorkspace *w = ctx->tc;
    const bool pair = use_pair(ctx);
    void (*kern)(BrArgs);
    if (pair)
        kern = level == 0 ? k_tc_blind_rotate<0, true>
             : (level == 1 ? k_tc_blind_rotate<1, true>
                           : (level == 2 ? k_tc_blind_rotate<2, true> : k_tc_blind_rotate<3, true>));
    else
        kern = level == 0 ? k_tc_blind_rotate<0, false>
             : (level == 1 ? k_tc_blind_rotate<1, false>
                           : (level == 2 ? k_tc_blind_rotate<2, false> : k_tc_blind_rotate<3, false>));
    const int smem = smem_bytes(ctx->p.N, pair);
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    TFHE_CUDA_TRY(ctx, cudaMemsetAsync(w->sync, 0, (2 + 3 * (size_t)args.tiles_pad) * 4, st));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(P_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    if (pair) {
        // as many SM pairs as can be resident at once (one block per SM)
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int &mp = w->max_pairs[level];
        if (mp < 0) {
            cfg.gridDim = dim3(2 * (w->sms / 2));
            int n = 0;
            TFHE_CUDA_TRY(ctx, cudaOccupancyMaxActiveClusters(&n, kern, &cfg));
            if (n < 1) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core SM pairs not schedulable");
            mp = n;
        }
        const long long pairs = args.total_e < mp ? args.total_e : mp;
        cfg.gridDim = dim3((unsigned)(2 * pairs));
    } else {
        cfg.gridDim = dim3((unsigned)(args.total_e < w->sms ? args.total_e : w->sms));
    }
    StageTimer tm(ctx, TFHE_STAGE_BLIND_ROTATE_TC, st);
    TFHE_CUDA_TRY(ctx, cudaLaunchKernelEx(&cfg, kern, args));
    tm.stop();
    return tfhe_check_launch(ctx, "tc blind rotate");
}

int tfhe_blind_rotate_tc(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                         cudaStream_t st, int level, const TcGateInputs *gates,
                         const uint32_t **tiled_acc) {
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    if (!tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form: unsupported parameters");
    int rc = tfhe_tc_ensure_level(ctx, level, st);
    if (rc != TFHE_OK) return rc;
    level = resolve_level(ctx, level);
    TcWorkspace *w = ctx->tc;
    const TcWorkspace::Level &V = w->lv[level];
    if (!V.ready) return tfhe_set_error(ctx, TFHE_ENOKEYS, "tensor-core form: key windows not prepared");
    BrArgs args;
    rc = persistent_args(ctx, G, p.n, level, V.win, V.win_cap, args);
    if (rc != TFHE_OK) return rc;
    args.bar = bar;
    args.in = gates ? gates->in : nullptr;
    args.num_in = gates ? gates->num_in : 0;
    args.types = gates ? gates->types : nullptr;
    args.idx = gates ? gates->idx : nullptr;
    args.bar_w = gates ? const_cast<uint32_t *>(bar) : nullptr;
    rc = launch_persistent(ctx, args, level, st);
    if (rc != TFHE_OK) return rc;
    if (tiled_acc) {  // the caller reads the tiled accumulators (the gate path's key switch)
        *tiled_acc = w->acc_t;
        return TFHE_OK;
    }
    StageTimer ta(ctx, TFHE_STAGE_TC_AUX, st);
    k_tc_untile_acc<<<dim3((unsigned)(p.N / 32), (unsigned)(4 * args.tiles), 2), dim3(32, 8), 0, st>>>(
        p.N, G, w->acc_t, acc);
    ta.stop();
    return tfhe_check_launch(ctx, "tc untile accumulators");
}

// Batched CMUX on the tensor cores: out(x, y) = d0 + C_y (.) (d1 - d0) for the geometry g
// (groups of g.nx CMUXes sharing selector C_y = sel + y * g.sy TRGSWs).  One step of the
// persistent kernel in CMUX mode over ceil(nx / 128) tiles per group; the selectors'
// windows are expanded for this call.  No keys are needed.
int tfhe_cmux_tc(tfhe_ctx *ctx, const uint32_t *sel, const CmuxGeom &g, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (g.count <= 0 || g.nx <= 0 || g.ny <= 0) return TFHE_OK;
    if (!tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form: unsupported parameters");
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    const int level = resolve_level(ctx, -1);
    if (!level_ok(p, level))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "Karatsuba level not supported for this N");
    int rc = ensure_plan(ctx, level, st);
    if (rc != TFHE_OK) return rc;
    TcWorkspace *w = ctx->tc;
    const TcWorkspace::Level &V = w->lv[level];
    const int T = (int)V.terms.size();
    const int s = p.N >> level;
    const int tpg = (g.nx + TILE_M - 1) / TILE_M;
    const int64_t tiles = (int64_t)tpg * g.ny;
    if (tiles * TILE_M > (int64_t)1 << 30)
        return tfhe_set_error(ctx, TFHE_EINVAL, "tensor-core CMUX: batch too large");
    const int ppk = 2 * p.l * 2;  // polynomials per selector
    const size_t npoly = (size_t)g.ny * ppk;
    rc = grow_dev(ctx, (void **)&w->cm_win, &w->cm_win_cap,
                  npoly * T * PLANES * 2 * (size_t)s * sizeof(uint4), "tensor-core CMUX windows");
    if (rc != TFHE_OK) return rc;
    {
        StageTimer ta(ctx, TFHE_STAGE_TC_AUX, st);
        k_tc_windows<<<dim3((unsigned)npoly, T), 256, 0, st>>>(sel, p.N, s, T, V.d_terms, w->cm_win,
                                                              ppk, g.sy * ppk);
        ta.stop();
        rc = tfhe_check_launch(ctx, "tc cmux windows");
        if (rc != TFHE_OK) return rc;
    }
    BrArgs args;
    rc = persistent_args(ctx, (int)(tiles * TILE_M), 1, level, w->cm_win, w->cm_win_cap, args);
    if (rc != TFHE_OK) return rc;
    args.cmux = 1;
    args.tpg = tpg;
    args.cm_d1 = g.d1;
    args.cm_d0 = g.d0;
    args.cm_dx = g.dx;
    args.cm_dy = g.dy;
    args.cm_nx = g.nx;
    args.cm_count = g.count;
    rc = launch_persistent(ctx, args, level, st);
    if (rc != TFHE_OK) return rc;
    StageTimer ta(ctx, TFHE_STAGE_TC_AUX, st);
    k_tc_untile_cmux<<<dim3((unsigned)(p.N / 32), (unsigned)(4 * tiles), 2), dim3(32, 8), 0, st>>>(
        p.N, tpg, g.nx, g.count, g.ox, g.oy, w->acc_t, g.out);
    ta.stop();
    return tfhe_check_launch(ctx, "tc cmux outputs");
}

int tfhe_tc_set_variant(tfhe_ctx *ctx, int variant) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    if (variant < -1 || variant > TFHE_TC_SM_PAIR)
        return tfhe_set_error(ctx, TFHE_EINVAL, "tensor-core variant");
    if (variant == TFHE_TC_SM_PAIR) {
        int cl = 0;
        TFHE_CUDA_TRY(ctx, cudaDeviceGetAttribute(&cl, cudaDevAttrClusterLaunch, ctx->device));
        if (!cl) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "device cannot launch SM pairs");
    }
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    ctx->tc->want_variant = variant;
    return TFHE_OK;
}

int tfhe_tc_set_pass_limit(tfhe_ctx *ctx, int limit) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    if (limit < -1 || limit > ONE_PASS_LIMIT)
        return tfhe_set_error(ctx, TFHE_EINVAL, "one-pass limit above 2^17 is not exact");
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    ctx->tc->one_pass_limit = limit < 0 ? ONE_PASS_LIMIT : limit;
    return TFHE_OK;
}

int tfhe_tc_variant(tfhe_ctx *ctx) {
    if (!tfhe_tc_supported(ctx)) return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no tensor-core form");
    return use_pair(ctx) ? TFHE_TC_SM_PAIR : TFHE_TC_SINGLE_SM;
}


