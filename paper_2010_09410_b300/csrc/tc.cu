// tc.cu -- the tensor-core form of BlindRotate (and of batched CMUXes).
//
// One BlindRotate step over a tile of 128 gates is the dense contraction
//   Y[g][c][n] = sum_{r < 2l} sum_{k < N} D_g[r][k] * T_{r,c}[n][k]   (mod 2^32)
// of the gadget digits D (|d| <= Bg/2 <= 32) by the negacyclic Toeplitz matrices of the
// key polynomials q = BSK_i[r][c]: T[n][k] = q[n-k] for n >= k, -q[n-k+N] otherwise.
// It runs on the sm_103a tensor cores (tcgen05.mma kind::f16, bf16 operands, fp32
// accumulators in TMEM).  bf16 holds the digits and signed byte planes of the key
// (q = sum_p 2^{8p} q_p, q_p in [-128, 128)) exactly; one K-half covers the l rows of one
// polynomial of the TRLWE (l*N <= 4096 terms), so every partial sum is an integer below
// l*N*32*128 <= 2^24 and the fp32 accumulation is exact.  Each half is read out of TMEM,
// rounded to int32 and recombined mod 2^32 as sum_p 2^{8p} Y_p.
//
// The Toeplitz operand is never materialised.  Row n of T (as a function of k) is the
// window r_vec[N-1-n+k] of one vector of length 2N,
//   r_vec[x] = q[N-1-x]  (x < N),   r_vec[x] = -q[2N-1-x]  (N <= x < 2N).
// Shared memory holds "units": unit u is the 16 bytes r_vec[u .. u+7] (one byte plane,
// bf16).  For an output block n in [c0-NB+1, c0] (column idx = c0 - n) and digits
// k in [k0, k0+KS), the element (idx, k) is r_vec[P0 + idx + k] with P0 = N-1-c0, i.e.
// element t of unit (P0 + k0) + idx + (k - k0 - t).  A K-major, no-swizzle UMMA
// descriptor reads row idx's 8-element core-matrix row at base + 16*idx and the next
// 8 k's at +128 B, so LBO = SBO = 128 B walk the windows directly.
//
// Kernels per BlindRotate step: k_tc_digits (rotation X^{a} ACC - ACC and gadget
// digits, written in the A-operand layout) then k_tc_extprod (tensor-core product,
// ACC += Y).  Warp roles in k_tc_extprod (192 threads): warps 0-3 build the key
// windows and read out TMEM (warp w owns TMEM lanes 32w..32w+31 = gates), warp 4
// streams the digit tiles with cp.async.bulk, warp 5 allocates TMEM and one lane
// issues the MMAs.  Every wait polls a bounded number of times; on time-out the block
// records TFHE_ETIMEOUT in the context's error word and winds down.
#include "common.cuh"

namespace {

constexpr int TILE_M = 128;  // gates per tile (TMEM lanes)
constexpr int NB = 128;      // output columns per tile and MMA N
constexpr int KS = 128;      // digits (K) per pipeline stage
constexpr int PLANES = 4;    // byte planes of the key
constexpr int STAGES = 4;
constexpr int A_STAGE_BYTES = TILE_M * KS * 2;            // 32 KB
constexpr int B_UNITS = NB + KS;                          // units per plane and stage
constexpr int B_PLANE_BYTES = B_UNITS * 16;               // 4 KB
constexpr int B_STAGE_BYTES = PLANES * B_PLANE_BYTES;     // 16 KB
constexpr int KEY_BYTES_MAX = 6 * 1024 * 4;                // 2l x N key words (l*N <= 3072)
constexpr int SMEM_BYTES = STAGES * (A_STAGE_BYTES + B_STAGE_BYTES) + KEY_BYTES_MAX + 1024;
constexpr int THREADS = 192;
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

// Bounded wait for the phase with the given parity to complete.  Returns false (and
// raises the block's abort flag and the error word) on time-out or when another role
// has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort,
                                          int *err) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            *abort = 1;
            atomicCAS(err, 0, TFHE_ETIMEOUT);
            return false;
        }
    }
    return true;
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

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// bf16 bit pattern of a small integer |x| <= 256: its fp32 pattern has at most 8
// significant bits, so the upper half is the exact bf16 value.
__device__ __forceinline__ uint32_t bf16_bits(int x) {
    return __float_as_uint((float)x) >> 16;
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

// r_vec[x] of the key polynomial q held in shared memory (zero past 2N: never read by
// an MMA).
__device__ __forceinline__ uint32_t rvec(const uint32_t *q, int N, int x) {
    if (x < N) return q[N - 1 - x];
    if (x < 2 * N) return 0u - q[2 * N - 1 - x];
    return 0u;
}

// ---------------------------------------------------------------------------
// Step kernel 1: digits of X^{a_g} ACC_g - ACC_g in the A-operand layout.
// Layout of the digit buffer: [tile][row r < 2l][stage s < N/KS] blocks of 32 KB,
// each block [mg < 16][kb < 16][m8 < 8][8 bf16]: gate m = 8 mg + m8 of the tile,
// digit index k = s*KS + 8 kb + e.  One thread produces 8 consecutive k of one gate
// and one polynomial (c) for all l digit rows.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tc_digits(int N, int l, int Bgbit, int n1, int G,
                                                   int step, const uint32_t *__restrict__ bar,
                                                   const uint32_t *__restrict__ acc,
                                                   uint4 *__restrict__ digits,
                                                   const uint32_t *__restrict__ d1,
                                                   const uint32_t *__restrict__ d0,
                                                   const CmuxGeom *geom) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int kstages = N / KS;
    // thread -> (tile, c, stage, kb, mg, m8), m8 fastest so 8 threads write 128 B
    int t = tid;
    const int m8 = t & 7; t >>= 3;
    const int mg = t & 15; t >>= 4;
    const int kb = t & 15; t >>= 4;
    const int s = t % kstages; t /= kstages;
    const int c = t & 1; t >>= 1;
    const int tile = t;
    const int ntiles = (G + TILE_M - 1) / TILE_M;
    if (tile >= ntiles) return;
    const int m = mg * 8 + m8;
    const int g = tile * TILE_M + m;
    const int k0 = s * KS + kb * 8;
    uint32_t x[8];
    if (g < G) {
        const uint32_t *p = acc + (size_t)g * 2 * N + (size_t)c * N;
        const int a = (int)(bar[(size_t)g * n1 + step] % (uint32_t)(2 * N));
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = rot_coef(p, N, a, k0 + e) - p[k0 + e];
    } else {
#pragma unroll
        for (int e = 0; e < 8; e++) x[e] = 0;
    }
    const uint32_t off = gadget_offset(l, Bgbit);
    for (int j = 0; j < l; j++) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const uint32_t lo = bf16_bits(gadget_digit(x[e] + off, j + 1, Bgbit));
            const uint32_t hi = bf16_bits(gadget_digit(x[e + 1] + off, j + 1, Bgbit));
            w[e / 2] = lo | (hi << 16);
        }
        const int r = c * l + j;
        const size_t blk = ((size_t)tile * 2 * l + r) * kstages + s;
        digits[blk * (A_STAGE_BYTES / 16) + ((size_t)mg * 16 + kb) * 8 + m8] =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ACC = X^{-b~} (0, v), v_j = mu: coefficient j of X^{-b~} v is +mu when (j + b~) mod 2N < N.
__global__ void k_tc_init_acc(int N, int n1, int G, const uint32_t *__restrict__ bar,
                              uint32_t *__restrict__ acc) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)G * 2 * N) return;
    const size_t g = e / (2 * N);
    const int j = (int)(e % (2 * N));
    const uint32_t mu = 1u << 29;
    if (j < N) {
        acc[e] = 0;
    } else {
        const int bb = (int)(bar[g * n1 + n1 - 1] % (uint32_t)(2 * N));
        acc[e] = (((j - N) + bb) % (2 * N)) < N ? mu : 0u - mu;
    }
}

// ---------------------------------------------------------------------------
// Step kernel 2: ACC[tile gates][c][block columns] += sum over the 2l rows of digits x
// Toeplitz(key), on the tensor cores.  blockIdx.x = gate tile, blockIdx.y = column
// block (c = y / (N/NB), columns [b*NB, b*NB + NB)).
// keys: the 2l x 2 key polynomials of this step, key(r, c) = keys + (r*2 + c)*N.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS, 1) k_tc_extprod(int N, int l, int G,
                                                           const uint4 *__restrict__ digits,
                                                           const uint32_t *__restrict__ keys,
                                                           uint32_t *__restrict__ acc, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *a_st = smem;                                   // STAGES x 32 KB
    uint8_t *b_st = smem + STAGES * A_STAGE_BYTES;          // STAGES x 16 KB
    uint32_t *key_s = (uint32_t *)(b_st + STAGES * B_STAGE_BYTES);  // [2l][N], column c
    __shared__ __align__(8) uint64_t full_a[STAGES], full_b[STAGES], empty[STAGES];
    __shared__ __align__(8) uint64_t acc_full, acc_empty, drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int blocks_per_poly = N / NB;
    const int c = blockIdx.y / blocks_per_poly;
    const int bcol = blockIdx.y % blocks_per_poly;
    const int c0 = bcol * NB + NB - 1;    // highest output column of the block
    const int P0 = N - 1 - c0;
    const int kstages = N / KS;
    const int half_stages = l * kstages;  // stages per K-half (one polynomial's l rows)
    const int total_stages = 2 * half_stages;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full_a[s], 1);
            mbar_init(&full_b[s], 128);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 128);
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    volatile int *abort = &abort_flag;

    if (warp == 4) {
        // ---- digit tiles: one 32 KB bulk copy per stage ----
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < total_stages; t++) {
                const int s = t % STAGES;
                if (t >= STAGES && !mbar_wait(&empty[s], ((t / STAGES) - 1) & 1, abort, err)) break;
                const int r = t / kstages, ks = t % kstages;
                const size_t blk = ((size_t)tile * 2 * l + r) * kstages + ks;
                mbar_arrive_tx(&full_a[s], A_STAGE_BYTES);
                bulk_g2s(a_st + s * A_STAGE_BYTES, digits + blk * (A_STAGE_BYTES / 16),
                         A_STAGE_BYTES, &full_a[s]);
                issued = t + 1;
            }
            // let this block's last copies land before it can exit
            for (int t = issued - STAGES; t < issued; t++)
                if (t >= 0) mbar_wait_settle(&full_a[t % STAGES], (t / STAGES) & 1);
        }
    } else if (warp == 5) {
        // ---- MMA issue ----
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(TILE_M, NB);
            for (int t = 0; t < total_stages; t++) {
                const int s = t % STAGES;
                const uint32_t par = (t / STAGES) & 1;
                if (t == half_stages && !mbar_wait(&acc_empty, 0, abort, err)) break;
                if (!mbar_wait(&full_a[s], par, abort, err)) break;
                if (!mbar_wait(&full_b[s], par, abort, err)) break;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(a_st + s * A_STAGE_BYTES);
                const uint32_t b_addr = smem_u32(b_st + s * B_STAGE_BYTES);
                const bool first = (t % half_stages) == 0;
#pragma unroll
                for (int kk = 0; kk < KS / 16; kk++) {
                    const uint64_t ad = make_desc(a_addr + kk * 256, 128, 2048);
#pragma unroll
                    for (int p = 0; p < PLANES; p++) {
                        const uint64_t bd = make_desc(b_addr + p * B_PLANE_BYTES + kk * 256, 128, 128);
                        mma_bf16(tmem + p * NB, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
                    }
                }
                mma_commit(&empty[s]);
                if ((t + 1) % half_stages == 0) mma_commit(&acc_full);
            }
            // drain: wait until every MMA issued above has finished with TMEM
            mma_commit(&drain);
            mbar_wait_settle(&drain, 0);
        }
    } else {
        // ---- warps 0-3: key windows, then TMEM read-out per K-half ----
        const int tid = threadIdx.x;  // 0..127, also the TMEM lane = gate of the tile
        const int g = tile * TILE_M + tid;
        uint32_t *acc_row = acc + (size_t)g * 2 * N + (size_t)c * N;
        // the 2l key polynomials of column c, into shared memory (named barrier 1 = warps 0-3)
        for (int w = tid; w < 2 * l * N / 4; w += 128) {
            const int r = (w * 4) / N, k = (w * 4) % N;
            *(uint4 *)(key_s + r * N + k) = __ldg((const uint4 *)(keys + ((size_t)r * 2 + c) * N + k));
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        bool ok = true;
        for (int h = 0; h < 2 && ok; h++) {
            // build the key windows of this half (and, for h = 0, run ahead into h = 1)
            const int t_begin = (h == 0) ? 0 : half_stages + STAGES;
            const int t_end = (h == 0) ? min(total_stages, half_stages + STAGES) : total_stages;
            for (int t = t_begin; t < t_end && ok; t++) {
                const int s = t % STAGES;
                if (t >= STAGES && !mbar_wait(&empty[s], ((t / STAGES) - 1) & 1, abort, err)) {
                    ok = false;
                    break;
                }
                const int r = t / kstages, ks = t % kstages;
                const uint32_t *q = key_s + (size_t)r * N;
                const int U0 = P0 + ks * KS;
                uint8_t *bs = b_st + s * B_STAGE_BYTES;
                for (int v = tid; v < B_UNITS; v += 128) {
                    uint32_t w[PLANES][4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        int pl0[PLANES], pl1[PLANES];
                        byte_planes(rvec(q, N, U0 + v + e), pl0);
                        byte_planes(rvec(q, N, U0 + v + e + 1), pl1);
#pragma unroll
                        for (int p = 0; p < PLANES; p++)
                            w[p][e / 2] = bf16_bits(pl0[p]) | (bf16_bits(pl1[p]) << 16);
                    }
#pragma unroll
                    for (int p = 0; p < PLANES; p++)
                        *(uint4 *)(bs + p * B_PLANE_BYTES + v * 16) =
                            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
                }
                fence_proxy_async();
                mbar_arrive(&full_b[s]);
            }
            if (!ok) break;
            // read-out of half h: chunk j holds columns idx = 32j..32j+31, i.e. the words
            // n = nb..nb+31 (nb = c0 - 32j - 31, a multiple of 32) of this gate's row, word
            // n = nb + w taking the sum of column 31 - w.  The old words of the next chunk
            // are loaded before this chunk's TMEM values are needed.
            uint4 cur[8];
            const bool live = g < G;
            if (live) {
                const uint4 *src = (const uint4 *)(acc_row + (c0 - 31));
#pragma unroll
                for (int q = 0; q < 8; q++) cur[q] = src[q];
            }
            if (!mbar_wait(&acc_full, h, abort, err)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t lane_base = tmem + (((uint32_t)(warp * 32)) << 16);
#pragma unroll 1
            for (int j = 0; j < NB / 32; j++) {
                uint4 nxt[8];
                if (live && j + 1 < NB / 32) {
                    const uint4 *src = (const uint4 *)(acc_row + (c0 - 32 * (j + 1) - 31));
#pragma unroll
                    for (int q = 0; q < 8; q++) nxt[q] = src[q];
                }
                uint32_t sum[32];
#pragma unroll
                for (int e = 0; e < 32; e++) sum[e] = 0;
#pragma unroll
                for (int p = 0; p < PLANES; p++) {
                    uint32_t v[32];
                    tmem_ld32(lane_base + p * NB + j * 32, v);
#pragma unroll
                    for (int e = 0; e < 32; e++)
                        sum[e] += (uint32_t)__float2int_rn(__uint_as_float(v[e])) << (8 * p);
                }
                if (live) {
                    uint4 *dst = (uint4 *)(acc_row + (c0 - 32 * j - 31));
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        uint4 o = cur[q];
                        o.x += sum[31 - (4 * q + 0)];
                        o.y += sum[31 - (4 * q + 1)];
                        o.z += sum[31 - (4 * q + 2)];
                        o.w += sum[31 - (4 * q + 3)];
                        dst[q] = o;
                    }
#pragma unroll
                    for (int q = 0; q < 8; q++) cur[q] = nxt[q];
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

}  // namespace

struct TcWorkspace {
    uint4 *digits = nullptr;
    size_t digits_cap = 0;  // bytes
};

int tfhe_tc_supported(const tfhe_ctx *ctx) {
    const tfhe_params &p = ctx->p;
    return p.N >= 256 && p.N <= 1024 && p.N % NB == 0 && p.N % KS == 0 && p.Bgbit <= 6 &&
           (int64_t)p.l * p.N * 32 * 128 <= (1 << 24) && 2 * p.l * p.N * 4 <= KEY_BYTES_MAX;
}

void tfhe_tc_free(tfhe_ctx *ctx) {
    if (!ctx->tc) return;
    if (ctx->tc->digits) cudaFree(ctx->tc->digits);
    delete ctx->tc;
    ctx->tc = nullptr;
}

static int ensure_digits(tfhe_ctx *ctx, int G) {
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    const size_t tiles = (size_t)(G + TILE_M - 1) / TILE_M;
    const size_t bytes = tiles * 2 * ctx->p.l * ctx->p.N * TILE_M * 2;
    if (bytes <= ctx->tc->digits_cap) return TFHE_OK;
    if (ctx->tc->digits) cudaFree(ctx->tc->digits);
    ctx->tc->digits = nullptr;
    ctx->tc->digits_cap = 0;
    if (cudaMalloc(&ctx->tc->digits, bytes) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core digit buffer");
    ctx->tc->digits_cap = bytes;
    return TFHE_OK;
}

int tfhe_blind_rotate_tc(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                         cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    if (!tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form: unsupported parameters");
    int rc = ensure_digits(ctx, G);
    if (rc != TFHE_OK) return rc;
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_extprod,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            SMEM_BYTES));
    const int n1 = p.n + 1;
    {
        const size_t total = (size_t)G * 2 * p.N;
        k_tc_init_acc<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(p.N, n1, G, bar, acc);
        rc = tfhe_check_launch(ctx, "tc_init_acc");
        if (rc != TFHE_OK) return rc;
    }
    const int tiles = (G + TILE_M - 1) / TILE_M;
    const size_t dig_threads = (size_t)tiles * 2 * (p.N / KS) * 16 * 16 * 8;
    const unsigned dig_blocks = (unsigned)((dig_threads + 255) / 256);
    const dim3 grid(tiles, 2 * p.N / NB);
    const size_t per = (size_t)2 * p.l * 2 * p.N;
    for (int i = 0; i < p.n; i++) {
        {
            StageTimer tm(ctx, TFHE_STAGE_DECOMPOSE_TC, st);
            k_tc_digits<<<dig_blocks, 256, 0, st>>>(p.N, p.l, p.Bgbit, n1, G, i, bar, acc,
                                                    ctx->tc->digits, nullptr, nullptr, nullptr);
            tm.stop();
        }
        {
            StageTimer tm(ctx, TFHE_STAGE_EXTPROD_TC, st);
            k_tc_extprod<<<grid, THREADS, SMEM_BYTES, st>>>(p.N, p.l, G, ctx->tc->digits,
                                                            ctx->bsk_raw + (size_t)i * per, acc,
                                                            ctx->d_err);
            tm.stop();
        }
        rc = tfhe_check_launch(ctx, "tc step");
        if (rc != TFHE_OK) return rc;
    }
    return TFHE_OK;
}

int tfhe_cmux_tc(tfhe_ctx *ctx, const uint32_t *, const CmuxGeom &, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core CMUX not built yet");
}

int tfhe_ram_write_tc(tfhe_ctx *ctx, const uint32_t *, const uint32_t *, int, const uint32_t *,
                      uint32_t *, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core RAM write not built yet");
}
