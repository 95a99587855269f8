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
// The units of every key polynomial and byte plane (2N units of 16 B each) are expanded
// once when the keys are loaded (k_tc_windows: 1 GB for the n = 630, N = 1024 BSK), so a
// B stage is four contiguous bulk copies, like the digit (A) stage.
//
// The digits of X^{a_i} ACC - ACC are written per 128-gate tile in the A-operand layout:
// [tile][row r < 2l][stage s < N/KS] blocks of 32 KB, each [mg < 16][kb < 16][m8 < 8]
// [8 bf16] for gate m = 8 mg + m8 and digit index k = s*KS + 8 kb + e.  One launch of
// k_tc_blind_rotate runs all n steps (see below).  Every wait polls a bounded number of times; on time-out the block
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
constexpr int SMEM_BYTES = STAGES * (A_STAGE_BYTES + B_STAGE_BYTES) + 1024;
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

// r_vec[x] of the key polynomial q (zero past 2N: never read by an MMA).
__device__ __forceinline__ uint32_t rvec(const uint32_t *__restrict__ q, int N, int x) {
    if (x < N) return __ldg(q + (N - 1 - x));
    if (x < 2 * N) return 0u - __ldg(q + (2 * N - 1 - x));
    return 0u;
}

// Window units of `npoly` key polynomials: win[(poly * 4 + p) * 2N + u] holds byte plane p
// of r_vec[u .. u+7] as 8 bf16.  One block per polynomial.
__global__ void k_tc_windows(const uint32_t *__restrict__ polys, int N, uint4 *__restrict__ win) {
    const size_t poly = blockIdx.x;
    const uint32_t *q = polys + poly * N;
    for (int u = threadIdx.x; u < 2 * N; u += blockDim.x) {
        uint32_t w[PLANES][4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            int pl0[PLANES], pl1[PLANES];
            byte_planes(rvec(q, N, u + e), pl0);
            byte_planes(rvec(q, N, u + e + 1), pl1);
#pragma unroll
            for (int p = 0; p < PLANES; p++) w[p][e / 2] = bf16_bits(pl0[p]) | (bf16_bits(pl1[p]) << 16);
        }
#pragma unroll
        for (int p = 0; p < PLANES; p++)
            win[(poly * PLANES + p) * 2 * N + u] = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
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
// Persistent BlindRotate: all n steps in one launch, one block per SM.
//
// Jobs: D(i, gt, part) writes the digits of gates 8*part .. 8*part+7 of gate tile gt for
// step i (16 parts per tile); E(i, gt, cb) is the tensor-core product of column block
// cb (ACC += Y).  Order: all D(0, ., .), then for each step i and tile gt:
// E(i, gt, 0..cbs-1) followed by D(i+1, gt, 0..15).  Blocks take jobs from a global
// counter, so a job only ever waits for jobs with smaller indices, which running
// blocks hold: E(i, gt, .) waits for done_D[gt] >= 16 (i+1); D(i+1, gt, .) waits for
// done_E[gt] >= cbs (i+1).  Every wait is bounded.
//
// Warp roles (320 threads): warps 0-3 read TMEM out (warp w owns lanes 32w..32w+31),
// warp 4 fetches jobs and streams stages with cp.async.bulk, warp 5 owns TMEM and one
// lane issues the MMAs, warps 6-9 compute digits.  The four planes of TMEM are handed
// back one by one after each K-half's read-out, so the next half's MMAs on plane p start
// as soon as plane p has been read; both halves of a job accumulate in registers and the
// accumulator row is updated once per job.
// ---------------------------------------------------------------------------
constexpr int P_THREADS = 320;
constexpr int JQ = 8;  // job ring depth

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
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

constexpr int DPARTS = 16;  // digit parts per gate tile (8 gates each)

struct BrArgs {
    int N, l, Bgbit, G, n, n1;
    int tiles, cbs;             // gate tiles, column blocks (2N / NB)
    long long total_jobs;
    const uint32_t *bar;        // [G][n+1]
    uint32_t *acc;              // [G][2][N]
    uint4 *digits;              // [tiles][2l][N/KS] x 32 KB
    const uint4 *win;           // [n][2l][2][4][2N] units
    uint32_t *sync;             // [0] job counter, [1 .. tiles] done_D, [1+tiles ..] done_E
    int *err;
};

struct Job {
    int kind;  // 0 = stop, 1 = digits D(i, gt, part), 2 = product E(i, gt, cb)
    int i, gt, sub;
};

__device__ __forceinline__ Job decode_job(const BrArgs &a, int job) {
    Job J{0, 0, 0, 0};
    if (job < 0) return J;
    const int d0 = a.tiles * DPARTS;
    if (job < d0) {
        J.kind = 1; J.i = 0; J.gt = job / DPARTS; J.sub = job % DPARTS;
        return J;
    }
    int j = job - d0;
    const int per = a.tiles * (a.cbs + DPARTS);
    int i = j / per;
    if (i < a.n - 1) {
        j %= per;
        J.gt = j / (a.cbs + DPARTS);
        const int x = j % (a.cbs + DPARTS);
        if (x < a.cbs) { J.kind = 2; J.i = i; J.sub = x; }
        else { J.kind = 1; J.i = i + 1; J.sub = x - a.cbs; }
        return J;
    }
    j -= (a.n - 1) * per;  // last step: products only
    J.kind = 2; J.i = a.n - 1; J.gt = j / a.cbs; J.sub = j % a.cbs;
    return J;
}

__global__ void __launch_bounds__(P_THREADS, 1) k_tc_blind_rotate(BrArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *a_st = smem;
    uint8_t *b_st = smem + STAGES * A_STAGE_BYTES;
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
    __shared__ __align__(8) uint64_t acc_full, acc_empty[PLANES], drain;
    __shared__ __align__(8) uint64_t job_full[JQ], job_empty[JQ];
    __shared__ int jobs[JQ];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N = a.N, l = a.l;
    const int kstages = N / KS;
    const int half_stages = l * kstages;
    const int total_stages = 2 * half_stages;
    const long long total_jobs = a.total_jobs;
    uint32_t *job_counter = a.sync;
    uint32_t *done_D = a.sync + 1;
    uint32_t *done_E = a.sync + 1 + a.tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        for (int p = 0; p < PLANES; p++) mbar_init(&acc_empty[p], 128);
        mbar_init(&drain, 1);
        for (int q = 0; q < JQ; q++) {
            mbar_init(&job_full[q], 1);
            mbar_init(&job_empty[q], 3);  // MMA lane, read-out leader, digit leader
        }
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
    int *err = a.err;

    if (warp == 4) {
        // ---- job fetch + stage loads ----
        if (lane == 0) {
            int t_global = 0, issued = 0;
            for (int q = 0;; q++) {
                const int slot = q % JQ;
                if (q >= JQ && !mbar_wait(&job_empty[slot], ((q / JQ) - 1) & 1, abort, err)) break;
                const unsigned j = atomicAdd(job_counter, 1u);
                const int job = (long long)j < total_jobs ? (int)j : -1;
                jobs[slot] = job;
                mbar_arrive(&job_full[slot]);
                if (job < 0) break;
                const Job J = decode_job(a, job);
                if (J.kind != 2) continue;  // digit job: nothing to load
                const int i = J.i, gt = J.gt, cb = J.sub;
                const int c = cb / (N / NB), bcol = cb % (N / NB);
                const int P0 = N - NB - bcol * NB;
                if (!wait_count(&done_D[gt], (uint32_t)(DPARTS * (i + 1)), abort, err)) break;
                asm volatile("fence.proxy.async.global;" ::: "memory");
                const uint4 *win = a.win + (size_t)i * (2 * l * 2) * PLANES * 2 * N;
                bool ok = true;
                for (int ts = 0; ts < total_stages; ts++, t_global++) {
                    const int s = t_global % STAGES;
                    if (t_global >= STAGES &&
                        !mbar_wait(&empty[s], ((t_global / STAGES) - 1) & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    const int r = ts / kstages, ks = ts % kstages;
                    const size_t blk = ((size_t)gt * 2 * l + r) * kstages + ks;
                    mbar_arrive_tx(&full[s], A_STAGE_BYTES + B_STAGE_BYTES);
                    bulk_g2s(a_st + s * A_STAGE_BYTES, a.digits + blk * (A_STAGE_BYTES / 16),
                             A_STAGE_BYTES, &full[s]);
                    const uint4 *wsrc = win + ((size_t)(r * 2 + c) * PLANES) * 2 * N + (P0 + ks * KS);
#pragma unroll
                    for (int p = 0; p < PLANES; p++)
                        bulk_g2s(b_st + s * B_STAGE_BYTES + p * B_PLANE_BYTES,
                                 wsrc + (size_t)p * 2 * N, B_PLANE_BYTES, &full[s]);
                    issued = t_global + 1;
                }
                if (!ok) break;
            }
            for (int t = issued - STAGES; t < issued; t++)
                if (t >= 0) mbar_wait_settle(&full[t % STAGES], (t / STAGES) & 1);
        }
    } else if (warp == 5) {
        // ---- MMA issue ----
        if (lane == 0) {
            constexpr uint32_t idesc = make_idesc(TILE_M, NB);
            int t_global = 0, khalf = 0;
            bool ok = true;
            for (int q = 0; ok; q++) {
                const int slot = q % JQ;
                if (!mbar_wait(&job_full[slot], (q / JQ) & 1, abort, err)) break;
                const int job = jobs[slot];
                mbar_arrive(&job_empty[slot]);
                if (job < 0) break;
                if (decode_job(a, job).kind != 2) continue;  // digit job
                for (int ts = 0; ts < total_stages && ok; ts++, t_global++) {
                    const int s = t_global % STAGES;
                    if (!mbar_wait(&full[s], (t_global / STAGES) & 1, abort, err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = smem_u32(a_st + s * A_STAGE_BYTES);
                    const uint32_t b_addr = smem_u32(b_st + s * B_STAGE_BYTES);
                    if (ts % half_stages == 0) {
                        // first stage of a half: plane p starts once its previous contents
                        // have been read out
#pragma unroll
                        for (int p = 0; p < PLANES; p++) {
                            if (khalf > 0 && !mbar_wait(&acc_empty[p], (khalf - 1) & 1, abort, err)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
#pragma unroll
                            for (int kk = 0; kk < KS / 16; kk++)
                                mma_bf16(tmem + p * NB, make_desc(a_addr + kk * 256, 128, 2048),
                                         make_desc(b_addr + p * B_PLANE_BYTES + kk * 256, 128, 128),
                                         idesc, kk == 0 ? 0u : 1u);
                        }
                        if (!ok) break;
                    } else {
#pragma unroll
                        for (int kk = 0; kk < KS / 16; kk++) {
                            const uint64_t ad = make_desc(a_addr + kk * 256, 128, 2048);
#pragma unroll
                            for (int p = 0; p < PLANES; p++)
                                mma_bf16(tmem + p * NB, ad,
                                         make_desc(b_addr + p * B_PLANE_BYTES + kk * 256, 128, 128),
                                         idesc, 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                    if ((ts + 1) % half_stages == 0) {
                        mma_commit(&acc_full);
                        khalf++;
                    }
                }
            }
            mma_commit(&drain);
            mbar_wait_settle(&drain, 0);
        }
    } else if (warp < 4) {
        // ---- TMEM read-out: thread = TMEM lane = gate of the tile ----
        const int tid = threadIdx.x;
        const uint32_t lane_base = tmem + (((uint32_t)(warp * 32)) << 16);
        int khalf = 0;
        for (int q = 0;; q++) {
            const int slot = q % JQ;
            if (!mbar_wait(&job_full[slot], (q / JQ) & 1, abort, err)) break;
            const int job = jobs[slot];
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (tid == 0) mbar_arrive(&job_empty[slot]);
            if (job < 0) break;
            const Job J = decode_job(a, job);
            if (J.kind != 2) continue;
            const int i = J.i, gt = J.gt, cb = J.sub;
            const int c = cb / (N / NB), bcol = cb % (N / NB);
            const int c0 = bcol * NB + NB - 1;
            uint32_t sum[NB];
#pragma unroll
            for (int e = 0; e < NB; e++) sum[e] = 0;
            bool ok = true;
            for (int h = 0; h < 2 && ok; h++, khalf++) {
                if (!mbar_wait(&acc_full, khalf & 1, abort, err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
#pragma unroll
                for (int p = 0; p < PLANES; p++) {
#pragma unroll
                    for (int j = 0; j < NB / 16; j += 2) {
                        uint32_t v[32];
                        tmem_ld16(lane_base + p * NB + j * 16, v);
                        tmem_ld16(lane_base + p * NB + (j + 1) * 16, v + 16);
                        tmem_wait_ld();
#pragma unroll
                        for (int e = 0; e < 32; e++)
                            sum[j * 16 + e] += (uint32_t)__float2int_rn(__uint_as_float(v[e])) << (8 * p);
                    }
                    tc_fence_before();
                    mbar_arrive(&acc_empty[p]);
                }
            }
            if (!ok) break;
            // ACC row update: word n = c0 - idx receives column idx.  The leader's acquire of
            // done_D (already satisfied) orders these accesses after the previous step's
            // updates of the same words by other blocks.
            if (tid == 0) wait_count(&done_D[gt], (uint32_t)(DPARTS * (i + 1)), abort, err);
            asm volatile("bar.sync 1, 128;" ::: "memory");
            const int g = gt * TILE_M + tid;
            if (g < a.G) {
                uint4 *row = (uint4 *)(a.acc + (size_t)g * 2 * N + (size_t)c * N + (c0 - NB + 1));
#pragma unroll
                for (int q4 = 0; q4 < NB / 4; q4++) {
                    uint4 o = row[q4];
                    o.x += sum[NB - 1 - (4 * q4 + 0)];
                    o.y += sum[NB - 1 - (4 * q4 + 1)];
                    o.z += sum[NB - 1 - (4 * q4 + 2)];
                    o.w += sum[NB - 1 - (4 * q4 + 3)];
                    row[q4] = o;
                }
            }
            __threadfence();
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (tid == 0) atomicAdd(&done_E[gt], 1u);
        }
    } else {
        // ---- warps 6-9: digit jobs ----
        const int tid = threadIdx.x - 192;
        const uint32_t off = gadget_offset(l, a.Bgbit);
        for (int q = 0;; q++) {
            const int slot = q % JQ;
            if (!mbar_wait(&job_full[slot], (q / JQ) & 1, abort, err)) break;
            const int job = jobs[slot];
            asm volatile("bar.sync 2, 128;" ::: "memory");
            if (tid == 0) mbar_arrive(&job_empty[slot]);
            if (job < 0) break;
            const Job J = decode_job(a, job);
            if (J.kind != 1) continue;
            const int i = J.i, gt = J.gt, mg = J.sub;
            if (tid == 0) wait_count(&done_E[gt], (uint32_t)(a.cbs * i), abort, err);
            asm volatile("bar.sync 2, 128;" ::: "memory");
            if (*abort) break;
            // items of this part: (c, stage s, kb, m8), m8 fastest so 8 threads write 128 B
            const int items = 2 * kstages * 16 * 8;
#pragma unroll 4
            for (int it = tid; it < items; it += 128) {
                int t = it;
                const int m8 = t & 7; t >>= 3;
                const int kb = t & 15; t >>= 4;
                const int s = t % kstages;
                const int c = t / kstages;
                const int g = gt * TILE_M + mg * 8 + m8;
                const int k0 = s * KS + kb * 8;
                uint32_t xv[8];
                if (g < a.G) {
                    const uint32_t *pr = a.acc + (size_t)g * 2 * N + (size_t)c * N;
                    const int rot = (int)(__ldg(a.bar + (size_t)g * a.n1 + i) % (uint32_t)(2 * N));
                    const uint4 own0 = *(const uint4 *)(pr + k0);
                    const uint4 own1 = *(const uint4 *)(pr + k0 + 4);
                    const uint32_t own[8] = {own0.x, own0.y, own0.z, own0.w,
                                             own1.x, own1.y, own1.z, own1.w};
#pragma unroll
                    for (int e = 0; e < 8; e++) xv[e] = rot_coef(pr, N, rot, k0 + e) - own[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 8; e++) xv[e] = 0;
                }
                for (int jd = 0; jd < l; jd++) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const uint32_t lo = bf16_bits(gadget_digit(xv[e] + off, jd + 1, a.Bgbit));
                        const uint32_t hi = bf16_bits(gadget_digit(xv[e + 1] + off, jd + 1, a.Bgbit));
                        w[e / 2] = lo | (hi << 16);
                    }
                    const int r = c * l + jd;
                    const size_t blk = ((size_t)gt * 2 * l + r) * kstages + s;
                    a.digits[blk * (A_STAGE_BYTES / 16) + ((size_t)mg * 16 + kb) * 8 + m8] =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            __threadfence();
            asm volatile("bar.sync 2, 128;" ::: "memory");
            if (tid == 0) atomicAdd(&done_D[gt], 1u);
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
    uint4 *win = nullptr;   // BSK window units, [n][2l][2][4 planes][2N]
    uint32_t *sync = nullptr;  // job counter and per-tile progress counters
    size_t sync_cap = 0;       // words
    int sms = 0;
};

int tfhe_tc_supported(const tfhe_ctx *ctx) {
    const tfhe_params &p = ctx->p;
    return p.N >= 256 && p.N <= 1024 && p.N % NB == 0 && p.N % KS == 0 && p.Bgbit <= 6 &&
           (int64_t)p.l * p.N * 32 * 128 <= (1 << 24);
}

void tfhe_tc_free(tfhe_ctx *ctx) {
    if (!ctx->tc) return;
    if (ctx->tc->digits) cudaFree(ctx->tc->digits);
    if (ctx->tc->win) cudaFree(ctx->tc->win);
    if (ctx->tc->sync) cudaFree(ctx->tc->sync);
    delete ctx->tc;
    ctx->tc = nullptr;
}

static int ensure_digits(tfhe_ctx *ctx, int G) {
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    const size_t tiles = (size_t)(G + TILE_M - 1) / TILE_M;
    const size_t bytes = tiles * 2 * ctx->p.l * ctx->p.N * TILE_M * 2;
    const size_t words = 1 + 2 * tiles;
    if (words > ctx->tc->sync_cap) {
        if (ctx->tc->sync) cudaFree(ctx->tc->sync);
        ctx->tc->sync = nullptr;
        ctx->tc->sync_cap = 0;
        if (cudaMalloc(&ctx->tc->sync, words * 4) != cudaSuccess)
            return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core progress counters");
        ctx->tc->sync_cap = words;
    }
    if (bytes <= ctx->tc->digits_cap) return TFHE_OK;
    if (ctx->tc->digits) cudaFree(ctx->tc->digits);
    ctx->tc->digits = nullptr;
    ctx->tc->digits_cap = 0;
    if (cudaMalloc(&ctx->tc->digits, bytes) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core digit buffer");
    ctx->tc->digits_cap = bytes;
    return TFHE_OK;
}

// Expand the window units of the whole BSK (called when the keys are loaded).
int tfhe_tc_prepare_keys(tfhe_ctx *ctx, const uint32_t *bsk, cudaStream_t st) {
    if (!tfhe_tc_supported(ctx)) return TFHE_OK;
    const tfhe_params &p = ctx->p;
    if (!ctx->tc) ctx->tc = new TcWorkspace();
    const size_t npoly = (size_t)p.n * 2 * p.l * 2;
    if (!ctx->tc->win &&
        cudaMalloc(&ctx->tc->win, npoly * PLANES * 2 * p.N * sizeof(uint4)) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "tensor-core key windows");
    k_tc_windows<<<(unsigned)npoly, 256, 0, st>>>(bsk, p.N, ctx->tc->win);
    return tfhe_check_launch(ctx, "tc_windows");
}

int tfhe_blind_rotate_tc(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                         cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    if (!tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form: unsupported parameters");
    if (!ctx->tc || !ctx->tc->win)
        return tfhe_set_error(ctx, TFHE_ENOKEYS, "tensor-core form: key windows not prepared");
    int rc = ensure_digits(ctx, G);
    if (rc != TFHE_OK) return rc;
    const int n1 = p.n + 1;
    {
        const size_t total = (size_t)G * 2 * p.N;
        k_tc_init_acc<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(p.N, n1, G, bar, acc);
        rc = tfhe_check_launch(ctx, "tc_init_acc");
        if (rc != TFHE_OK) return rc;
    }
    const int tiles = (G + TILE_M - 1) / TILE_M;
    if (!ctx->tc->sms) {
        int sms = 0;
        TFHE_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        ctx->tc->sms = sms;
    }
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_tc_blind_rotate,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            SMEM_BYTES));
    TFHE_CUDA_TRY(ctx, cudaMemsetAsync(ctx->tc->sync, 0, (1 + 2 * (size_t)tiles) * 4, st));
    BrArgs args;
    args.N = p.N;
    args.l = p.l;
    args.Bgbit = p.Bgbit;
    args.G = G;
    args.n = p.n;
    args.n1 = n1;
    args.tiles = tiles;
    args.cbs = 2 * p.N / NB;
    args.bar = bar;
    args.acc = acc;
    args.digits = ctx->tc->digits;
    args.win = ctx->tc->win;
    args.sync = ctx->tc->sync;
    args.err = ctx->d_err;
    args.total_jobs = (long long)tiles * DPARTS +
                      (long long)(p.n - 1) * tiles * (args.cbs + DPARTS) + (long long)tiles * args.cbs;
    const long long jobs = args.total_jobs;
    const int grid = (int)(jobs < ctx->tc->sms ? jobs : ctx->tc->sms);
    StageTimer tm(ctx, TFHE_STAGE_EXTPROD_TC, st);
    k_tc_blind_rotate<<<grid, P_THREADS, SMEM_BYTES, st>>>(args);
    tm.stop();
    return tfhe_check_launch(ctx, "tc blind rotate");
}

int tfhe_cmux_tc(tfhe_ctx *ctx, const uint32_t *, const CmuxGeom &, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core CMUX not built yet");
}

int tfhe_ram_write_tc(tfhe_ctx *ctx, const uint32_t *, const uint32_t *, int, const uint32_t *,
                      uint32_t *, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core RAM write not built yet");
}
