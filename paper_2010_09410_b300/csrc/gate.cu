// gate.cu -- the bootstrapped-gate path around BlindRotate: the gate's linear
// combination with ModSwitch (first kernel), and SampleExtract with the identity key
// switch (last kernel); plus the public gate, blind-rotate, CMUX-batch and host-buffer
// entry points.
#include "common.cuh"

// One block per gate: bar[g][k] = ModSwitch(combination_k), k <= n.  ModSwitch rounds
// x * 2N / 2^32 half up with 32-bit wrap (shift s = 32 - log2(2N)).
__global__ void k_combine_modswitch(int n, int shift, const uint32_t *__restrict__ in,
                                    int64_t num_in, const uint8_t *__restrict__ types,
                                    const int32_t *__restrict__ idx, uint32_t *__restrict__ bar,
                                    int *err) {
    const int64_t g = blockIdx.x;
    uint32_t *o = bar + g * (n + 1);
    if (!gate_ok(types, idx, num_in, g)) {
        if (threadIdx.x == 0) atomicCAS(err, 0, TFHE_EINVAL);
        for (int k = threadIdx.x; k <= n; k += blockDim.x) o[k] = 0;
        return;
    }
    const int t = types[g];
    const uint32_t *c1 = in + (int64_t)idx[2 * g] * (n + 1);
    const uint32_t *c2 = in + (int64_t)idx[2 * g + 1] * (n + 1);
    uint32_t kappa, s1, s2;
    gate_coeffs(t, kappa, s1, s2);
    const uint32_t half = 1u << (shift - 1);
    for (int k = threadIdx.x; k <= n; k += blockDim.x) {
        uint32_t x = s1 * c1[k] + s2 * c2[k];
        if (k == n) x += kappa;
        o[k] = (x + half) >> shift;
    }
}

// bar[g][k] = ModSwitch(in[g][k]) for G rows of n+1 words (a bootstrap of the TLWE
// itself: the refresh of Section 8.2's write bars).
__global__ void k_modswitch_rows(int n1, int shift, int64_t G, const uint32_t *__restrict__ in,
                                 uint32_t *__restrict__ bar) {
    const size_t total = (size_t)G * n1;
    const uint32_t rnd = 1u << (shift - 1);
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x)
        bar[e] = (in[e] + rnd) >> shift;
}

int tfhe_launch_modswitch_rows(tfhe_ctx *ctx, const uint32_t *in, uint32_t *bar, int64_t G,
                               cudaStream_t st) {
    k_modswitch_rows<<<1184, 256, 0, st>>>(ctx->p.n + 1, 32 - (ctx->logN + 1), G, in, bar);
    return tfhe_check_launch(ctx, "modswitch_rows");
}

int tfhe_blind_rotate_form(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G, int form,
                           cudaStream_t st);

// ---- HomMUX: c ? a : b as two bootstraps, c AND a and (not c) AND b, whose TRLWEs are
// summed with (0, 1/8 X^0) (Section 2.1.2 "HomMUX without SE and IKS"); SampleExtract
// and the identity key switch of the sum give the TLWE gate output.
__device__ __forceinline__ bool mux_ok(const int32_t *idx3, int64_t num_in, int64_t g) {
    const int32_t s = idx3[3 * g], a = idx3[3 * g + 1], b = idx3[3 * g + 2];
    return s >= 0 && a >= 0 && b >= 0 && s < num_in && a < num_in && b < num_in;
}

// Block h: half h & 1 of MUX h >> 1 (0: c AND a, 1: (not c) AND b), combined and
// ModSwitched like k_combine_modswitch.
__global__ void k_mux_combine_modswitch(int n, int shift, const uint32_t *__restrict__ in,
                                        int64_t num_in, const int32_t *__restrict__ idx3,
                                        uint32_t *__restrict__ bar, int *err) {
    const int64_t h = blockIdx.x, g = h >> 1;
    const int half = (int)(h & 1);
    uint32_t *o = bar + h * (n + 1);
    if (!mux_ok(idx3, num_in, g)) {
        if (threadIdx.x == 0) atomicCAS(err, 0, TFHE_EINVAL);
        for (int k = threadIdx.x; k <= n; k += blockDim.x) o[k] = 0;
        return;
    }
    const uint32_t *cs = in + (int64_t)idx3[3 * g] * (n + 1);
    const uint32_t *x = in + (int64_t)idx3[3 * g + 1 + half] * (n + 1);
    const uint32_t sc = half ? 0xFFFFFFFFu : 1u;  // -c for the (not c) half
    const uint32_t kappa = 0u - (1u << 29);       // -1/8 (AND, ANDNY)
    const uint32_t rnd = 1u << (shift - 1);
    for (int k = threadIdx.x; k <= n; k += blockDim.x) {
        uint32_t v = sc * cs[k] + x[k];
        if (k == n) v += kappa;
        o[k] = (v + rnd) >> shift;
    }
}

// out[g] = acc[2g] + acc[2g+1] + (0, mu X^0); all zero for a MUX with a bad index.
__global__ void k_mux_sum(int N, int G, const uint32_t *__restrict__ acc, int64_t num_in,
                          const int32_t *__restrict__ idx3, uint32_t *__restrict__ out) {
    const size_t total = (size_t)G * 2 * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t g = e / (2 * N);
        const int w = (int)(e % (2 * N));
        uint32_t v = 0;
        if (mux_ok(idx3, num_in, (int64_t)g)) {
            v = acc[(2 * g) * 2 * N + w] + acc[(2 * g + 1) * 2 * N + w];
            if (w == N) v += 1u << 29;
        }
        out[e] = v;
    }
}

// SampleExtract + identity key switch for GT gates per block.  Thread c owns the
// 16-byte column c of the lvl0 ciphertext (words 4c..4c+3 of the padded row).
//   phase 1: unsigned key-switching digits of every extracted mask coefficient
//            a'_0 = a_0, a'_i = -a_{N-i}, rounded to t digits of basebit bits;
//   phase 2: res -= KSK[i][j][digit] over all (i, j) with a nonzero digit;
//   phase 3: out = (0, b') - ... with b' = b_0.
// Gates with a bad type or index (when types != nullptr) get an all-zero output.
template <int GT>
__global__ void __launch_bounds__(160) k_extract_keyswitch(
    int n, int N, int t, int bb, int n_pad, const uint32_t *__restrict__ acc,
    const uint4 *__restrict__ ksk, uint32_t *__restrict__ out, int G,
    const uint8_t *__restrict__ types, const int32_t *__restrict__ idx, int64_t num_in) {
    extern __shared__ uint8_t dig[];  // [N * t][GT]
    const int g0 = blockIdx.x * GT;
    const uint32_t prec = 1u << (32 - (1 + bb * t));
    const uint32_t mask = (1u << bb) - 1;
    for (int e = threadIdx.x; e < GT * N; e += blockDim.x) {
        const int g = e / N, i = e % N;
        uint32_t a = 0;
        bool live = g0 + g < G;
        if (live && types) live = gate_ok(types, idx, num_in, g0 + g);
        if (live) {
            const uint32_t *A = acc + (size_t)(g0 + g) * 2 * N;
            a = (i == 0) ? A[0] : 0u - A[N - i];
        }
        const uint32_t ab = a + prec;
        for (int j = 0; j < t; j++)
            dig[((size_t)i * t + j) * GT + g] = live ? (uint8_t)((ab >> (32 - (j + 1) * bb)) & mask) : 0;
    }
    __syncthreads();
    const int c = threadIdx.x;
    const int ncol = n_pad >> 2;
    if (c >= ncol) return;
    uint4 res[GT];
#pragma unroll
    for (int g = 0; g < GT; g++) res[g] = make_uint4(0, 0, 0, 0);
    const int base1 = (1 << bb) - 1;
    const int rows = N * t;
    for (int ij = 0; ij < rows; ij++) {
        uint8_t d[GT];
        if (GT == 8) {
            const uint64_t w = *(const uint64_t *)(dig + (size_t)ij * GT);
#pragma unroll
            for (int g = 0; g < GT; g++) d[g] = (uint8_t)(w >> (8 * g));
        } else {
#pragma unroll
            for (int g = 0; g < GT; g++) d[g] = dig[(size_t)ij * GT + g];
        }
        const uint4 *rowbase = ksk + ((size_t)ij * base1) * ncol + c;
#pragma unroll
        for (int g = 0; g < GT; g++) {
            if (d[g]) {
                const uint4 k = __ldg(rowbase + (size_t)(d[g] - 1) * ncol);
                res[g].x += k.x;
                res[g].y += k.y;
                res[g].z += k.z;
                res[g].w += k.w;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < GT; g++) {
        const int gg = g0 + g;
        if (gg >= G) break;
        bool live = true;
        if (types) live = gate_ok(types, idx, num_in, gg);
        const uint32_t bprime = live ? acc[(size_t)gg * 2 * N + N] : 0u;
        uint32_t *o = out + (size_t)gg * (n + 1);
        const uint32_t v[4] = {res[g].x, res[g].y, res[g].z, res[g].w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = 4 * c + q;
            if (k <= n) o[k] = live ? ((k == n ? bprime : 0u) - v[q]) : 0u;
        }
    }
}

static constexpr int KS_GT = 8;

// Key switching with basebit = 2: the per-gate kernel above with the block's 8 gates'
// 2-bit digits packed into one 16-bit word per key-switch row (gate g in bits 2g, 2g+1),
// so the block's digits take N*t*2 bytes of shared memory instead of N*t*8 and several
// blocks share an SM.  Digits, order and sums are those of the per-gate kernel.
constexpr int KS2_GT = 8;
__global__ void __launch_bounds__(160, 6) k_extract_keyswitch_b2(
    int n, int N, int t, int n_pad, const uint32_t *__restrict__ acc, const uint4 *__restrict__ ksk,
    uint32_t *__restrict__ out, int G, const uint8_t *__restrict__ types,
    const int32_t *__restrict__ idx, int64_t num_in) {
    extern __shared__ uint16_t dig16[];  // [N * t] packed digits
    __shared__ int live_s[KS2_GT];
    const int g0 = blockIdx.x * KS2_GT;
    if (threadIdx.x < KS2_GT) {
        const int g = g0 + threadIdx.x;
        bool live = g < G;
        if (live && types) live = gate_ok(types, idx, num_in, g);
        live_s[threadIdx.x] = live;
    }
    __syncthreads();
    const uint32_t prec = 1u << (32 - (1 + 2 * t));
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // t <= 8 (checked by the host)
#pragma unroll
        for (int g = 0; g < KS2_GT; g++) {
            if (!live_s[g]) continue;
            const uint32_t *A = acc + (size_t)(g0 + g) * 2 * N;
            const uint32_t ab = ((i == 0) ? A[0] : 0u - A[N - i]) + prec;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (j < t) w[j] |= ((ab >> (32 - (j + 1) * 2)) & 3u) << (2 * g);
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (j < t) dig16[i * t + j] = (uint16_t)w[j];
    }
    __syncthreads();
    const int c = threadIdx.x;
    const int ncol = n_pad >> 2;
    if (c >= ncol) return;
    uint4 res[KS2_GT];
#pragma unroll
    for (int g = 0; g < KS2_GT; g++) res[g] = make_uint4(0, 0, 0, 0);
    const int rows = N * t;
    for (int ij = 0; ij < rows; ij++) {
        const uint32_t w = dig16[ij];
        const uint4 *rowbase = ksk + (size_t)ij * 3 * ncol + c;
#pragma unroll
        for (int g = 0; g < KS2_GT; g++) {
            const uint32_t d = (w >> (2 * g)) & 3u;
            if (d) {
                const uint4 k = __ldg(rowbase + (size_t)(d - 1) * ncol);
                res[g].x += k.x;
                res[g].y += k.y;
                res[g].z += k.z;
                res[g].w += k.w;
            }
        }
    }
#pragma unroll
    for (int g = 0; g < KS2_GT; g++) {
        const int gg = g0 + g;
        if (gg >= G) break;
        const bool live = live_s[g];
        const uint32_t bprime = live ? acc[(size_t)gg * 2 * N + N] : 0u;
        uint32_t *o = out + (size_t)gg * (n + 1);
        const uint32_t v[4] = {res[g].x, res[g].y, res[g].z, res[g].w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = 4 * c + q;
            if (k <= n) o[k] = live ? ((k == n ? bprime : 0u) - v[q]) : 0u;
        }
    }
}

// Key switching with basebit = 2, KSK rows staged through shared memory: a block of 16
// gates streams the key rows of consecutive (i, j) pairs (the base - 1 = 3 nonzero-digit
// rows of a pair are contiguous, 7,584 bytes at n = 630) into a 4-slot ring with
// cp.async.bulk, and every gate of the block adds the row its digit selects from shared
// memory (two threads per 16-byte column, eight gates each, for latency hiding).  Four
// pairs per stage (30 KB copies) in two slots, two blocks per SM: on B300 this geometry
// took the 4096-gate key switch from 4.2 ms (L1 gathers, 8 gates per block) to 3.2 ms.  Each KSK row is read from L2 once per 16 gates, instead of once per gate
// through L1.  Digits, order and sums are those of the per-gate kernel above.
constexpr int KST_GT = 16;       // gates per block (2-bit digits packed in one u32)
constexpr int KST_IJ = 4;        // (i, j) pairs per stage (30 KB copies at n = 630)
constexpr int KST_STAGES = 2;
constexpr int KST_HALF = 8;      // gates per thread: thread (h, c) adds gates 8h .. 8h+7
constexpr int KST_COLS = 160;    // threads per gate half, one per 16-byte column, n + 1 <= 640
constexpr int KST_THREADS = 2 * KST_COLS;
constexpr long long KST_WAIT_CYCLES = 4000000000LL;  // about 2 s

__device__ __forceinline__ uint32_t ks_smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool ks_wait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(ks_smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > KST_WAIT_CYCLES) return false;
    }
}

// Word k of polynomial c of gate g in the accumulators: [G][2][N], or (tiled) the
// tensor-core form's gate-fastest tiles of TFHE_TC_TILE gates.
__device__ __forceinline__ size_t acc_at(bool tiled, int N, int g, int c, int k) {
    return tiled ? (((size_t)(g / TFHE_TC_TILE) * 2 + c) * N + k) * TFHE_TC_TILE + (g % TFHE_TC_TILE)
                 : ((size_t)g * 2 + c) * N + k;
}

__global__ void __launch_bounds__(KST_THREADS, 2) k_extract_keyswitch_staged(
    int n, int N, int t, int n_pad, const uint32_t *__restrict__ acc, const uint4 *__restrict__ ksk,
    uint32_t *__restrict__ out, int G, const uint8_t *__restrict__ types,
    const int32_t *__restrict__ idx, int64_t num_in, int *err, int tiled) {
    extern __shared__ __align__(128) uint8_t ks_smem[];
    const int ncol = n_pad >> 2;                // 16-byte columns of a key row
    const int pair_u4 = 3 * ncol;               // the three rows of one (i, j) pair
    const int stage_u4 = KST_IJ * pair_u4;
    uint4 *ring = reinterpret_cast<uint4 *>(ks_smem);                   // [STAGES][stage_u4]
    uint4 *zrow = ring + KST_STAGES * stage_u4;                         // [ncol] zeros (digit 0)
    uint32_t *dig = reinterpret_cast<uint32_t *>(zrow + ncol);          // [N t]
    __shared__ __align__(8) uint64_t full[KST_STAGES];
    __shared__ int live_s[KST_GT];
    const int g0 = blockIdx.x * KST_GT;
    const int rows = N * t;
    const int nst = (rows + KST_IJ - 1) / KST_IJ;
    if (threadIdx.x == 0) {
        for (int q = 0; q < KST_STAGES; q++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ks_smem_u32(&full[q])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < KST_GT) {
        const int g = g0 + threadIdx.x;
        bool live = g < G;
        if (live && types) live = gate_ok(types, idx, num_in, g);
        live_s[threadIdx.x] = live;
    }
    __syncthreads();
    // stage s holds the rows of pairs KST_IJ s .. KST_IJ s + KST_IJ - 1 (fewer at the end)
    auto issue = [&](int s) {
        const int slot = s % KST_STAGES;
        const int ij0 = s * KST_IJ;
        const int nij = min(KST_IJ, rows - ij0);
        const uint32_t bytes = (uint32_t)nij * pair_u4 * 16;
        const uint32_t bar = ks_smem_u32(&full[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                ks_smem_u32(ring + (size_t)slot * stage_u4)),
            "l"(ksk + (size_t)ij0 * pair_u4), "r"(bytes), "r"(bar)
            : "memory");
    };
    if (threadIdx.x == 0)
        for (int s = 0; s < KST_STAGES && s < nst; s++) issue(s);
    for (int q = threadIdx.x; q < ncol; q += blockDim.x) zrow[q] = make_uint4(0, 0, 0, 0);
    // digits of the block's gates, two bits per gate (gate g at bits 2g, 2g+1)
    const uint32_t prec = 1u << (32 - (1 + 2 * t));
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // t <= 8 (checked by the host)
        // a'_i of the block's 16 gates: tiled, they are 64 contiguous bytes (g0 is a
        // multiple of 16, so of 4 words); otherwise one word per gate
        uint32_t av[KST_GT];
        if (tiled) {
            const uint4 *src = reinterpret_cast<const uint4 *>(acc + acc_at(true, N, g0, 0, i == 0 ? 0 : N - i));
#pragma unroll
            for (int q = 0; q < KST_GT / 4; q++) {
                const uint4 v = src[q];
                av[4 * q] = v.x;
                av[4 * q + 1] = v.y;
                av[4 * q + 2] = v.z;
                av[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int g = 0; g < KST_GT; g++)
                av[g] = live_s[g] ? acc[acc_at(false, N, g0 + g, 0, i == 0 ? 0 : N - i)] : 0u;
        }
#pragma unroll
        for (int g = 0; g < KST_GT; g++) {
            if (!live_s[g]) continue;
            const uint32_t ab = ((i == 0) ? av[g] : 0u - av[g]) + prec;
#pragma unroll
            for (int j = 0; j < 8; j++)
                if (j < t) w[j] |= ((ab >> (32 - (j + 1) * 2)) & 3u) << (2 * g);
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (j < t) dig[i * t + j] = w[j];
    }
    __syncthreads();
    const int c = threadIdx.x % KST_COLS, h = threadIdx.x / KST_COLS;
    uint4 res[KST_HALF];
#pragma unroll
    for (int g = 0; g < KST_HALF; g++) res[g] = make_uint4(0, 0, 0, 0);
    int s = 0;
    bool failed = false;
    for (; s < nst; s++) {
        const int slot = s % KST_STAGES;
        const bool late = !ks_wait(&full[slot], (uint32_t)(s / KST_STAGES) & 1u);
        if (c < ncol && !late) {
            const uint4 *st = ring + (size_t)slot * stage_u4 + c;
            const int ij0 = s * KST_IJ;
#pragma unroll
            for (int q = 0; q < KST_IJ; q++) {
                if (ij0 + q >= rows) break;
                const uint32_t w = dig[ij0 + q] >> (2 * KST_HALF * h);
                const uint4 *rb = st + q * pair_u4;
                // branch-free: digit 0 reads a zero row, so all loads issue before the adds
                // (measured faster than skipping those loads by predication)
                uint4 kv[KST_HALF];
#pragma unroll
                for (int g = 0; g < KST_HALF; g++) {
                    const uint32_t d = (w >> (2 * g)) & 3u;
                    kv[g] = *(d ? rb + (d - 1) * ncol : zrow + c);
                }
#pragma unroll
                for (int g = 0; g < KST_HALF; g++) {
                    res[g].x += kv[g].x;
                    res[g].y += kv[g].y;
                    res[g].z += kv[g].z;
                    res[g].w += kv[g].w;
                }
            }
        }
        // every thread is done with the slot before it is refilled; the vote is uniform
        failed = __syncthreads_or(late) != 0;
        if (failed) break;
        if (threadIdx.x == 0 && s + KST_STAGES < nst) issue(s + KST_STAGES);
    }
    if (failed) {
        // a copy did not arrive in time: record it, let the copies still in flight land
        // (bounded), and leave the outputs untouched
        if (threadIdx.x == 0) {
            atomicCAS(err, 0, TFHE_ETIMEOUT);
            for (int q = s; q < nst && q < s + KST_STAGES; q++)
                ks_wait(&full[q % KST_STAGES], (uint32_t)(q / KST_STAGES) & 1u);
        }
        __syncthreads();
        return;
    }
    if (c >= ncol) return;
#pragma unroll
    for (int g = 0; g < KST_HALF; g++) {
        const int gb = KST_HALF * h + g;  // gate within the block
        const int gg = g0 + gb;
        if (gg >= G) break;
        const bool live = live_s[gb];
        const uint32_t bprime = live ? acc[acc_at(tiled, N, gg, 1, 0)] : 0u;
        uint32_t *o = out + (size_t)gg * (n + 1);
        const uint32_t v[4] = {res[g].x, res[g].y, res[g].z, res[g].w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int k = 4 * c + q;
            if (k <= n) o[k] = live ? ((k == n ? bprime : 0u) - v[q]) : 0u;
        }
    }
}

// The staged key switch (basebit 2, t <= 8, shared memory within 110 KB) reads either
// accumulator layout; the others read [G][2][N] only.
static size_t ks_staged_smem(const tfhe_ctx *ctx) {
    const tfhe_params &p = ctx->p;
    return (size_t)KST_STAGES * KST_IJ * 3 * ctx->n_pad * 4 + (size_t)ctx->n_pad * 4 +
           (size_t)p.N * p.ks_t * 4;
}

bool tfhe_ks_reads_tiled(const tfhe_ctx *ctx) {
    return ctx->p.ks_basebit == 2 && ctx->p.ks_t <= 8 && ctx->n_pad / 4 <= KST_COLS &&
           ks_staged_smem(ctx) <= 110 * 1024;
}

static int launch_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                    const uint8_t *types, const int32_t *idx, int64_t num_in,
                                    cudaStream_t st, bool tiled = false) {
    if (tiled && !tfhe_ks_reads_tiled(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "key switch: tiled accumulators need the staged kernel");
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    const size_t smem = (size_t)p.N * p.ks_t * KS_GT;
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_extract_keyswitch<KS_GT>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    if (ctx->n_pad / 4 > 160)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "key switch: n + 1 > 640");
    if (p.ks_basebit == 2 && p.ks_t <= 8) {
        const size_t smem_st = ks_staged_smem(ctx);
        if (smem_st <= 110 * 1024) {
            TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_extract_keyswitch_staged,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)smem_st));
            StageTimer tm(ctx, TFHE_STAGE_KEYSWITCH, st);
            k_extract_keyswitch_staged<<<(G + KST_GT - 1) / KST_GT, KST_THREADS, smem_st, st>>>(
                p.n, p.N, p.ks_t, ctx->n_pad, acc, (const uint4 *)ctx->ksk, out, G, types, idx,
                num_in, ctx->d_err, tiled ? 1 : 0);
            tm.stop();
            return tfhe_check_launch(ctx, "extract_keyswitch");
        }
        const size_t smem2 = (size_t)p.N * p.ks_t * 2;
        TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_extract_keyswitch_b2,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem2));
        StageTimer tm(ctx, TFHE_STAGE_KEYSWITCH, st);
        k_extract_keyswitch_b2<<<(G + KS2_GT - 1) / KS2_GT, 160, smem2, st>>>(
            p.n, p.N, p.ks_t, ctx->n_pad, acc, (const uint4 *)ctx->ksk, out, G, types, idx, num_in);
        tm.stop();
        return tfhe_check_launch(ctx, "extract_keyswitch");
    }
    const int blocks = (G + KS_GT - 1) / KS_GT;
    StageTimer tm(ctx, TFHE_STAGE_KEYSWITCH, st);
    k_extract_keyswitch<KS_GT><<<blocks, 160, smem, st>>>(
        p.n, p.N, p.ks_t, p.ks_basebit, ctx->n_pad, acc, (const uint4 *)ctx->ksk, out, G, types,
        idx, num_in);
    tm.stop();
    return tfhe_check_launch(ctx, "extract_keyswitch");
}

static int check_form(tfhe_ctx *ctx, int form) {
    if (form == TFHE_FORM_NTT) return TFHE_OK;
    if (form == TFHE_FORM_NTT2) {
        if (!tfhe_cmux_exact(ctx) || !ctx->bsk_ntt2)
            return tfhe_set_error(ctx, TFHE_EUNSUPPORTED,
                                  "two-prime NTT form needs 2l N Bg/2 2^32 <= 2^58");
        return TFHE_OK;
    }
    if (form == TFHE_FORM_TC) {
        if (!tfhe_tc_supported(ctx))
            return tfhe_set_error(ctx, TFHE_EUNSUPPORTED,
                                  "tensor-core form needs 256 <= N <= 1024, Bgbit <= 6 and "
                                  "l * N * 32 * 128 <= 2^24");
        return TFHE_OK;
    }
    return tfhe_set_error(ctx, TFHE_EINVAL, "unknown form");
}

static int blind_rotate_dispatch(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                                 int form, cudaStream_t st, int tc_level = -1) {
    if (form == TFHE_FORM_TC) return tfhe_blind_rotate_tc(ctx, bar, acc, G, st, tc_level);
    if (form == TFHE_FORM_NTT2) return tfhe_blind_rotate_ntt2(ctx, bar, acc, G, st);
    return tfhe_blind_rotate_ntt(ctx, bar, acc, G, st);
}

int tfhe_blind_rotate_form(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G, int form,
                           cudaStream_t st) {
    return blind_rotate_dispatch(ctx, bar, acc, G, form, st);
}

extern "C" int tfhe_gate_batch(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                               const uint8_t *types, const int32_t *in_idx, uint32_t *out, int G,
                               int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    return tfhe_gate_batch_cfg(ctx, in, num_in, types, in_idx, out, G, form, -1,
                               (cudaStream_t)stream);
}

int tfhe_gate_batch_cfg(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                        const int32_t *in_idx, uint32_t *out, int G, int form, int tc_level,
                        cudaStream_t stream) {
    if (G < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch: G < 0");
    if (G == 0) return TFHE_OK;
    if (!in || !types || !in_idx || !out || num_in < 1)
        return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch: null pointer or num_in < 1");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "gate_batch: keys not set");
    if (form == -1) tfhe_pick_form(ctx, G, &form, &tc_level);  // chosen for the batch width
    int rc = check_form(ctx, form);
    if (rc != TFHE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = tfhe_ensure_workspace(ctx, G);
    if (rc != TFHE_OK) return rc;
    const tfhe_params &p = ctx->p;
    if (form == TFHE_FORM_TC && tfhe_ks_reads_tiled(ctx)) {
        // two launches: the persistent BlindRotate (its step-0 digit jobs form the gate
        // combinations and the accumulators), then the key switch reading the tiled
        // accumulators
        const TcGateInputs gin{in, num_in, types, in_idx};
        const uint32_t *acc_t = nullptr;
        rc = tfhe_blind_rotate_tc(ctx, ctx->ws_bar, nullptr, G, st, tc_level, &gin, &acc_t);
        if (rc != TFHE_OK) return rc;
        return launch_extract_keyswitch(ctx, acc_t, out, G, types, in_idx, num_in, st, true);
    }
    const int shift = 32 - (ctx->logN + 1);
    StageTimer tm(ctx, TFHE_STAGE_COMBINE, st);
    k_combine_modswitch<<<G, 256, 0, st>>>(p.n, shift, in, num_in, types, in_idx, ctx->ws_bar,
                                           ctx->d_err);
    tm.stop();
    rc = tfhe_check_launch(ctx, "combine_modswitch");
    if (rc != TFHE_OK) return rc;
    rc = blind_rotate_dispatch(ctx, ctx->ws_bar, ctx->ws_acc, G, form, st, tc_level);
    if (rc != TFHE_OK) return rc;
    return launch_extract_keyswitch(ctx, ctx->ws_acc, out, G, types, in_idx, num_in, st);
}

extern "C" int tfhe_blind_rotate(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                                 int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (G < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "blind_rotate: G < 0");
    if (G == 0) return TFHE_OK;
    if (!bar || !acc) return tfhe_set_error(ctx, TFHE_EINVAL, "blind_rotate: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "blind_rotate: keys not set");
    int level = -1;
    if (form == -1) tfhe_pick_form(ctx, G, &form, &level);  // chosen for the batch width
    int rc = check_form(ctx, form);
    if (rc != TFHE_OK) return rc;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return blind_rotate_dispatch(ctx, bar, acc, G, form, (cudaStream_t)stream, level);
}

extern "C" int tfhe_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                      void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (G < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "extract_keyswitch: G < 0");
    if (G == 0) return TFHE_OK;
    if (!acc || !out) return tfhe_set_error(ctx, TFHE_EINVAL, "extract_keyswitch: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "extract_keyswitch: no keys");
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return launch_extract_keyswitch(ctx, acc, out, G, nullptr, nullptr, 0, (cudaStream_t)stream);
}

extern "C" int tfhe_cmux_batch(tfhe_ctx *ctx, const uint32_t *trgsw, int group,
                               const uint32_t *d1, const uint32_t *d0, uint32_t *out, int B,
                               int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (B < 0 || group < 1) return tfhe_set_error(ctx, TFHE_EINVAL, "cmux_batch: B < 0 or group < 1");
    if (B == 0) return TFHE_OK;
    if (!trgsw || !d1 || !d0 || !out)
        return tfhe_set_error(ctx, TFHE_EINVAL, "cmux_batch: null pointer");
    int rc = check_form(ctx, form);
    if (rc != TFHE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int64_t N2 = 2 * (int64_t)ctx->p.N;
    const int gx = group < B ? group : B;
    const int ny = (B + group - 1) / group;
    CmuxGeom g{d1, d0, out, N2, (int64_t)group * N2, N2, (int64_t)group * N2, 1, gx, ny, B};
    // tensor-core form for groups of at least one 128-CMUX tile, else the NTT form
    if (form == TFHE_FORM_TC && gx >= TFHE_TC_TILE) return tfhe_cmux_tc(ctx, trgsw, g, st);
    rc = tfhe_ensure_trgsw_ws(ctx, (size_t)ny);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_sel_to_ntt(ctx, trgsw, ctx->ws_trgsw_ntt, (size_t)ny, st);
    if (rc != TFHE_OK) return rc;
    return tfhe_cmux_ntt(ctx, ctx->ws_trgsw_ntt, g, st);
}

static int grow(tfhe_ctx *ctx, void **ptr, size_t *cap, size_t need) {
    return tfhe_grow(ctx, ptr, cap, need, "host-API staging allocation");
}

extern "C" int tfhe_gate_batch_host(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                                    const uint8_t *types, const int32_t *in_idx, uint32_t *out,
                                    int G, int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (G < 0 || num_in < 1) return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch_host: sizes");
    if (G == 0) return TFHE_OK;
    if (!in || !types || !in_idx || !out)
        return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch_host: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t w = (size_t)ctx->p.n + 1;
    size_t in_cap = ctx->st_in_cap, gate_cap = ctx->st_gate_cap, tcap = ctx->st_gate_cap,
           icap = ctx->st_gate_cap;
    int rc = grow(ctx, (void **)&ctx->st_in, &in_cap, (size_t)num_in * w * 4);
    if (rc != TFHE_OK) return rc;
    ctx->st_in_cap = in_cap;
    if ((size_t)G * w * 4 > ctx->st_gate_cap) {
        rc = grow(ctx, (void **)&ctx->st_out, &gate_cap, (size_t)G * w * 4);
        if (rc == TFHE_OK) rc = grow(ctx, (void **)&ctx->st_types, &tcap, (size_t)G * w * 4);
        if (rc == TFHE_OK) rc = grow(ctx, (void **)&ctx->st_idx, &icap, (size_t)G * w * 4);
        if (rc != TFHE_OK) {
            ctx->st_gate_cap = 0;
            return rc;
        }
        ctx->st_gate_cap = gate_cap;
    }
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->st_in, in, (size_t)num_in * w * 4,
                                       cudaMemcpyHostToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->st_types, types, (size_t)G, cudaMemcpyHostToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->st_idx, in_idx, (size_t)G * 8, cudaMemcpyHostToDevice,
                                       st));
    rc = tfhe_gate_batch(ctx, ctx->st_in, num_in, ctx->st_types, ctx->st_idx, ctx->st_out, G, form,
                         stream);
    if (rc != TFHE_OK) return rc;
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->st_out, (size_t)G * w * 4,
                                       cudaMemcpyDeviceToHost, st));
    TFHE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return TFHE_OK;
}

// Launch helpers for entry points that supply their own scratch (noalloc.cu): the
// same launches tfhe_gate_batch makes, on caller-chosen buffers.
int tfhe_launch_combine(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                        const int32_t *in_idx, uint32_t *bar, int G, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    const int shift = 32 - (ctx->logN + 1);
    StageTimer tm(ctx, TFHE_STAGE_COMBINE, st);
    k_combine_modswitch<<<G, 256, 0, st>>>(p.n, shift, in, num_in, types, in_idx, bar, ctx->d_err);
    tm.stop();
    return tfhe_check_launch(ctx, "combine_modswitch");
}

int tfhe_launch_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                  const uint8_t *types, const int32_t *idx, int64_t num_in,
                                  cudaStream_t st) {
    return launch_extract_keyswitch(ctx, acc, out, G, types, idx, num_in, st);
}

// Load the combination and key-switch kernels now (lazy module loading would otherwise
// load their code, allocating device memory, at their first launch).
int tfhe_preload_gate_kernels(tfhe_ctx *ctx) {
    cudaFuncAttributes fa;
    TFHE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_combine_modswitch));
    TFHE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_extract_keyswitch_staged));
    TFHE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_extract_keyswitch_b2));
    TFHE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_extract_keyswitch<KS_GT>));
    return TFHE_OK;
}

// ---- HomMUX batches ----------------------------------------------------------------

static int mux_batch(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const int32_t *idx3,
                     uint32_t *out, int G, int form, bool noks, cudaStream_t st) {
    if (G < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "mux_batch: G < 0");
    if (G == 0) return TFHE_OK;
    if (!in || !idx3 || !out || num_in < 1)
        return tfhe_set_error(ctx, TFHE_EINVAL, "mux_batch: null pointer or num_in < 1");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "mux_batch: keys not set");
    if ((int64_t)G * 2 > 0x7FFFFFFF) return tfhe_set_error(ctx, TFHE_EINVAL, "mux_batch: G too large");
    if (form == -1) {  // chosen for the width of the 2G bootstraps
        int lv = -1;
        tfhe_pick_form(ctx, 2 * (int64_t)G, &form, &lv);
    }
    int rc = check_form(ctx, form);
    if (rc != TFHE_OK) return rc;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    rc = tfhe_ensure_workspace(ctx, 2 * G);  // two bootstraps per MUX
    if (rc != TFHE_OK) return rc;
    const tfhe_params &p = ctx->p;
    const int shift = 32 - (ctx->logN + 1);
    {
        StageTimer tm(ctx, TFHE_STAGE_COMBINE, st);
        k_mux_combine_modswitch<<<2 * G, 256, 0, st>>>(p.n, shift, in, num_in, idx3, ctx->ws_bar,
                                                       ctx->d_err);
        tm.stop();
        rc = tfhe_check_launch(ctx, "mux_combine_modswitch");
        if (rc != TFHE_OK) return rc;
    }
    rc = blind_rotate_dispatch(ctx, ctx->ws_bar, ctx->ws_acc, 2 * G, form, st);
    if (rc != TFHE_OK) return rc;
    uint32_t *sum = noks ? out : ctx->ws_tmp;
    {
        StageTimer tm(ctx, TFHE_STAGE_COMBINE, st);
        k_mux_sum<<<1184, 256, 0, st>>>(p.N, G, ctx->ws_acc, num_in, idx3, sum);
        tm.stop();
        rc = tfhe_check_launch(ctx, "mux_sum");
        if (rc != TFHE_OK) return rc;
    }
    if (noks) return TFHE_OK;
    return launch_extract_keyswitch(ctx, ctx->ws_tmp, out, G, nullptr, nullptr, 0, st);
}

int tfhe_mux_batch_impl(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const int32_t *idx3,
                        uint32_t *out, int G, int form, bool noks, cudaStream_t st) {
    return mux_batch(ctx, in, num_in, idx3, out, G, form, noks, st);
}

extern "C" int tfhe_mux_batch(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                              const int32_t *idx3, uint32_t *out, int G, int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    return mux_batch(ctx, in, num_in, idx3, out, G, form, false, (cudaStream_t)stream);
}

extern "C" int tfhe_mux_batch_noks(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                                   const int32_t *idx3, uint32_t *out_trlwe, int G, int form,
                                   void *stream) {
    if (!ctx) return TFHE_EINVAL;
    return mux_batch(ctx, in, num_in, idx3, out_trlwe, G, form, true, (cudaStream_t)stream);
}
