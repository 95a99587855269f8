// cb.cu -- circuit bootstrapping (Section 2.1.2 "Circuit Bootstrapping"): a lvl0 TLWE
// of bit m becomes a lvl1 TRGSW of m, the form in which the CMUX Memory takes its
// addresses (Section 8.2).  Section 6.2(a) leaves it to the CPU because its lvl2 ring
// lives on the 64-bit torus, beyond what a 64-bit NTT prime multiplies exactly.
//
// Step 1 (k_cb_blind_rotate, one thread block per (input r, level u)): ModSwitch to
// Z_{2 N2}, BlindRotate of the test vector 1/(2 Bg^u) sum_j X^j over the lvl2 ring,
// SampleExtract, + 1/(2 Bg^u) on b: a lvl2 TLWE of m / Bg^u.
//
// Exact Torus64 external products with the NTT over P = 2^64 - 2^32 + 1: each key word
// K = K_lo + 2^32 K_hi is kept as the transforms of its two 32-bit halves.  With digits
// |d| <= Bg2/2, each half's product sum over 2 l2 rows of N2 terms is below
// 2 l2 N2 (Bg2/2) 2^32 (2^54 at l2 = 4, N2 = 2048, Bg2 = 512) < P/2 in magnitude, so its
// residue identifies the integer; the result is (V_lo + 2^32 V_hi) mod 2^64.  The
// accumulator, the l2 digit polynomials of one TRLWE column and the four product
// polynomials (a/b column x lo/hi half) stay in shared memory (160 KB at N2 = 2048).
//
// Step 2 (k_private_ks, one block per (lvl2 TLWE, function z)): the private functional
// key switch out = - sum_{i <= N2} sum_k PKSK[z][i][k][digit_k(a_i)] (a_{N2} = b), the
// digits staged in shared memory, the PKSK rows (8 KB TRLWEs at N = 1024) gathered with
// 16-byte loads.
#include "ntt.cuh"

namespace {

// Coefficient j of X^k p over Torus64 (k in [0, 2N)).
__device__ __forceinline__ uint64_t rot_coef64(const uint64_t *p, int N, int k, int j) {
    int neg = 0;
    if (k >= N) { k -= N; neg = 1; }
    const uint64_t v = j >= k ? p[j - k] : 0ull - p[j - k + N];
    return neg ? 0ull - v : v;
}

// Signed gadget digits of a Torus64 value (l levels of Bgbit bits, round to nearest,
// digits in [-Bg/2, Bg/2)) by bit extraction from u = t + offset.
__device__ __forceinline__ uint64_t gadget_offset64(int l, int Bgbit) {
    uint64_t off = 1ull << (64 - l * Bgbit - 1);
    for (int j = 1; j <= l; j++) off += (1ull << (Bgbit - 1)) << (64 - j * Bgbit);
    return off;
}

__device__ __forceinline__ int32_t gadget_digit64(uint64_t u, int j /*1-based*/, int Bgbit) {
    return (int32_t)((u >> (64 - j * Bgbit)) & ((1ull << Bgbit) - 1)) - (1 << (Bgbit - 1));
}

// residue of an integer V with |V| < P/2 -> V mod 2^64 (V - P wraps to V + 2^32 - 1)
__device__ __forceinline__ uint64_t gl_lift_u64(uint64_t v) {
    return v > (GL_P >> 1) ? v - GL_P : v;
}

// BSK2 polynomials u64[polys][N] -> NTT domain of their 32-bit halves, u64[polys][2][N]
// (lo, hi), scaled by N^{-1}.
__global__ void k_bsk2_to_ntt(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int N,
                              int logN, uint64_t n_inv, const uint64_t *__restrict__ psi) {
    extern __shared__ uint64_t sm[];  // [2][N]
    const size_t poly = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const uint64_t w = src[poly * N + k];
        sm[k] = (uint32_t)w;
        sm[N + k] = w >> 32;
    }
    __syncthreads();
    ntt_fwd(sm, 2, N, logN, psi);
    for (int k = threadIdx.x; k < 2 * N; k += blockDim.x)
        dst[poly * 2 * N + k] = gl_mul(sm[k], n_inv);
}

// PKSK [2][N2+1][t][base][W] -> [2][N2+1][t][base-1][W]: drop the v = 0 entries.
__global__ void k_pksk_relayout(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                size_t rows, int base, int W) {
    for (size_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const size_t g = r / (base - 1);
        const int v = (int)(r % (base - 1)) + 1;
        const uint32_t *s = src + (g * base + v) * (size_t)W;
        uint32_t *d = dst + r * (size_t)W;
        for (int k = threadIdx.x; k < W; k += blockDim.x) d[k] = s[k];
    }
}

// Step 1 for job = r * l + (u - 1): in u32[R][n+1] -> out u64[R][l][N2+1].
__global__ void __launch_bounds__(1024) k_cb_blind_rotate(
    int n, int N2, int logN2, int l2, int Bg2bit, int l, int Bgbit,
    const uint32_t *__restrict__ in, uint64_t *__restrict__ out,
    const uint64_t *__restrict__ bsk2, const uint64_t *__restrict__ psi_f,
    const uint64_t *__restrict__ psi_i) {
    extern __shared__ uint64_t sm[];
    uint64_t *acc = sm;                      // [2][N2]
    uint64_t *dig = acc + 2 * N2;            // [l2][N2]
    uint64_t *prod = dig + (size_t)l2 * N2;  // [2 columns][2 halves][N2]
    const int job = blockIdx.x;
    const int r = job / l, u = job % l + 1;
    const uint32_t *c = in + (size_t)r * (n + 1);
    const int M = 2 * N2;
    const int sh = 32 - (logN2 + 1);  // ModSwitch to Z_{2 N2}: round half up, 32-bit wrap
    const uint64_t mu = 1ull << (64 - u * Bgbit - 1);  // 1 / (2 Bg^u)
    const int bb = (int)((uint32_t)(c[n] + (1u << (sh - 1))) >> sh);
    for (int j = threadIdx.x; j < N2; j += blockDim.x) {
        acc[j] = 0;
        acc[N2 + j] = ((j + bb) % M) < N2 ? mu : 0ull - mu;
    }
    __syncthreads();
    const uint64_t off = gadget_offset64(l2, Bg2bit);
    const size_t per = (size_t)2 * l2 * 4 * N2;  // words of one NTT-domain BSK2_i
    for (int i = 0; i < n; i++) {
        const int a = (int)((uint32_t)(__ldg(c + i) + (1u << (sh - 1))) >> sh);
        if (a == 0) continue;  // X^0 ACC - ACC = 0: all-zero digits, the step is the identity
        const uint64_t *key = bsk2 + (size_t)i * per;
        for (int cc = 0; cc < 2; cc++) {
            const uint64_t *p = acc + (size_t)cc * N2;
            for (int j = threadIdx.x; j < N2; j += blockDim.x) {
                const uint64_t uu = rot_coef64(p, N2, a, j) - p[j] + off;
                for (int q = 0; q < l2; q++)
                    dig[(size_t)q * N2 + j] = gl_from_i32(gadget_digit64(uu, q + 1, Bg2bit));
            }
            __syncthreads();
            ntt_fwd(dig, l2, N2, logN2, psi_f);
            for (int k = threadIdx.x; k < N2; k += blockDim.x) {
                uint64_t s00 = 0, s01 = 0, s10 = 0, s11 = 0;
                if (cc) {
                    s00 = prod[k];
                    s01 = prod[N2 + k];
                    s10 = prod[2 * N2 + k];
                    s11 = prod[3 * N2 + k];
                }
                for (int q = 0; q < l2; q++) {
                    const uint64_t dv = dig[(size_t)q * N2 + k];
                    const uint64_t *kr = key + (size_t)(cc * l2 + q) * 4 * N2 + k;
                    s00 = gl_add(s00, gl_mul(dv, __ldg(kr)));           // a column, lo half
                    s01 = gl_add(s01, gl_mul(dv, __ldg(kr + N2)));      // a column, hi half
                    s10 = gl_add(s10, gl_mul(dv, __ldg(kr + 2 * N2)));  // b column, lo half
                    s11 = gl_add(s11, gl_mul(dv, __ldg(kr + 3 * N2)));  // b column, hi half
                }
                prod[k] = s00;
                prod[N2 + k] = s01;
                prod[2 * N2 + k] = s10;
                prod[3 * N2 + k] = s11;
            }
            __syncthreads();
        }
        ntt_inv(prod, 4, N2, logN2, psi_i);
        for (int j = threadIdx.x; j < N2; j += blockDim.x) {
            acc[j] += gl_lift_u64(prod[j]) + (gl_lift_u64(prod[N2 + j]) << 32);
            acc[N2 + j] += gl_lift_u64(prod[2 * N2 + j]) + (gl_lift_u64(prod[3 * N2 + j]) << 32);
        }
        __syncthreads();
    }
    // SampleExtract (coefficient 0) and + mu on b
    uint64_t *o = out + (size_t)job * (N2 + 1);
    for (int j = threadIdx.x; j < N2; j += blockDim.x) o[j] = j == 0 ? acc[0] : 0ull - acc[N2 - j];
    if (threadIdx.x == 0) o[N2] = acc[N2] + mu;
}

constexpr int PKS_THREADS = 256;
constexpr int PKS_MAXQ = 2;  // 16-byte words per thread: 2N / 4 <= PKS_THREADS * PKS_MAXQ

// Step 2: block (j, y) switches lvl2 TLWE j with function z = z0 + y and writes the
// TRLWE at out + (j / per) s_r + (j % per) s_u + z s_z (word offsets).
__global__ void __launch_bounds__(PKS_THREADS) k_private_ks(
    int N2, int t, int bb, int N, const uint64_t *__restrict__ in,
    const uint32_t *__restrict__ pksk, uint32_t *__restrict__ out, int per, int64_t s_r,
    int64_t s_u, int64_t s_z, int z0) {
    extern __shared__ uint8_t dsm[];  // digits [N2+1][t]
    const int j = blockIdx.x, z = z0 + blockIdx.y;
    const uint64_t *a = in + (size_t)j * (N2 + 1);
    const int base1 = (1 << bb) - 1;
    const uint64_t prec = 1ull << (64 - (1 + bb * t));
    for (int x = threadIdx.x; x < (N2 + 1) * t; x += blockDim.x) {
        const int i = x / t, k = x - i * t;
        dsm[x] = (uint8_t)(((a[i] + prec) >> (64 - (k + 1) * bb)) & (uint64_t)base1);
    }
    __syncthreads();
    const int W4 = (2 * N) / 4;  // 16-byte words per TRLWE
    const size_t row4 = (size_t)W4;
    const uint4 *kz = reinterpret_cast<const uint4 *>(pksk) + (size_t)z * (N2 + 1) * t * base1 * row4;
    uint4 acc[PKS_MAXQ];
#pragma unroll
    for (int q = 0; q < PKS_MAXQ; q++) acc[q] = make_uint4(0, 0, 0, 0);
    for (int x = 0; x < (N2 + 1) * t; x++) {
        const int v = dsm[x];  // the same for every thread of the block
        if (v == 0) continue;
        const uint4 *row = kz + ((size_t)x * base1 + (v - 1)) * row4;
#pragma unroll
        for (int q = 0; q < PKS_MAXQ; q++) {
            const int w = threadIdx.x + q * PKS_THREADS;
            if (w < W4) {
                const uint4 y = __ldg(row + w);
                acc[q].x -= y.x;
                acc[q].y -= y.y;
                acc[q].z -= y.z;
                acc[q].w -= y.w;
            }
        }
    }
    uint32_t *o = out + (int64_t)(j / per) * s_r + (int64_t)(j % per) * s_u + (int64_t)z * s_z;
#pragma unroll
    for (int q = 0; q < PKS_MAXQ; q++) {
        const int w = threadIdx.x + q * PKS_THREADS;
        if (w < W4) {
            o[4 * w] = acc[q].x;
            o[4 * w + 1] = acc[q].y;
            o[4 * w + 2] = acc[q].z;
            o[4 * w + 3] = acc[q].w;
        }
    }
}

size_t cb_br_smem(const tfhe_cb_params &q) { return (size_t)(2 + q.l2 + 4) * q.N2 * 8; }
size_t cb_ks_smem(const tfhe_cb_params &q) { return (size_t)(q.N2 + 1) * q.pks_t; }

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

int cb_check(tfhe_ctx *ctx, const char *what) {
    if (!ctx->has_cb_keys)
        return tfhe_set_error(ctx, TFHE_ENOKEYS, std::string(what) + ": circuit-bootstrapping keys not set");
    return TFHE_OK;
}

int launch_cb_blind_rotate(tfhe_ctx *ctx, const uint32_t *in, uint64_t *out, int R,
                           cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    const tfhe_cb_params &q = ctx->cbp;
    const size_t smem = cb_br_smem(q);
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_cb_blind_rotate,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    StageTimer tm(ctx, TFHE_STAGE_CB_BLIND_ROTATE, st);
    k_cb_blind_rotate<<<R * p.l, 1024, smem, st>>>(p.n, q.N2, ctx->logN2, q.l2, q.Bg2bit, p.l,
                                                   p.Bgbit, in, out, ctx->bsk2_ntt, ctx->psi2_fwd,
                                                   ctx->psi2_inv);
    tm.stop();
    return tfhe_check_launch(ctx, "cb_blind_rotate");
}

int launch_private_ks(tfhe_ctx *ctx, const uint64_t *in, uint32_t *out, int J, int nz, int z0,
                      int per, int64_t s_r, int64_t s_u, int64_t s_z, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    const tfhe_cb_params &q = ctx->cbp;
    const size_t smem = cb_ks_smem(q);
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_private_ks,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    StageTimer tm(ctx, TFHE_STAGE_CB_KEYSWITCH, st);
    k_private_ks<<<dim3(J, nz), PKS_THREADS, smem, st>>>(q.N2, q.pks_t, q.pks_basebit, p.N, in,
                                                         ctx->pksk, out, per, s_r, s_u, s_z, z0);
    tm.stop();
    return tfhe_check_launch(ctx, "private_keyswitch");
}

}  // namespace

extern "C" int tfhe_ctx_set_cb_keys(tfhe_ctx *ctx, const tfhe_cb_params *cbp, const uint64_t *bsk2,
                                    const uint32_t *pksk, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (!cbp || !bsk2 || !pksk)
        return tfhe_set_error(ctx, TFHE_EINVAL, "set_cb_keys: null argument");
    const tfhe_params &p = ctx->p;
    const tfhe_cb_params q = *cbp;
    int logN2 = 0;
    while ((1 << logN2) < q.N2) logN2++;
    // exactness of the split-key products: 2 l2 N2 2^(Bg2bit-1) 2^32 < 2^63
    int log2l2 = 0;
    while ((1 << log2l2) < 2 * q.l2) log2l2++;
    if (!is_pow2(q.N2) || q.N2 < 256 || q.N2 > 2048 || q.l2 < 1 || q.l2 > 8 || q.Bg2bit < 1 ||
        q.Bg2bit > 16 || q.l2 * q.Bg2bit > 63 || log2l2 + logN2 + q.Bg2bit - 1 + 32 > 62 ||
        q.pks_t < 1 || q.pks_basebit < 1 || q.pks_basebit > 8 || q.pks_t * q.pks_basebit > 32 ||
        p.l * p.Bgbit > 62 || cb_br_smem(q) > 227 * 1024 || cb_ks_smem(q) > 64 * 1024 ||
        2 * p.N > 4 * PKS_THREADS * PKS_MAXQ)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "set_cb_keys: parameters out of range");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    ctx->has_cb_keys = false;
    if (ctx->psi2_fwd && ctx->cbp.N2 != q.N2) {
        cudaFree(ctx->psi2_fwd);
        cudaFree(ctx->psi2_inv);
        ctx->psi2_fwd = ctx->psi2_inv = nullptr;
    }
    if (!ctx->psi2_fwd) {
        const int rc = tfhe_make_twiddles(ctx, q.N2, &ctx->psi2_fwd, &ctx->psi2_inv, &ctx->n2_inv);
        if (rc != TFHE_OK) return rc;
    }
    const size_t polys = (size_t)p.n * 2 * q.l2 * 2;
    const int base = 1 << q.pks_basebit;
    const size_t W = (size_t)2 * p.N;
    const size_t pk_rows = (size_t)2 * (q.N2 + 1) * q.pks_t * (base - 1);
    if (ctx->bsk2_ntt) cudaFree(ctx->bsk2_ntt);
    if (ctx->pksk) cudaFree(ctx->pksk);
    ctx->bsk2_ntt = nullptr;
    ctx->pksk = nullptr;
    if (cudaMalloc(&ctx->bsk2_ntt, polys * 2 * q.N2 * 8) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_cb_keys: NTT-domain BSK2");
    if (cudaMalloc(&ctx->pksk, pk_rows * W * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_cb_keys: private key-switching keys");
    ctx->cbp = q;
    ctx->logN2 = logN2;
    k_bsk2_to_ntt<<<(unsigned)polys, 512, 2 * q.N2 * 8, st>>>(bsk2, ctx->bsk2_ntt, q.N2, logN2,
                                                             ctx->n2_inv, ctx->psi2_fwd);
    int rc = tfhe_check_launch(ctx, "bsk2_to_ntt");
    if (rc != TFHE_OK) return rc;
    k_pksk_relayout<<<8192, 256, 0, st>>>(pksk, ctx->pksk, pk_rows, base, (int)W);
    rc = tfhe_check_launch(ctx, "pksk relayout");
    if (rc != TFHE_OK) return rc;
    ctx->has_cb_keys = true;
    return TFHE_OK;
}

extern "C" int tfhe_cb_tlwe2(tfhe_ctx *ctx, const uint32_t *in, uint64_t *out, int R,
                             void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (R < 0 || (R > 0 && (!in || !out)))
        return tfhe_set_error(ctx, TFHE_EINVAL, "cb_tlwe2: bad arguments");
    int rc = cb_check(ctx, "cb_tlwe2");
    if (rc != TFHE_OK || R == 0) return rc;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return launch_cb_blind_rotate(ctx, in, out, R, (cudaStream_t)stream);
}

extern "C" int tfhe_private_keyswitch(tfhe_ctx *ctx, const uint64_t *in, uint32_t *out, int J,
                                      int z, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (J < 0 || (z != 0 && z != 1) || (J > 0 && (!in || !out)))
        return tfhe_set_error(ctx, TFHE_EINVAL, "private_keyswitch: bad arguments");
    int rc = cb_check(ctx, "private_keyswitch");
    if (rc != TFHE_OK || J == 0) return rc;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return launch_private_ks(ctx, in, out, J, 1, z, 1, 2 * ctx->p.N, 0, 0, (cudaStream_t)stream);
}

extern "C" int tfhe_circuit_bootstrap(tfhe_ctx *ctx, const uint32_t *in, uint32_t *out, int R,
                                      void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (R < 0 || (R > 0 && (!in || !out)))
        return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_bootstrap: bad arguments");
    int rc = cb_check(ctx, "circuit_bootstrap");
    if (rc != TFHE_OK || R == 0) return rc;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const tfhe_params &p = ctx->p;
    const int J = R * p.l;
    rc = tfhe_grow(ctx, (void **)&ctx->ws_cb, &ctx->ws_cb_cap,
                   (size_t)J * (ctx->cbp.N2 + 1) * 8, "circuit_bootstrap workspace");
    if (rc != TFHE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = launch_cb_blind_rotate(ctx, in, ctx->ws_cb, R, st);
    if (rc != TFHE_OK) return rc;
    const int64_t W = 2 * p.N;
    return launch_private_ks(ctx, ctx->ws_cb, out, J, 2, 0, p.l, 2 * p.l * W, W, p.l * W, st);
}
