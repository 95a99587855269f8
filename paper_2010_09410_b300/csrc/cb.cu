// cb.cu -- circuit bootstrapping (Section 2.1.2 "Circuit Bootstrapping"): a lvl0 TLWE
// of bit m becomes a lvl1 TRGSW of m, the form in which the CMUX Memory takes its
// addresses (Section 8.2).  Section 6.2(a) leaves it to the CPU because its lvl2 ring
// lives on the 64-bit torus, beyond what a 64-bit NTT prime multiplies exactly.
//
// Step 1 (k_cb_blind_rotate, one thread block per (input r, level u)): ModSwitch to
// Z_{2 N2}, BlindRotate of the test vector 1/(2 Bg^u) sum_j X^j over the lvl2 ring,
// SampleExtract, + 1/(2 Bg^u) on b: a lvl2 TLWE of m / Bg^u.
//
// Exact Torus64 external products: each key word K = K_lo + 2^32 K_hi is kept as the
// transforms of its two 32-bit halves.  With digits |d| <= Bg2/2, each half's product sum
// over 2 l2 rows of N2 terms is below 2 l2 N2 (Bg2/2) 2^32 (2^54 at l2 = 4, N2 = 2048,
// Bg2 = 512).  It is computed by NTTs modulo two 30-bit primes and recombined by the CRT
// (ntt32.cuh; the modulus, about 2^59.4, exceeds twice the bound), so it is the integer
// itself, and (V_lo + 2^32 V_hi) mod 2^64 is the product.  The accumulator (2 x N2 u64),
// the 2 l2 digit polynomials of both TRLWE columns for both primes (transformed together;
// the four product polynomials, a/b column x lo/hi half, then overwrite the first four),
// and the twiddles stay in shared memory (224 KB at N2 = 2048); digit and product
// polynomials are stored swizzled (swz).
//
// Step 2 (k_private_ks, one block per (lvl2 TLWE, function z)): the private functional
// key switch out = - sum_{i <= N2} sum_k PKSK[z][i][k][digit_k(a_i)] (a_{N2} = b), the
// digits staged in shared memory, the PKSK rows (8 KB TRLWEs at N = 1024) gathered with
// 16-byte loads.
#include <vector>

#include "ntt32.cuh"

namespace {

// Coefficient j of X^k p over Torus64 (k in [0, 2N)).
__device__ __forceinline__ uint64_t rot_coef64(const uint64_t *p, int N, int k, int j) {
    // s = j - k in (-2N, N): p[s mod N], negated once exactly when -N <= s < 0
    const int s = j - k;
    const uint64_t neg = (uint64_t)(int64_t)((s >> 31) & ~((s + N) >> 31));  // all ones or zero
    return (p[s & (N - 1)] ^ neg) - neg;
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

// BSK2 polynomials u64[polys][N] -> the NTT-domain residues of their 32-bit halves,
// u32[polys][2 primes][2 halves][N], in Montgomery form and scaled by N^{-1}:
// f_p = N^{-1} 2^32 mod p.
__global__ void k_bsk2_to_ntt32(const uint64_t *__restrict__ src, uint32_t *__restrict__ dst,
                                int N, int logN, const uint32_t *__restrict__ tw, uint32_t f1,
                                uint32_t f2) {
    extern __shared__ uint32_t sm32[];  // [2 primes][2 halves][N]
    const size_t poly = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const uint64_t w = src[poly * N + k];
        const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
        sm32[k] = lo % NP1;
        sm32[N + k] = hi % NP1;
        sm32[2 * N + k] = lo % NP2;
        sm32[3 * N + k] = hi % NP2;
    }
    __syncthreads();
    ntt32_fwd(sm32, 2, N, logN, tw);
    for (int x = threadIdx.x; x < 4 * N; x += blockDim.x) {
        const bool pr = x >= 2 * N;
        const uint32_t p = pr ? NP2 : NP1;
        const uint32_t v = red_below(sm32[x], p);
        dst[poly * 4 * N + x] = (uint32_t)((uint64_t)v * (pr ? f2 : f1) % p);
    }
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
constexpr int CB_THREADS = 512;  // 128 registers a thread: more key loads in flight

__host__ __device__ constexpr int cb_rows(int l2) { return 2 * l2 > 4 ? 2 * l2 : 4; }

__global__ void __launch_bounds__(CB_THREADS, 1) k_cb_blind_rotate(
    int n, int N2, int logN2, int l2, int Bg2bit, int l, int Bgbit,
    const uint32_t *__restrict__ in, uint64_t *__restrict__ out,
    const uint32_t *__restrict__ bsk2, const uint32_t *__restrict__ tw) {
    extern __shared__ __align__(16) uint64_t sm[];
    const int rows = cb_rows(l2);
    uint64_t *acc = sm;                                      // [2][N2]
    uint32_t *dig = (uint32_t *)(acc + 2 * N2);              // [2 primes][rows][N2]
    uint32_t *tws = dig + (size_t)2 * rows * N2;             // twiddles [2 primes][2][N2][2]
    for (int x = threadIdx.x; x < 2 * N2; x += blockDim.x)
        reinterpret_cast<uint4 *>(tws)[x] = __ldg(reinterpret_cast<const uint4 *>(tw) + x);
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
    const size_t per = (size_t)2 * l2 * 2 * 4 * N2;  // words of one NTT-domain BSK2_i
    const size_t pplane = (size_t)rows * N2;          // words of one prime's rows
    // Every block reads the same key row at about the same time; each starts its pointwise
    // sweep at its own offset (a multiple of 32 items, so warps stay coalesced) to spread
    // the concurrent requests over the L2 slices.
    const int rot = ((blockIdx.x * 37) & ((N2 >> 5) - 1)) << 5;
    for (int i = 0; i < n; i++) {
        const int a = (int)((uint32_t)(__ldg(c + i) + (1u << (sh - 1))) >> sh);
        if (a == 0) continue;  // X^0 ACC - ACC = 0: all-zero digits, the step is the identity
        const uint32_t *key = bsk2 + (size_t)i * per;
        // digits of both columns, rows cc * l2 + q; two consecutive coefficients per thread
        for (int j = 2 * threadIdx.x; j < N2; j += 2 * blockDim.x) {
            for (int cc = 0; cc < 2; cc++) {
                const uint64_t *pa = acc + (size_t)cc * N2;
                const ulonglong2 own = *reinterpret_cast<const ulonglong2 *>(pa + j);
                const uint64_t u0 = rot_coef64(pa, N2, a, j) - own.x + off;
                const uint64_t u1 = rot_coef64(pa, N2, a, j + 1) - own.y + off;
                for (int q = 0; q < l2; q++) {
                    const int32_t d0 = gadget_digit64(u0, q + 1, Bg2bit);
                    const int32_t d1 = gadget_digit64(u1, q + 1, Bg2bit);
                    uint32_t *dr = dig + (size_t)(cc * l2 + q) * N2 + swz(j);
                    *reinterpret_cast<uint2 *>(dr) = make_uint2(res_of_i32(d0, NP1), res_of_i32(d1, NP1));
                    *reinterpret_cast<uint2 *>(dr + pplane) =
                        make_uint2(res_of_i32(d0, NP2), res_of_i32(d1, NP2));
                }
            }
        }
        __syncthreads();
        ntt32_fwd_r8(dig, 2 * l2, logN2, tws, (int)pplane);
        // pointwise: per prime and pair of coefficients, the sums over the 2 l2 rows of
        // digit x key for the four outputs (a/b column x lo/hi half), Montgomery-reduced
        // every 4 rows; the outputs overwrite rows 0..3 of the same coefficients, which
        // only this thread reads.
        for (int it0 = threadIdx.x; it0 < N2; it0 += blockDim.x) {
            const int it = (it0 + rot) & (N2 - 1);
            const int pr = it >= (N2 >> 1);
            const int k = 2 * (it - (pr ? (N2 >> 1) : 0));
            const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p, ninv = pr ? NP2_NINV : NP1_NINV;
            uint32_t *pp = dig + pr * pplane + swz(k);
            uint2 rs[4];
#pragma unroll
            for (int o = 0; o < 4; o++) rs[o] = make_uint2(0, 0);
            uint64_t ta[4] = {0, 0, 0, 0}, tb[4] = {0, 0, 0, 0};
#pragma unroll 4
            for (int rr = 0; rr < 2 * l2; rr++) {
                const uint2 dd = *reinterpret_cast<const uint2 *>(pp + (size_t)rr * N2);
                const uint32_t d0 = red_below(dd.x, p), d1 = red_below(dd.y, p);
                // key words of row rr, this prime: a column lo/hi, b column lo/hi
                const uint32_t *kr = key + ((size_t)rr * 2 * 4 + pr * 2) * N2 + k;
                const uint2 k0 = __ldg(reinterpret_cast<const uint2 *>(kr));
                const uint2 k1 = __ldg(reinterpret_cast<const uint2 *>(kr + N2));
                const uint2 k2 = __ldg(reinterpret_cast<const uint2 *>(kr + 4 * N2));
                const uint2 k3 = __ldg(reinterpret_cast<const uint2 *>(kr + 5 * N2));
                ta[0] += (uint64_t)d0 * k0.x;
                tb[0] += (uint64_t)d1 * k0.y;
                ta[1] += (uint64_t)d0 * k1.x;
                tb[1] += (uint64_t)d1 * k1.y;
                ta[2] += (uint64_t)d0 * k2.x;
                tb[2] += (uint64_t)d1 * k2.y;
                ta[3] += (uint64_t)d0 * k3.x;
                tb[3] += (uint64_t)d1 * k3.y;
                if ((rr & 3) == 3 || rr == 2 * l2 - 1) {  // < 4 p^2 < p 2^32: reduce
#pragma unroll
                    for (int o = 0; o < 4; o++) {
                        rs[o].x = red_below(rs[o].x + redc32(ta[o], p, ninv), p2);
                        rs[o].y = red_below(rs[o].y + redc32(tb[o], p, ninv), p2);
                        ta[o] = tb[o] = 0;
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 4; o++) *reinterpret_cast<uint2 *>(pp + (size_t)o * N2) = rs[o];
        }
        __syncthreads();
        ntt32_inv_r8(dig, 4, logN2, tws, (int)pplane);
        for (int j = threadIdx.x; j < N2; j += blockDim.x) {
#pragma unroll
            for (int col = 0; col < 2; col++) {
                const size_t o_lo = (size_t)(col * 2) * N2 + swz(j), o_hi = o_lo + N2;
                const int64_t vlo = crt_centred(red_below(dig[o_lo], NP1),
                                                red_below(dig[pplane + o_lo], NP2));
                const int64_t vhi = crt_centred(red_below(dig[o_hi], NP1),
                                                red_below(dig[pplane + o_hi], NP2));
                acc[(size_t)col * N2 + j] += (uint64_t)vlo + ((uint64_t)vhi << 32);
            }
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

int bitrev32(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// smallest generator of Z_p^*: g^((p-1)/f) != 1 for every prime factor f of p - 1
uint32_t primitive_root(uint32_t p) {
    std::vector<uint32_t> fs;
    uint32_t m = p - 1;
    for (uint32_t f = 2; f * f <= m; f++)
        if (m % f == 0) {
            fs.push_back(f);
            while (m % f == 0) m /= f;
        }
    if (m > 1) fs.push_back(m);
    for (uint32_t g = 2;; g++) {
        bool ok = true;
        for (uint32_t f : fs) ok = ok && powmod64(g, (p - 1) / f, p) != 1;
        if (ok) return g;
    }
}

// u64 accumulator, digits (then products) of both primes (u32), twiddles [2][2][N2][2] (u32)
size_t cb_br_smem(const tfhe_cb_params &q) { return (size_t)(2 + cb_rows(q.l2) + 4) * q.N2 * 8; }
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
    k_cb_blind_rotate<<<R * p.l, CB_THREADS, smem, st>>>(p.n, q.N2, ctx->logN2, q.l2, q.Bg2bit, p.l,
                                                   p.Bgbit, in, out, ctx->bsk2_ntt, ctx->cb_tw);
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

int tfhe_make_twiddles32(tfhe_ctx *ctx, int N, uint32_t **tw) {
    int logN = 0;
    while ((1 << logN) < N) logN++;
    std::vector<uint32_t> h((size_t)2 * 4 * N);
    const uint32_t primes[2] = {NP1, NP2};
    for (int pr = 0; pr < 2; pr++) {
        const uint32_t p = primes[pr];
        if ((p - 1) % (2 * (uint32_t)N) != 0)
            return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no 2N-th root of unity mod the NTT prime");
        const uint64_t psi = powmod64(primitive_root(p), (p - 1) / (2 * (uint64_t)N), p);
        if (powmod64(psi, N, p) != p - 1)
            return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no primitive 2N-th root of unity");
        const uint64_t psi_inv = powmod64(psi, p - 2, p);
        uint32_t *T = h.data() + (size_t)pr * 4 * N;
        for (int k = 0; k < N; k++) {
            const uint32_t w = (uint32_t)powmod64(psi, bitrev32(k, logN), p);
            const uint32_t wi = (uint32_t)powmod64(psi_inv, bitrev32(k, logN), p);
            T[2 * k] = w;
            T[2 * k + 1] = (uint32_t)(((uint64_t)w << 32) / p);
            T[2 * N + 2 * k] = wi;
            T[2 * N + 2 * k + 1] = (uint32_t)(((uint64_t)wi << 32) / p);
        }
    }
    if (cudaMalloc(tw, h.size() * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "twiddle tables");
    TFHE_CUDA_TRY(ctx, cudaMemcpy(*tw, h.data(), h.size() * 4, cudaMemcpyHostToDevice));
    return TFHE_OK;
}

extern "C" int tfhe_ctx_set_cb_keys(tfhe_ctx *ctx, const tfhe_cb_params *cbp, const uint64_t *bsk2,
                                    const uint32_t *pksk, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (!cbp || !bsk2 || !pksk)
        return tfhe_set_error(ctx, TFHE_EINVAL, "set_cb_keys: null argument");
    const tfhe_params &p = ctx->p;
    const tfhe_cb_params q = *cbp;
    int logN2 = 0;
    while ((1 << logN2) < q.N2) logN2++;
    // exactness of the split-key products: 2 l2 N2 2^(Bg2bit-1) 2^32 <= 2^58 < P1 P2 / 2
    int log2l2 = 0;
    while ((1 << log2l2) < 2 * q.l2) log2l2++;
    if (!is_pow2(q.N2) || q.N2 < 256 || q.N2 > 2048 || q.l2 < 1 || q.l2 > 8 || q.Bg2bit < 1 ||
        q.Bg2bit > 16 || q.l2 * q.Bg2bit > 63 || log2l2 + logN2 + q.Bg2bit - 1 + 32 > 58 ||
        q.pks_t < 1 || q.pks_basebit < 1 || q.pks_basebit > 8 || q.pks_t * q.pks_basebit > 32 ||
        p.l * p.Bgbit > 62 || cb_br_smem(q) > 227 * 1024 || cb_ks_smem(q) > 64 * 1024 ||
        2 * p.N > 4 * PKS_THREADS * PKS_MAXQ)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "set_cb_keys: parameters out of range");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    ctx->has_cb_keys = false;
    if (ctx->cb_tw && ctx->cbp.N2 != q.N2) {
        cudaFree(ctx->cb_tw);
        ctx->cb_tw = nullptr;
    }
    if (!ctx->cb_tw) {
        const int rc = tfhe_make_twiddles32(ctx, q.N2, &ctx->cb_tw);
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
    if (cudaMalloc(&ctx->bsk2_ntt, polys * 4 * q.N2 * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_cb_keys: NTT-domain BSK2");
    if (cudaMalloc(&ctx->pksk, pk_rows * W * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_cb_keys: private key-switching keys");
    ctx->cbp = q;
    ctx->logN2 = logN2;
    const uint32_t ninv1 = (uint32_t)powmod64(q.N2, NP1 - 2, NP1);
    const uint32_t ninv2 = (uint32_t)powmod64(q.N2, NP2 - 2, NP2);
    const uint32_t f1 = (uint32_t)(((uint64_t)ninv1 << 32) % NP1);  // N2^{-1} 2^32 mod P1
    const uint32_t f2 = (uint32_t)(((uint64_t)ninv2 << 32) % NP2);
    k_bsk2_to_ntt32<<<(unsigned)polys, 512, 4 * q.N2 * 4, st>>>(bsk2, ctx->bsk2_ntt, q.N2, logN2,
                                                               ctx->cb_tw, f1, f2);
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
