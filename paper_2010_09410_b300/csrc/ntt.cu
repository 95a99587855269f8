// ntt.cu -- the plain per-gate form: BlindRotate and CMUX with each external product
// computed by an exact negacyclic NTT over P = 2^64 - 2^32 + 1 (the GPU TFHE library
// form of Section 6.2(a)).  One thread block owns one gate (or one CMUX): its
// accumulator, digit polynomials and transforms live in shared memory for all n steps.
//
// Exactness: a product sum_r d_r * k_r with |d| <= Bg/2, key words < 2^32 and 2l rows
// of N terms is below 2l * N * (Bg/2) * 2^32 (< 2^50 for l = 3, N = 1024, Bg = 64) <
// P/2 in magnitude, so its residue mod P identifies the integer, which is then
// reduced mod 2^32 (gl_lift_u32).
#include "ntt.cuh"
#include "ntt32.cuh"

// ---------------------------------------------------------------------------
// Host: twiddles
// ---------------------------------------------------------------------------

static uint64_t h_mulmod(uint64_t a, uint64_t b) {
    return (uint64_t)((unsigned __int128)a * b % GL_P);
}

static uint64_t h_powmod(uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
        if (e & 1) r = h_mulmod(r, a);
        a = h_mulmod(a, a);
        e >>= 1;
    }
    return r;
}

static int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

int tfhe_make_twiddles(tfhe_ctx *ctx, int N, uint64_t **fwd, uint64_t **inv, uint64_t *n_inv) {
    int logN = 0;
    while ((1 << logN) < N) logN++;
    // 7 generates the multiplicative group of Z_P (order 2^32 (2^32 - 1)).
    const uint64_t psi = h_powmod(7, (GL_P - 1) / (2 * (uint64_t)N));
    if (h_powmod(psi, N) != GL_P - 1)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "no primitive 2N-th root of unity");
    const uint64_t psi_inv = h_powmod(psi, GL_P - 2);
    std::vector<uint64_t> f(N), g(N);
    for (int k = 0; k < N; k++) {
        f[k] = h_powmod(psi, (uint64_t)bitrev(k, logN));
        g[k] = h_powmod(psi_inv, (uint64_t)bitrev(k, logN));
    }
    *n_inv = h_powmod((uint64_t)N, GL_P - 2);
    if (cudaMalloc(fwd, N * 8) != cudaSuccess || cudaMalloc(inv, N * 8) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "twiddle tables");
    TFHE_CUDA_TRY(ctx, cudaMemcpy(*fwd, f.data(), N * 8, cudaMemcpyHostToDevice));
    TFHE_CUDA_TRY(ctx, cudaMemcpy(*inv, g.data(), N * 8, cudaMemcpyHostToDevice));
    return TFHE_OK;
}

int tfhe_ntt_setup(tfhe_ctx *ctx) {
    const int rc = tfhe_make_twiddles(ctx, ctx->p.N, &ctx->psi_fwd, &ctx->psi_inv, &ctx->n_inv);
    if (rc != TFHE_OK) return rc;
    return tfhe_make_twiddles32(ctx, ctx->p.N, &ctx->tw32);
}

// Polynomials (u32 words as integers in [0, 2^32)) -> NTT domain scaled by N^{-1}.
__global__ void k_polys_to_ntt(const uint32_t *__restrict__ src, uint64_t *__restrict__ dst,
                               int N, int logN, uint64_t n_inv,
                               const uint64_t *__restrict__ psi) {
    extern __shared__ uint64_t sm[];
    const size_t poly = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) sm[k] = src[poly * N + k];
    __syncthreads();
    ntt_fwd(sm, 1, N, logN, psi);
    for (int k = threadIdx.x; k < N; k += blockDim.x) dst[poly * N + k] = gl_mul(sm[k], n_inv);
}

// External product of the TRLWE `d` (u32[2][N] in shared memory) by an NTT-domain
// TRGSW `key` (u64[2l][2][N]): prod (u64[2][N], shared) receives C (.) d in
// coefficient form, as residues.  `dig` is u64[2l][N] shared scratch.  Digit rows:
// j < l from the a-polynomial (paired with TRGSW row j), l + j from b.
__device__ __forceinline__ void extprod_ntt(const uint32_t *d, const uint64_t *__restrict__ key,
                                            uint64_t *dig, uint64_t *prod, int N, int logN,
                                            int l, int Bgbit, const uint64_t *__restrict__ psi_f,
                                            const uint64_t *__restrict__ psi_i) {
    const uint32_t off = gadget_offset(l, Bgbit);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        for (int c = 0; c < 2; c++) {
            const uint32_t u = d[c * N + j] + off;
            for (int r = 0; r < l; r++)
                dig[(size_t)(c * l + r) * N + j] = gl_from_i32(gadget_digit(u, r + 1, Bgbit));
        }
    }
    __syncthreads();
    ntt_fwd(dig, 2 * l, N, logN, psi_f);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        uint64_t s0 = 0, s1 = 0;
        for (int r = 0; r < 2 * l; r++) {
            const uint64_t dv = dig[(size_t)r * N + k];
            s0 = gl_add(s0, gl_mul(dv, __ldg(key + (size_t)(r * 2 + 0) * N + k)));
            s1 = gl_add(s1, gl_mul(dv, __ldg(key + (size_t)(r * 2 + 1) * N + k)));
        }
        prod[k] = s0;
        prod[N + k] = s1;
    }
    __syncthreads();
    ntt_inv(prod, 2, N, logN, psi_i);
}

// One block per gate: BlindRotate of the test vector by (a~, b~) = bar[g].
__global__ void __launch_bounds__(1024) k_blind_rotate_ntt(
    int n, int N, int logN, int l, int Bgbit, const uint32_t *__restrict__ bar,
    uint32_t *__restrict__ acc_out, const uint64_t *__restrict__ bsk,
    const uint64_t *__restrict__ psi_f, const uint64_t *__restrict__ psi_i) {
    extern __shared__ uint64_t sm[];
    uint64_t *dig = sm;                                  // [2l][N]
    uint64_t *prod = sm + (size_t)2 * l * N;             // [2][N]
    uint32_t *acc = (uint32_t *)(prod + (size_t)2 * N);  // [2][N]
    uint32_t *diff = acc + 2 * N;                        // [2][N]
    const size_t g = blockIdx.x;
    const uint32_t *mb = bar + g * (n + 1);
    const uint32_t mu = 1u << 29;
    const int N2 = 2 * N;
    const int bb = (int)(mb[n] % (uint32_t)N2);
    // ACC = X^{-b~} (0, v): coefficient j of X^{-b~} v is +mu when (j + b~) mod 2N < N.
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        acc[j] = 0;
        acc[N + j] = ((j + bb) % N2) < N ? mu : 0u - mu;
    }
    __syncthreads();
    const size_t per = (size_t)2 * l * 2 * N;
    for (int i = 0; i < n; i++) {
        const int a = (int)(mb[i] % (uint32_t)N2);
        if (a == 0) continue;  // X^0 ACC - ACC = 0 has all-zero digits: the step is the identity
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            diff[j] = rot_coef(acc, N, a, j) - acc[j];
            diff[N + j] = rot_coef(acc + N, N, a, j) - acc[N + j];
        }
        __syncthreads();
        extprod_ntt(diff, bsk + (size_t)i * per, dig, prod, N, logN, l, Bgbit, psi_f, psi_i);
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            acc[j] += gl_lift_u32(prod[j]);
            acc[N + j] += gl_lift_u32(prod[N + j]);
        }
        __syncthreads();
    }
    uint32_t *o = acc_out + g * 2 * N;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) o[j] = acc[j];
}

// CMUX external products (tree reads, write bars, CMUX batches) use the two-prime NTT of
// ntt32.cuh: selectors are kept as u32[2l][2][2 primes][N] residues of their NTT-domain
// polynomials (Montgomery form, scaled by N^{-1}; tfhe_sel_to_ntt).  A product sum
// sum_r d_r k_r with |d| <= Bg/2 and k < 2^32 over 2l rows of N terms is below
// 2l N (Bg/2) 2^32 (2^49.6 at l = 3, N = 1024, Bg = 64) < P1 P2 / 2, so the CRT gives it
// exactly and its residue mod 2^32 is taken.

// prod (u32[2 primes][2][N], swizzled) receives the residues of C (.) d for the TRLWE d
// (u32[2][N] in shared memory) and the selector `key`; dig is u32[2 primes][2l][N].
// The pointwise sweep starts at item rot (a multiple of 32 below N, so warps stay
// coalesced): blocks that read the same selector at about the same time pass different
// offsets (sweep_rot) and spread their requests over the L2 slices.
__device__ __forceinline__ int sweep_rot(int N) {
    return (((int)blockIdx.x * 37 + (int)blockIdx.y * 11) & ((N >> 5) - 1)) << 5;
}

__device__ __forceinline__ void extprod32(const uint32_t *d, const uint32_t *__restrict__ key,
                                          uint32_t *dig, uint32_t *prod, int N, int logN, int l,
                                          int Bgbit, const uint32_t *tw, int rot) {
    const uint32_t off = gadget_offset(l, Bgbit);
    const size_t dplane = (size_t)2 * l * N, pplane = (size_t)2 * N;
    // digits, two consecutive coefficients per thread; rows c*l + q (a, then b)
    for (int j = 2 * threadIdx.x; j < N; j += 2 * blockDim.x) {
        for (int c = 0; c < 2; c++) {
            const uint2 dv = *reinterpret_cast<const uint2 *>(d + (size_t)c * N + j);
            const uint32_t u0 = dv.x + off, u1 = dv.y + off;
            for (int q = 0; q < l; q++) {
                const int32_t d0 = gadget_digit(u0, q + 1, Bgbit), d1 = gadget_digit(u1, q + 1, Bgbit);
                const size_t row = (size_t)(c * l + q) * N + swz(j);
                *reinterpret_cast<uint2 *>(dig + row) = make_uint2(res_of_i32(d0, NP1), res_of_i32(d1, NP1));
                *reinterpret_cast<uint2 *>(dig + dplane + row) =
                    make_uint2(res_of_i32(d0, NP2), res_of_i32(d1, NP2));
            }
        }
    }
    __syncthreads();
    ntt32_fwd_r8(dig, 2 * l, logN, tw);
    // pointwise, two consecutive coefficients per thread, Montgomery-reduced every 4 rows
    for (int it0 = threadIdx.x; it0 < N; it0 += blockDim.x) {
        const int it = (it0 + rot) & (N - 1);
        const int pr = it >= (N >> 1);
        const int k = 2 * (it - (pr ? (N >> 1) : 0));
        const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p, ninv = pr ? NP2_NINV : NP1_NINV;
        uint2 rs[2] = {make_uint2(0, 0), make_uint2(0, 0)};
        uint64_t ta[2] = {0, 0}, tb[2] = {0, 0};
#pragma unroll 6
        for (int r = 0; r < 2 * l; r++) {
            const uint2 dd = *reinterpret_cast<const uint2 *>(dig + pr * dplane + (size_t)r * N + swz(k));
            const uint32_t d0 = red_below(dd.x, p), d1 = red_below(dd.y, p);
            const uint32_t *kr = key + ((size_t)r * 4 + pr) * N + k;  // [r][column][prime][N]
            const uint2 k0 = __ldg(reinterpret_cast<const uint2 *>(kr));
            const uint2 k1 = __ldg(reinterpret_cast<const uint2 *>(kr + 2 * N));
            ta[0] += (uint64_t)d0 * k0.x;
            tb[0] += (uint64_t)d1 * k0.y;
            ta[1] += (uint64_t)d0 * k1.x;
            tb[1] += (uint64_t)d1 * k1.y;
            if ((r & 3) == 3 || r == 2 * l - 1) {  // < 4 p^2 < p 2^32: reduce
#pragma unroll
                for (int o = 0; o < 2; o++) {
                    rs[o].x = red_below(rs[o].x + redc32(ta[o], p, ninv), p2);
                    rs[o].y = red_below(rs[o].y + redc32(tb[o], p, ninv), p2);
                    ta[o] = tb[o] = 0;
                }
            }
        }
        *reinterpret_cast<uint2 *>(prod + pr * pplane + swz(k)) = rs[0];
        *reinterpret_cast<uint2 *>(prod + pr * pplane + N + swz(k)) = rs[1];
    }
    __syncthreads();
    ntt32_inv_r8(prod, 2, logN, tw);
}

// word j of polynomial c of the product, mod 2^32
__device__ __forceinline__ uint32_t prod32_word(const uint32_t *prod, int N, int c, int j) {
    const size_t o = (size_t)c * N + swz(j);
    return crt_lo32(red_below(prod[o], NP1), red_below(prod[(size_t)2 * N + o], NP2));
}

// One block per CMUX (x, y) = (blockIdx.x, blockIdx.y) of the geometry g:
// out = d0 + C_y (.) (d1 - d0).  out may alias d0 or d1 of the same CMUX.
__global__ void __launch_bounds__(256) k_cmux_ntt(int N, int logN, int l, int Bgbit,
                                                  const uint64_t *__restrict__ sel, CmuxGeom g,
                                                  const uint32_t *__restrict__ tw) {
    extern __shared__ __align__(16) uint32_t smc[];
    uint32_t *dig = smc;                          // [2][2l][N]
    uint32_t *prod = dig + (size_t)2 * 2 * l * N;  // [2][2][N]
    uint32_t *diff = prod + (size_t)4 * N;         // [2][N]
    uint32_t *base = diff + 2 * N;                 // [2][N]
    const int64_t x = blockIdx.x, y = blockIdx.y;
    if (y * g.nx + x >= g.count) return;
    const uint32_t *a1 = g.d1 + x * g.dx + y * g.dy, *a0 = g.d0 + x * g.dx + y * g.dy;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) {
        const uint32_t x0 = a0[j];
        base[j] = x0;
        diff[j] = a1[j] - x0;
    }
    __syncthreads();
    const size_t per = (size_t)2 * l * 2 * N;  // one selector, in u64 units
    extprod32(diff, reinterpret_cast<const uint32_t *>(sel + (size_t)y * g.sy * per), dig, prod, N,
              logN, l, Bgbit, tw, sweep_rot(N));
    uint32_t *o = g.out + x * g.ox + y * g.oy;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x)
        o[j] = base[j] + prod32_word(prod, N, j >= N, j >= N ? j - N : j);
}

// BlindRotate of one gate by the whole block in the two-prime NTT form: ACC (shared,
// u32[2][N]) <- X^{-b~}(0, v), then for i < n: ACC += BSK_i (.) (X^{a~_i} ACC - ACC).  mb is
// the ModSwitched combination (u32[n+1], global: a~_0 .. a~_{n-1}, b~); dig, prod, diff
// are shared work areas, tws the block's twiddle copy.
__device__ __forceinline__ void br_ntt2_block(int n, int N, int logN, int l, int Bgbit,
                                              const uint32_t *mb, uint32_t *acc, uint32_t *dig,
                                              uint32_t *prod, uint32_t *diff,
                                              const uint32_t *__restrict__ bsk2p,
                                              const uint32_t *tws) {
    const uint32_t mu = 1u << 29;
    const int M = 2 * N;
    const int bb = (int)(mb[n] % (uint32_t)M);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        acc[j] = 0;
        acc[N + j] = ((j + bb) % M) < N ? mu : 0u - mu;
    }
    __syncthreads();
    const size_t per = (size_t)2 * l * 2 * 2 * N;  // words of one BSK_i
    for (int i = 0; i < n; i++) {
        const int a = (int)(mb[i] % (uint32_t)M);
        if (a == 0) continue;  // X^0 ACC - ACC = 0 has all-zero digits: the step is the identity
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            diff[j] = rot_coef(acc, N, a, j) - acc[j];
            diff[N + j] = rot_coef(acc + N, N, a, j) - acc[N + j];
        }
        __syncthreads();
        extprod32(diff, bsk2p + (size_t)i * per, dig, prod, N, logN, l, Bgbit, tws, 0);
        for (int j = threadIdx.x; j < 2 * N; j += blockDim.x)
            acc[j] += prod32_word(prod, N, j >= N, j >= N ? j - N : j);
        __syncthreads();
    }
}

// Per-gate BlindRotate in the two-prime NTT form (TFHE_FORM_NTT2): as k_blind_rotate_ntt,
// with each external product computed by extprod32 against the BSK in the two-prime NTT
// form (u32[n][2l][2][2 primes][N]).  Shared memory: digits, products, accumulator,
// rotation difference and the twiddle table (112 KB at N = 1024, l = 3).
template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_blind_rotate_ntt2(
    int n, int N, int logN, int l, int Bgbit, const uint32_t *__restrict__ bar,
    uint32_t *__restrict__ acc_out, const uint32_t *__restrict__ bsk2p,
    const uint32_t *__restrict__ tw) {
    extern __shared__ __align__(16) uint32_t smb[];
    uint32_t *dig = smb;                          // [2][2l][N]
    uint32_t *prod = dig + (size_t)4 * l * N;      // [2][2][N]
    uint32_t *acc = prod + (size_t)4 * N;          // [2][N]
    uint32_t *diff = acc + 2 * N;                  // [2][N]
    uint32_t *tws = diff + 2 * N;                  // [2][2][N][2]
    for (int x = threadIdx.x; x < 2 * N; x += blockDim.x)
        reinterpret_cast<uint4 *>(tws)[x] = __ldg(reinterpret_cast<const uint4 *>(tw) + x);
    const size_t g = blockIdx.x;
    br_ntt2_block(n, N, logN, l, Bgbit, bar + g * (n + 1), acc, dig, prod, diff, bsk2p, tws);
    uint32_t *o = acc_out + g * 2 * N;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) o[j] = acc[j];
}

// ---- dataflow engine (TfheDataflow) ------------------------------------------------

__device__ __forceinline__ int df_ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void df_st_release(int32_t *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int df_sub_acq_rel(int32_t *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(-v) : "memory");
    return old;
}
// give up a wait for a queue slot after this many cycles without any gate being queued
// (about 2 s at 2 GHz)
constexpr long long DF_STALL_CYCLES = 4000000000LL;

// SampleExtract (coefficient 0) and identity key switch of the block's accumulator
// (shared, u32[2][N]) into the TLWE `out` (u32[n+1]): a'_0 = a_0, a'_i = -a_{N-i}, b' = b_0;
// out = (0, b') - sum_{i, j} KSK[i][j][digit_j(a'_i)].  Thread (c, grp) sums 16-byte column
// c of the key rows for i = grp, grp + ngrp, ...; the groups' sums meet in `part` (shared,
// uint4[ngrp][ncol]).  KSK rows: u32[N][t][base-1][n_pad] (v = 0 dropped).
__device__ __forceinline__ void ks_block(const uint32_t *acc, int n, int N, int t, int bb,
                                         int n_pad, const uint4 *__restrict__ ksk, uint32_t *out,
                                         uint4 *part) {
    const int ncol = n_pad >> 2, ngrp = (int)blockDim.x / ncol;
    const int c = threadIdx.x % ncol, grp = threadIdx.x / ncol;
    const int base1 = (1 << bb) - 1;
    const uint32_t prec = 1u << (32 - (1 + bb * t)), mask = (1u << bb) - 1;
    if (grp < ngrp) {
        uint4 r = make_uint4(0, 0, 0, 0);
        for (int i = grp; i < N; i += ngrp) {
            const uint32_t ab = (i == 0 ? acc[0] : 0u - acc[N - i]) + prec;
            const uint4 *rows = ksk + (size_t)i * t * base1 * ncol + c;
#pragma unroll 8
            for (int j = 0; j < t; j++) {
                const uint32_t d = (ab >> (32 - (j + 1) * bb)) & mask;
                if (d) {
                    const uint4 k = __ldg(rows + ((size_t)j * base1 + d - 1) * ncol);
                    r.x += k.x;
                    r.y += k.y;
                    r.z += k.z;
                    r.w += k.w;
                }
            }
        }
        part[grp * ncol + c] = r;
    }
    __syncthreads();
    if (grp == 0) {
        uint4 r = part[c];
        for (int q = 1; q < ngrp; q++) {
            const uint4 o = part[q * ncol + c];
            r.x += o.x;
            r.y += o.y;
            r.z += o.z;
            r.w += o.w;
        }
        const uint32_t v[4] = {r.x, r.y, r.z, r.w};
        for (int q = 0; q < 4; q++) {
            const int k = 4 * c + q;
            if (k <= n) out[k] = (k == n ? acc[N] : 0u) - v[q];
        }
    }
}

// The engine: every block loops { take a ticket t; wait until queue[t] holds a gate (or
// t >= G: done); evaluate the gate; queue its consumers that became ready }.  Every gate
// is queued exactly once, after its inputs are written, and the DAG is acyclic, so a
// block that waits always has a gate coming unless the run has failed; a wait gives up
// (TFHE_ETIMEOUT) only when no gate has been queued for DF_STALL_CYCLES.
__global__ void __launch_bounds__(512, 2) k_dataflow_ntt2(
    TfheDataflow df, int n, int N, int logN, int l, int Bgbit, int t, int bb, int n_pad,
    int ms_shift, const uint32_t *__restrict__ bsk2p, const uint32_t *__restrict__ tw,
    const uint4 *__restrict__ ksk, int *err) {
    extern __shared__ __align__(16) uint32_t smb[];
    uint32_t *dig = smb;                          // [2][2l][N]
    uint32_t *prod = dig + (size_t)4 * l * N;      // [2][2][N]
    uint32_t *acc = prod + (size_t)4 * N;          // [2][N]
    uint32_t *diff = acc + 2 * N;                  // [2][N]
    uint32_t *tws = diff + 2 * N;                  // [2][2][N][2]
    __shared__ int s_gate;
    for (int x = threadIdx.x; x < 2 * N; x += blockDim.x)
        reinterpret_cast<uint4 *>(tws)[x] = __ldg(reinterpret_cast<const uint4 *>(tw) + x);
    const int n1 = n + 1;
    uint32_t *mb = df.scratch + (size_t)blockIdx.x * n1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t tk = atomicAdd(&df.ctr[0], 1u);
            int gate = -1;
            if ((int64_t)tk < df.G) {
                long long t0 = clock64();
                uint32_t seen = *(volatile uint32_t *)&df.ctr[1];
                while ((gate = df_ld_acquire(df.queue + tk)) < 0) {
                    const uint32_t now = *(volatile uint32_t *)&df.ctr[1];
                    if (now != seen) {
                        seen = now;
                        t0 = clock64();
                    } else if (clock64() - t0 > DF_STALL_CYCLES || *(volatile int *)err) {
                        atomicCAS(err, 0, TFHE_ETIMEOUT);
                        break;
                    }
                    __nanosleep(256);
                }
            }
            s_gate = gate;
        }
        __syncthreads();
        const int g = s_gate;
        if (g < 0) break;
        // combination (inputs written by other blocks of this launch: coherent loads) and
        // ModSwitch into the block's scratch row
        {
            uint32_t kappa, s1, s2;
            gate_coeffs(df.types[g], kappa, s1, s2);
            int64_t i0 = df.idx[2 * g], i1 = df.idx[2 * g + 1];
            const int64_t wires = df.num_in + df.G;
            if (!tfhe_in_bounds((size_t)i0, (size_t)wires, err)) i0 = 0;
            if (!tfhe_in_bounds((size_t)i1, (size_t)wires, err)) i1 = 0;
            const uint32_t *w0 = df.wires + (size_t)i0 * n1;
            const uint32_t *w1 = df.wires + (size_t)i1 * n1;
            for (int k = threadIdx.x; k < n1; k += blockDim.x) {
                uint32_t x = s1 * __ldcg(w0 + k) + s2 * __ldcg(w1 + k);
                if (k == n) x += kappa;
                mb[k] = (x + (1u << (ms_shift - 1))) >> ms_shift;
            }
        }
        __syncthreads();
        br_ntt2_block(n, N, logN, l, Bgbit, mb, acc, dig, prod, diff, bsk2p, tws);
        ks_block(acc, n, N, t, bb, n_pad, ksk, df.wires + (size_t)(df.num_in + g) * n1,
                 reinterpret_cast<uint4 *>(dig));
        // publish: the barrier orders the block's output stores before the leader's fence
        // (cumulative); each consumer whose last gate input this was is queued
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            for (int e = df.cons_off[g]; e < df.cons_off[g + 1]; e++) {
                const int cg = df.cons[e];
                if (!tfhe_in_bounds((size_t)cg, (size_t)df.G, err)) continue;
                if (df_sub_acq_rel(df.pending + cg, 1) == 1) {
                    const uint32_t slot = atomicAdd(&df.ctr[1], 1u);
                    if (tfhe_in_bounds(slot, (size_t)df.G, err)) df_st_release(df.queue + slot, cg);
                }
            }
        }
    }
}

// One block per RAM cell c (write bar, Section 8.2): r = new; for j < v:
// r = CMUX(S_j, r, cell_c) with S_j = C_j when bit j of c is 1 and G - C_j otherwise.
// blockIdx.y is the bit block: its controlled data is new_cell + y * new_stride and its
// cells start at cells + y * 2^v * 2N.
__global__ void __launch_bounds__(256) k_ram_write_ntt(int N, int logN, int l, int Bgbit, int v,
                                                       const uint64_t *__restrict__ c_ntt,
                                                       const uint64_t *__restrict__ gmc_ntt,
                                                       const uint32_t *__restrict__ new_cell,
                                                       int64_t new_stride, uint32_t *cells,
                                                       const uint32_t *__restrict__ tw) {
    extern __shared__ __align__(16) uint32_t smc[];
    uint32_t *dig = smc;
    uint32_t *prod = dig + (size_t)2 * 2 * l * N;
    uint32_t *diff = prod + (size_t)4 * N;
    uint32_t *r = diff + 2 * N;
    uint32_t *old = r + 2 * N;
    const size_t c = blockIdx.x;
    uint32_t *cell = cells + (((size_t)blockIdx.y << v) + c) * 2 * N;
    const uint32_t *nc = new_cell + (size_t)blockIdx.y * new_stride;
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) {
        r[j] = nc[j];
        old[j] = cell[j];
    }
    __syncthreads();
    const size_t per = (size_t)2 * l * 2 * N;
    for (int b = 0; b < v; b++) {
        for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) diff[j] = r[j] - old[j];
        __syncthreads();
        const uint64_t *S = (((c >> b) & 1) ? c_ntt : gmc_ntt) + (size_t)b * per;
        extprod32(diff, reinterpret_cast<const uint32_t *>(S), dig, prod, N, logN, l, Bgbit, tw,
                  sweep_rot(N));
        for (int j = threadIdx.x; j < 2 * N; j += blockDim.x)
            r[j] = old[j] + prod32_word(prod, N, j >= N, j >= N ? j - N : j);
        __syncthreads();
    }
    for (int j = threadIdx.x; j < 2 * N; j += blockDim.x) cell[j] = r[j];
}

// Polynomials (u32 words) -> the residues of their NTT-domain values mod both primes,
// u32[poly][2 primes][N], Montgomery form, scaled by N^{-1} (f_p = N^{-1} 2^32 mod p).
__global__ void k_polys_to_ntt32(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                 int N, int logN, const uint32_t *__restrict__ tw, uint32_t f1,
                                 uint32_t f2) {
    extern __shared__ uint32_t sp[];  // [2 primes][N]
    const size_t poly = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const uint32_t w = src[poly * N + k];
        sp[k] = w % NP1;
        sp[N + k] = w % NP2;
    }
    __syncthreads();
    ntt32_fwd(sp, 1, N, logN, tw);
    for (int x = threadIdx.x; x < 2 * N; x += blockDim.x) {
        const bool pr = x >= N;
        const uint32_t p = pr ? NP2 : NP1;
        dst[poly * 2 * N + x] = (uint32_t)((uint64_t)red_below(sp[x], p) * (pr ? f2 : f1) % p);
    }
}

int tfhe_sel_to_ntt(tfhe_ctx *ctx, const uint32_t *trgsw, uint64_t *out, size_t count,
                    cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    const size_t polys = count * 2 * p.l * 2;
    if (polys == 0) return TFHE_OK;
    const uint32_t f1 = (uint32_t)((powmod64(p.N, NP1 - 2, NP1) << 32) % NP1);
    const uint32_t f2 = (uint32_t)((powmod64(p.N, NP2 - 2, NP2) << 32) % NP2);
    k_polys_to_ntt32<<<(unsigned)polys, 256, 2 * p.N * 4, st>>>(
        trgsw, reinterpret_cast<uint32_t *>(out), p.N, ctx->logN, ctx->tw32, f1, f2);
    return tfhe_check_launch(ctx, "polys_to_ntt32");
}

bool tfhe_cmux_exact(const tfhe_ctx *ctx) {
    const tfhe_params &p = ctx->p;
    int lg = 0;
    while ((1 << lg) < 2 * p.l) lg++;
    return lg + ctx->logN + p.Bgbit - 1 + 32 <= 58;  // 2l N (Bg/2) 2^32 <= 2^58 < P1 P2 / 2
}

int tfhe_trgsw_to_ntt(tfhe_ctx *ctx, const uint32_t *trgsw, uint64_t *out, size_t count,
                      cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    const size_t polys = count * 2 * p.l * 2;
    if (polys == 0) return TFHE_OK;
    k_polys_to_ntt<<<(unsigned)polys, 256, p.N * 8, st>>>(trgsw, out, p.N, ctx->logN, ctx->n_inv,
                                                         ctx->psi_fwd);
    return tfhe_check_launch(ctx, "polys_to_ntt");
}

// Load the per-gate NTT BlindRotate kernel now (see tfhe_preload_gate_kernels).
int tfhe_preload_ntt_kernels(tfhe_ctx *ctx) {
    cudaFuncAttributes fa;
    TFHE_CUDA_TRY(ctx, cudaFuncGetAttributes(&fa, k_blind_rotate_ntt));
    return TFHE_OK;
}

int tfhe_blind_rotate_ntt(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                          cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    const size_t smem = (size_t)2 * p.l * p.N * 8 + (size_t)2 * p.N * 8 + (size_t)4 * p.N * 4;
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_blind_rotate_ntt,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    // threads per gate: measured on B300 at N = 1024 (per-level ms for 64 / 148 / 296 /
    // 512 / 2048 gates): 256 threads 30.2 / 29.4 / 38.9 / 71.5 / 230; 512 threads 24.0 /
    // 23.2 / 36.8 / 67.0 / 218; 1024 threads 22.1 / 21.5 / 38.1 / 71.1 / 237
    if (!ctx->sms)
        TFHE_CUDA_TRY(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount,
                                                  ctx->device));
    const int threads = G <= ctx->sms ? 1024 : 512;
    StageTimer tm(ctx, TFHE_STAGE_BLIND_ROTATE_NTT, st);
    k_blind_rotate_ntt<<<G, threads, smem, st>>>(p.n, p.N, ctx->logN, p.l, p.Bgbit, bar, acc,
                                                 ctx->bsk_ntt, ctx->psi_fwd, ctx->psi_inv);
    tm.stop();
    return tfhe_check_launch(ctx, "blind_rotate_ntt");
}

int tfhe_blind_rotate_ntt2(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                           cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (G == 0) return TFHE_OK;
    if (!ctx->bsk_ntt2)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "two-prime NTT form not available here");
    const size_t smem = ((size_t)4 * p.l * p.N + (size_t)16 * p.N) * 4;
    if (!ctx->sms)
        TFHE_CUDA_TRY(ctx, cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount,
                                                  ctx->device));
    StageTimer tm(ctx, TFHE_STAGE_BLIND_ROTATE_NTT, st);
    if (G <= ctx->sms) {
        // one block per SM while there are SMs to spare: 512 threads with up to 128
        // registers each
        TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_blind_rotate_ntt2<512>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem));
        k_blind_rotate_ntt2<512><<<G, 512, smem, st>>>(p.n, p.N, ctx->logN, p.l, p.Bgbit, bar,
                                                       acc, ctx->bsk_ntt2, ctx->tw32);
    } else {
        // two blocks of 512 threads per SM (64 registers each)
        TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_blind_rotate_ntt2<1024>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem));
        k_blind_rotate_ntt2<1024><<<G, 512, smem, st>>>(p.n, p.N, ctx->logN, p.l, p.Bgbit, bar,
                                                        acc, ctx->bsk_ntt2, ctx->tw32);
    }
    tm.stop();
    return tfhe_check_launch(ctx, "blind_rotate_ntt2");
}

int tfhe_dataflow_blocks(tfhe_ctx *ctx) {
    if (!ctx->sms && cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return 0;
    return 2 * ctx->sms;
}

int tfhe_dataflow_ntt2(tfhe_ctx *ctx, const TfheDataflow &df, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (df.G == 0) return TFHE_OK;
    if (!ctx->bsk_ntt2)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "dataflow: two-prime NTT form not available here");
    if (ctx->n_pad / 4 > 512)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "dataflow: key rows wider than the block");
    const size_t smem = ((size_t)4 * p.l * p.N + (size_t)16 * p.N) * 4;
    if ((size_t)(ctx->n_pad / 4) * (512 / (ctx->n_pad / 4)) * 16 > (size_t)4 * p.l * p.N * 4)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "dataflow: key-switch partial sums do not fit");
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_dataflow_ntt2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    StageTimer tm(ctx, TFHE_STAGE_BLIND_ROTATE_NTT, st);
    k_dataflow_ntt2<<<df.blocks, 512, smem, st>>>(df, p.n, p.N, ctx->logN, p.l, p.Bgbit, p.ks_t,
                                                  p.ks_basebit, ctx->n_pad, 32 - (ctx->logN + 1),
                                                  ctx->bsk_ntt2, ctx->tw32,
                                                  (const uint4 *)ctx->ksk, ctx->d_err);
    tm.stop();
    return tfhe_check_launch(ctx, "dataflow_ntt2");
}

static size_t cmux_smem(const tfhe_params &p) {
    // digits and products for both primes, difference and base (or r and old) polynomials
    return (size_t)2 * 2 * p.l * p.N * 4 + (size_t)4 * p.N * 4 + (size_t)4 * p.N * 4;
}

int tfhe_cmux_ntt(tfhe_ctx *ctx, const uint64_t *sel_ntt, const CmuxGeom &g, cudaStream_t st) {
    const tfhe_params &p = ctx->p;
    if (g.count == 0) return TFHE_OK;
    if (!tfhe_cmux_exact(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "CMUX: 2l N Bg/2 2^32 exceeds the NTT bound");
    const size_t smem = cmux_smem(p);
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_cmux_ntt,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    dim3 grid(g.nx, g.ny);
    StageTimer tm(ctx, TFHE_STAGE_CMUX, st);
    k_cmux_ntt<<<grid, 256, smem, st>>>(p.N, ctx->logN, p.l, p.Bgbit, sel_ntt, g, ctx->tw32);
    tm.stop();
    return tfhe_check_launch(ctx, "cmux_ntt");
}

int tfhe_ram_write_ntt(tfhe_ctx *ctx, const uint64_t *c_ntt, const uint64_t *gmc_ntt, int v,
                       const uint32_t *new_cell, uint32_t *cells, cudaStream_t st, int blocks,
                       int64_t new_stride) {
    const tfhe_params &p = ctx->p;
    if (!tfhe_cmux_exact(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "RAM write: 2l N Bg/2 2^32 exceeds the NTT bound");
    const size_t smem = cmux_smem(p) + (size_t)2 * p.N * 4;
    TFHE_CUDA_TRY(ctx, cudaFuncSetAttribute(k_ram_write_ntt,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    StageTimer tm(ctx, TFHE_STAGE_CMUX, st);
    k_ram_write_ntt<<<dim3(1u << v, blocks), 256, smem, st>>>(p.N, ctx->logN, p.l, p.Bgbit, v, c_ntt,
                                                            gmc_ntt, new_cell, new_stride, cells,
                                                            ctx->tw32);
    tm.stop();
    return tfhe_check_launch(ctx, "ram_write_ntt");
}
