// ntt32.cuh -- exact negacyclic polynomial products with 32-bit lanes: NTTs over two
// 30-bit primes P1 = 119 * 2^23 + 1 and P2 = 45 * 2^24 + 1 and a CRT back to the integer.
//
// Each product sum V = sum_r d_r * k_r (small signed digits d, key words k < 2^32) is
// computed modulo P1 and modulo P2 and recombined by the Chinese remainder theorem.  The
// modulus M = P1 P2 (about 2^59.4) exceeds 2|V|, so the centred CRT value is V itself,
// whose residue mod 2^32 or mod 2^64 the callers take.  This replaces the 64-bit
// arithmetic mod 2^64 - 2^32 + 1: 30-bit residues fit one 32-bit register, a twiddle
// multiply is three 32-bit multiplies (Shoup's precomputed quotient), and butterflies
// keep values lazily in [0, 2p) (Harvey's bounds), so there are few compare-and-subtract
// steps.
//
// Layout: the transforms work in place on shared memory a[2 primes][np][N], prime-major;
// the twiddle table is tw[2 primes][4][N]: psi^{brv(k)}, its Shoup quotient,
// psi^{-brv(k)} and its quotient, psi a primitive 2N-th root of unity mod the prime.
#pragma once

#include "common.cuh"

constexpr uint32_t NP1 = 998244353u;  // 119 * 2^23 + 1
constexpr uint32_t NP2 = 754974721u;  // 45 * 2^24 + 1

// -p^{-1} mod 2^32 by Newton's iteration (each step doubles the correct low bits)
__host__ __device__ constexpr uint32_t neg_inv32(uint32_t p) {
    uint32_t x = p;  // correct mod 2^3 for odd p
    for (int i = 0; i < 4; i++) x *= 2u - p * x;
    return 0u - x;
}

__host__ __device__ constexpr uint64_t powmod64(uint64_t a, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1) r = r * a % m;  // m < 2^32: products fit 64 bits
        a = a * a % m;
        e >>= 1;
    }
    return r;
}

constexpr uint32_t NP1_NINV = neg_inv32(NP1);
constexpr uint32_t NP2_NINV = neg_inv32(NP2);
constexpr uint32_t CRT_C = (uint32_t)powmod64(NP1 % NP2, NP2 - 2, NP2);  // P1^{-1} mod P2
constexpr uint32_t CRT_CS = (uint32_t)(((uint64_t)CRT_C << 32) / NP2);  // its Shoup quotient
constexpr uint64_t CRT_M = (uint64_t)NP1 * NP2;

// x * w mod p in [0, 2p) for any x < 2^32 (ws = floor(w 2^32 / p), p < 2^31)
__device__ __forceinline__ uint32_t shoup_mul(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
    return x * w - __umulhi(x, ws) * p;
}

__device__ __forceinline__ uint32_t red_below(uint32_t a, uint32_t b) { return a >= b ? a - b : a; }

// Montgomery reduction: T / 2^32 mod p in [0, 2p) for T < p 2^32
__device__ __forceinline__ uint32_t redc32(uint64_t T, uint32_t p, uint32_t ninv) {
    const uint32_t m = (uint32_t)T * ninv;
    return (uint32_t)((T + (uint64_t)m * p) >> 32);
}

// signed integer below 2^31 in magnitude -> residue in [0, p)
__device__ __forceinline__ uint32_t res_of_i32(int32_t d, uint32_t p) {
    return d >= 0 ? (uint32_t)d : p - (uint32_t)(-d);
}

// CRT of canonical residues (r1 mod P1, r2 mod P2) -> the centred integer V, |V| < M/2
__device__ __forceinline__ int64_t crt_centred(uint32_t r1, uint32_t r2) {
    const uint32_t r1m = red_below(r1, NP2);  // r1 < P1 < 2 P2
    const uint32_t dlt = red_below(r2 + NP2 - r1m, NP2);
    const uint32_t h = red_below(shoup_mul(dlt, CRT_C, CRT_CS, NP2), NP2);
    const uint64_t v = (uint64_t)r1 + (uint64_t)NP1 * h;  // in [0, M)
    return v > CRT_M / 2 ? (int64_t)(v - CRT_M) : (int64_t)v;
}

// Cooley-Tukey, natural order in, bit-reversed evaluations out; values in [0, 2p).
__device__ __forceinline__ void ntt32_fwd(uint32_t *a, int np, int N, int logN,
                                          const uint32_t *__restrict__ tw) {
    const int half = N >> 1;
    for (int s = 0; s < logN; s++) {
        const int m = 1 << s, logt = logN - 1 - s, t = 1 << logt;
        for (int idx = threadIdx.x; idx < 2 * np * half; idx += blockDim.x) {
            const int poly = idx >> (logN - 1), b = idx & (half - 1);
            const int pr = poly >= np;
            const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
            const int i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            uint32_t *x = a + (size_t)poly * N;
            const uint32_t *T = tw + (size_t)pr * 4 * N;
            const uint32_t V = shoup_mul(x[j + t], __ldg(T + m + i), __ldg(T + N + m + i), p);
            const uint32_t U = x[j];
            x[j] = red_below(U + V, p2);
            x[j + t] = red_below(U - V + p2, p2);
        }
        __syncthreads();
    }
}

// Gentleman-Sande, bit-reversed in, natural out (without the factor N^{-1}); [0, 2p).
__device__ __forceinline__ void ntt32_inv(uint32_t *a, int np, int N, int logN,
                                          const uint32_t *__restrict__ tw) {
    const int half = N >> 1;
    for (int s = 0; s < logN; s++) {
        const int logt = s, t = 1 << s, h = N >> (s + 1);
        for (int idx = threadIdx.x; idx < 2 * np * half; idx += blockDim.x) {
            const int poly = idx >> (logN - 1), b = idx & (half - 1);
            const int pr = poly >= np;
            const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
            const int i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            uint32_t *x = a + (size_t)poly * N;
            const uint32_t *T = tw + (size_t)pr * 4 * N;
            const uint32_t U = x[j], V = x[j + t];
            x[j] = red_below(U + V, p2);
            x[j + t] = shoup_mul(U - V + p2, __ldg(T + 2 * N + h + i), __ldg(T + 3 * N + h + i), p);
        }
        __syncthreads();
    }
}

// ---- register-blocked transforms: radix-2^R passes (R <= 3 stages per pass) ------------
// (tw may point to global or to shared memory)
//
// The polynomials these transforms work on are stored swizzled: coefficient e of a
// polynomial sits at word swz(e) = e ^ (((e >> 5) & 7) << 2), which permutes aligned
// 4-word groups inside each 32-word row.  Strided passes then spread a warp's accesses
// over all banks, and groups of 2 or 4 consecutive coefficients stay contiguous and
// aligned, so the passes whose groups are contiguous use 16-byte accesses.
//
// A forward pass over stages s .. s+R-1 (t = N >> (s+1) at stage s) works on groups of
// 2^R elements e_k = 2t i + x0 + k t / 2^(R-1), i < 2^s the stage-s block, x0 < t / 2^(R-1);
// stage s + q pairs k and k + 2^(R-1-q) with the twiddle of its block 2^q i + (k >> (R-q)).
// An inverse pass over stages s .. s+R-1 (t = 2^s at stage s) works on groups
// e_k = 2^R t i + x0 + k t, x0 < t; stage s + q pairs k and k + 2^q, block 2^(R-1-q) i +
// (k >> (q+1)), twiddle index (N >> (s+q+1)) + block.  One barrier per pass; the same
// butterflies, twiddles and order within each group as the stage-by-stage loops above.
__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 5) & 7) << 2); }

// load / store the 2^R coefficients e0 + k*st of a group (contiguous when st == 1)
template <int G>
__device__ __forceinline__ void grp_load(const uint32_t *x, int e0, int st, uint32_t *v) {
    if (G >= 4 && st == 1) {
#pragma unroll
        for (int k = 0; k < G; k += 4) {
            const uint4 w = *reinterpret_cast<const uint4 *>(x + swz(e0 + k));
            v[k] = w.x; v[k + 1] = w.y; v[k + 2] = w.z; v[k + 3] = w.w;
        }
    } else if (G == 2 && st == 1) {
        const uint2 w = *reinterpret_cast<const uint2 *>(x + swz(e0));
        v[0] = w.x; v[1] = w.y;
    } else {
#pragma unroll
        for (int k = 0; k < G; k++) v[k] = x[swz(e0 + k * st)];
    }
}

template <int G>
__device__ __forceinline__ void grp_store(uint32_t *x, int e0, int st, const uint32_t *v) {
    if (G >= 4 && st == 1) {
#pragma unroll
        for (int k = 0; k < G; k += 4)
            *reinterpret_cast<uint4 *>(x + swz(e0 + k)) = make_uint4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else if (G == 2 && st == 1) {
        *reinterpret_cast<uint2 *>(x + swz(e0)) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < G; k++) x[swz(e0 + k * st)] = v[k];
    }
}

template <int R>
__device__ __forceinline__ void ntt32_fwd_pass(uint32_t *a, int np, int N, int logN, int s,
                                               const uint32_t *tw) {
    constexpr int G = 1 << R;
    const int t = N >> (s + 1);
    const int logst = logN - s - R;          // log2 of the element stride inside a group
    const int st = 1 << logst;
    const int lgroups = logN - R;            // log2 of the groups per polynomial
    for (int idx = threadIdx.x; idx < (2 * np) << lgroups; idx += blockDim.x) {
        const int poly = idx >> lgroups, gidx = idx & ((1 << lgroups) - 1);
        const int pr = poly >= np;
        const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
        const int i = gidx >> logst, x0 = gidx & (st - 1);
        uint32_t *x = a + (size_t)poly * N;
        const int e0 = i * 2 * t + x0;
        const uint32_t *T = tw + (size_t)pr * 4 * N;
        uint32_t v[G];
        grp_load<G>(x, e0, st, v);
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int half = G >> (q + 1);
#pragma unroll
            for (int k = 0; k < G; k++) {
                if (k & half) continue;
                const int blk = ((1 << s) << q) + (i << q) + (k >> (R - q));
                const uint32_t V = shoup_mul(v[k + half], T[blk], T[N + blk], p);
                const uint32_t U = v[k];
                v[k] = red_below(U + V, p2);
                v[k + half] = red_below(U - V + p2, p2);
            }
        }
        grp_store<G>(x, e0, st, v);
    }
    __syncthreads();
}

template <int R>
__device__ __forceinline__ void ntt32_inv_pass(uint32_t *a, int np, int N, int logN, int s,
                                               const uint32_t *tw) {
    constexpr int G = 1 << R;
    const int t = 1 << s;
    const int lgroups = logN - R;
    for (int idx = threadIdx.x; idx < (2 * np) << lgroups; idx += blockDim.x) {
        const int poly = idx >> lgroups, gidx = idx & ((1 << lgroups) - 1);
        const int pr = poly >= np;
        const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
        const int i = gidx >> s, x0 = gidx & (t - 1);
        uint32_t *x = a + (size_t)poly * N;
        const int e0 = (i << (s + R)) + x0;
        const uint32_t *T = tw + (size_t)pr * 4 * N;
        uint32_t v[G];
        grp_load<G>(x, e0, t, v);
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int dist = 1 << q;
#pragma unroll
            for (int k = 0; k < G; k++) {
                if (k & dist) continue;
                const int blk = (N >> (s + q + 1)) + (i << (R - 1 - q)) + (k >> (q + 1));
                const uint32_t U = v[k], V = v[k + dist];
                v[k] = red_below(U + V, p2);
                v[k + dist] = shoup_mul(U - V + p2, T[2 * N + blk], T[3 * N + blk], p);
            }
        }
        grp_store<G>(x, e0, t, v);
    }
    __syncthreads();
}

// Whole transforms by passes of three stages (and one shorter pass at the end).
__device__ __forceinline__ void ntt32_fwd_r8(uint32_t *a, int np, int N, int logN,
                                             const uint32_t *tw) {
    int s = 0;
    for (; s + 3 <= logN; s += 3) ntt32_fwd_pass<3>(a, np, N, logN, s, tw);
    if (logN - s == 2) ntt32_fwd_pass<2>(a, np, N, logN, s, tw);
    else if (logN - s == 1) ntt32_fwd_pass<1>(a, np, N, logN, s, tw);
}

__device__ __forceinline__ void ntt32_inv_r8(uint32_t *a, int np, int N, int logN,
                                             const uint32_t *tw) {
    int s = 0;
    for (; s + 3 <= logN; s += 3) ntt32_inv_pass<3>(a, np, N, logN, s, tw);
    if (logN - s == 2) ntt32_inv_pass<2>(a, np, N, logN, s, tw);
    else if (logN - s == 1) ntt32_inv_pass<1>(a, np, N, logN, s, tw);
}

// host: the twiddle table tw[2][4][N] (device allocation) for ring degree N
int tfhe_make_twiddles32(tfhe_ctx *ctx, int N, uint32_t **tw);
