// ntt32.cuh -- exact negacyclic polynomial products with 32-bit lanes: NTTs over two
// 30-bit primes P1 = 119 * 2^23 + 1 and P2 = 45 * 2^24 + 1 and a CRT back to the integer.
//
// Each product sum V = sum_r d_r * k_r (small signed digits d, key words k < 2^32) is
// computed modulo P1 and modulo P2 and recombined by the Chinese remainder theorem.  The
// modulus M = P1 P2 (about 2^59.4) exceeds 2|V|, so the centred CRT value is V itself,
// whose residue mod 2^32 or mod 2^64 the callers take.  This replaces the 64-bit
// arithmetic mod 2^64 - 2^32 + 1: 30-bit residues fit one 32-bit register, a twiddle
// multiply is three 32-bit multiplies (Shoup's precomputed quotient), and butterflies
// keep values lazily below 2p or 4p (Harvey's bounds), so there are few conditional
// subtractions, each an unsigned min.
//
// Layout: the transforms work in place on shared memory a[2 primes][np][N], prime-major
// (or with a given stride between the primes); the twiddle table is tw[2 primes][2][N][2]:
// for each prime the forward pairs (psi^{brv(k)}, its Shoup quotient), then the inverse
// pairs (psi^{-brv(k)}, quotient), psi a primitive 2N-th root of unity mod the prime.  A
// pair is one 8-byte load, and the consecutive pairs of a group's stages are one 8-byte
// load or one to four 16-byte loads.
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

// a - b if a >= b, else a (any a, b > 0): when a < b, a - b wraps above a, so the unsigned
// minimum picks a; one subtraction and one min, no compare-and-select
__device__ __forceinline__ uint32_t red_below(uint32_t a, uint32_t b) { return min(a, a - b); }

// Montgomery reduction: T / 2^32 mod p in [0, 2p) for T < p 2^32
__device__ __forceinline__ uint32_t redc32(uint64_t T, uint32_t p, uint32_t ninv) {
    const uint32_t m = (uint32_t)T * ninv;
    return (uint32_t)((T + (uint64_t)m * p) >> 32);
}

// signed integer d, |d| < p, -> residue in [0, p): for d >= 0 the bit pattern u = d is
// below u + p; for d < 0, u >= 2^31 exceeds u + p = p - |d|; the unsigned min picks it
__device__ __forceinline__ uint32_t res_of_i32(int32_t d, uint32_t p) {
    const uint32_t u = (uint32_t)d;
    return min(u, u + p);
}

// CRT of canonical residues (r1 mod P1, r2 mod P2): v = r1 + P1 h in [0, M) with
// h = (r2 - r1) P1^{-1} mod P2.  The centred integer V is v - M when v > M/2.  As M is
// odd and 0 <= r1 < P1, that holds exactly when h > (P2-1)/2, or h = (P2-1)/2 and
// r1 > (P1-1)/2, so it is decided on 32-bit words.
__device__ __forceinline__ uint32_t crt_digit(uint32_t r1, uint32_t r2) {
    const uint32_t r1m = red_below(r1, NP2);  // r1 < P1 < 2 P2
    const uint32_t dlt = red_below(r2 + NP2 - r1m, NP2);
    return red_below(shoup_mul(dlt, CRT_C, CRT_CS, NP2), NP2);
}

__device__ __forceinline__ bool crt_negative(uint32_t r1, uint32_t h) {
    return h > (NP2 - 1) / 2 || (h == (NP2 - 1) / 2 && r1 > (NP1 - 1) / 2);
}

// -> the centred integer V, |V| < M/2
__device__ __forceinline__ int64_t crt_centred(uint32_t r1, uint32_t r2) {
    const uint32_t h = crt_digit(r1, r2);
    const uint64_t v = (uint64_t)r1 + (uint64_t)NP1 * h;  // in [0, M)
    return (int64_t)(v - (crt_negative(r1, h) ? CRT_M : 0ull));
}

// -> V mod 2^32
__device__ __forceinline__ uint32_t crt_lo32(uint32_t r1, uint32_t r2) {
    const uint32_t h = crt_digit(r1, r2);
    return r1 + NP1 * h - (crt_negative(r1, h) ? (uint32_t)CRT_M : 0u);
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
            const uint32_t V = shoup_mul(x[j + t], __ldg(T + 2 * (m + i)), __ldg(T + 2 * (m + i) + 1), p);
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
            x[j + t] = shoup_mul(U - V + p2, __ldg(T + 2 * N + 2 * (h + i)),
                                 __ldg(T + 2 * N + 2 * (h + i) + 1), p);
        }
        __syncthreads();
    }
}

// ---- register-blocked transforms: radix-2^R passes (R <= 4 stages per pass) ------------
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
//
// The ring degree and the stage are template parameters, so a group's addresses are
// swz(e_0) combined with constants: the swizzle is linear over GF(2) and the bits of
// k * stride are disjoint from those of e_0, so swz(e_k) = swz(e_0) ^ swz(k * stride),
// an add folded into the access wherever the constant cannot meet the bits of swz(e_0).
//
// Forward butterflies are Harvey's lazy form: values stay in [0, 4p) between stages (4p <
// 2^32 for both primes), only U is brought below 2p, and the last pass brings every output
// below 2p.  Inverse butterflies keep [0, 2p).  Callers see [0, 2p) in and out as before.
__device__ __forceinline__ int swz(int e) { return e ^ (((e >> 5) & 7) << 2); }

template <int LOGST, int R>
__device__ __forceinline__ int grp_off(int sb, int k) {
    const int c = swz(k << LOGST);  // a constant once k is unrolled
    const int m = ((1 << LOGST) - 1) | ~((1 << (LOGST + R)) - 1) | 0x1c;  // bits swz(e_0) may hold
    return (c & m) == 0 ? sb + c : sb ^ c;
}

// load / store the 2^R coefficients of a group, sb = swz(e_0), stride 2^LOGST
template <int LOGST, int R>
__device__ __forceinline__ void grp_load(const uint32_t *x, int sb, uint32_t *v) {
    constexpr int G = 1 << R;
    if constexpr (LOGST == 0 && G >= 4) {
#pragma unroll
        for (int k = 0; k < G; k += 4) {
            const uint4 w = *reinterpret_cast<const uint4 *>(x + grp_off<0, R>(sb, k));
            v[k] = w.x; v[k + 1] = w.y; v[k + 2] = w.z; v[k + 3] = w.w;
        }
    } else if constexpr (LOGST == 0 && G == 2) {
        const uint2 w = *reinterpret_cast<const uint2 *>(x + sb);
        v[0] = w.x; v[1] = w.y;
    } else {
#pragma unroll
        for (int k = 0; k < G; k++) v[k] = x[grp_off<LOGST, R>(sb, k)];
    }
}

template <int LOGST, int R>
__device__ __forceinline__ void grp_store(uint32_t *x, int sb, const uint32_t *v) {
    constexpr int G = 1 << R;
    if constexpr (LOGST == 0 && G >= 4) {
#pragma unroll
        for (int k = 0; k < G; k += 4)
            *reinterpret_cast<uint4 *>(x + grp_off<0, R>(sb, k)) =
                make_uint4(v[k], v[k + 1], v[k + 2], v[k + 3]);
    } else if constexpr (LOGST == 0 && G == 2) {
        *reinterpret_cast<uint2 *>(x + sb) = make_uint2(v[0], v[1]);
    } else {
#pragma unroll
        for (int k = 0; k < G; k++) x[grp_off<LOGST, R>(sb, k)] = v[k];
    }
}

// np consecutive (twiddle, quotient) pairs starting at pair index b (b a multiple of np;
// np is a constant once the callers' stage loops are unrolled)
__device__ __forceinline__ void tw_pairs(const uint32_t *T, int b, int np, uint32_t *w) {
    if (np == 1) {
        const uint2 x = *reinterpret_cast<const uint2 *>(T + 2 * b);
        w[0] = x.x; w[1] = x.y;
    } else {
#pragma unroll
        for (int m = 0; m < 2 * np; m += 4) {
            const uint4 x = *reinterpret_cast<const uint4 *>(T + 2 * b + m);
            w[m] = x.x; w[m + 1] = x.y; w[m + 2] = x.z; w[m + 3] = x.w;
        }
    }
}

template <int LOGN, int S, int R, bool LAST>
__device__ __forceinline__ void ntt32_fwd_pass(uint32_t *a, int np, int pst, const uint32_t *tw) {
    constexpr int N = 1 << LOGN, G = 1 << R;
    constexpr int LOGST = LOGN - S - R;  // log2 of the element stride inside a group
    constexpr int LG = LOGN - R;         // log2 of the groups per polynomial
    for (int idx = threadIdx.x; idx < (2 * np) << LG; idx += blockDim.x) {
        const int poly = idx >> LG, gidx = idx & ((1 << LG) - 1);
        const int pr = poly >= np;
        const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
        const int i = gidx >> LOGST;
        const int sb = swz((i << (LOGST + R)) | (gidx & ((1 << LOGST) - 1)));
        uint32_t *x = a + (size_t)pr * pst + (size_t)(poly - (pr ? np : 0)) * N;
        const uint32_t *T = tw + (size_t)pr * 4 * N;  // forward pairs
        uint32_t v[G];
        grp_load<LOGST, R>(x, sb, v);
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int half = G >> (q + 1);
            uint32_t w[G];  // 2^q pairs: blocks ((2^S + i) << q) + j, j < 2^q
            tw_pairs(T, ((1 << S) + i) << q, 1 << q, w);
#pragma unroll
            for (int k = 0; k < G; k++) {
                if (k & half) continue;
                const int j = k >> (R - q);
                const uint32_t V = shoup_mul(v[k + half], w[2 * j], w[2 * j + 1], p);
                // inputs of the first stage are below 2p already (the transform's contract)
                const uint32_t U = (S == 0 && q == 0) ? v[k] : red_below(v[k], p2);
                v[k] = U + V;
                v[k + half] = U - V + p2;
            }
        }
        if constexpr (LAST) {
#pragma unroll
            for (int k = 0; k < G; k++) v[k] = red_below(v[k], p2);
        }
        grp_store<LOGST, R>(x, sb, v);
    }
    __syncthreads();
}

template <int LOGN, int S, int R>
__device__ __forceinline__ void ntt32_inv_pass(uint32_t *a, int np, int pst, const uint32_t *tw) {
    constexpr int N = 1 << LOGN, G = 1 << R;
    constexpr int LG = LOGN - R;
    for (int idx = threadIdx.x; idx < (2 * np) << LG; idx += blockDim.x) {
        const int poly = idx >> LG, gidx = idx & ((1 << LG) - 1);
        const int pr = poly >= np;
        const uint32_t p = pr ? NP2 : NP1, p2 = 2 * p;
        const int i = gidx >> S;
        const int sb = swz((i << (S + R)) | (gidx & ((1 << S) - 1)));
        uint32_t *x = a + (size_t)pr * pst + (size_t)(poly - (pr ? np : 0)) * N;
        const uint32_t *T = tw + (size_t)pr * 4 * N + 2 * N;  // inverse pairs
        uint32_t v[G];
        grp_load<S, R>(x, sb, v);
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int dist = 1 << q;
            uint32_t w[G];  // 2^(R-1-q) pairs from (N >> (S+q+1)) + (i << (R-1-q))
            tw_pairs(T, (N >> (S + q + 1)) + (i << (R - 1 - q)), 1 << (R - 1 - q), w);
#pragma unroll
            for (int k = 0; k < G; k++) {
                if (k & dist) continue;
                const int j = k >> (q + 1);
                const uint32_t U = v[k], V = v[k + dist];
                v[k] = red_below(U + V, p2);
                v[k + dist] = shoup_mul(U - V + p2, w[2 * j], w[2 * j + 1], p);
            }
        }
        grp_store<S, R>(x, sb, v);
    }
    __syncthreads();
}

// Stages per pass.  Radix-16 passes cut the per-group overhead where the swizzle keeps
// them free of bank conflicts: forward 4+3+4 (N = 2048), 4+3+3 (N = 1024); inverse 4+3+4,
// 3+3+4; otherwise passes of three stages and a shorter one at the end.
template <int LOGN, int S, bool FWD>
__host__ __device__ constexpr int ntt32_pass_r() {
    if (LOGN == 11 && (S == 0 || S == 7)) return 4;
    if (LOGN == 10 && ((FWD && S == 0) || (!FWD && S == 6))) return 4;
    return LOGN - S < 3 ? LOGN - S : 3;
}

// Whole transforms by passes.
template <int LOGN, int S>
__device__ __forceinline__ void ntt32_fwd_from(uint32_t *a, int np, int pst, const uint32_t *tw) {
    constexpr int R = ntt32_pass_r<LOGN, S, true>();
    if constexpr (R > 0) {
        ntt32_fwd_pass<LOGN, S, R, S + R == LOGN>(a, np, pst, tw);
        ntt32_fwd_from<LOGN, S + R>(a, np, pst, tw);
    }
}

template <int LOGN, int S>
__device__ __forceinline__ void ntt32_inv_from(uint32_t *a, int np, int pst, const uint32_t *tw) {
    constexpr int R = ntt32_pass_r<LOGN, S, false>();
    if constexpr (R > 0) {
        ntt32_inv_pass<LOGN, S, R>(a, np, pst, tw);
        ntt32_inv_from<LOGN, S + R>(a, np, pst, tw);
    }
}

// Ring degrees are validated to 256 .. 2048 where contexts and lvl2 keys are set up.  The
// np polynomials of prime 2 start pst words after those of prime 1 (default: np N).
__device__ __forceinline__ void ntt32_fwd_r8(uint32_t *a, int np, int logN, const uint32_t *tw,
                                             int pst = -1) {
    if (pst < 0) pst = np << logN;
    switch (logN) {
    case 8: ntt32_fwd_from<8, 0>(a, np, pst, tw); break;
    case 9: ntt32_fwd_from<9, 0>(a, np, pst, tw); break;
    case 10: ntt32_fwd_from<10, 0>(a, np, pst, tw); break;
    case 11: ntt32_fwd_from<11, 0>(a, np, pst, tw); break;
    }
}

__device__ __forceinline__ void ntt32_inv_r8(uint32_t *a, int np, int logN, const uint32_t *tw,
                                             int pst = -1) {
    if (pst < 0) pst = np << logN;
    switch (logN) {
    case 8: ntt32_inv_from<8, 0>(a, np, pst, tw); break;
    case 9: ntt32_inv_from<9, 0>(a, np, pst, tw); break;
    case 10: ntt32_inv_from<10, 0>(a, np, pst, tw); break;
    case 11: ntt32_inv_from<11, 0>(a, np, pst, tw); break;
    }
}

// host: the twiddle table tw[2][2][N][2] (device allocation) for ring degree N
int tfhe_make_twiddles32(tfhe_ctx *ctx, int N, uint32_t **tw);
