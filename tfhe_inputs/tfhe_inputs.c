/*
 * tfhe_inputs.c -- seeded synthetic inputs for the TFHE gate-bootstrapping path.
 *
 * This module draws every random number the scheme needs (secret keys, uniform
 * masks, Gaussian noise, plaintext bits) and performs the client-side
 * encryptions that turn them into the evaluator's inputs: the bootstrapping key
 * (BSK), the key-switching key (KSK), TLWE/TRLWE/TRGSW ciphertexts.  It never
 * evaluates anything the server computes (no gate, CMUX, external product,
 * bootstrap, sample extraction or key switch), so the CPU oracle and the CUDA
 * library can both consume its bytes without sharing any of the evaluated
 * arithmetic.
 *
 * Conventions (paper, Section 2.1.2 "TFHE"):
 *   Torus32: a torus element x in [-1/2, 1/2) is stored as round(x * 2^32) mod 2^32.
 *   mu = 1/8 = 2^29.  A bit m is encoded as mu * (2m - 1).
 *   TLWE (lvl0):   u32[n + 1]   = a[0..n-1], b        b = <a, s> + mu(2m-1) + e
 *   TRLWE (lvl1):  u32[2][N]    = a[X], b[X]          b = a*s + mu(2m[X]-1[X]) + e[X]
 *   TRGSW (lvl1):  u32[2l][2][N] rows of TRLWE encryptions of 0 with m/Bg^j added
 *                  to a (rows 0..l-1) or b (rows l..2l-1) at coefficient 0.
 *   BSK:           u32[n][2l][2][N],  BSK[i] = TRGSW_{s1}(s0[i])
 *   KSK:           u32[N][t][base][n+1],
 *                  KSK[i][j][v] = TLWE_{s0}(v * s1[i] / base^(j+1)),  KSK[i][j][0] = 0
 *
 * Random streams: xoshiro256** (Blackman & Vigna 2018) seeded through SplitMix64
 * (Steele, Lea & Flood 2014).  Each object draws from its own stream, identified
 * by (seed, label, index), so the bytes of an object do not depend on what else
 * was generated before it.  Gaussian noise uses the Box-Muller transform and is
 * rounded to the nearest Torus32 integer.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n, N, l, Bgbit, ks_t, ks_basebit;
    double sigma0, sigma1; /* noise standard deviations on the torus, lvl0 and lvl1 */
} tin_params;

/* stream labels */
enum {
    TIN_S0 = 1, TIN_S1 = 2, TIN_BSK = 3, TIN_KSK = 4, TIN_TLWE0 = 5,
    TIN_TRLWE = 6, TIN_TRGSW = 7, TIN_BITS = 8, TIN_TLWE1 = 9
};

typedef struct { uint64_t s[4]; } tin_rng;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t rng_next(tin_rng *r) {
    uint64_t *s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static void rng_init(tin_rng *r, uint64_t seed, uint64_t label, uint64_t index) {
    uint64_t x = seed;
    uint64_t mix = splitmix64(&x);
    x = mix ^ (label * 0xD1B54A32D192ED03ULL) ^ (index * 0x8CB92BA72F3D8DD7ULL);
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}

static inline uint32_t rng_torus(tin_rng *r) { return (uint32_t)(rng_next(r) >> 32); }
static inline uint32_t rng_bit(tin_rng *r) { return (uint32_t)(rng_next(r) >> 63); }

/* Box-Muller normal sample, scaled to Torus32 and rounded. */
static int32_t rng_noise(tin_rng *r, double sigma) {
    if (sigma <= 0.0) return 0;
    double u1 = ((double)((rng_next(r) >> 11) + 1)) * 0x1.0p-53; /* (0, 1] */
    double u2 = ((double)(rng_next(r) >> 11)) * 0x1.0p-53;       /* [0, 1) */
    double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
    return (int32_t)llround(sigma * g * 4294967296.0);
}

/* ---- secret keys ------------------------------------------------------- */

/* s0 in B^n (lvl0 TLWE key), s1 in B_N[X] (lvl1 TRLWE key), both uniform binary. */
void tin_keygen(const tin_params *p, uint64_t seed, uint32_t *s0, uint32_t *s1) {
    tin_rng r;
    rng_init(&r, seed, TIN_S0, 0);
    for (int i = 0; i < p->n; i++) s0[i] = rng_bit(&r);
    rng_init(&r, seed, TIN_S1, 0);
    for (int i = 0; i < p->N; i++) s1[i] = rng_bit(&r);
}

/* ---- client-side encryption -------------------------------------------- */

/* b[X] += a[X] * s[X] mod (X^N + 1), s binary, arithmetic mod 2^32. */
static void add_mask_times_key(int N, const uint32_t *a, const uint32_t *s, uint32_t *b) {
    for (int j = 0; j < N; j++) {
        if (!s[j]) continue;
        /* X^j * a: coefficient k receives a[k - j] for k >= j, -a[k - j + N] below. */
        for (int k = 0; k < j; k++) b[k] -= a[k - j + N];
        for (int k = j; k < N; k++) b[k] += a[k - j];
    }
}

/* TLWE encryption of the torus value `msg` under key s (length n). */
static void tlwe_encrypt(int n, const uint32_t *s, uint32_t msg, double sigma, tin_rng *r,
                         uint32_t *c) {
    uint32_t b = 0;
    for (int i = 0; i < n; i++) {
        c[i] = rng_torus(r);
        b += c[i] * s[i];
    }
    b += msg + (uint32_t)rng_noise(r, sigma);
    c[n] = b;
}

/* TRLWE encryption of the torus polynomial `msg` (may be NULL for zero). */
static void trlwe_encrypt(int N, const uint32_t *s, const uint32_t *msg, double sigma,
                          tin_rng *r, uint32_t *c) {
    uint32_t *a = c, *b = c + N;
    for (int k = 0; k < N; k++) a[k] = rng_torus(r);
    for (int k = 0; k < N; k++) b[k] = (msg ? msg[k] : 0u) + (uint32_t)rng_noise(r, sigma);
    add_mask_times_key(N, a, s, b);
}

/* TRGSW encryption of the integer m (0 or 1), paper Section 2.1.2 "TRGSW". */
static void trgsw_encrypt(const tin_params *p, const uint32_t *s1, uint32_t m, tin_rng *r,
                          uint32_t *C) {
    const int N = p->N, l = p->l;
    for (int row = 0; row < 2 * l; row++) {
        uint32_t *c = C + (size_t)row * 2 * N;
        trlwe_encrypt(N, s1, NULL, p->sigma1, r, c);
        int j = (row < l ? row : row - l) + 1;              /* gadget level 1..l */
        uint32_t g = (uint32_t)1u << (32 - j * p->Bgbit);   /* 1 / Bg^j in Torus32 */
        if (row < l) c[0] += m * g;                          /* a-column */
        else c[N] += m * g;                                  /* b-column */
    }
}

/* BSK[i] = TRGSW_{s1}(s0[i]) for i < n.  Output u32[n][2l][2][N]. */
void tin_bsk(const tin_params *p, uint64_t seed, const uint32_t *s0, const uint32_t *s1,
             uint32_t *bsk) {
    const size_t per = (size_t)2 * p->l * 2 * p->N;
    for (int i = 0; i < p->n; i++) {
        tin_rng r;
        rng_init(&r, seed, TIN_BSK, (uint64_t)i);
        trgsw_encrypt(p, s1, s0[i], &r, bsk + (size_t)i * per);
    }
}

/* KSK[i][j][v] = TLWE_{s0}(v * s1[i] * 2^(32 - (j+1) basebit)), v = 1..base-1;
 * KSK[i][j][0] = 0.  Output u32[N][t][base][n+1]. */
void tin_ksk(const tin_params *p, uint64_t seed, const uint32_t *s0, const uint32_t *s1,
             uint32_t *ksk) {
    const int n = p->n, t = p->ks_t, base = 1 << p->ks_basebit;
    for (int i = 0; i < p->N; i++) {
        tin_rng r;
        rng_init(&r, seed, TIN_KSK, (uint64_t)i);
        for (int j = 0; j < t; j++) {
            for (int v = 0; v < base; v++) {
                uint32_t *c = ksk + ((((size_t)i * t + j) * base + v) * (size_t)(n + 1));
                if (v == 0) {
                    memset(c, 0, sizeof(uint32_t) * (size_t)(n + 1));
                    continue;
                }
                uint32_t msg = (uint32_t)v * s1[i] * ((uint32_t)1u << (32 - (j + 1) * p->ks_basebit));
                tlwe_encrypt(n, s0, msg, p->sigma0, &r, c);
            }
        }
    }
}

/* count TLWE lvl0 encryptions of bits[k] (0/1), out u32[count][n+1]. */
void tin_tlwe0_encrypt_bits(const tin_params *p, uint64_t seed, uint64_t stream,
                            const uint32_t *s0, const uint8_t *bits, int64_t count,
                            uint32_t *out) {
    const uint32_t mu = 1u << 29;
    for (int64_t k = 0; k < count; k++) {
        tin_rng r;
        rng_init(&r, seed, TIN_TLWE0, (stream << 32) ^ (uint64_t)k);
        uint32_t msg = bits[k] ? mu : (uint32_t)(0u - mu);
        tlwe_encrypt(p->n, s0, msg, p->sigma0, &r, out + (size_t)k * (p->n + 1));
    }
}

/* count TRLWE encryptions of bit polynomials msg[k][N] (0/1 per coefficient),
 * out u32[count][2][N]. */
void tin_trlwe_encrypt_bits(const tin_params *p, uint64_t seed, uint64_t stream,
                            const uint32_t *s1, const uint8_t *msg, int64_t count,
                            uint32_t *out) {
    const int N = p->N;
    const uint32_t mu = 1u << 29;
    uint32_t buf[65536];
    if (N > 65536) return;
    for (int64_t k = 0; k < count; k++) {
        tin_rng r;
        rng_init(&r, seed, TIN_TRLWE, (stream << 32) ^ (uint64_t)k);
        for (int j = 0; j < N; j++) buf[j] = msg[(size_t)k * N + j] ? mu : (uint32_t)(0u - mu);
        trlwe_encrypt(N, s1, buf, p->sigma1, &r, out + (size_t)k * 2 * N);
    }
}

/* count TRGSW encryptions of bits[k], out u32[count][2l][2][N]. */
void tin_trgsw_encrypt_bits(const tin_params *p, uint64_t seed, uint64_t stream,
                            const uint32_t *s1, const uint8_t *bits, int64_t count,
                            uint32_t *out) {
    const size_t per = (size_t)2 * p->l * 2 * p->N;
    for (int64_t k = 0; k < count; k++) {
        tin_rng r;
        rng_init(&r, seed, TIN_TRGSW, (stream << 32) ^ (uint64_t)k);
        trgsw_encrypt(p, s1, bits[k] ? 1u : 0u, &r, out + (size_t)k * per);
    }
}

/* Uniform random bytes from one stream (plaintext bits, gate types, indices). */
void tin_random_u64(uint64_t seed, uint64_t stream, int64_t count, uint64_t *out) {
    tin_rng r;
    rng_init(&r, seed, TIN_BITS, stream);
    for (int64_t k = 0; k < count; k++) out[k] = rng_next(&r);
}

/* ==== Circuit-bootstrapping keys (Section 2.1.2 "Circuit Bootstrapping") ================
 *
 * Circuit bootstrapping (TLWE lvl0 -> TRGSW lvl1) goes through a level-2 ring over the
 * 64-bit torus (Torus64: x -> round(x * 2^64) mod 2^64) and back to lvl1 by private
 * functional key switching.  Its keys:
 *   s2:    B_{N2}[X], uniform binary (lvl2 TRLWE key)
 *   BSK2:  u64[n][2 l2][2][N2],  BSK2[i] = TRGSW_{s2}(s0[i]) over Torus64 (rows as for
 *          the lvl1 TRGSW, 1/Bg2^j = 2^(64 - j Bg2bit) at coefficient 0)
 *   PKSK:  u32[2][N2 + 1][t][base][2][N],
 *          PKSK[z][i][j][v] = TRLWE_{s1}(f_z(v * k_i / base^(j+1))), k_i = s2[i] for i < N2
 *          and k_{N2} = -1, with f_0(x) = -s1[X] * x and f_1(x) = x; v = 0 is the zero
 *          ciphertext.
 * Each TRGSW (per i) and each PKSK block (per z, i) draws from its own stream, so the
 * objects are generated in parallel with identical bytes. */

typedef struct {
    int32_t N2, l2, Bg2bit, pks_t, pks_basebit;
    double sigma2, sigma_pks; /* noise stdev: lvl2 keys (Torus64), PKSK (Torus32) */
} tin_cb_params;

enum { TIN_S2 = 10, TIN_BSK2 = 11, TIN_PKSK = 12 };

static inline uint64_t rng_torus64(tin_rng *r) { return rng_next(r); }

/* Box-Muller normal sample, scaled to Torus64 and rounded. */
static int64_t rng_noise64(tin_rng *r, double sigma) {
    if (sigma <= 0.0) return 0;
    double u1 = ((double)((rng_next(r) >> 11) + 1)) * 0x1.0p-53;
    double u2 = ((double)(rng_next(r) >> 11)) * 0x1.0p-53;
    double g = sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
    return (int64_t)llround(sigma * g * 18446744073709551616.0);
}

void tin_keygen2(const tin_cb_params *q, uint64_t seed, uint32_t *s2) {
    tin_rng r;
    rng_init(&r, seed, TIN_S2, 0);
    for (int i = 0; i < q->N2; i++) s2[i] = rng_bit(&r);
}

/* b[X] += a[X] * s[X] mod (X^N + 1) over Torus64, s binary. */
static void add_mask_times_key64(int N, const uint64_t *a, const uint32_t *s, uint64_t *b) {
    for (int j = 0; j < N; j++) {
        if (!s[j]) continue;
        for (int k = 0; k < j; k++) b[k] -= a[k - j + N];
        for (int k = j; k < N; k++) b[k] += a[k - j];
    }
}

/* BSK2[i] = TRGSW_{s2}(s0[i]) over Torus64, i < n. */
void tin_bsk2(const tin_params *p, const tin_cb_params *q, uint64_t seed, const uint32_t *s0,
              const uint32_t *s2, uint64_t *bsk2) {
    const int N2 = q->N2, l2 = q->l2;
    const size_t per = (size_t)2 * l2 * 2 * N2;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < p->n; i++) {
        tin_rng r;
        rng_init(&r, seed, TIN_BSK2, (uint64_t)i);
        uint64_t *C = bsk2 + (size_t)i * per;
        for (int row = 0; row < 2 * l2; row++) {
            uint64_t *a = C + (size_t)row * 2 * N2, *b = a + N2;
            for (int k = 0; k < N2; k++) a[k] = rng_torus64(&r);
            for (int k = 0; k < N2; k++) b[k] = (uint64_t)rng_noise64(&r, q->sigma2);
            add_mask_times_key64(N2, a, s2, b);
            const int j = (row < l2 ? row : row - l2) + 1;
            const uint64_t g = (uint64_t)1u << (64 - j * q->Bg2bit);
            if (row < l2) a[0] += (uint64_t)s0[i] * g;
            else b[0] += (uint64_t)s0[i] * g;
        }
    }
}

/* PKSK[z][i][j][v], layout u32[2][N2+1][t][base][2][N]. */
void tin_pksk(const tin_params *p, const tin_cb_params *q, uint64_t seed, const uint32_t *s1,
              const uint32_t *s2, uint32_t *pksk) {
    const int N = p->N, N2 = q->N2, t = q->pks_t, bb = q->pks_basebit, base = 1 << bb;
    const size_t row_words = (size_t)2 * N;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int z = 0; z < 2; z++) {
        for (int i = 0; i <= N2; i++) {
            tin_rng r;
            rng_init(&r, seed, TIN_PKSK, ((uint64_t)z << 32) ^ (uint64_t)i);
            uint32_t *msg = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
            const uint32_t key = i < N2 ? s2[i] : 0xFFFFFFFFu; /* k_{N2} = -1 */
            for (int j = 0; j < t; j++) {
                for (int v = 0; v < base; v++) {
                    uint32_t *c =
                        pksk + ((((size_t)z * (N2 + 1) + i) * t + j) * base + v) * row_words;
                    if (v == 0) {
                        memset(c, 0, sizeof(uint32_t) * row_words);
                        continue;
                    }
                    const uint32_t x = (uint32_t)v * key * ((uint32_t)1u << (32 - (j + 1) * bb));
                    if (z == 0)
                        for (int k = 0; k < N; k++) msg[k] = (uint32_t)(0u - x * s1[k]);
                    else {
                        memset(msg, 0, sizeof(uint32_t) * (size_t)N);
                        msg[0] = x;
                    }
                    uint32_t *a = c, *b = c + N;
                    for (int k = 0; k < N; k++) a[k] = rng_torus(&r);
                    for (int k = 0; k < N; k++) b[k] = msg[k] + (uint32_t)rng_noise(&r, q->sigma_pks);
                    add_mask_times_key(N, a, s1, b);
                }
            }
            free(msg);
        }
    }
}
