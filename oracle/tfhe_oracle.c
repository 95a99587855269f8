/*
 * tfhe_oracle.c -- plain, slow, obviously correct CPU oracle for TFHE gate
 * bootstrapping and the CMUX-tree memory of
 *   "Virtual Secure Platform: A Five-Stage Pipeline Processor over TFHE".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * executes this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator with
 * the CUDA path.
 *
 * Everything is integer arithmetic modulo 2^32 on uint32 (Torus32): a torus value
 * x in [-1/2, 1/2) (Section 2.1.2, Notations) is stored as round(x * 2^32) mod 2^32
 * and its sign is the sign of the int32 view.  Polynomials live in
 * Z[X]/(X^N + 1) and are multiplied by the schoolbook definition.  No blocking,
 * transforms or reordering: each function follows the definition it cites.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   R1 sgn(0): a phase that is >= 0 as int32 decrypts to 1.
 *   R2 gadget decomposition (implied by the TRGSW rows m/Bg^j, Section 2.1.2
 *      "TRGSW"): l signed digits in [-Bg/2, Bg/2), rounding to nearest with ties
 *      upward, digit j (1-based) paired with TRGSW row j (weight 1/Bg^j).
 *   R3 ModSwitch to Z_{2N}: round half up with 32-bit wrap.
 *   R4 BlindRotate (Section 2.1.2 "Bootstrapping in TFHE", "CMUX"): accumulator
 *      starts at X^{-b~} (0, v) with every coefficient of v equal to mu = 1/8, then
 *      ACC <- CMUX(BK_i, X^{a~_i} ACC, ACC) for i = 0..n-1.
 *   R5 Identity key switching (Section 2.1.2 "Sample Extraction and Identity Key
 *      Switching"): unsigned base-2^basebit digits of each extracted mask
 *      coefficient rounded to t digits; a zero digit contributes nothing.
 *   R6 gate constants (Section 2.1.2 "Homomorphic Gates"; TFHE's standard linear
 *      combinations); "NY" negates the first input, "YN" the second.
 *   R7 CMUX tree (Section 8.2 "Read Unit"): address bit j selects at tree level j,
 *      least significant bit at the leaves.
 *   R8 RAM write bar (Section 8.2 "Write Unit" and its Remark): for cell c the
 *      controlled data passes through v CMUXes, bit j ascending; the selector is
 *      C_j when bit j of c is 1 and G - C_j otherwise (G the gadget TRGSW of 1).
 *   R15 ROM with vertical and horizontal packing (Section 8.3 "ROM"; Table "The number
 *      of CMUXs in CMUX Memory": 8 for the ROM): M words of w bits, P = N / w words per
 *      TRLWE with word q of a TRLWE in coefficients q w .. q w + w - 1 (bit i at q w + i),
 *      T = M / P TRLWEs.  Address bits 0 .. log2 P - 1 pick the word inside a TRLWE, the
 *      rest the TRLWE.  A read first runs the CMUX tree (R7) over the TRLWE bits, then
 *      the blind rotation ACC <- CMUX(C_j, X^{-w 2^j} ACC, ACC) for the low bits j
 *      ascending, which brings the word to coefficients 0 .. w-1; bit i is SE at
 *      coefficient i (the TRLWE times X^{-i}, then R5's extraction) followed by IKS.
 *      512 words of bytes at N = 1024, i.e. 128 words of 32 bits in 4 TRLWEs, take
 *      3 + 5 = 8 CMUXes.
 *   R14 RAM cycle (Section 8.2 "Control Unit" and "Write Unit"): one address per cycle
 *      for read and write; the w bit blocks are read by CMUX trees sharing the address
 *      (R7), the read words go through SE and IKS (returned as the read data), the
 *      controlled data is HomMUX without SE and IKS of (write flag, write data, read
 *      data) (R13), each block's write bar takes it (R8), and every cell is refreshed by
 *      SE, IKS, ModSwitch and BlindRotate (R4) back to a TRLWE whose coefficient 0
 *      carries the bit.
 *   R16 Circuit Bootstrapping (Section 2.1.2 "Circuit Bootstrapping"; steps from the TFHE
 *      construction the paper cites): l BlindRotates over a lvl2 ring on the 64-bit
 *      torus with test vectors 1/(2 Bg^u), then private functional key switching to the
 *      2l TRGSW rows with f(x) = -s1[X] x (rows 0..l-1) and f(x) = x (rows l..2l-1).
 *   R13 HomMUX (Section 2.1.2 "Homomorphic Gates", "HomMUX without SE and IKS"; the
 *      paper names the gate but not its steps): MUX(c, a, b) = c ? a : b as
 *      u = BlindRotate(AND(c, a)) + BlindRotate(ANDNY(c, b)) + (0, mu X^0), the two
 *      gate combinations as in R6 and mu = 1/8; "without SE and IKS" is u itself
 *      (three TLWE in, one TRLWE out); HomMUX is IKS(SE(u)).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { int32_t n, N, l, Bgbit, ks_t, ks_basebit; } orc_params;

/* Counts external products evaluated by this thread (for the CMUX-count pin). */
static _Thread_local uint64_t orc_extprod_calls = 0;
uint64_t orc_extprod_count(void) { return orc_extprod_calls; }
void orc_extprod_count_reset(void) { orc_extprod_calls = 0; }

/* ---- Torus polynomials (Section 2.1.2, Notations: T_N[X], Z_N[X]) ---------- */

/* out = a * b in Z[X]/(X^N+1), a with integer coefficients, b on the torus.
 * Schoolbook: term a_i b_j lands on X^{i+j}; X^N = -1 folds i+j >= N with a minus. */
void orc_poly_mul(int N, const int32_t *a, const uint32_t *b, uint32_t *out) {
    uint32_t *acc = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    for (int i = 0; i < N; i++) {
        const uint32_t ai = (uint32_t)a[i];
        for (int j = 0; j < N - i; j++) acc[i + j] += ai * b[j];     /* i + j < N */
        for (int j = N - i; j < N; j++) acc[i + j - N] -= ai * b[j]; /* X^N = -1 */
    }
    memcpy(out, acc, sizeof(uint32_t) * (size_t)N);
    free(acc);
}

/* out = X^k * p in T_N[X], k in [0, 2N).  X^k p has coefficient p_{j-k} at X^j for
 * j >= k; the wrapped terms carry X^N = -1.  For k >= N, X^k = -X^{k-N}. */
void orc_rotate(int N, int k, const uint32_t *p, uint32_t *out) {
    int neg = 0;
    k %= 2 * N;
    if (k < 0) k += 2 * N;
    if (k >= N) { k -= N; neg = 1; }
    for (int j = 0; j < N; j++) {
        uint32_t v = (j >= k) ? p[j - k] : (uint32_t)(0u - p[j - k + N]);
        out[j] = neg ? (uint32_t)(0u - v) : v;
    }
}

/* ---- TLWE / TRLWE phase and decryption (Section 2.1.2 "TLWE", "TRLWE") ----- */

/* phase = b - <a, s> */
uint32_t orc_tlwe_phase(int n, const uint32_t *s, const uint32_t *c) {
    uint32_t as = 0;
    for (int i = 0; i < n; i++) as += c[i] * s[i];
    return c[n] - as;
}

/* Decryption returns (1 + sgn(phase)) / 2 with reading R1. */
int orc_tlwe_decrypt(int n, const uint32_t *s, const uint32_t *c) {
    return (int32_t)orc_tlwe_phase(n, s, c) >= 0 ? 1 : 0;
}

/* phase[X] = b[X] - a[X] s[X]; s binary (taken as an integer polynomial). */
void orc_trlwe_phase(int N, const uint32_t *s, const uint32_t *c, uint32_t *phase) {
    int32_t *si = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint32_t *as = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    for (int i = 0; i < N; i++) si[i] = (int32_t)s[i];
    orc_poly_mul(N, si, c, as); /* a[X] is the first polynomial of c */
    for (int i = 0; i < N; i++) phase[i] = c[N + i] - as[i];
    free(si);
    free(as);
}

void orc_trlwe_decrypt(int N, const uint32_t *s, const uint32_t *c, uint8_t *bits) {
    uint32_t *ph = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    orc_trlwe_phase(N, s, c, ph);
    for (int i = 0; i < N; i++) bits[i] = (int32_t)ph[i] >= 0 ? 1 : 0;
    free(ph);
}

/* ---- Gadget decomposition (reading R2) ------------------------------------ */

/* Digits d_1..d_l in [-Bg/2, Bg/2) with sum_j d_j 2^{32 - j Bgbit} = t rounded to
 * the nearest multiple of 2^{32 - l Bgbit}.  Adding Bg/2 to every digit position
 * and half of the last weight turns signed rounding into unsigned truncation. */
void orc_decompose(int l, int Bgbit, uint32_t t, int32_t *digits) {
    const uint32_t Bg = 1u << Bgbit, half = Bg / 2;
    uint32_t offset = 1u << (32 - l * Bgbit - 1);
    for (int j = 1; j <= l; j++) offset += half << (32 - j * Bgbit);
    uint32_t u = t + offset;
    for (int j = 1; j <= l; j++)
        digits[j - 1] = (int32_t)((u >> (32 - j * Bgbit)) & (Bg - 1)) - (int32_t)half;
}

/* ---- External product and CMUX (Section 2.1.2 "TRGSW", "CMUX") -------------- */

/* out = C (.) d = sum_{j<l} Dec_j(a) * C[j] + sum_{j<l} Dec_j(b) * C[l+j],
 * C a TRGSW u32[2l][2][N], d a TRLWE u32[2][N]; each product is in T_N[X]. */
void orc_external_product(const orc_params *p, const uint32_t *C, const uint32_t *d,
                          uint32_t *out) {
    const int N = p->N, l = p->l;
    int32_t *dig = (int32_t *)malloc(sizeof(int32_t) * (size_t)2 * l * N);
    uint32_t *prod = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *res = (uint32_t *)calloc((size_t)2 * N, sizeof(uint32_t));
    int32_t tmp[64];
    /* digit polynomials: row j < l from the a-polynomial, row l + j from b */
    for (int c = 0; c < 2; c++)
        for (int k = 0; k < N; k++) {
            orc_decompose(l, p->Bgbit, d[c * N + k], tmp);
            for (int j = 0; j < l; j++) dig[(size_t)(c * l + j) * N + k] = tmp[j];
        }
    for (int row = 0; row < 2 * l; row++)
        for (int col = 0; col < 2; col++) {
            orc_poly_mul(N, dig + (size_t)row * N, C + ((size_t)row * 2 + col) * N, prod);
            for (int k = 0; k < N; k++) res[col * N + k] += prod[k];
        }
    memcpy(out, res, sizeof(uint32_t) * (size_t)2 * N);
    free(dig);
    free(prod);
    free(res);
    orc_extprod_calls++;
}

/* CMUX(C, d1, d0) = d0 + C (.) (d1 - d0): selects d1 when C encrypts 1. */
void orc_cmux(const orc_params *p, const uint32_t *C, const uint32_t *d1, const uint32_t *d0,
              uint32_t *out) {
    const int N2 = 2 * p->N;
    uint32_t *diff = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N2);
    uint32_t *ep = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N2);
    for (int k = 0; k < N2; k++) diff[k] = d1[k] - d0[k];
    orc_external_product(p, C, diff, ep);
    for (int k = 0; k < N2; k++) out[k] = d0[k] + ep[k];
    free(diff);
    free(ep);
}

/* ---- Bootstrapping: ModSwitch, BlindRotate, SampleExtract, IKS ------------- */

/* Reading R3: x~ = round(x * 2N / 2^32) mod 2N. */
uint32_t orc_modswitch(int N, uint32_t x) {
    int logN2 = 0;
    while ((1 << logN2) < 2 * N) logN2++;
    const int s = 32 - logN2;
    return (uint32_t)(x + (1u << (s - 1))) >> s;
}

/* Reading R4.  bar = (a~_0..a~_{n-1}, b~) in Z_{2N}; bsk u32[n][2l][2][N];
 * acc u32[2][N] receives the rotated test vector. */
void orc_blind_rotate(const orc_params *p, const uint32_t *bsk, const uint32_t *bar,
                      uint32_t *acc) {
    const int N = p->N, n = p->n;
    const size_t per = (size_t)2 * p->l * 2 * N;
    const uint32_t mu = 1u << 29;
    uint32_t *tv = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *rot = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)2 * N);
    for (int k = 0; k < N; k++) tv[k] = mu;
    memset(acc, 0, sizeof(uint32_t) * (size_t)N);                      /* a = 0 */
    orc_rotate(N, (int)((2 * N - bar[n] % (2 * N)) % (2 * N)), tv, acc + N); /* b = X^{-b~} v */
    for (int i = 0; i < n; i++) {
        orc_rotate(N, (int)bar[i], acc, rot);
        orc_rotate(N, (int)bar[i], acc + N, rot + N);
        orc_cmux(p, bsk + (size_t)i * per, rot, acc, acc);
    }
    free(tv);
    free(rot);
}

/* TRLWE -> TLWE lvl1 (coefficient 0): a'_0 = a_0, a'_j = -a_{N-j}, b' = b_0. */
void orc_sample_extract(int N, const uint32_t *c, uint32_t *out) {
    out[0] = c[0];
    for (int j = 1; j < N; j++) out[j] = 0u - c[N - j];
    out[N] = c[N];
}

/* Reading R5: digits v_1..v_t in [0, base) with sum_j v_j 2^{32 - j basebit} equal to
 * a rounded to the nearest multiple of 2^{32 - t basebit} (ties upward). */
void orc_ks_digits(int t, int bb, uint32_t a, uint32_t *digits) {
    const uint32_t prec = 1u << (32 - (1 + bb * t));
    const uint32_t abar = a + prec;
    for (int j = 0; j < t; j++)
        digits[j] = (abar >> (32 - (j + 1) * bb)) & ((1u << bb) - 1u);
}

/* ksk u32[N][t][base][n+1]; in: TLWE lvl1 u32[N+1]; out u32[n+1].
 * res = (0, b') - sum_i sum_j KSK[i][j][digit_ij(a'_i)]. */
void orc_keyswitch(const orc_params *p, const uint32_t *ksk, const uint32_t *in, uint32_t *out) {
    const int n = p->n, N = p->N, t = p->ks_t, bb = p->ks_basebit, base = 1 << bb;
    uint32_t dig[32];
    memset(out, 0, sizeof(uint32_t) * (size_t)(n + 1));
    out[n] = in[N];
    for (int i = 0; i < N; i++) {
        orc_ks_digits(t, bb, in[i], dig);
        for (int j = 0; j < t; j++) {
            const uint32_t v = dig[j];
            if (v == 0) continue;
            const uint32_t *row = ksk + ((((size_t)i * t + j) * base + v) * (size_t)(n + 1));
            for (int k = 0; k <= n; k++) out[k] -= row[k];
        }
    }
}

/* ---- Homomorphic gates (Section 2.1.2 "Homomorphic Gates"; reading R6) ----- */

/* c = (0, kappa) + s1 c1 + s2 c2 for gate type `type` (enum order NAND, AND, OR, NOR,
 * XOR, XNOR, ANDNY, ANDYN, ORNY, ORYN).  Returns 0, or -1 for an unknown type. */
int orc_gate_combine(int n, int type, const uint32_t *c1, const uint32_t *c2, uint32_t *out) {
    const uint32_t e8 = 1u << 29, e4 = 1u << 30;
    uint32_t kappa;
    int32_t s1, s2;
    switch (type) {
        case 0: kappa = e8;        s1 = -1; s2 = -1; break; /* NAND */
        case 1: kappa = 0u - e8;   s1 = 1;  s2 = 1;  break; /* AND */
        case 2: kappa = e8;        s1 = 1;  s2 = 1;  break; /* OR */
        case 3: kappa = 0u - e8;   s1 = -1; s2 = -1; break; /* NOR */
        case 4: kappa = e4;        s1 = 2;  s2 = 2;  break; /* XOR */
        case 5: kappa = 0u - e4;   s1 = -2; s2 = -2; break; /* XNOR */
        case 6: kappa = 0u - e8;   s1 = -1; s2 = 1;  break; /* ANDNY = (not a) and b */
        case 7: kappa = 0u - e8;   s1 = 1;  s2 = -1; break; /* ANDYN = a and (not b) */
        case 8: kappa = e8;        s1 = -1; s2 = 1;  break; /* ORNY = (not a) or b */
        case 9: kappa = e8;        s1 = 1;  s2 = -1; break; /* ORYN = a or (not b) */
        default: return -1;
    }
    for (int k = 0; k <= n; k++) out[k] = (uint32_t)s1 * c1[k] + (uint32_t)s2 * c2[k];
    out[n] += kappa;
    return 0;
}

/* One bootstrapped gate: combine -> ModSwitch -> BlindRotate -> SampleExtract -> IKS.
 * Returns 0, or -1 for an unknown gate type. */
int orc_homgate(const orc_params *p, const uint32_t *bsk, const uint32_t *ksk, int type,
                const uint32_t *c1, const uint32_t *c2, uint32_t *out) {
    const int n = p->n, N = p->N;
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t *bar = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)2 * N);
    uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    int rc = orc_gate_combine(n, type, c1, c2, lin);
    if (rc == 0) {
        for (int k = 0; k <= n; k++) bar[k] = orc_modswitch(N, lin[k]);
        orc_blind_rotate(p, bsk, bar, acc);
        orc_sample_extract(N, acc, ext);
        orc_keyswitch(p, ksk, ext, out);
    }
    free(lin);
    free(bar);
    free(acc);
    free(ext);
    return rc;
}

/* Gates g in [g_begin, g_end) of a batch: out[g] = gate(types[g], in[idx[g][0]], in[idx[g][1]]).
 * Returns 0, or -1 on a bad type or index. */
int orc_gate_batch(const orc_params *p, const uint32_t *bsk, const uint32_t *ksk,
                   const uint32_t *in, int64_t num_in, const uint8_t *types,
                   const int32_t *idx, uint32_t *out, int64_t g_begin, int64_t g_end) {
    const size_t w = (size_t)p->n + 1;
    for (int64_t g = g_begin; g < g_end; g++) {
        int32_t a = idx[2 * g], b = idx[2 * g + 1];
        if (a < 0 || b < 0 || a >= num_in || b >= num_in) return -1;
        if (orc_homgate(p, bsk, ksk, types[g], in + (size_t)a * w, in + (size_t)b * w,
                        out + (size_t)g * w) != 0)
            return -1;
    }
    return 0;
}

/* ---- HomMUX (reading R13) ---------------------------------------------------- */

/* HomMUX without SE and IKS: TLWE c, a, b -> TRLWE out u32[2][N]. */
void orc_hommux_noks(const orc_params *p, const uint32_t *bsk, const uint32_t *c,
                     const uint32_t *a, const uint32_t *b, uint32_t *out) {
    const int n = p->n, N = p->N;
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t *bar = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)2 * N);
    /* c AND a (type 1) */
    orc_gate_combine(n, 1, c, a, lin);
    for (int k = 0; k <= n; k++) bar[k] = orc_modswitch(N, lin[k]);
    orc_blind_rotate(p, bsk, bar, out);
    /* (not c) AND b (type 6, ANDNY) */
    orc_gate_combine(n, 6, c, b, lin);
    for (int k = 0; k <= n; k++) bar[k] = orc_modswitch(N, lin[k]);
    orc_blind_rotate(p, bsk, bar, acc);
    for (int k = 0; k < 2 * N; k++) out[k] += acc[k];
    out[N] += 1u << 29; /* + (0, mu X^0) */
    free(lin);
    free(bar);
    free(acc);
}

/* HomMUX: TLWE c, a, b -> TLWE out u32[n+1] = IKS(SE(u)). */
void orc_hommux(const orc_params *p, const uint32_t *bsk, const uint32_t *ksk, const uint32_t *c,
                const uint32_t *a, const uint32_t *b, uint32_t *out) {
    const int N = p->N;
    uint32_t *u = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)2 * N);
    uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    orc_hommux_noks(p, bsk, c, a, b, u);
    orc_sample_extract(N, u, ext);
    orc_keyswitch(p, ksk, ext, out);
    free(u);
    free(ext);
}

/* MUXes g in [g_begin, g_end): out[g] = MUX(in[idx[g][0]], in[idx[g][1]], in[idx[g][2]])
 * (selector, then the input chosen when it is 1, then the other), TLWE (noks = 0) or
 * TRLWE (noks = 1) outputs.  Returns 0, or -1 on a bad index. */
int orc_mux_batch(const orc_params *p, const uint32_t *bsk, const uint32_t *ksk,
                  const uint32_t *in, int64_t num_in, const int32_t *idx, int noks, uint32_t *out,
                  int64_t g_begin, int64_t g_end) {
    const size_t w = (size_t)p->n + 1;
    const size_t wo = noks ? (size_t)2 * p->N : w;
    for (int64_t g = g_begin; g < g_end; g++) {
        const int32_t s = idx[3 * g], a = idx[3 * g + 1], b = idx[3 * g + 2];
        if (s < 0 || a < 0 || b < 0 || s >= num_in || a >= num_in || b >= num_in) return -1;
        if (noks)
            orc_hommux_noks(p, bsk, in + (size_t)s * w, in + (size_t)a * w, in + (size_t)b * w,
                            out + (size_t)g * wo);
        else
            orc_hommux(p, bsk, ksk, in + (size_t)s * w, in + (size_t)a * w, in + (size_t)b * w,
                       out + (size_t)g * wo);
    }
    return 0;
}

/* ---- CMUX Memory (Section 8.2) ---------------------------------------------- */

/* Read unit, reading R7: addr u32[v][2l][2][N] (TRGSW of address bit j at [j]),
 * table u32[2^v][2][N]; out u32[2][N] = row at the encrypted address.
 * Level j halves the candidates: node_j[k] = CMUX(C_j, node_{j-1}[2k+1], node_{j-1}[2k]). */
void orc_cmux_tree_read(const orc_params *p, const uint32_t *addr, const uint32_t *table, int v,
                        uint32_t *out) {
    const size_t tr = (size_t)2 * p->N, gsw = (size_t)2 * p->l * tr;
    size_t rows = (size_t)1 << v;
    uint32_t *cur = (uint32_t *)malloc(sizeof(uint32_t) * rows * tr);
    memcpy(cur, table, sizeof(uint32_t) * rows * tr);
    for (int j = 0; j < v; j++) {
        rows >>= 1;
        for (size_t k = 0; k < rows; k++)
            orc_cmux(p, addr + (size_t)j * gsw, cur + (2 * k + 1) * tr, cur + (2 * k) * tr,
                     cur + k * tr);
    }
    memcpy(out, cur, sizeof(uint32_t) * tr);
    free(cur);
}

/* Write unit, reading R8: cells u32[2^v][2][N] updated in place.  For every cell c,
 * r <- new_cell; for j = 0..v-1: r <- CMUX(S_j, r, old_c), S_j = C_j if bit j of c is 1
 * else G - C_j; cell c <- r.  G has 2^{32 - (j+1) Bgbit} at coefficient 0 of the a
 * column of row j and of the b column of row l + j, zero elsewhere. */
void orc_ram_write(const orc_params *p, const uint32_t *addr, int v, const uint32_t *new_cell,
                   uint32_t *cells) {
    const int N = p->N, l = p->l;
    const size_t tr = (size_t)2 * N, gsw = (size_t)2 * l * tr;
    uint32_t *gmc = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)v * gsw);
    uint32_t *r = (uint32_t *)malloc(sizeof(uint32_t) * tr);
    /* G - C_j for every address bit (Remark, Section 8.2) */
    for (int j = 0; j < v; j++) {
        uint32_t *dst = gmc + (size_t)j * gsw;
        const uint32_t *src = addr + (size_t)j * gsw;
        for (size_t k = 0; k < gsw; k++) dst[k] = 0u - src[k];
        for (int row = 0; row < 2 * l; row++) {
            int lev = (row < l ? row : row - l) + 1;
            int col = row < l ? 0 : 1;
            dst[((size_t)row * 2 + col) * N] += 1u << (32 - lev * p->Bgbit);
        }
    }
    for (size_t c = 0; c < ((size_t)1 << v); c++) {
        uint32_t *old = cells + c * tr;
        memcpy(r, new_cell, sizeof(uint32_t) * tr);
        for (int j = 0; j < v; j++) {
            const uint32_t *S = ((c >> j) & 1) ? addr + (size_t)j * gsw : gmc + (size_t)j * gsw;
            orc_cmux(p, S, r, old, r);
        }
        memcpy(old, r, sizeof(uint32_t) * tr);
    }
    free(gmc);
    free(r);
}

/* RAM cycle, reading R14.  cells u32[w][2^v][2][N] (bit block b, cell x) updated in
 * place; addr u32[v][2l][2][N]; flag u32[n+1]; wdata u32[w][n+1]; rdata u32[w][n+1]
 * receives the read word (TLWE lvl0, before the write). */
void orc_ram_cycle(const orc_params *p, const uint32_t *bsk, const uint32_t *ksk,
                   const uint32_t *addr, int v, int w, const uint32_t *flag, const uint32_t *wdata,
                   uint32_t *cells, uint32_t *rdata) {
    const int n = p->n, N = p->N;
    const size_t tr = (size_t)2 * N, w1 = (size_t)n + 1, rows = (size_t)1 << v;
    uint32_t *rd = (uint32_t *)malloc(sizeof(uint32_t) * tr);
    uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    uint32_t *ctl = (uint32_t *)malloc(sizeof(uint32_t) * tr);
    uint32_t *lvl0 = (uint32_t *)malloc(sizeof(uint32_t) * w1);
    uint32_t *bar = (uint32_t *)malloc(sizeof(uint32_t) * w1);
    for (int b = 0; b < w; b++) {
        uint32_t *block = cells + (size_t)b * rows * tr;
        /* read unit + control unit */
        orc_cmux_tree_read(p, addr, block, v, rd);
        orc_sample_extract(N, rd, ext);
        orc_keyswitch(p, ksk, ext, rdata + (size_t)b * w1);
        orc_hommux_noks(p, bsk, flag, wdata + (size_t)b * w1, rdata + (size_t)b * w1, ctl);
        /* write unit: write bars, then the refresh of every cell */
        orc_ram_write(p, addr, v, ctl, block);
        for (size_t x = 0; x < rows; x++) {
            uint32_t *cell = block + x * tr;
            orc_sample_extract(N, cell, ext);
            orc_keyswitch(p, ksk, ext, lvl0);
            for (int k = 0; k <= n; k++) bar[k] = orc_modswitch(N, lvl0[k]);
            orc_blind_rotate(p, bsk, bar, cell);
        }
    }
    free(rd);
    free(ext);
    free(ctl);
    free(lvl0);
    free(bar);
}

/* ROM read, reading R15.  addr u32[v][2l][2][N]; table u32[T][2][N] with T = M / (N / w)
 * a power of two, v = log2 M; out_trlwe u32[2][N] (word at coefficients 0..w-1, may be
 * NULL); out_bits u32[w][n+1] (TLWE lvl0 of each bit, may be NULL). */
void orc_rom_read(const orc_params *p, const uint32_t *ksk, const uint32_t *addr,
                  const uint32_t *table, int v, int w, uint32_t *out_trlwe, uint32_t *out_bits) {
    const int N = p->N, l = p->l;
    const size_t tr = (size_t)2 * N, gsw = (size_t)2 * l * tr;
    int lo = 0;
    while ((w << lo) < N) lo++;             /* log2 (N / w) */
    const int hi = v - lo;                  /* TRLWE-selecting bits */
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * tr);
    uint32_t *rot = (uint32_t *)malloc(sizeof(uint32_t) * tr);
    uint32_t *ext = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N + 1));
    orc_cmux_tree_read(p, addr + (size_t)lo * gsw, table, hi, acc);
    for (int j = 0; j < lo; j++) {
        const int k = (2 * N - ((w << j) % (2 * N))) % (2 * N);  /* X^{-w 2^j} */
        orc_rotate(N, k, acc, rot);
        orc_rotate(N, k, acc + N, rot + N);
        orc_cmux(p, addr + (size_t)j * gsw, rot, acc, acc);
    }
    if (out_trlwe) memcpy(out_trlwe, acc, sizeof(uint32_t) * tr);
    if (out_bits)
        for (int i = 0; i < w; i++) {
            const int k = (2 * N - i) % (2 * N);                  /* X^{-i} */
            orc_rotate(N, k, acc, rot);
            orc_rotate(N, k, acc + N, rot + N);
            orc_sample_extract(N, rot, ext);
            orc_keyswitch(p, ksk, ext, out_bits + (size_t)i * (p->n + 1));
        }
    free(acc);
    free(rot);
    free(ext);
}

/* ==== Circuit Bootstrapping (Section 2.1.2 "Circuit Bootstrapping"; reading R16) ======
 *
 * TLWE lvl0 -> TRGSW lvl1.  The paper names the operation and its source (the TFHE
 * construction) and notes (Section 6.2(a)) that it needs a modulus above 64 bits in an
 * NTT; its steps, in the TFHE construction's order:
 *   1. for u = 1..l: BlindRotate the ModSwitched input (to Z_{2 N2}) over the lvl2 ring
 *      on the 64-bit torus with the test vector mu_u sum_j X^j, mu_u = 1/(2 Bg^u);
 *      SampleExtract; add mu_u to b.  The result is a lvl2 TLWE of m / Bg^u (m the input
 *      bit: phase >= 0 is 1, reading R1).
 *   2. row u-1 of the TRGSW = private functional key switch of that TLWE with
 *      f_0(x) = -s1[X] x (a TRLWE of phase -m s1 / Bg^u, i.e. m / Bg^u on the a column);
 *      row l+u-1 = the same with f_1(x) = x (m / Bg^u on the b column).
 * Torus64 functions mirror the Torus32 ones above with uint64 arithmetic. */

typedef struct { int32_t N2, l2, Bg2bit, pks_t, pks_basebit; } orc_cb_params;

/* out = a * b in Z[X]/(X^N+1) over Torus64 (schoolbook). */
void orc64_poly_mul(int N, const int32_t *a, const uint64_t *b, uint64_t *out) {
    uint64_t *acc = (uint64_t *)calloc((size_t)N, sizeof(uint64_t));
    for (int i = 0; i < N; i++) {
        const uint64_t ai = (uint64_t)(int64_t)a[i];
        for (int j = 0; j < N - i; j++) acc[i + j] += ai * b[j];
        for (int j = N - i; j < N; j++) acc[i + j - N] -= ai * b[j];
    }
    memcpy(out, acc, sizeof(uint64_t) * (size_t)N);
    free(acc);
}

/* out = X^k * p over Torus64, k in [0, 2N). */
void orc64_rotate(int N, int k, const uint64_t *p, uint64_t *out) {
    int neg = 0;
    k %= 2 * N;
    if (k < 0) k += 2 * N;
    if (k >= N) { k -= N; neg = 1; }
    for (int j = 0; j < N; j++) {
        uint64_t v = (j >= k) ? p[j - k] : (uint64_t)(0u - p[j - k + N]);
        out[j] = neg ? (uint64_t)(0u - v) : v;
    }
}

/* phase = b - <a, s> over Torus64 (lvl2 TLWE, s = s2). */
uint64_t orc64_tlwe_phase(int n, const uint32_t *s, const uint64_t *c) {
    uint64_t as = 0;
    for (int i = 0; i < n; i++) as += c[i] * (uint64_t)s[i];
    return c[n] - as;
}

/* phase[X] = b[X] - a[X] s[X] over Torus64. */
void orc64_trlwe_phase(int N, const uint32_t *s, const uint64_t *c, uint64_t *phase) {
    int32_t *si = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    uint64_t *as = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    for (int i = 0; i < N; i++) si[i] = (int32_t)s[i];
    orc64_poly_mul(N, si, c, as);
    for (int i = 0; i < N; i++) phase[i] = c[N + i] - as[i];
    free(si);
    free(as);
}

/* Reading R2 on Torus64: digits d_1..d_l in [-Bg/2, Bg/2), sum_j d_j 2^{64 - j Bgbit} =
 * t rounded to the nearest multiple of 2^{64 - l Bgbit} (ties upward). */
void orc64_decompose(int l, int Bgbit, uint64_t t, int32_t *digits) {
    const uint64_t Bg = (uint64_t)1 << Bgbit, half = Bg / 2;
    uint64_t offset = (uint64_t)1 << (64 - l * Bgbit - 1);
    for (int j = 1; j <= l; j++) offset += half << (64 - j * Bgbit);
    const uint64_t u = t + offset;
    for (int j = 1; j <= l; j++)
        digits[j - 1] = (int32_t)((u >> (64 - j * Bgbit)) & (Bg - 1)) - (int32_t)half;
}

/* out = C (.) d over Torus64: C u64[2l][2][N], d u64[2][N]. */
void orc64_external_product(int N, int l, int Bgbit, const uint64_t *C, const uint64_t *d,
                            uint64_t *out) {
    int32_t *dig = (int32_t *)malloc(sizeof(int32_t) * (size_t)2 * l * N);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *res = (uint64_t *)calloc((size_t)2 * N, sizeof(uint64_t));
    int32_t tmp[64];
    for (int c = 0; c < 2; c++)
        for (int k = 0; k < N; k++) {
            orc64_decompose(l, Bgbit, d[c * N + k], tmp);
            for (int j = 0; j < l; j++) dig[(size_t)(c * l + j) * N + k] = tmp[j];
        }
    for (int row = 0; row < 2 * l; row++)
        for (int col = 0; col < 2; col++) {
            orc64_poly_mul(N, dig + (size_t)row * N, C + ((size_t)row * 2 + col) * N, prod);
            for (int k = 0; k < N; k++) res[col * N + k] += prod[k];
        }
    memcpy(out, res, sizeof(uint64_t) * (size_t)2 * N);
    free(dig);
    free(prod);
    free(res);
    orc_extprod_calls++;
}

/* CMUX over Torus64: out = d0 + C (.) (d1 - d0). */
void orc64_cmux(int N, int l, int Bgbit, const uint64_t *C, const uint64_t *d1,
                const uint64_t *d0, uint64_t *out) {
    uint64_t *diff = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)2 * N);
    uint64_t *ep = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)2 * N);
    for (int k = 0; k < 2 * N; k++) diff[k] = d1[k] - d0[k];
    orc64_external_product(N, l, Bgbit, C, diff, ep);
    for (int k = 0; k < 2 * N; k++) out[k] = d0[k] + ep[k];
    free(diff);
    free(ep);
}

/* Reading R4 on the lvl2 ring: bar = (a~, b~) in Z_{2 N2} (length n + 1); bsk2
 * u64[n][2 l2][2][N2]; acc u64[2][N2] = BlindRotate of the test vector mu sum_j X^j. */
void orc64_blind_rotate(const orc_params *p, const orc_cb_params *q, const uint64_t *bsk2,
                        const uint32_t *bar, uint64_t mu, uint64_t *acc) {
    const int N = q->N2, n = p->n;
    const size_t per = (size_t)2 * q->l2 * 2 * N;
    uint64_t *tv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t *rot = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)2 * N);
    for (int k = 0; k < N; k++) tv[k] = mu;
    memset(acc, 0, sizeof(uint64_t) * (size_t)N);
    orc64_rotate(N, (int)((2 * N - bar[n] % (2 * N)) % (2 * N)), tv, acc + N);
    for (int i = 0; i < n; i++) {
        orc64_rotate(N, (int)bar[i], acc, rot);
        orc64_rotate(N, (int)bar[i], acc + N, rot + N);
        orc64_cmux(N, q->l2, q->Bg2bit, bsk2 + (size_t)i * per, rot, acc, acc);
    }
    free(tv);
    free(rot);
}

/* TRLWE -> TLWE (coefficient 0) over Torus64. */
void orc64_sample_extract(int N, const uint64_t *c, uint64_t *out) {
    out[0] = c[0];
    for (int j = 1; j < N; j++) out[j] = 0u - c[N - j];
    out[N] = c[N];
}

/* Step 1 for one u: lvl0 TLWE in u32[n+1] -> lvl2 TLWE out u64[N2+1] of m / Bg^u. */
void orc_cb_tlwe2(const orc_params *p, const orc_cb_params *q, const uint64_t *bsk2,
                  const uint32_t *in, int u, uint64_t *out) {
    const int n = p->n, N2 = q->N2;
    uint32_t *bar = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n + 1));
    uint64_t *acc = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)2 * N2);
    const uint64_t mu = (uint64_t)1 << (64 - u * p->Bgbit - 1); /* 1 / (2 Bg^u) */
    for (int k = 0; k <= n; k++) bar[k] = orc_modswitch(N2, in[k]);
    orc64_blind_rotate(p, q, bsk2, bar, mu, acc);
    orc64_sample_extract(N2, acc, out);
    out[N2] += mu;
    free(bar);
    free(acc);
}

/* Unsigned base-2^bb digits of a Torus64 value rounded to t digits (reading R5). */
void orc_pks_digits(int t, int bb, uint64_t a, uint32_t *digits) {
    const uint64_t prec = (uint64_t)1 << (64 - (1 + bb * t));
    const uint64_t abar = a + prec;
    for (int j = 0; j < t; j++)
        digits[j] = (uint32_t)((abar >> (64 - (j + 1) * bb)) & (((uint64_t)1 << bb) - 1));
}

/* Private functional key switch (reading R16): lvl2 TLWE in u64[N2+1] -> TRLWE lvl1
 * out u32[2][N] with phase f_z(phase(in)).  pksk u32[2][N2+1][t][base][2][N].  With
 * a_{N2} = b and k_{N2} = -1: out = -sum_{i <= N2} sum_j PKSK[z][i][j][digit_j(a_i)]. */
void orc_private_keyswitch(const orc_params *p, const orc_cb_params *q, const uint32_t *pksk,
                           int z, const uint64_t *in, uint32_t *out) {
    const int N = p->N, N2 = q->N2, t = q->pks_t, bb = q->pks_basebit, base = 1 << bb;
    const size_t tr = (size_t)2 * N;
    uint32_t dig[64];
    memset(out, 0, sizeof(uint32_t) * tr);
    for (int i = 0; i <= N2; i++) {
        orc_pks_digits(t, bb, in[i], dig);
        for (int j = 0; j < t; j++) {
            const uint32_t v = dig[j];
            if (v == 0) continue;
            const uint32_t *row =
                pksk + ((((size_t)z * (N2 + 1) + i) * t + j) * base + v) * tr;
            for (size_t k = 0; k < tr; k++) out[k] -= row[k];
        }
    }
}

/* Circuit bootstrapping of one lvl0 TLWE: out u32[2l][2][N], a TRGSW of the input bit. */
void orc_circuit_bootstrap(const orc_params *p, const orc_cb_params *q, const uint64_t *bsk2,
                           const uint32_t *pksk, const uint32_t *in, uint32_t *out) {
    const int l = p->l;
    const size_t tr = (size_t)2 * p->N;
    uint64_t *t2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(q->N2 + 1));
    for (int u = 1; u <= l; u++) {
        orc_cb_tlwe2(p, q, bsk2, in, u, t2);
        orc_private_keyswitch(p, q, pksk, 0, t2, out + (size_t)(u - 1) * tr);
        orc_private_keyswitch(p, q, pksk, 1, t2, out + (size_t)(l + u - 1) * tr);
    }
    free(t2);
}
