/*
 * Exhaustive checks over all 2^32 Torus32 values of the oracle's rounding steps.
 * The oracle functions are called through the pointers the test passes in; this
 * file states only the properties the scheme fixes (digit ranges and rounding
 * bounds), never the oracle's own formulas.
 */
#include <stdint.h>

typedef void (*decomp_fn)(int, int, uint32_t, int32_t *);
typedef void (*ksdig_fn)(int, int, uint32_t, uint32_t *);
typedef uint32_t (*modsw_fn)(int, uint32_t);

/* Gadget digits: every d_j in [-Bg/2, Bg/2) and t - sum_j d_j 2^{32-j Bgbit}
 * (as a signed 32-bit difference) in [-2^{31 - l Bgbit}, 2^{31 - l Bgbit}). */
uint64_t chk_decompose(void *fp, int l, int Bgbit, uint64_t lo, uint64_t hi) {
    decomp_fn f = (decomp_fn)fp;
    const int32_t half = 1 << (Bgbit - 1);
    const int64_t bound = (int64_t)1 << (31 - l * Bgbit);
    uint64_t bad = 0;
    int32_t d[16];
    for (uint64_t x = lo; x < hi; x++) {
        uint32_t t = (uint32_t)x;
        f(l, Bgbit, t, d);
        uint32_t rec = 0;
        for (int j = 1; j <= l; j++) {
            if (d[j - 1] < -half || d[j - 1] >= half) { bad++; break; }
            rec += (uint32_t)d[j - 1] * (1u << (32 - j * Bgbit));
        }
        int64_t err = (int32_t)(t - rec);
        if (err < -bound || err >= bound) bad++;
    }
    return bad;
}

/* Key-switching digits: every v_j in [0, 2^bb) and a - sum_j v_j 2^{32 - j bb} in
 * [-2^{31 - t bb}, 2^{31 - t bb}). */
uint64_t chk_ks_digits(void *fp, int t, int bb, uint64_t lo, uint64_t hi) {
    ksdig_fn f = (ksdig_fn)fp;
    const int64_t bound = (int64_t)1 << (31 - t * bb);
    uint64_t bad = 0;
    uint32_t v[32];
    for (uint64_t x = lo; x < hi; x++) {
        uint32_t a = (uint32_t)x;
        f(t, bb, a, v);
        uint32_t rec = 0;
        for (int j = 1; j <= t; j++) {
            if (v[j - 1] >= (1u << bb)) { bad++; break; }
            rec += v[j - 1] * (1u << (32 - j * bb));
        }
        int64_t err = (int32_t)(a - rec);
        if (err < -bound || err >= bound) bad++;
    }
    return bad;
}

/* ModSwitch: result in [0, 2N) and x - r 2^{32}/(2N) in [-2^{s-1}, 2^{s-1}),
 * s = 32 - log2(2N). */
uint64_t chk_modswitch(void *fp, int N, uint64_t lo, uint64_t hi) {
    modsw_fn f = (modsw_fn)fp;
    int logN2 = 0;
    while ((1 << logN2) < 2 * N) logN2++;
    const int s = 32 - logN2;
    const int64_t bound = (int64_t)1 << (s - 1);
    uint64_t bad = 0;
    for (uint64_t x = lo; x < hi; x++) {
        uint32_t r = f(N, (uint32_t)x);
        if (r >= (uint32_t)(2 * N)) { bad++; continue; }
        int64_t err = (int32_t)((uint32_t)x - (r << s));
        if (err < -bound || err >= bound) bad++;
    }
    return bad;
}
