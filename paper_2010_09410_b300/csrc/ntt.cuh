// ntt.cuh -- in-place negacyclic NTTs over P = 2^64 - 2^32 + 1 on polynomials held in
// shared memory (used by the per-gate NTT form and by circuit bootstrapping).
#pragma once

#include "common.cuh"

// ---------------------------------------------------------------------------
// Device: in-place negacyclic transforms of `np` polynomials a[np][N] in shared memory
// ---------------------------------------------------------------------------

// Cooley-Tukey butterflies with twiddles psi^{brv(m+i)}: natural order in,
// evaluations at the odd powers of psi (bit-reversed order) out.
__device__ __forceinline__ void ntt_fwd(uint64_t *a, int np, int N, int logN,
                                        const uint64_t *__restrict__ psi) {
    const int half = N >> 1;
    for (int s = 0; s < logN; s++) {
        const int m = 1 << s, logt = logN - 1 - s, t = 1 << logt;
        for (int idx = threadIdx.x; idx < np * half; idx += blockDim.x) {
            const int poly = idx >> (logN - 1), b = idx & (half - 1);
            const int i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            uint64_t *x = a + (size_t)poly * N;
            const uint64_t S = __ldg(psi + m + i);
            const uint64_t U = x[j], V = gl_mul(x[j + t], S);
            x[j] = gl_add(U, V);
            x[j + t] = gl_sub(U, V);
        }
        __syncthreads();
    }
}

// Gentleman-Sande butterflies with psi^{-brv(h+i)}: bit-reversed in, natural out.
// The factor N^{-1} is folded into the NTT-domain keys.
__device__ __forceinline__ void ntt_inv(uint64_t *a, int np, int N, int logN,
                                        const uint64_t *__restrict__ psi_inv) {
    const int half = N >> 1;
    for (int s = 0; s < logN; s++) {
        const int logt = s, t = 1 << s, h = N >> (s + 1);
        for (int idx = threadIdx.x; idx < np * half; idx += blockDim.x) {
            const int poly = idx >> (logN - 1), b = idx & (half - 1);
            const int i = b >> logt, j = (i << (logt + 1)) + (b & (t - 1));
            uint64_t *x = a + (size_t)poly * N;
            const uint64_t S = __ldg(psi_inv + h + i);
            const uint64_t U = x[j], V = x[j + t];
            x[j] = gl_add(U, V);
            x[j + t] = gl_mul(gl_sub(U, V), S);
        }
        __syncthreads();
    }
}

