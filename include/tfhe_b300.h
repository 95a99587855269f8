/*
 * tfhe_b300.h -- C ABI of a B300 (sm_103a) library for TFHE gate bootstrapping and
 * CMUX-tree memory, following "Virtual Secure Platform: A Five-Stage Pipeline
 * Processor over TFHE" (Matsuoka et al.).
 *
 * Scope: the server-side hot path of the paper's encrypted processor -- every
 * two-input Homomorphic Gate of a circuit level (Section 2.1.2 "Homomorphic
 * Gates", "Bootstrapping in TFHE"), the CMUX Memory read and write units
 * (Section 8.2) and the circuit bootstrapping that feeds them TRGSW addresses.  Key generation and encryption are client-side and not part of
 * this library.
 *
 * Data conventions (all values Torus32 = uint32, arithmetic mod 2^32):
 *   TLWE lvl0   u32[n + 1]         a[0..n-1], b                    (Section 2.1.2 "TLWE")
 *   TLWE lvl1   u32[N + 1]         a[0..N-1], b
 *   TRLWE       u32[2][N]          a[X], b[X]                      (Section 2.1.2 "TRLWE")
 *   TRGSW       u32[2l][2][N]      row j < l carries m/Bg^{j+1} on a, row l+j on b
 *                                                                  (Section 2.1.2 "TRGSW")
 *   BSK         u32[n][2l][2][N]   BSK[i] = TRGSW(s0[i]) under the lvl1 key
 *   KSK         u32[N][t][2^basebit][n + 1]
 *                                  KSK[i][j][v] = TLWE_lvl0(v s1[i] / 2^{(j+1) basebit});
 *                                  entries with v = 0 are never read (a zero digit
 *                                  contributes nothing).
 *
 * Memory: every ciphertext pointer is a DEVICE pointer owned by the caller unless a
 * function says otherwise.  The context owns only its own re-laid-out key copies
 * and workspaces.  Calls are asynchronous on the given stream (a cudaStream_t
 * passed as void*, NULL for the legacy default stream) and return after
 * enqueueing.
 *
 * Errors: functions return TFHE_OK (0) or a negative TFHE_E* code.  Arguments are
 * validated on the host before anything is enqueued; on error nothing is
 * enqueued and tfhe_last_error() describes the cause.  No call aborts the process.
 * Device-side checks (gate types and input indices that live in device memory)
 * record a code in a device error word that tfhe_ctx_sync() reports.
 */
#ifndef TFHE_B300_H
#define TFHE_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tfhe_params {
    int32_t n;          /* lvl0 TLWE dimension, 1..4096 */
    int32_t N;          /* lvl1 ring degree: power of two, 256..2048 */
    int32_t l;          /* gadget levels, 1..4 */
    int32_t Bgbit;      /* log2 of the gadget base, l * Bgbit <= 31 */
    int32_t ks_t;       /* key-switching levels */
    int32_t ks_basebit; /* log2 of the key-switching base, t * basebit <= 31 */
} tfhe_params;

typedef struct tfhe_ctx tfhe_ctx;
typedef struct tfhe_plan tfhe_plan;

enum {
    TFHE_OK = 0,
    TFHE_EINVAL = -1,       /* bad argument (null pointer, size, type, index range) */
    TFHE_ENOMEM = -2,       /* device allocation failed */
    TFHE_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    TFHE_ETIMEOUT = -4,     /* a device-side wait gave up (bounded spin) */
    TFHE_EUNSUPPORTED = -5, /* parameters or form not supported by this build */
    TFHE_ENOKEYS = -6,      /* tfhe_ctx_set_keys has not been called */
    TFHE_EBOUNDS = -7       /* debug builds only (compiled with TFHE_BOUNDS_CHECK): a device
                               index check failed; the access was skipped or redirected */
};

/* Two-input gate types (uint8 in gate-type arrays).  NY negates the first input,
 * YN the second: ANDNY = (not a) and b, ORYN = a or (not b). */
enum {
    TFHE_NAND = 0, TFHE_AND = 1, TFHE_OR = 2, TFHE_NOR = 3, TFHE_XOR = 4,
    TFHE_XNOR = 5, TFHE_ANDNY = 6, TFHE_ANDYN = 7, TFHE_ORNY = 8, TFHE_ORYN = 9
};

/* How the external products of BlindRotate are computed.  Both give bit-identical
 * ciphertexts.
 *   TFHE_FORM_NTT: one thread block per gate (or CMUX); each external product is an
 *     exact negacyclic NTT over the prime 2^64 - 2^32 + 1 (the GPU library form of
 *     Section 6.2(a)).
 *   TFHE_FORM_TC: the gates of a batch share each BSK_i, so one BlindRotate step
 *     over B gates is a dense [B x 2lN] x [2lN x 2N] contraction of signed digits
 *     by negacyclic Toeplitz blocks of the key, run on the tcgen05 tensor cores
 *     with the key split into byte planes (exact in fp16, fp32 accumulation kept
 *     below 2^24, recombined mod 2^32).  Needs 256 <= N <= 1024, Bgbit <= 6 and
 *     l N 32 128 <= 2^24 (the exactness budget of a pass); otherwise the call returns
 *     TFHE_EUNSUPPORTED. */
enum { TFHE_FORM_NTT = 0, TFHE_FORM_TC = 1, TFHE_FORM_NTT2 = 2 };
/*   TFHE_FORM_NTT2: one thread block per gate like TFHE_FORM_NTT, with each external
 *     product computed by NTTs modulo the two 30-bit primes 998244353 and 754974721 in
 *     32-bit lanes and recombined by the Chinese remainder theorem (exact while
 *     2l N (Bg/2) 2^32 <= 2^58, else TFHE_EUNSUPPORTED).  The fastest form for narrow
 *     levels; the CMUX batches, trees and RAM writes always use this arithmetic. */

/* Library version (major * 10000 + minor * 100 + patch). */
int tfhe_version(void);

/* Create a context for `params` on CUDA device `device`; *out receives it.
 * TFHE_EUNSUPPORTED for parameters outside the documented ranges. */
int tfhe_ctx_create(const tfhe_params *params, int device, tfhe_ctx **out);

/* Release every device buffer the context owns.  NULL is ignored. */
void tfhe_ctx_destroy(tfhe_ctx *ctx);

/* Text of the last error recorded on this context (never NULL; "" if none).
 * Valid until the next call on the context. */
const char *tfhe_last_error(const tfhe_ctx *ctx);

/* The same text copied into a caller buffer: writes at most len - 1 bytes of it and a
 * terminating NUL into buf (nothing if buf is NULL or len <= 0) and returns the text's
 * full length in bytes, so a return value >= len means it was truncated.  Safe to keep
 * after later calls on the context.  TFHE_EINVAL for a NULL context (buf, if usable,
 * receives ""). */
int tfhe_last_error_string(const tfhe_ctx *ctx, char *buf, int len);

/* Load the bootstrapping and key-switching keys (device pointers, layouts above).
 * The context copies and re-lays them out on `stream` (NTT-domain BSK for the NTT
 * form, raw BSK for the TC form, KSK rows without the v = 0 entries and padded to
 * 16-byte multiples); the caller keeps ownership of its buffers and may free them
 * once the stream has passed this call. */
int tfhe_ctx_set_keys(tfhe_ctx *ctx, const uint32_t *bsk, const uint32_t *ksk, void *stream);

/* Pre-size the context's workspaces for batches of up to `max_gates` gates (or
 * CMUXes), so that later calls do not allocate, and build the tensor-core job table
 * for exactly `max_gates` gates (tables are per batch size, in tiles of 128 gates).
 * Required before capturing calls into a CUDA graph yourself: a call that would have
 * to allocate or upload while its stream is capturing fails with TFHE_ECUDA or
 * TFHE_EINVAL instead.  Calls with larger batches grow the workspaces themselves;
 * growing reallocates, so a graph captured earlier must not be replayed after it. */
int tfhe_ctx_reserve(tfhe_ctx *ctx, int max_gates);

/* Wait for `stream` and report device-side errors recorded by this context's
 * kernels (TFHE_EINVAL, TFHE_ETIMEOUT) or CUDA errors (TFHE_ECUDA); clears the
 * device error word. */
int tfhe_ctx_sync(tfhe_ctx *ctx, void *stream);

/* Failure-detection probe (the paper has no counterpart).  Enqueues on `stream` one
 * bounded device wait of the kind the library's persistent kernels use between blocks:
 * poll *flag (device u32) with acquire loads until it is >= target, and give up after
 * max_cycles SM clock cycles (0 .. 8e9; about 2 GHz on B300), recording TFHE_ETIMEOUT
 * in the context's device error word.  tfhe_ctx_sync then returns TFHE_ETIMEOUT and clears
 * the word; the context stays usable.  Meant for testing the time-out path with a flag
 * that nothing sets, or with one set by the host or by work ordered before this call;
 * waiting for a kernel running concurrently on another stream is not supported (nothing
 * guarantees that the two run at the same time).  TFHE_EINVAL for a null flag or
 * max_cycles out of range. */
int tfhe_ctx_probe_wait(tfhe_ctx *ctx, const uint32_t *flag, uint32_t target, int64_t max_cycles,
                        void *stream);

/* Karatsuba levels of the tensor-core form (0 .. 3; -1 selects the default: 2 for
 * N >= 1024, 1 for N = 512, else 0).  Level L computes each negacyclic product as 3^L Toeplitz products of
 * size N / 2^L (3/4 of the multiply-adds per level); results are identical for every
 * level.  Needs N / 2^L >= 128.  If keys are loaded, re-expands the key windows on the
 * legacy default stream.  TFHE_EUNSUPPORTED if the tensor-core form or level is not
 * available for these parameters. */
int tfhe_ctx_set_tc_level(tfhe_ctx *ctx, int levels);

/* The Karatsuba level the tensor-core form runs with (>= 0), or TFHE_EUNSUPPORTED if the
 * form is not available for these parameters. */
int tfhe_ctx_tc_level(tfhe_ctx *ctx);

/* How the tensor-core BlindRotate maps onto SMs.  TFHE_TC_SINGLE_SM: each SM multiplies
 * 128-gate tiles on its own (M = 128 MMAs).  TFHE_TC_SM_PAIR: thread-block clusters of
 * two SMs multiply 256-gate tile pairs together (M = 256 MMAs over both SMs' shared
 * memory and TMEM), so each SM stages only half of every key window.  -1 selects the
 * default, TFHE_TC_SINGLE_SM (faster on B300 at N = 1024).  Results are identical.
 * Applies to calls made after it (a captured plan graph keeps the variant it was
 * recorded with until it is recorded again).  tfhe_ctx_tc_variant returns the variant
 * in use.  TFHE_EUNSUPPORTED if the tensor-core form is not available. */
enum { TFHE_TC_SINGLE_SM = 0, TFHE_TC_SM_PAIR = 1 };
int tfhe_ctx_set_tc_variant(tfhe_ctx *ctx, int variant);
int tfhe_ctx_tc_variant(tfhe_ctx *ctx);

/* The tensor-core BlindRotate accumulates a product job's whole K (2l rows of the key
 * polynomial) in one pass of fp32 TMEM accumulators when, for every gate of the tile,
 * the sum of |digit| over that K is at most `limit`: with key byte planes |q| <= 128 every
 * partial sum then stays within 2^24, where fp32 holds integers exactly.  Steps of a tile
 * where some gate exceeds it take two passes of l rows (always exact for the supported
 * parameters).  limit: 0 .. 2^17 (the default, and the largest exact value); 0 forces two
 * passes everywhere; -1 restores the default.  Results are identical for every limit.
 * TFHE_EINVAL above 2^17, TFHE_EUNSUPPORTED without the tensor-core form. */
int tfhe_ctx_set_tc_pass_limit(tfhe_ctx *ctx, int limit);

/* Per-kernel timing (tracing).  When enabled, the context brackets the kernel launches of
 * each stage with CUDA events on the launching stream (not while the stream is being
 * captured into a graph).  tfhe_ctx_stage_times waits for the recorded events, writes
 * the summed device time in milliseconds and the number of kernel launches of each stage
 * into ms[TFHE_NUM_STAGES] and launches[TFHE_NUM_STAGES] (either may be NULL), and
 * resets the counters. */
enum {
    TFHE_STAGE_COMBINE = 0,          /* gate linear combination + ModSwitch (one launch) */
    TFHE_STAGE_BLIND_ROTATE_NTT = 1, /* whole BlindRotate, NTT form (one launch) */
    TFHE_STAGE_TC_AUX = 2,           /* TC form: re-layout of the accumulators to [G][2][N]
                                        (one launch; not on the gate path, whose key
                                        switch reads the tensor-core layout directly) */
    TFHE_STAGE_BLIND_ROTATE_TC = 3,  /* TC form: the persistent BlindRotate launch (on the
                                        gate path it also forms the gate combinations, and
                                        no combine launch is made) */
    TFHE_STAGE_KEYSWITCH = 4,        /* SampleExtract + identity key switch (one launch) */
    TFHE_STAGE_CMUX = 5,             /* CMUX batches, tree levels, RAM write */
    TFHE_STAGE_CB_BLIND_ROTATE = 6,  /* circuit bootstrapping: lvl2 BlindRotates (one launch) */
    TFHE_STAGE_CB_KEYSWITCH = 7,     /* circuit bootstrapping: private key switches */
    TFHE_NUM_STAGES = 8
};
int tfhe_ctx_enable_timing(tfhe_ctx *ctx, int on);
int tfhe_ctx_stage_times(tfhe_ctx *ctx, double *ms, int64_t *launches);

/* Bootstrapped two-input gates (Section 2.1.2 "Homomorphic Gates"; a circuit level
 * of independent gates, Section 6.2(d)):
 *   out[g] = HomGate(types[g], in[in_idx[2g]], in[in_idx[2g+1]])   for g < G
 * in:      device u32[num_in][n+1] lvl0 TLWE
 * types:   device u8[G], each < 10
 * in_idx:  device i32[G][2], each in [0, num_in).  Both are checked on the device:
 *          a bad type or index gives that gate an all-zero output and records
 *          TFHE_EINVAL in the device error word (see tfhe_ctx_sync)
 * out:     device u32[G][n+1]; must not overlap rows of `in` read by this call
 * form:    TFHE_FORM_NTT, TFHE_FORM_TC, TFHE_FORM_NTT2, or -1 for the form (and Karatsuba
 *          level) chosen for the batch width: tfhe_ctx_autotune's table when present, else
 *          the level scheduler's fixed rule (the two-prime form below about 1,280 gates)
 * Each gate: linear combination, ModSwitch to Z_2N, BlindRotate of the test vector
 * (n CMUXes against BSK), SampleExtract, identity key switch. */
int tfhe_gate_batch(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                    const int32_t *in_idx, uint32_t *out, int G, int form, void *stream);

/* HomMUX (Section 2.1.2 "Homomorphic Gates": the three-operand MUX; "HomMUX without SE
 * and IKS"): out[g] = MUX(in[idx3[g][0]], in[idx3[g][1]], in[idx3[g][2]]), i.e. the
 * selector's plaintext chooses the second input when it is 1 and the third when it is 0.
 * Two bootstraps per MUX: BlindRotate of (selector AND second) and of ((not selector)
 * AND third), whose TRLWEs are summed with (0, 1/8 X^0); tfhe_mux_batch then applies
 * SampleExtract and the identity key switch (out: device u32[G][n+1] TLWE lvl0), while
 * tfhe_mux_batch_noks returns the summed TRLWE (out_trlwe: device u32[G][2][N]).
 * in: device u32[num_in][n+1]; idx3: device int32[G][3]; form as for tfhe_gate_batch
 * (-1 chooses by the width 2G).
 * Host-detectable errors return before launch; a MUX with an index outside
 * [0, num_in) gets an all-zero output and TFHE_EINVAL at the next tfhe_ctx_sync.
 * Asynchronous on `stream`; workspaces for 2G bootstraps are grown as needed. */
int tfhe_mux_batch(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const int32_t *idx3,
                   uint32_t *out, int G, int form, void *stream);
int tfhe_mux_batch_noks(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const int32_t *idx3,
                        uint32_t *out_trlwe, int G, int form, void *stream);

/* tfhe_gate_batch with HOST buffers (pinned or pageable): copies the inputs in,
 * evaluates, copies the outputs back, and returns once `out` holds the result.
 * Uses context-owned device staging buffers. */
int tfhe_gate_batch_host(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                         const uint8_t *types, const int32_t *in_idx, uint32_t *out, int G,
                         int form, void *stream);

/* tfhe_gate_batch (NTT form) without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not call cudaMalloc
 * while they run -- for example a process whose device memory is all owned by
 * another allocator (a framework's caching pool, or an arena reserved at start-up),
 * where a fresh allocation can fail even though the work fits, or a serving loop that
 * cannot let an allocation or free stall the device in the middle of a request.
 * Arguments and results are those of tfhe_gate_batch with form TFHE_FORM_NTT; the
 * context must already hold its keys (created and loaded beforehand, when allocating
 * is still allowed).  Instead of the context's workspaces, the call uses a fixed
 * 2 MiB scratch array compiled into the library, which every GPU that loads the
 * library holds until the process exits.  It therefore accepts at most
 * G * ((n+1) + 2N) * 4 bytes (rounded) of scratch: 195 gates at n = 630, N = 1024;
 * larger batches return TFHE_EINVAL without enqueueing anything.  tfhe_ctx_create
 * looks up the array's device address (cudaGetSymbolAddress, which under lazy module
 * loading loads the array's module and so allocates it) and loads the kernels this
 * entry point launches; a call then only reads the stored address.  The address belongs
 * to the CUDA context current at tfhe_ctx_create: after a device reset, create new
 * contexts.  All calls on a device share the one array: calls whose work overlaps on
 * the GPU (other streams, other contexts) race and must be serialised by the caller.
 * Calls no cudaMalloc, cudaFree or allocating routine. */
int tfhe_gate_batch_noalloc(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                            const uint8_t *types, const int32_t *in_idx, uint32_t *out, int G,
                            void *stream);

/* The stages of tfhe_gate_batch, exposed for testing and for callers that build
 * their own schedules.
 *   tfhe_blind_rotate: bar device u32[G][n+1] with values in [0, 2N) (ModSwitched
 *     a~_0..a~_{n-1}, b~); acc device u32[G][2][N] receives the accumulator
 *     encrypting X^{-b~ + sum a~_i s_i} v, v the test vector with every coefficient
 *     1/8 (Section 2.1.2 "Bootstrapping in TFHE", "CMUX").
 *   tfhe_extract_keyswitch: acc device u32[G][2][N] -> out device u32[G][n+1]:
 *     SampleExtract of coefficient 0 and identity key switch (Section 2.1.2
 *     "Sample Extraction and Identity Key Switching"). */
/* (form as for tfhe_gate_batch, -1 included) */
int tfhe_blind_rotate(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G, int form,
                      void *stream);
int tfhe_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                           void *stream);

/* Batched CMUX (Section 2.1.2 "CMUX"): out[k] = d0[k] + C_k (.) (d1[k] - d0[k]) with
 * C_k = trgsw + (k / group) * (2l * 2 * N) -- consecutive runs of `group` CMUXes
 * share one TRGSW selector.  d1, d0, out: device u32[B][2][N]; out may alias d0 or
 * d1 (same k only).  trgsw: device u32[ceil(B / group)][2l][2][N].
 * form TFHE_FORM_NTT or TFHE_FORM_NTT2: the two-prime NTT arithmetic of TFHE_FORM_NTT2.
 * TFHE_FORM_TC: groups of at least 128 CMUXes sharing a selector run on the tensor cores
 * (the selector takes the place of BSK_i in one BlindRotate step; its key windows are
 * expanded on each call, 3.5 MB per selector at N = 1024), smaller groups in the
 * two-prime NTT form.  Results are identical in every form. */
int tfhe_cmux_batch(tfhe_ctx *ctx, const uint32_t *trgsw, int group, const uint32_t *d1,
                    const uint32_t *d0, uint32_t *out, int B, int form, void *stream);

/* CMUX-tree read unit (Section 8.2 "Read Unit"): R independent reads of a table of
 * 2^v TRLWE rows.  Address bit j (least significant first) selects at tree level j:
 *   node_j[k] = CMUX(C_{r,j}, node_{j-1}[2k+1], node_{j-1}[2k]),  node_{-1} = table.
 * addr_trgsw: device u32[R][v][2l][2][N]; table: device u32[2^v][2][N];
 * out: device u32[R][2][N].  1 <= v <= 16.  form as for tfhe_cmux_batch: with
 * TFHE_FORM_TC the levels with at least 128 CMUXes per read run on the tensor cores. */
int tfhe_cmux_tree_read(tfhe_ctx *ctx, const uint32_t *addr_trgsw, const uint32_t *table, int v,
                        uint32_t *out, int R, int form, void *stream);

/* RAM write unit, CMUX part (Section 8.2 "Write Unit" and its Remark): for every
 * cell c of the 2^v cells, r <- new_cell; for j = 0..v-1: r <- CMUX(S_j, r, cell_c)
 * with S_j = C_j if bit j of c is 1 else G - C_j (G the gadget TRGSW of 1); then
 * cell_c <- r.  addr_trgsw: device u32[v][2l][2][N]; new_cell: device u32[2][N];
 * cells: device u32[2^v][2][N], updated in place.  1 <= v <= 16.  Every form runs the
 * write bars in the two-prime NTT arithmetic: at step j a cell takes C_j or G - C_j by
 * bit j of its index, so the cells that share a selector are not contiguous tiles. */
int tfhe_ram_write(tfhe_ctx *ctx, const uint32_t *addr_trgsw, int v, const uint32_t *new_cell,
                   uint32_t *cells, int form, void *stream);

/* ---- Circuit Bootstrapping (Section 2.1.2 "Circuit Bootstrapping"; Section 8.2: the
 * memory controller feeds TLWE address bits, which circuit bootstrapping turns into the
 * TRGSW selectors of the CMUX Memory; Section 6.2(a) names it an open problem on GPUs
 * because its modulus exceeds the 64-bit NTT prime).
 *
 * A lvl0 TLWE c of bit m becomes a lvl1 TRGSW of m in two steps:
 *   1. for u = 1..l: ModSwitch c to Z_{2 N2}; BlindRotate over the lvl2 ring (degree N2,
 *      64-bit torus: x -> round(x 2^64) mod 2^64) with BSK2 and the test vector
 *      1/(2 Bg^u) sum_j X^j; SampleExtract; add 1/(2 Bg^u) to b.  Result: a lvl2 TLWE
 *      u64[N2 + 1] of m / Bg^u.
 *   2. TRGSW row u-1 = private functional key switch of that TLWE with f_0(x) = -s1[X] x
 *      (phase -m s1 / Bg^u, i.e. m / Bg^u on the a column); row l+u-1 = the same with
 *      f_1(x) = x (m / Bg^u on the b column).
 * The lvl2 products are exact: each 64-bit key word is split into 32-bit halves, and
 * each half's product with the digits (|sum| < 2^63) goes through the NTT over
 * 2^64 - 2^32 + 1; the halves recombine mod 2^64.
 *
 * Key layouts (device pointers, caller-owned):
 *   BSK2  u64[n][2 l2][2][N2]   BSK2[i] = TRGSW_lvl2(s0[i]) over the 64-bit torus, rows as
 *                               for the lvl1 TRGSW with 1/Bg2^j = 2^(64 - j Bg2bit)
 *   PKSK  u32[2][N2 + 1][t][2^basebit][2][N]
 *                               PKSK[z][i][j][v] = TRLWE_lvl1(f_z(v k_i / 2^{(j+1) basebit})),
 *                               k_i = s2[i] for i < N2, k_{N2} = -1 (so that the TLWE's b is
 *                               input N2); entries with v = 0 are never read. */
typedef struct tfhe_cb_params {
    int32_t N2;          /* lvl2 ring degree: power of two, N..2048 */
    int32_t l2;          /* lvl2 gadget levels, 1..8 */
    int32_t Bg2bit;      /* log2 of the lvl2 gadget base, l2 * Bg2bit <= 63, 2 l2 N2 Bg2/2 < 2^31 */
    int32_t pks_t;       /* private key-switching levels */
    int32_t pks_basebit; /* log2 of its base, 1..8, pks_t * pks_basebit <= 32 */
} tfhe_cb_params;

/* Load the circuit-bootstrapping keys (layouts above) for the context's lvl0/lvl1
 * parameters.  The context copies them (BSK2 as the NTT-domain transforms of its two
 * 32-bit halves, u64[n][2 l2][2][2][N2]; PKSK without the v = 0 entries) on `stream`;
 * the caller keeps ownership of its buffers.  TFHE_EUNSUPPORTED for parameters outside
 * the ranges above; TFHE_ENOMEM if the copies do not fit (about 2.7 GB at N2 = 2048,
 * N = 1024, t = 10, basebit = 3). */
int tfhe_ctx_set_cb_keys(tfhe_ctx *ctx, const tfhe_cb_params *cbp, const uint64_t *bsk2,
                         const uint32_t *pksk, void *stream);

/* Circuit bootstrapping of R lvl0 TLWEs: in device u32[R][n+1] -> out device
 * u32[R][2l][2][N] lvl1 TRGSWs (usable as CMUX selectors, e.g. tfhe_cmux_tree_read's
 * addr_trgsw).  R*l lvl2 BlindRotates (one thread block each) then 2*R*l private key
 * switches.  TFHE_ENOKEYS without tfhe_ctx_set_cb_keys.  Workspace u64[R][l][N2+1] is
 * grown as needed.  Asynchronous on `stream`. */
int tfhe_circuit_bootstrap(tfhe_ctx *ctx, const uint32_t *in, uint32_t *out, int R, void *stream);

/* The two steps separately (for testing and custom schedules).
 *   tfhe_cb_tlwe2: in device u32[R][n+1] -> out device u64[R][l][N2+1], the lvl2 TLWE of
 *     m / Bg^u at [r][u-1].
 *   tfhe_private_keyswitch: in device u64[J][N2+1] lvl2 TLWEs -> out device u32[J][2][N]
 *     TRLWEs with phase f_z(phase of in[j]), z = 0 (f_0(x) = -s1[X] x) or 1 (f_1(x) = x):
 *     out[j] = - sum_{i <= N2} sum_{k < t} PKSK[z][i][k][digit_k(a_i)] with a_{N2} = b and
 *     the unsigned base-2^basebit digits of a_i rounded to t digits. */
int tfhe_cb_tlwe2(tfhe_ctx *ctx, const uint32_t *in, uint64_t *out, int R, void *stream);
int tfhe_private_keyswitch(tfhe_ctx *ctx, const uint64_t *in, uint32_t *out, int J, int z,
                           void *stream);

/* ---- Level scheduler (Section 6.2(d): circuit -> DAG -> levels of independent gates) */

/* One circuit, HOST arrays.  Wire w < num_inputs is primary input w; wire
 * num_inputs + g is the output of gate g.  Gates must be listed in topological
 * order: both inputs of gate g are wires < num_inputs + g. */
typedef struct tfhe_circuit {
    int32_t num_inputs;
    int32_t num_gates;
    const uint8_t *types;   /* host u8[num_gates] */
    const int32_t *in_idx;  /* host i32[num_gates][2] */
} tfhe_circuit;

/* ROM read with vertical and horizontal packing (Section 8.3 "ROM"): a ROM of 2^v words
 * of w bits (w a power of two <= N) stored as T = 2^v * w / N TRLWEs, word q of a TRLWE
 * in coefficients q w .. q w + w - 1 (bit i at q w + i).  table: device u32[T][2][N];
 * addr_trgsw: device u32[R][v][2l][2][N] (bit j of read r's address at [r][j]).  Address
 * bits 0 .. log2(N/w)-1 pick the word inside a TRLWE, the rest the TRLWE.  Per read: a
 * CMUX tree over the TRLWE bits, then a blind rotation ACC <- CMUX(C_j, X^{-w 2^j} ACC,
 * ACC) over the low bits (T - 1 + log2(N/w) CMUXes: 8 for 512 bytes at N = 1024), which
 * leaves the word at coefficients 0 .. w-1.  out_trlwe: device u32[R][2][N] or NULL;
 * out_bits: device u32[R][w][n+1] TLWE lvl0 (SampleExtract at coefficient i + identity
 * key switch) or NULL; not both NULL.  CMUXes run in the NTT form.  Asynchronous. */
int tfhe_rom_read(tfhe_ctx *ctx, const uint32_t *addr_trgsw, const uint32_t *table, int v, int w,
                  uint32_t *out_trlwe, uint32_t *out_bits, int R, void *stream);

/* One cycle of the CMUX-Memory RAM (Section 8.2: read unit, control unit, write unit)
 * at one encrypted address.  cells: device u32[w][2^v][2][N], in/out: bit block b of
 * word x at [b][x], the bit at coefficient 0 (the other coefficients are not used).
 * addr_trgsw: device u32[v][2l][2][N] (address bit j at [j]); flag: device u32[n+1] TLWE
 * lvl0 write flag; wdata: device u32[w][n+1] TLWE lvl0 write word; rdata: device
 * u32[w][n+1] out, the word read at the address before the write.  Steps: the w bit
 * blocks' CMUX trees (sharing the address) read the word; SampleExtract and the
 * identity key switch give rdata; HomMUX without SE and IKS of (flag, write bit, read
 * bit) gives the controlled data; each block's write bar takes it at the address; every
 * cell is refreshed by SampleExtract, key switching, ModSwitch and BlindRotate.  The
 * CMUX steps run in the NTT form; `form` selects the BlindRotate form of the MUX and
 * refresh bootstraps (w * 2^v + 2w bootstraps per cycle), or -1 to let each of the two
 * bootstrap batches take the form chosen for its width (tfhe_ctx_autotune's table when
 * present, else the level scheduler's fixed rule: e.g. the two-prime form for the 2w MUX
 * bootstraps and the tensor-core form for the 4096 refreshes).  w * 2^v <= 2^24. */
int tfhe_ram_cycle(tfhe_ctx *ctx, const uint32_t *addr_trgsw, int v, int w, const uint32_t *flag,
                   const uint32_t *wdata, uint32_t *cells, uint32_t *rdata, int form, void *stream);

/* Build a schedule for `num_circuits` independent circuits evaluated together:
 * gates are grouped by level (longest path from the primary inputs) and level k of
 * every circuit runs in one batch.  `form` as for tfhe_gate_batch, or -1 to let the
 * plan pick a form and Karatsuba level per level width (tfhe_ctx_autotune's table, or
 * a fixed rule before autotuning).  The plan owns its device
 * copies of the wiring; the context must outlive the plan. */
int tfhe_circuit_plan(tfhe_ctx *ctx, const tfhe_circuit *circuits, int num_circuits, int form,
                      tfhe_plan **out);

/* Number of levels of the plan, and for circuit c the (0-based) level after which
 * all of its gates are done (for per-circuit completion times). */
int tfhe_plan_num_levels(const tfhe_plan *plan);
int tfhe_plan_circuit_last_level(const tfhe_plan *plan, int c);

/* Evaluate the plan.  primary_in: device u32[sum of num_inputs][n+1], circuits in
 * order; gate_out: device u32[sum of num_gates][n+1], circuits in order, gates in
 * each circuit's original order.  With use_graph != 0 the level schedule is
 * captured once into a CUDA graph and replayed on later runs with the same
 * pointers; it is re-recorded when the pointers change or when another call has
 * reallocated a context workspace since (the graph holds their addresses).  level_events (optional, may be NULL): array of
 * tfhe_plan_num_levels() cudaEvent_t (as void*), recorded after each level when
 * use_graph == 0. */
int tfhe_plan_run(tfhe_plan *plan, const uint32_t *primary_in, uint32_t *gate_out, int use_graph,
                  void **level_events, void *stream);

/* Evaluate the plan as a dataflow (Section 6.2(d): list scheduling over the gate DAG)
 * instead of level by level: one persistent launch of two blocks per SM, in which each
 * block takes the next ready gate, evaluates it end to end in the two-prime per-gate
 * form (combination, ModSwitch, BlindRotate, SampleExtract, key switch) and makes ready
 * every consumer whose last input it produced; a wide level's last wave then overlaps the
 * next level's first gates.  Same arguments and outputs as tfhe_plan_run (the words are
 * identical: every form is exact); the plan's form choice is not used.  A block that
 * finds no ready gate waits, and gives up with TFHE_ETIMEOUT (at the next sync) only
 * after about 2 s in which no gate became ready.  TFHE_EUNSUPPORTED without the
 * two-prime form.  Asynchronous on `stream`. */
int tfhe_plan_run_dataflow(tfhe_plan *plan, const uint32_t *primary_in, uint32_t *gate_out,
                           void *stream);

void tfhe_plan_destroy(tfhe_plan *plan);

/* Plan autotuner (the level scheduler's choice of form and Karatsuba level per batch
 * width).  Times every form and tensor-core Karatsuba level on batches of 64, 128, ...
 * and max_gates gates of pseudo-random ciphertexts (one warm-up and two timed runs on
 * `stream`; the NTT form stops being timed at larger widths once it is twice as slow as
 * the best) and keeps the fastest per width; plans built afterwards with form = -1 use the
 * entry at the nearest width (log scale).  Without it plans use a fixed rule measured on
 * B300 at N = 1024.  Allocates scratch for 3 * max_gates ciphertexts; keeps the key
 * windows of the levels the table uses.  Blocks until done (seconds).  Results of every
 * form and level are identical; only speed differs. */
int tfhe_ctx_autotune(tfhe_ctx *ctx, int max_gates, void *stream);
/* The autotuner's table: fills up to `cap` entries (any pointer may be NULL) with
 * width, form, Karatsuba level (-1 for the NTT form) and milliseconds per batch; returns
 * the number of entries (0 before tfhe_ctx_autotune). */
int tfhe_ctx_tune_table(const tfhe_ctx *ctx, int *widths, int *forms, int *levels, float *ms,
                        int cap);

#ifdef __cplusplus
}
#endif

#endif /* TFHE_B300_H */
