// common.cuh -- internal definitions shared by the library's translation units:
// the context, error helpers, Torus32 polynomial helpers and arithmetic modulo the
// prime P = 2^64 - 2^32 + 1 used by the NTT form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tfhe_b300.h"

#define TFHE_VERSION 10000

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

struct TcWorkspace;  // tensor-core form buffers (tc.cu)

struct tfhe_ctx {
    tfhe_params p{};
    int device = 0;
    int sms = 0;    // multiprocessors of the device (queried on first use)
    int logN = 0;
    int n_pad = 0;  // KSK row length in words, (n + 1) rounded up to a multiple of 4
    std::string err;

    // keys
    bool has_keys = false;
    uint64_t *bsk_ntt = nullptr;  // [n][2l][2][N] NTT domain (bit-reversed), scaled by N^-1
    uint32_t *bsk_raw = nullptr;  // [n][2l][2][N] as given
    uint32_t *ksk = nullptr;      // [N][t][base - 1][n_pad], rows v = 1..base-1
    uint32_t *bsk_ntt2 = nullptr; // [n][2l][2][2 primes][N] two-prime NTT form (TFHE_FORM_NTT2)

    // NTT twiddles: psi^{brv(k)} and psi^{-brv(k)}, psi a primitive 2N-th root of unity
    uint64_t *psi_fwd = nullptr;
    uint64_t *psi_inv = nullptr;
    uint64_t n_inv = 0;
    // two-prime twiddles for CMUX products at ring degree N ([2][2][N][2], ntt32.cuh)
    uint32_t *tw32 = nullptr;

    // per-batch workspaces (grown on demand)
    int ws_cap = 0;              // capacity in gates / CMUXes
    uint32_t *ws_bar = nullptr;  // [cap][n+1] ModSwitched combination
    uint32_t *ws_acc = nullptr;  // [cap][2][N] accumulators
    uint32_t *ws_tmp = nullptr;  // [cap][2][N] scratch TRLWE (CMUX tree / RAM)
    uint64_t *ws_trgsw_ntt = nullptr;  // NTT-domain TRGSW selectors (CMUX batches)
    size_t ws_trgsw_cap = 0;           // in TRGSWs
    uint32_t *ws_gmc = nullptr;        // G - C_j selectors for the RAM write
    int ws_gmc_cap = 0;                // in TRGSWs
    uint32_t *ws_ram = nullptr;        // RAM-cycle scratch (read words, controlled data,
    size_t ws_ram_cap = 0;             //  MUX inputs, refreshed lvl0 and ModSwitched rows)

    // host-API staging (device side)
    size_t st_in_cap = 0, st_gate_cap = 0;
    uint32_t *st_in = nullptr, *st_out = nullptr;
    uint8_t *st_types = nullptr;
    int32_t *st_idx = nullptr;

    // circuit bootstrapping (cb.cu)
    bool has_cb_keys = false;
    tfhe_cb_params cbp{};
    int logN2 = 0;
    uint32_t *bsk2_ntt = nullptr;  // [n][2 l2][2][2 primes][2 halves][N2] residues, NTT domain,
                                   // Montgomery form, scaled by N2^-1
    uint32_t *pksk = nullptr;      // [2][N2+1][t][base - 1][2N], rows v = 1..base-1
    uint32_t *cb_tw = nullptr;     // two-prime twiddles for the lvl2 ring [2][2][N2][2]
    uint64_t *ws_cb = nullptr;  // lvl2 TLWEs [R][l][N2+1] between the two steps
    size_t ws_cb_cap = 0;       // bytes

    TcWorkspace *tc = nullptr;
    // plan autotuner: the fastest (form, Karatsuba level) measured per batch width
    struct TuneEntry {
        int width, form, level;
        float ms;
    };
    std::vector<TuneEntry> tune;

    // Workspace generation: bumped by every reallocation of a context-owned buffer, so a
    // captured plan graph (which holds raw addresses) knows to re-record itself.  While
    // `capturing` is set no buffer may be reallocated.
    uint64_t mem_gen = 0;
    bool capturing = false;

    int *d_err = nullptr;  // device error word (0 = ok, else a TFHE_E* code)

    // device address of the no-allocation entry point's fixed scratch array (noalloc.cu),
    // resolved at context creation; null (with the cause) if that failed
    uint32_t *noalloc_scratch = nullptr;
    std::string noalloc_err;

    // per-kernel timing (tfhe_ctx_enable_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct StageRecord {
        cudaEvent_t a, b;
        int kernels;  // kernel launches between the two events
    };
    std::vector<StageRecord> ev_pending[TFHE_NUM_STAGES];
};

// Brackets kernel launches with events when timing is on and the stream is not
// being captured.  Usage: StageTimer t(ctx, stage, st); launches; t.stop(kernels);
struct StageTimer {
    tfhe_ctx *ctx;
    int stage;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    StageTimer(tfhe_ctx *c, int s, cudaStream_t stream);
    void stop(int kernels = 1);
    ~StageTimer();  // an unstopped timer (error path) returns its events to the pool
};

// Addressing of a 2-D grid of CMUXes (x within a group sharing one selector, y the
// group): CMUX (x, y) reads d1 + x*dx + y*dy and d0 + x*dx + y*dy, writes
// out + x*ox + y*oy (word offsets) and uses selector sel + y*sy (in TRGSWs).  Only
// CMUXes with y*nx + x < count exist.
struct CmuxGeom {
    const uint32_t *d1, *d0;
    uint32_t *out;
    int64_t dx, dy, ox, oy, sy;
    int nx, ny;
    int64_t count;
};

// error recording helpers (ctx.cu)
int tfhe_set_error(tfhe_ctx *ctx, int code, const std::string &msg);
int tfhe_check_launch(tfhe_ctx *ctx, const char *what);
int tfhe_ensure_workspace(tfhe_ctx *ctx, int gates);
int tfhe_ensure_trgsw_ws(tfhe_ctx *ctx, size_t count);

// noalloc.cu: resolve the fixed scratch array and load the kernels of its entry point
int tfhe_noalloc_prepare(tfhe_ctx *ctx);

// ntt.cu
int tfhe_ntt_setup(tfhe_ctx *ctx);
// psi^{brv(k)}, psi^{-brv(k)} (psi a primitive 2N-th root of unity mod P) and N^{-1}
int tfhe_make_twiddles(tfhe_ctx *ctx, int N, uint64_t **fwd, uint64_t **inv, uint64_t *n_inv);
int tfhe_trgsw_to_ntt(tfhe_ctx *ctx, const uint32_t *trgsw, uint64_t *out, size_t count,
                      cudaStream_t st);
// CMUX selectors -> the two-prime NTT form read by tfhe_cmux_ntt and tfhe_ram_write_ntt
// (same size as tfhe_trgsw_to_ntt's output: per TRGSW 2l * 2 * N words of 8 bytes)
int tfhe_sel_to_ntt(tfhe_ctx *ctx, const uint32_t *trgsw, uint64_t *out, size_t count,
                    cudaStream_t st);
int tfhe_blind_rotate_ntt(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                          cudaStream_t st);
int tfhe_blind_rotate_ntt2(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                           cudaStream_t st);
// products of the CMUX / two-prime forms are exact for these parameters
bool tfhe_cmux_exact(const tfhe_ctx *ctx);
int tfhe_cmux_ntt(tfhe_ctx *ctx, const uint64_t *sel_ntt, const CmuxGeom &g, cudaStream_t st);
// write bars of `blocks` RAM bit blocks of 2^v cells each: block b takes new_cell +
// b * new_stride and updates cells + b * 2^v * 2N (words)
int tfhe_ram_write_ntt(tfhe_ctx *ctx, const uint64_t *c_ntt, const uint64_t *gmc_ntt, int v,
                       const uint32_t *new_cell, uint32_t *cells, cudaStream_t st,
                       int blocks = 1, int64_t new_stride = 0);

// tc.cu
int tfhe_tc_supported(const tfhe_ctx *ctx);
int tfhe_tc_prepare_keys(tfhe_ctx *ctx, const uint32_t *bsk, cudaStream_t st);
int tfhe_tc_set_level(tfhe_ctx *ctx, int level);
int tfhe_tc_level(tfhe_ctx *ctx);
// key windows of Karatsuba `level` (-1: the context's level) expanded for the loaded keys
int tfhe_tc_ensure_level(tfhe_ctx *ctx, int level, cudaStream_t st);
void tfhe_tc_keep_levels(tfhe_ctx *ctx, unsigned mask);
// tensor-core buffers and the job table of a `gates`-gate BlindRotate at `level`
int tfhe_tc_reserve(tfhe_ctx *ctx, int gates, int level);
int tfhe_tc_set_variant(tfhe_ctx *ctx, int variant);
int tfhe_tc_variant(tfhe_ctx *ctx);
int tfhe_tc_set_pass_limit(tfhe_ctx *ctx, int limit);
// Gate inputs for the tensor-core BlindRotate's fused combination: its step-0 digit jobs
// compute bar = ModSwitch(gate combination) from these (into the `bar` buffer) and
// initialise the accumulators.
// Dataflow evaluation of a gate DAG (Section 6.2(d) list scheduling) in the two-prime
// per-gate form: a persistent grid of blocks takes ready gates from a queue, evaluates
// each end to end (combination, ModSwitch, BlindRotate, SampleExtract, key switch) and
// queues every consumer whose last input it completed.  Gates are numbered 0 .. G-1;
// gate g reads wires idx[2g], idx[2g+1] and writes wire num_in + g of `wires`
// ([num_in + G][n+1]).  Consumers of g: cons[cons_off[g] .. cons_off[g+1]) (a gate that
// reads g twice appears twice); pending[g] counts g's inputs that are gates; queue holds
// the ready gates in the order they became ready (-1: not yet), its first `ready0` entries
// set; ctr = {tickets taken, gates queued}.  The caller resets pending, queue and ctr
// before each run.
// Debug builds (-DTFHE_BOUNDS_CHECK, libtfhe_b300_bounds.so): device index checks on the
// hot path.  A failed check records TFHE_EBOUNDS in the context's error word (read at the
// next sync) and the caller skips the access, or points a bulk copy at an in-bounds
// source so that its barrier still completes; nothing traps.  In normal builds every
// check is the constant true and compiles away.
#ifdef TFHE_BOUNDS_CHECK
__device__ __forceinline__ bool tfhe_in_bounds(size_t i, size_t n, int *err) {
    if (i < n) return true;
    atomicCAS(err, 0, TFHE_EBOUNDS);
    return false;
}
#else
__device__ __forceinline__ constexpr bool tfhe_in_bounds(size_t, size_t, int *) { return true; }
#endif

struct TfheDataflow {
    uint32_t *wires;
    int64_t num_in, G;
    const uint8_t *types;
    const int32_t *idx;
    const int32_t *cons_off, *cons;
    int32_t *pending, *queue;
    uint32_t *ctr;
    uint32_t *scratch;  // [blocks][n+1]: ModSwitched combination of each block's gate
    int blocks;         // grid size (two per SM); scratch holds this many rows
};
int tfhe_dataflow_ntt2(tfhe_ctx *ctx, const TfheDataflow &df, cudaStream_t st);
// the grid size the dataflow engine runs with on this context's device
int tfhe_dataflow_blocks(tfhe_ctx *ctx);

struct TcGateInputs {
    const uint32_t *in;
    int64_t num_in;
    const uint8_t *types;
    const int32_t *idx;
};
// Accumulators of the tensor-core form stay gate-fastest within tiles of this many gates:
// word k of polynomial c of gate g at [((g / TFHE_TC_TILE) * 2 + c) * N + k][g % TFHE_TC_TILE].
constexpr int TFHE_TC_TILE = 128;
// gates: NULL (bar given) or the inputs of a fused combination (bar receives it).
// tiled_acc: NULL (acc receives [G][2][N]) or receives the context's tiled accumulators
// (valid until the next tensor-core call; acc unused).
int tfhe_blind_rotate_tc(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G,
                         cudaStream_t st, int level, const TcGateInputs *gates = nullptr,
                         const uint32_t **tiled_acc = nullptr);
int tfhe_cmux_tc(tfhe_ctx *ctx, const uint32_t *sel, const CmuxGeom &g, cudaStream_t st);
// Reallocate a context-owned device buffer to at least `need` bytes (no copy); refused
// while a plan graph is being recorded; bumps mem_gen.
int tfhe_grow(tfhe_ctx *ctx, void **ptr, size_t *cap_bytes, size_t need, const char *what);
// gate.cu: building blocks of the RAM cycle (cmux.cu)
int tfhe_mux_batch_impl(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const int32_t *idx3,
                        uint32_t *out, int G, int form, bool noks, cudaStream_t st);
int tfhe_launch_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                  const uint8_t *types, const int32_t *idx, int64_t num_in,
                                  cudaStream_t st);
// true when the key switch can read the tensor-core form's tiled accumulators directly
bool tfhe_ks_reads_tiled(const tfhe_ctx *ctx);
int tfhe_launch_modswitch_rows(tfhe_ctx *ctx, const uint32_t *in, uint32_t *bar, int64_t G,
                               cudaStream_t st);
int tfhe_blind_rotate_form(tfhe_ctx *ctx, const uint32_t *bar, uint32_t *acc, int G, int form,
                           cudaStream_t st);
// plan.cu: the form (and Karatsuba level, -1 for the context's) a batch of `width` gates
// runs in when the caller lets the library choose: the autotuner's table, else a fixed rule
void tfhe_pick_form(tfhe_ctx *ctx, int64_t width, int *form, int *level);
// gate.cu: tfhe_gate_batch with the tensor-core Karatsuba level chosen per call (-1: the
// context's level)
int tfhe_gate_batch_cfg(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                        const int32_t *in_idx, uint32_t *out, int G, int form, int tc_level,
                        cudaStream_t st);
void tfhe_tc_free(tfhe_ctx *ctx);

#define TFHE_CUDA_TRY(ctx, call)                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return tfhe_set_error((ctx), TFHE_ECUDA,                                    \
                                  std::string(#call ": ") + cudaGetErrorString(e_));    \
    } while (0)

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Coefficient j of X^k * p (k in [0, 2N)) for a Torus32 polynomial p of degree < N:
// X^k p has p_{j-k} at X^j for j >= k and -p_{j-k+N} below; X^k = -X^{k-N} for k >= N.
__device__ __forceinline__ uint32_t rot_coef(const uint32_t *p, int N, int k, int j) {
    // s = j - k in (-2N, N): the source is p[s mod N], negated once exactly when
    // -N <= s < 0 (X^N = -1; two wraps cancel).  N is a power of two.
    const int s = j - k;
    const uint32_t neg = (uint32_t)((s >> 31) & ~((s + N) >> 31));  // all ones or zero
    return (p[s & (N - 1)] ^ neg) - neg;
}

// Gate constants (Section 2.1.2 "Homomorphic Gates"): c = (0, kappa) + s1 c1 + s2 c2, in
// Torus32 with 1/8 = 2^29 and 1/4 = 2^30; enum order NAND, AND, OR, NOR, XOR, XNOR,
// ANDNY, ANDYN, ORNY, ORYN (NY negates the first input, YN the second).  t < 10.
__device__ __forceinline__ void gate_coeffs(int t, uint32_t &kappa, uint32_t &s1, uint32_t &s2) {
    const int8_t k8[10] = {1, -1, 1, -1, 2, -2, -1, -1, 1, 1};  // kappa in units of 2^29
    const int8_t a1[10] = {-1, 1, 1, -1, 2, -2, -1, 1, -1, 1};
    const int8_t a2[10] = {-1, 1, 1, -1, 2, -2, 1, -1, 1, -1};
    kappa = (uint32_t)(int32_t)k8[t] << 29;
    s1 = (uint32_t)(int32_t)a1[t];
    s2 = (uint32_t)(int32_t)a2[t];
}

__device__ __forceinline__ bool gate_ok(const uint8_t *types, const int32_t *idx, int64_t num_in,
                                        int64_t g) {
    const int32_t a = idx[2 * g], b = idx[2 * g + 1];
    return types[g] < 10 && a >= 0 && b >= 0 && a < num_in && b < num_in;
}

// Signed gadget digits of t (l levels of Bgbit bits, rounding to nearest, digits in
// [-Bg/2, Bg/2)): adding Bg/2 at every level and half a unit of the last level turns
// the signed rounding into plain bit extraction of u = t + offset.
__device__ __forceinline__ uint32_t gadget_offset(int l, int Bgbit) {
    uint32_t off = 1u << (32 - l * Bgbit - 1);
    for (int j = 1; j <= l; j++) off += (1u << (Bgbit - 1)) << (32 - j * Bgbit);
    return off;
}

__device__ __forceinline__ int32_t gadget_digit(uint32_t u, int j /*1-based*/, int Bgbit) {
    return (int32_t)((u >> (32 - j * Bgbit)) & ((1u << Bgbit) - 1)) - (1 << (Bgbit - 1));
}

// ---- arithmetic modulo P = 2^64 - 2^32 + 1 (2^64 = 2^32 - 1 mod P) ----------------

static constexpr uint64_t GL_P = 0xFFFFFFFF00000001ull;
static constexpr uint64_t GL_EPS = 0xFFFFFFFFull;  // 2^64 mod P

__device__ __forceinline__ uint64_t gl_add(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    if (s < a) s += GL_EPS;  // wrapped past 2^64: add 2^64 mod P
    if (s >= GL_P) s -= GL_P;
    return s;
}

__device__ __forceinline__ uint64_t gl_sub(uint64_t a, uint64_t b) {
    uint64_t d = a - b;
    if (a < b) d -= GL_EPS;  // borrowed 2^64: subtract 2^64 mod P
    return d;
}

__device__ __forceinline__ uint64_t gl_mul(uint64_t a, uint64_t b) {
    const uint64_t lo = a * b;
    const uint64_t hi = __umul64hi(a, b);
    const uint32_t h0 = (uint32_t)hi, h1 = (uint32_t)(hi >> 32);
    // a*b = lo + h0 2^64 + h1 2^96 = lo + h0 (2^32 - 1) - h1  (mod P)
    uint64_t t = lo - h1;
    if (lo < h1) t -= GL_EPS;
    const uint64_t m = (uint64_t)h0 * GL_EPS;
    uint64_t r = t + m;
    if (r < t) r += GL_EPS;
    if (r >= GL_P) r -= GL_P;
    return r;
}

// signed digit -> residue
__device__ __forceinline__ uint64_t gl_from_i32(int32_t d) {
    return d >= 0 ? (uint64_t)d : GL_P - (uint64_t)(-(int64_t)d);
}

// residue of an integer V with |V| < P/2 -> V mod 2^32 (P = 1 mod 2^32)
__device__ __forceinline__ uint32_t gl_lift_u32(uint64_t v) {
    return (uint32_t)v - (v > (GL_P >> 1) ? 1u : 0u);
}
