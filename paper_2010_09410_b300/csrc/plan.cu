// plan.cu -- level scheduler (Section 6.2(d)): circuits -> DAG -> levels of independent
// gates; level k of every circuit runs as one tfhe_gate_batch; the whole level
// schedule is optionally captured into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

struct tfhe_plan {
    tfhe_ctx *ctx = nullptr;
    int num_levels = 0;
    int64_t total_inputs = 0, total_gates = 0, total_wires = 0;
    std::vector<int64_t> level_off;   // [num_levels + 1] offsets into the level-major gate list
    std::vector<int> level_form;      // form per level
    std::vector<int> level_tc;        // Karatsuba level per level (tensor-core form)
    std::vector<int> circuit_last;    // last level of each circuit
    uint8_t *d_types = nullptr;       // level-major gate types
    int32_t *d_idx = nullptr;         // level-major input wire indices (internal numbering)
    int64_t *d_perm = nullptr;        // output slot (circuit order) -> internal wire
    uint32_t *d_wires = nullptr;      // [total_wires][n+1]
    // dataflow runs (tfhe_plan_run_dataflow): consumers of each gate (CSR over the
    // level-major gate positions), gate inputs per gate, the initial queue (the gates
    // without gate inputs, then -1) and counters, reset from these copies before each run
    int32_t *d_cons_off = nullptr, *d_cons = nullptr;
    int32_t *d_pending0 = nullptr, *d_pending = nullptr;
    int32_t *d_queue0 = nullptr, *d_queue = nullptr;
    uint32_t *d_ctr0 = nullptr, *d_ctr = nullptr;
    uint32_t *d_scratch = nullptr;
    int df_blocks = 0;
    // graph cache
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const uint32_t *g_in = nullptr;
    uint32_t *g_out = nullptr;
    uint64_t g_gen = 0;  // context workspace generation the graph was recorded with
    cudaStream_t g_stream = nullptr;
};

// gate_out[s] = wires[perm[s]] for every output slot s; one block per slot.
__global__ void k_gather_rows(const uint32_t *__restrict__ wires, const int64_t *__restrict__ perm,
                              uint32_t *__restrict__ out, int w) {
    const int64_t s = blockIdx.x;
    const uint32_t *src = wires + perm[s] * w;
    uint32_t *dst = out + s * w;
    for (int k = threadIdx.x; k < w; k += blockDim.x) dst[k] = src[k];
}

extern "C" void tfhe_plan_destroy(tfhe_plan *plan) {
    if (!plan) return;
    if (plan->ctx) cudaSetDevice(plan->ctx->device);
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    if (plan->d_types) cudaFree(plan->d_types);
    if (plan->d_idx) cudaFree(plan->d_idx);
    if (plan->d_perm) cudaFree(plan->d_perm);
    if (plan->d_wires) cudaFree(plan->d_wires);
    for (void *q : {(void *)plan->d_cons_off, (void *)plan->d_cons, (void *)plan->d_pending0,
                    (void *)plan->d_pending, (void *)plan->d_queue0, (void *)plan->d_queue,
                    (void *)plan->d_ctr0, (void *)plan->d_ctr, (void *)plan->d_scratch})
        if (q) cudaFree(q);
    delete plan;
}

// Form and Karatsuba level for a level of `width` gates when the caller lets the plan
// choose (form = -1).  After tfhe_ctx_autotune: the measured winner at the nearest tuned
// width (log scale).  Before: a rule from a B300 sweep at N = 1024, n = 630 (ms per
// level; two-prime per-gate NTT / tensor core L1 / L2): 512 gates 21.1 / 43.9 / 37.1;
// 1024: 35.0 / 45.9 / 39.9; 1280: 44.2 / 47.0 / 43.7; 1536: 53.5 / 50.1 / 46.2;
// 2048: 67.4 / 63.2 / 56.3.  So the two-prime per-gate form below 1,280 gates and the
// tensor cores at the context's Karatsuba level from there (the per-gate NTT form over
// 2^64 - 2^32 + 1 when the two-prime form is not available: up to about 400 gates).
void tfhe_pick_form(tfhe_ctx *ctx, int64_t width, int *form, int *level) {
    *level = -1;
    const int ntt = ctx->bsk_ntt2 ? TFHE_FORM_NTT2 : TFHE_FORM_NTT;  // the faster per-gate form
    if (!tfhe_tc_supported(ctx)) {
        *form = ntt;
        return;
    }
    if (!ctx->tune.empty()) {
        const tfhe_ctx::TuneEntry *best = &ctx->tune[0];
        double bd = 1e30;
        for (const auto &e : ctx->tune) {
            const double d = std::fabs(std::log2((double)e.width) - std::log2((double)std::max<int64_t>(width, 1)));
            if (d < bd || (d == bd && e.width > best->width)) {
                bd = d;
                best = &e;
            }
        }
        *form = best->form;
        *level = best->level;
        return;
    }
    if (width < (ctx->bsk_ntt2 ? 1280 : 384)) {
        *form = ntt;
        return;
    }
    *form = TFHE_FORM_TC;
    *level = tfhe_tc_level(ctx);
}

// Size the context's workspaces for every level of the plan (a later call of another
// size may have changed them since the plan was built).
static int plan_reserve(tfhe_plan *plan) {
    tfhe_ctx *ctx = plan->ctx;
    int64_t max_w = 0;
    for (int L = 0; L < plan->num_levels; L++)
        max_w = std::max(max_w, plan->level_off[L + 1] - plan->level_off[L]);
    int rc = tfhe_ensure_workspace(ctx, (int)max_w);
    for (int L = 0; L < plan->num_levels && rc == TFHE_OK; L++)
        if (plan->level_form[L] == TFHE_FORM_TC)
            rc = tfhe_tc_reserve(ctx, (int)(plan->level_off[L + 1] - plan->level_off[L]),
                                 plan->level_tc[L]);
    return rc;
}

extern "C" int tfhe_circuit_plan(tfhe_ctx *ctx, const tfhe_circuit *circuits, int num_circuits,
                                 int form, tfhe_plan **out) {
    if (!ctx || !out) return TFHE_EINVAL;
    *out = nullptr;
    if (!circuits || num_circuits < 1)
        return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_plan: no circuits");
    if (form != -1 && form != TFHE_FORM_NTT && form != TFHE_FORM_TC && form != TFHE_FORM_NTT2)
        return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_plan: unknown form");
    if (form == TFHE_FORM_NTT2 && !ctx->bsk_ntt2)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "circuit_plan: two-prime NTT form unsupported");
    if (form == TFHE_FORM_TC && !tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "circuit_plan: tensor-core form unsupported");
    // levels per gate: level(g) = 1 + max(level of its input wires), primaries at -1
    std::vector<std::vector<int>> lvl(num_circuits);
    int64_t total_in = 0, total_g = 0;
    int num_levels = 0;
    for (int c = 0; c < num_circuits; c++) {
        const tfhe_circuit &C = circuits[c];
        if (C.num_inputs < 0 || C.num_gates < 0 || (C.num_gates > 0 && (!C.types || !C.in_idx)))
            return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_plan: bad circuit arrays");
        lvl[c].assign(C.num_gates, 0);
        for (int g = 0; g < C.num_gates; g++) {
            if (C.types[g] >= 10)
                return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_plan: bad gate type");
            int L = 0;
            for (int s = 0; s < 2; s++) {
                const int32_t w = C.in_idx[2 * g + s];
                if (w < 0 || w >= C.num_inputs + g)
                    return tfhe_set_error(ctx, TFHE_EINVAL,
                                          "circuit_plan: gate input is not an earlier wire");
                if (w >= C.num_inputs) L = std::max(L, lvl[c][w - C.num_inputs] + 1);
            }
            lvl[c][g] = L;
            num_levels = std::max(num_levels, L + 1);
        }
        total_in += C.num_inputs;
        total_g += C.num_gates;
    }
    tfhe_plan *plan = new tfhe_plan();
    plan->ctx = ctx;
    plan->num_levels = num_levels;
    plan->total_inputs = total_in;
    plan->total_gates = total_g;
    plan->total_wires = total_in + total_g;
    // level-major order: level, then circuit, then original gate index
    std::vector<int64_t> count(num_levels + 1, 0);
    for (int c = 0; c < num_circuits; c++)
        for (int g = 0; g < circuits[c].num_gates; g++) count[lvl[c][g] + 1]++;
    plan->level_off.assign(num_levels + 1, 0);
    for (int L = 0; L < num_levels; L++) plan->level_off[L + 1] = plan->level_off[L] + count[L + 1];
    std::vector<int64_t> fill(plan->level_off.begin(), plan->level_off.end() - 1);
    std::vector<std::vector<int64_t>> internal(num_circuits);  // gate -> internal wire
    std::vector<int64_t> in_off(num_circuits, 0);
    for (int c = 1; c < num_circuits; c++) in_off[c] = in_off[c - 1] + circuits[c - 1].num_inputs;
    std::vector<uint8_t> h_types(total_g);
    std::vector<int32_t> h_idx(2 * total_g);
    plan->circuit_last.assign(num_circuits, -1);
    for (int c = 0; c < num_circuits; c++) {
        internal[c].resize(circuits[c].num_gates);
        for (int g = 0; g < circuits[c].num_gates; g++) {
            const int64_t pos = fill[lvl[c][g]]++;
            internal[c][g] = total_in + pos;
            plan->circuit_last[c] = std::max(plan->circuit_last[c], lvl[c][g]);
        }
    }
    if (plan->total_wires >= INT32_MAX) {
        tfhe_plan_destroy(plan);
        return tfhe_set_error(ctx, TFHE_EINVAL, "circuit_plan: too many wires");
    }
    std::vector<int64_t> perm(total_g);
    int64_t slot = 0;
    for (int c = 0; c < num_circuits; c++) {
        const tfhe_circuit &C = circuits[c];
        for (int g = 0; g < C.num_gates; g++) {
            const int64_t pos = internal[c][g] - total_in;
            h_types[pos] = C.types[g];
            for (int s = 0; s < 2; s++) {
                const int32_t w = C.in_idx[2 * g + s];
                h_idx[2 * pos + s] = (int32_t)(w < C.num_inputs ? in_off[c] + w
                                                                 : internal[c][w - C.num_inputs]);
            }
            perm[slot++] = internal[c][g];
        }
    }
    plan->level_form.assign(num_levels, form);
    plan->level_tc.assign(num_levels, -1);
    int64_t max_w = 0;
    for (int L = 0; L < num_levels; L++) {
        const int64_t w = plan->level_off[L + 1] - plan->level_off[L];
        max_w = std::max(max_w, w);
        if (form == -1) tfhe_pick_form(ctx, w, &plan->level_form[L], &plan->level_tc[L]);
    }
    const size_t wb = (size_t)ctx->p.n + 1;
    if (cudaSetDevice(ctx->device) != cudaSuccess ||
        cudaMalloc(&plan->d_types, std::max<int64_t>(total_g, 1)) != cudaSuccess ||
        cudaMalloc(&plan->d_idx, std::max<int64_t>(2 * total_g, 1) * 4) != cudaSuccess ||
        cudaMalloc(&plan->d_perm, std::max<int64_t>(total_g, 1) * 8) != cudaSuccess ||
        cudaMalloc(&plan->d_wires, std::max<int64_t>(plan->total_wires, 1) * wb * 4) != cudaSuccess) {
        tfhe_plan_destroy(plan);
        return tfhe_set_error(ctx, TFHE_ENOMEM, "circuit_plan: device allocation");
    }
    if (total_g > 0 &&
        (cudaMemcpy(plan->d_types, h_types.data(), total_g, cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(plan->d_idx, h_idx.data(), 2 * total_g * 4, cudaMemcpyHostToDevice) !=
             cudaSuccess ||
         cudaMemcpy(plan->d_perm, perm.data(), total_g * 8, cudaMemcpyHostToDevice) != cudaSuccess)) {
        tfhe_plan_destroy(plan);
        return tfhe_set_error(ctx, TFHE_ECUDA, "circuit_plan: upload");
    }
    const int rc = plan_reserve(plan);  // tensor-core levels: a job table for every width
    if (rc != TFHE_OK) {
        tfhe_plan_destroy(plan);
        return rc;
    }
    // dataflow tables: consumers (CSR), gate inputs per gate, initial queue
    {
        std::vector<int32_t> pend(total_g, 0), cnt(total_g + 1, 0);
        for (int64_t q = 0; q < total_g; q++)
            for (int s = 0; s < 2; s++) {
                const int64_t w = h_idx[2 * q + s];
                if (w >= total_in) {
                    cnt[w - total_in + 1]++;
                    pend[q]++;
                }
            }
        for (int64_t q = 0; q < total_g; q++) cnt[q + 1] += cnt[q];
        std::vector<int32_t> cons(std::max<int64_t>(cnt[total_g], 1), 0), fillc(cnt.begin(), cnt.end() - 1);
        for (int64_t q = 0; q < total_g; q++)
            for (int s = 0; s < 2; s++) {
                const int64_t w = h_idx[2 * q + s];
                if (w >= total_in) cons[fillc[w - total_in]++] = (int32_t)q;
            }
        std::vector<int32_t> queue0(std::max<int64_t>(total_g, 1), -1);
        uint32_t ready = 0;
        for (int64_t q = 0; q < total_g; q++)
            if (pend[q] == 0) queue0[ready++] = (int32_t)q;
        const uint32_t ctr0[2] = {0u, ready};
        plan->df_blocks = tfhe_dataflow_blocks(ctx);
        const size_t gq = (size_t)std::max<int64_t>(total_g, 1);
        bool ok = plan->df_blocks > 0 &&
                  cudaMalloc(&plan->d_cons_off, (gq + 1) * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_cons, cons.size() * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_pending0, gq * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_pending, gq * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_queue0, gq * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_queue, gq * 4) == cudaSuccess &&
                  cudaMalloc(&plan->d_ctr0, 8) == cudaSuccess && cudaMalloc(&plan->d_ctr, 8) == cudaSuccess &&
                  cudaMalloc(&plan->d_scratch, (size_t)plan->df_blocks * wb * 4) == cudaSuccess;
        if (!ok) {
            tfhe_plan_destroy(plan);
            return tfhe_set_error(ctx, TFHE_ENOMEM, "circuit_plan: dataflow tables");
        }
        ok = cudaMemcpy(plan->d_cons_off, cnt.data(), (total_g + 1) * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(plan->d_cons, cons.data(), cons.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             (total_g == 0 || cudaMemcpy(plan->d_pending0, pend.data(), total_g * 4, cudaMemcpyHostToDevice) == cudaSuccess) &&
             cudaMemcpy(plan->d_queue0, queue0.data(), gq * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(plan->d_ctr0, ctr0, 8, cudaMemcpyHostToDevice) == cudaSuccess;
        if (!ok) {
            tfhe_plan_destroy(plan);
            return tfhe_set_error(ctx, TFHE_ECUDA, "circuit_plan: dataflow upload");
        }
    }
    *out = plan;
    return TFHE_OK;
}

// Dataflow run: every gate in the two-prime per-gate form, each started as soon as its
// inputs are written (TfheDataflow), instead of level by level.
extern "C" int tfhe_plan_run_dataflow(tfhe_plan *plan, const uint32_t *primary_in, uint32_t *gate_out,
                                      void *stream) {
    if (!plan) return TFHE_EINVAL;
    tfhe_ctx *ctx = plan->ctx;
    if ((plan->total_inputs > 0 && !primary_in) || (plan->total_gates > 0 && !gate_out))
        return tfhe_set_error(ctx, TFHE_EINVAL, "plan_run_dataflow: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "plan_run_dataflow: keys not set");
    if (!ctx->bsk_ntt2)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "plan_run_dataflow: two-prime NTT form not available here");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t wb = (size_t)ctx->p.n + 1;
    const int64_t G = plan->total_gates;
    if (plan->total_inputs > 0)
        TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(plan->d_wires, primary_in, plan->total_inputs * wb * 4,
                                           cudaMemcpyDeviceToDevice, st));
    if (G == 0) return TFHE_OK;
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(plan->d_pending, plan->d_pending0, G * 4, cudaMemcpyDeviceToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(plan->d_queue, plan->d_queue0, G * 4, cudaMemcpyDeviceToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(plan->d_ctr, plan->d_ctr0, 8, cudaMemcpyDeviceToDevice, st));
    TfheDataflow df{};
    df.wires = plan->d_wires;
    df.num_in = plan->total_inputs;
    df.G = G;
    df.types = plan->d_types;
    df.idx = plan->d_idx;
    df.cons_off = plan->d_cons_off;
    df.cons = plan->d_cons;
    df.pending = plan->d_pending;
    df.queue = plan->d_queue;
    df.ctr = plan->d_ctr;
    df.scratch = plan->d_scratch;
    df.blocks = plan->df_blocks;
    int rc = tfhe_dataflow_ntt2(ctx, df, st);
    if (rc != TFHE_OK) return rc;
    k_gather_rows<<<(unsigned)G, 128, 0, st>>>(plan->d_wires, plan->d_perm, gate_out, (int)wb);
    return tfhe_check_launch(ctx, "gather_rows");
}

extern "C" int tfhe_plan_num_levels(const tfhe_plan *plan) { return plan ? plan->num_levels : -1; }

extern "C" int tfhe_plan_circuit_last_level(const tfhe_plan *plan, int c) {
    if (!plan || c < 0 || c >= (int)plan->circuit_last.size()) return -1;
    return plan->circuit_last[c];
}

// Enqueue the whole schedule on `st`.
static int plan_enqueue(tfhe_plan *plan, const uint32_t *primary_in, uint32_t *gate_out,
                        void **events, cudaStream_t st) {
    tfhe_ctx *ctx = plan->ctx;
    const size_t wb = (size_t)ctx->p.n + 1;
    if (plan->total_inputs > 0)
        TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(plan->d_wires, primary_in,
                                           plan->total_inputs * wb * 4,
                                           cudaMemcpyDeviceToDevice, st));
    for (int L = 0; L < plan->num_levels; L++) {
        const int64_t off = plan->level_off[L];
        const int G = (int)(plan->level_off[L + 1] - off);
        int rc = tfhe_gate_batch_cfg(ctx, plan->d_wires, plan->total_wires, plan->d_types + off,
                                     plan->d_idx + 2 * off,
                                     plan->d_wires + (plan->total_inputs + off) * wb, G,
                                     plan->level_form[L], plan->level_tc[L], st);
        if (rc != TFHE_OK) return rc;
        if (events && events[L]) TFHE_CUDA_TRY(ctx, cudaEventRecord((cudaEvent_t)events[L], st));
    }
    if (plan->total_gates > 0) {
        k_gather_rows<<<(unsigned)plan->total_gates, 128, 0, st>>>(plan->d_wires, plan->d_perm,
                                                                   gate_out, (int)wb);
        return tfhe_check_launch(ctx, "gather_rows");
    }
    return TFHE_OK;
}

extern "C" int tfhe_plan_run(tfhe_plan *plan, const uint32_t *primary_in, uint32_t *gate_out,
                             int use_graph, void **level_events, void *stream) {
    if (!plan) return TFHE_EINVAL;
    tfhe_ctx *ctx = plan->ctx;
    if ((plan->total_inputs > 0 && !primary_in) || (plan->total_gates > 0 && !gate_out))
        return tfhe_set_error(ctx, TFHE_EINVAL, "plan_run: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "plan_run: keys not set");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (!use_graph) return plan_enqueue(plan, primary_in, gate_out, level_events, st);
    if (!plan->exec || plan->g_in != primary_in || plan->g_out != gate_out ||
        plan->g_gen != ctx->mem_gen) {
        if (plan->exec) cudaGraphExecDestroy(plan->exec);
        if (plan->graph) cudaGraphDestroy(plan->graph);
        plan->exec = nullptr;
        plan->graph = nullptr;
        if (!plan->cap_stream)
            TFHE_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking));
        // size every workspace first: nothing may be reallocated while recording
        int rc = plan_reserve(plan);
        if (rc != TFHE_OK) return rc;
        TFHE_CUDA_TRY(ctx, cudaStreamBeginCapture(plan->cap_stream,
                                                  cudaStreamCaptureModeThreadLocal));
        ctx->capturing = true;
        rc = plan_enqueue(plan, primary_in, gate_out, nullptr, plan->cap_stream);
        ctx->capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(plan->cap_stream, &g);
        if (rc != TFHE_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess)
            return tfhe_set_error(ctx, TFHE_ECUDA,
                                  std::string("plan graph capture: ") + cudaGetErrorString(e));
        plan->graph = g;
        TFHE_CUDA_TRY(ctx, cudaGraphInstantiate(&plan->exec, g, 0));
        plan->g_in = primary_in;
        plan->g_out = gate_out;
        plan->g_gen = ctx->mem_gen;
    }
    TFHE_CUDA_TRY(ctx, cudaGraphLaunch(plan->exec, st));
    return TFHE_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: time every form and Karatsuba level at a ladder of batch widths on
// pseudo-random ciphertexts and keep the fastest per width (used by plans, form = -1).
// ---------------------------------------------------------------------------

// in[i] = hashed words (uniform TLWEs: uniform rotations, so no BlindRotate step is
// trivial); gate g reads inputs 2g, 2g+1 and has type g mod 10.
__global__ void k_tune_inputs(uint32_t *in, size_t words, uint8_t *types, int32_t *idx, int G) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += stride) {
        uint64_t h = e * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
        h ^= h >> 31;
        h *= 0xD6E8FEB86659FD93ull;
        h ^= h >> 32;
        in[e] = (uint32_t)h;
    }
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < (size_t)G; g += stride) {
        types[g] = (uint8_t)(g % 10);
        idx[2 * g] = (int32_t)(2 * g);
        idx[2 * g + 1] = (int32_t)(2 * g + 1);
    }
}

extern "C" int tfhe_ctx_autotune(tfhe_ctx *ctx, int max_gates, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (max_gates < 1) return tfhe_set_error(ctx, TFHE_EINVAL, "autotune: max_gates < 1");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "autotune: keys not set");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t w1 = (size_t)ctx->p.n + 1;
    uint32_t *in = nullptr, *out = nullptr;
    uint8_t *types = nullptr;
    int32_t *idx = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TFHE_OK;
    if (cudaMalloc(&in, 2 * (size_t)max_gates * w1 * 4) != cudaSuccess ||
        cudaMalloc(&out, (size_t)max_gates * w1 * 4) != cudaSuccess ||
        cudaMalloc(&types, max_gates) != cudaSuccess ||
        cudaMalloc(&idx, 2 * (size_t)max_gates * 4) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = tfhe_set_error(ctx, TFHE_ENOMEM, "autotune: scratch allocation");
    }
    std::vector<tfhe_ctx::TuneEntry> table;
    if (rc == TFHE_OK) {
        k_tune_inputs<<<256, 256, 0, st>>>(in, 2 * (size_t)max_gates * w1, types, idx, max_gates);
        rc = tfhe_check_launch(ctx, "tune_inputs");
    }
    // candidates: the per-gate NTT forms, and the tensor-core form at every supported level
    std::vector<std::pair<int, int>> cand = {{TFHE_FORM_NTT, -1}};
    if (ctx->bsk_ntt2) cand.push_back({TFHE_FORM_NTT2, -1});
    if (tfhe_tc_supported(ctx))
        for (int L = 0; L <= 3; L++)
            if (tfhe_tc_ensure_level(ctx, L, st) == TFHE_OK) cand.push_back({TFHE_FORM_TC, L});
    ctx->err.clear();
    std::vector<int> widths;
    for (int w = 64; w < max_gates; w *= 2) widths.push_back(w);
    widths.push_back(max_gates);
    std::vector<bool> alive(cand.size(), true);
    for (int w : widths) {
        if (rc != TFHE_OK) break;
        tfhe_ctx::TuneEntry best{w, TFHE_FORM_NTT, -1, 1e30f};
        std::vector<float> ms(cand.size(), 1e30f);
        for (size_t ci = 0; ci < cand.size() && rc == TFHE_OK; ci++) {
            if (!alive[ci]) continue;
            float t = 1e30f;
            for (int rep = 0; rep < 3 && rc == TFHE_OK; rep++) {  // one warm-up, two timed
                cudaEventRecord(e0, st);
                rc = tfhe_gate_batch_cfg(ctx, in, 2 * (int64_t)w, types, idx, out, w,
                                         cand[ci].first, cand[ci].second, st);
                cudaEventRecord(e1, st);
                if (rc == TFHE_OK && cudaEventSynchronize(e1) != cudaSuccess)
                    rc = tfhe_set_error(ctx, TFHE_ECUDA, "autotune: timing");
                float x = 0;
                if (rc == TFHE_OK && rep > 0 && cudaEventElapsedTime(&x, e0, e1) == cudaSuccess)
                    t = std::min(t, x);
            }
            ms[ci] = t;
            if (t < best.ms) best = {w, cand[ci].first, cand[ci].second, t};
        }
        // the NTT form stops being timed once it is twice as slow as the best: its time
        // grows linearly with the width (one block per gate), while the tensor-core
        // form's per-gate cost falls as its tiles fill, so only the NTT form's standing
        // can only get worse at larger widths
        for (size_t ci = 0; ci < cand.size(); ci++)
            if (cand[ci].first != TFHE_FORM_TC && ms[ci] > 2 * best.ms) alive[ci] = false;
        table.push_back(best);
    }
    if (rc == TFHE_OK) rc = tfhe_ctx_sync(ctx, stream);
    if (rc == TFHE_OK) {
        ctx->tune = table;
        unsigned used = 0;
        for (const auto &e : table)
            if (e.form == TFHE_FORM_TC && e.level >= 0) used |= 1u << e.level;
        tfhe_tc_keep_levels(ctx, used);  // keep only the windows the table uses
    }
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (types) cudaFree(types);
    if (idx) cudaFree(idx);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

extern "C" int tfhe_ctx_tune_table(const tfhe_ctx *ctx, int *widths, int *forms, int *levels,
                                   float *ms, int cap) {
    if (!ctx) return TFHE_EINVAL;
    const int n = (int)ctx->tune.size();
    for (int i = 0; i < n && i < cap; i++) {
        if (widths) widths[i] = ctx->tune[i].width;
        if (forms) forms[i] = ctx->tune[i].form;
        if (levels) levels[i] = ctx->tune[i].level;
        if (ms) ms[i] = ctx->tune[i].ms;
    }
    return n;
}
