// ctx.cu -- context lifetime, key loading, workspaces and error reporting.
#include <cstdio>
#include <cstring>

#include "common.cuh"

int tfhe_set_error(tfhe_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int tfhe_check_launch(tfhe_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return TFHE_OK;
}

static void free_dev(void *p) {
    if (p) cudaFree(p);
}

extern "C" int tfhe_version(void) { return TFHE_VERSION; }

extern "C" const char *tfhe_last_error(const tfhe_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int tfhe_last_error_string(const tfhe_ctx *ctx, char *buf, int len) {
    if (!ctx) {
        if (buf && len > 0) buf[0] = 0;
        return TFHE_EINVAL;
    }
    const std::string &m = ctx->err;
    if (buf && len > 0) {
        const size_t k = m.size() < (size_t)(len - 1) ? m.size() : (size_t)(len - 1);
        memcpy(buf, m.data(), k);
        buf[k] = 0;
    }
    return (int)(m.size() < 0x7FFFFFFF ? m.size() : 0x7FFFFFFF);
}

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

extern "C" int tfhe_ctx_create(const tfhe_params *params, int device, tfhe_ctx **out) {
    if (!params || !out) return TFHE_EINVAL;
    *out = nullptr;
    const tfhe_params &p = *params;
    if (p.n < 1 || p.n > 4096 || !is_pow2(p.N) || p.N < 256 || p.N > 2048 || p.l < 1 ||
        p.l > 4 || p.Bgbit < 1 || p.Bgbit > 16 || p.l * p.Bgbit > 31 || p.ks_t < 1 ||
        p.ks_basebit < 1 || p.ks_basebit > 8 || p.ks_t * p.ks_basebit > 31)
        return TFHE_EUNSUPPORTED;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return TFHE_ECUDA;
    tfhe_ctx *ctx = new tfhe_ctx();
    ctx->p = p;
    ctx->device = device;
    while ((1 << ctx->logN) < p.N) ctx->logN++;
    ctx->n_pad = (p.n + 1 + 3) & ~3;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return TFHE_ECUDA;
    }
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        tfhe_ctx_destroy(ctx);
        return TFHE_ENOMEM;
    }
    int rc = tfhe_ntt_setup(ctx);
    if (rc != TFHE_OK) {
        tfhe_ctx_destroy(ctx);
        return rc;
    }
    // Loads the module of the no-allocation entry point's scratch array now, while the
    // caller may allocate (failure only disables that entry point).
    tfhe_noalloc_prepare(ctx);
    ctx->err.clear();
    *out = ctx;
    return TFHE_OK;
}

extern "C" void tfhe_ctx_destroy(tfhe_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    tfhe_tc_free(ctx);
    free_dev(ctx->bsk_ntt);
    free_dev(ctx->bsk_raw);
    free_dev(ctx->bsk_ntt2);
    free_dev(ctx->ksk);
    free_dev(ctx->psi_fwd);
    free_dev(ctx->psi_inv);
    free_dev(ctx->tw32);
    free_dev(ctx->ws_bar);
    free_dev(ctx->ws_acc);
    free_dev(ctx->ws_tmp);
    free_dev(ctx->ws_trgsw_ntt);
    free_dev(ctx->ws_gmc);
    free_dev(ctx->ws_ram);
    free_dev(ctx->bsk2_ntt);
    free_dev(ctx->pksk);
    free_dev(ctx->cb_tw);
    free_dev(ctx->ws_cb);
    free_dev(ctx->st_in);
    free_dev(ctx->st_out);
    free_dev(ctx->st_types);
    free_dev(ctx->st_idx);
    free_dev(ctx->d_err);
    for (auto &v : ctx->ev_pending)
        for (auto &pr : v) {
            cudaEventDestroy(pr.a);
            cudaEventDestroy(pr.b);
        }
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
}

// KSK [N][t][base][n+1] -> [N][t][base-1][n_pad]: drop the v = 0 entries (never read:
// a zero digit contributes nothing) and pad rows to 16-byte multiples with zeros.
__global__ void k_ksk_relayout(const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                               int N, int t, int base, int n1, int n_pad) {
    const size_t rows = (size_t)N * t * (base - 1);
    for (size_t r = blockIdx.x; r < rows; r += gridDim.x) {
        const size_t ij = r / (base - 1);
        const int v = (int)(r % (base - 1)) + 1;
        const uint32_t *s = src + (ij * base + v) * (size_t)n1;
        uint32_t *d = dst + r * (size_t)n_pad;
        for (int k = threadIdx.x; k < n_pad; k += blockDim.x) d[k] = k < n1 ? s[k] : 0u;
    }
}

extern "C" int tfhe_ctx_set_keys(tfhe_ctx *ctx, const uint32_t *bsk, const uint32_t *ksk,
                                 void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (!bsk || !ksk) return tfhe_set_error(ctx, TFHE_EINVAL, "set_keys: null key pointer");
    cudaStream_t st = (cudaStream_t)stream;
    const tfhe_params &p = ctx->p;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t trgsw_words = (size_t)2 * p.l * 2 * p.N;
    const size_t bsk_words = (size_t)p.n * trgsw_words;
    const int base = 1 << p.ks_basebit;
    const size_t ksk_words = (size_t)p.N * p.ks_t * (base - 1) * ctx->n_pad;
    if (!ctx->bsk_raw && cudaMalloc(&ctx->bsk_raw, bsk_words * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_keys: BSK copy");
    if (!ctx->bsk_ntt && cudaMalloc(&ctx->bsk_ntt, bsk_words * 8) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_keys: NTT-domain BSK");
    if (!ctx->ksk && cudaMalloc(&ctx->ksk, ksk_words * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "set_keys: KSK");
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->bsk_raw, bsk, bsk_words * 4,
                                       cudaMemcpyDeviceToDevice, st));
    int rc = tfhe_trgsw_to_ntt(ctx, bsk, ctx->bsk_ntt, (size_t)p.n, st);
    if (rc != TFHE_OK) return rc;
    if (tfhe_cmux_exact(ctx)) {  // BSK in the two-prime NTT form (TFHE_FORM_NTT2)
        if (!ctx->bsk_ntt2 && cudaMalloc(&ctx->bsk_ntt2, bsk_words * 8) != cudaSuccess)
            return tfhe_set_error(ctx, TFHE_ENOMEM, "set_keys: two-prime NTT-domain BSK");
        rc = tfhe_sel_to_ntt(ctx, bsk, reinterpret_cast<uint64_t *>(ctx->bsk_ntt2), (size_t)p.n, st);
        if (rc != TFHE_OK) return rc;
    }
    k_ksk_relayout<<<4096, 256, 0, st>>>(ksk, ctx->ksk, p.N, p.ks_t, base, p.n + 1, ctx->n_pad);
    rc = tfhe_check_launch(ctx, "ksk relayout");
    if (rc != TFHE_OK) return rc;
    rc = tfhe_tc_prepare_keys(ctx, bsk, st);
    if (rc != TFHE_OK) return rc;
    ctx->has_keys = true;
    return TFHE_OK;
}

int tfhe_grow(tfhe_ctx *ctx, void **ptr, size_t *cap_bytes, size_t need, const char *what) {
    if (need <= *cap_bytes) return TFHE_OK;
    if (ctx->capturing)
        return tfhe_set_error(ctx, TFHE_EINVAL,
                              std::string(what) + ": buffer too small while recording a graph");
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap_bytes = 0;
    ctx->mem_gen++;
    if (cudaMalloc(ptr, need) != cudaSuccess) return tfhe_set_error(ctx, TFHE_ENOMEM, what);
    *cap_bytes = need;
    return TFHE_OK;
}

int tfhe_ensure_workspace(tfhe_ctx *ctx, int gates) {
    if (gates <= ctx->ws_cap) return TFHE_OK;
    if (ctx->capturing)
        return tfhe_set_error(ctx, TFHE_EINVAL, "workspace too small while recording a graph");
    const tfhe_params &p = ctx->p;
    const int cap = gates;
    free_dev(ctx->ws_bar);
    free_dev(ctx->ws_acc);
    free_dev(ctx->ws_tmp);
    ctx->ws_bar = ctx->ws_acc = ctx->ws_tmp = nullptr;
    ctx->ws_cap = 0;
    ctx->mem_gen++;
    if (cudaMalloc(&ctx->ws_bar, (size_t)cap * (p.n + 1) * 4) != cudaSuccess ||
        cudaMalloc(&ctx->ws_acc, (size_t)cap * 2 * p.N * 4) != cudaSuccess ||
        cudaMalloc(&ctx->ws_tmp, (size_t)cap * 2 * p.N * 4) != cudaSuccess)
        return tfhe_set_error(ctx, TFHE_ENOMEM, "workspace allocation");
    ctx->ws_cap = cap;
    return TFHE_OK;
}

int tfhe_ensure_trgsw_ws(tfhe_ctx *ctx, size_t count) {
    size_t cap = ctx->ws_trgsw_cap * 2 * ctx->p.l * 2 * ctx->p.N * 8;
    const size_t need = count * 2 * ctx->p.l * 2 * ctx->p.N * 8;
    int rc = tfhe_grow(ctx, (void **)&ctx->ws_trgsw_ntt, &cap, need, "TRGSW workspace allocation");
    if (rc != TFHE_OK) {
        if (!ctx->ws_trgsw_ntt) ctx->ws_trgsw_cap = 0;
        return rc;
    }
    if (count > ctx->ws_trgsw_cap) ctx->ws_trgsw_cap = count;
    return TFHE_OK;
}

extern "C" int tfhe_ctx_reserve(tfhe_ctx *ctx, int max_gates) {
    if (!ctx || max_gates < 0) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int rc = tfhe_ensure_workspace(ctx, max_gates);
    if (rc != TFHE_OK) return rc;
    return tfhe_tc_reserve(ctx, max_gates, -1);
}

// One bounded device wait, the kind the persistent kernels use between blocks: poll
// *flag with acquire loads until it reaches `target`, give up after max_cycles SM clock
// cycles and record TFHE_ETIMEOUT in the context's error word.  One thread, no trap.
__global__ void k_probe_wait(const uint32_t *flag, uint32_t target, long long max_cycles,
                             int *err) {
    if (threadIdx.x != 0) return;
    const long long t0 = clock64();
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= target) return;
        if (clock64() - t0 > max_cycles) {
            atomicCAS(err, 0, TFHE_ETIMEOUT);
            return;
        }
        __nanosleep(1000);
    }
}

extern "C" int tfhe_ctx_probe_wait(tfhe_ctx *ctx, const uint32_t *flag, uint32_t target,
                                   int64_t max_cycles, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (!flag || max_cycles < 0 || max_cycles > 8000000000LL)
        return tfhe_set_error(ctx, TFHE_EINVAL, "probe_wait: null flag or max_cycles out of range");
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    k_probe_wait<<<1, 32, 0, (cudaStream_t)stream>>>(flag, target, (long long)max_cycles, ctx->d_err);
    return tfhe_check_launch(ctx, "probe_wait");
}

extern "C" int tfhe_ctx_sync(tfhe_ctx *ctx, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    TFHE_CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    TFHE_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        TFHE_CUDA_TRY(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
        return tfhe_set_error(ctx, h, h == TFHE_ETIMEOUT ? "device wait timed out"
                                                         : "device-side argument error");
    }
    return TFHE_OK;
}

// ---- per-kernel timing ------------------------------------------------------------

static cudaEvent_t take_event(tfhe_ctx *ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

StageTimer::StageTimer(tfhe_ctx *c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream) {
    if (!ctx->timing) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    a = take_event(ctx);
    b = take_event(ctx);
    if (a && b) cudaEventRecord(a, st);
}

void StageTimer::stop(int kernels) {
    if (!a || !b) return;
    cudaEventRecord(b, st);
    ctx->ev_pending[stage].push_back({a, b, kernels});
    a = b = nullptr;
}

StageTimer::~StageTimer() {
    if (a) ctx->ev_pool.push_back(a);
    if (b) ctx->ev_pool.push_back(b);
}

extern "C" int tfhe_ctx_enable_timing(tfhe_ctx *ctx, int on) {
    if (!ctx) return TFHE_EINVAL;
    ctx->timing = on != 0;
    return TFHE_OK;
}

extern "C" int tfhe_ctx_stage_times(tfhe_ctx *ctx, double *ms, int64_t *launches) {
    if (!ctx) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = TFHE_OK;
    for (int s = 0; s < TFHE_NUM_STAGES; s++) {
        double total = 0;
        int64_t kernels = 0;
        for (auto &pr : ctx->ev_pending[s]) {
            float t = 0;
            if (cudaEventSynchronize(pr.b) != cudaSuccess ||
                cudaEventElapsedTime(&t, pr.a, pr.b) != cudaSuccess)
                rc = tfhe_set_error(ctx, TFHE_ECUDA, "stage_times: event query failed");
            total += t;
            kernels += pr.kernels;
            ctx->ev_pool.push_back(pr.a);
            ctx->ev_pool.push_back(pr.b);
        }
        if (ms) ms[s] = total;
        if (launches) launches[s] = kernels;
        ctx->ev_pending[s].clear();
    }
    return rc;
}

extern "C" int tfhe_ctx_set_tc_level(tfhe_ctx *ctx, int levels) {
    if (!ctx) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return tfhe_tc_set_level(ctx, levels);
}

extern "C" int tfhe_ctx_tc_level(tfhe_ctx *ctx) {
    if (!ctx) return TFHE_EINVAL;
    return tfhe_tc_level(ctx);
}

extern "C" int tfhe_ctx_set_tc_variant(tfhe_ctx *ctx, int variant) {
    if (!ctx) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return tfhe_tc_set_variant(ctx, variant);
}

extern "C" int tfhe_ctx_set_tc_pass_limit(tfhe_ctx *ctx, int limit) {
    if (!ctx) return TFHE_EINVAL;
    return tfhe_tc_set_pass_limit(ctx, limit);
}

extern "C" int tfhe_ctx_tc_variant(tfhe_ctx *ctx) {
    if (!ctx) return TFHE_EINVAL;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    return tfhe_tc_variant(ctx);
}
