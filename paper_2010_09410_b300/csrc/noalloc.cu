// noalloc.cu -- tfhe_gate_batch_noalloc: the NTT-form gate batch with its scratch in a
// fixed device array compiled into the library, for callers that must not allocate
// device memory while they run.
//
// Under lazy module loading (the CUDA default) the array's module is loaded, and its
// memory allocated, the first time host code touches one of its symbols.  So
// tfhe_ctx_create calls tfhe_noalloc_prepare, which looks the array's device address up
// (loading the module) and loads the kernels the entry point launches, while the caller
// may still allocate; the address is kept in the context.  A call of the entry point
// then only reads it.  A context lives inside one CUDA context: after a device reset
// the caller creates new contexts, which resolve the address again.
//
// The scratch is one file-scope __device__ array shared by every call on a device:
// the ModSwitched combinations u32[G][n+1] followed (at a 256-byte boundary) by the
// accumulators u32[G][2][N].  Every word a call reads from it was written earlier in
// the same call (the combination kernel writes all of bar, BlindRotate writes all of
// acc), so nothing needs clearing between calls; but two calls whose kernels overlap
// on the GPU (different streams, or different contexts on the same device) share the
// array and race.
#include "common.cuh"

int tfhe_launch_combine(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                        const int32_t *in_idx, uint32_t *bar, int G, cudaStream_t st);
int tfhe_launch_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                  const uint8_t *types, const int32_t *idx, int64_t num_in,
                                  cudaStream_t st);

// 2 MiB of scratch per device (195 gates at n = 630, N = 1024).
static constexpr size_t kScratchWords = (size_t)1 << 19;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

int tfhe_preload_gate_kernels(tfhe_ctx *ctx);
int tfhe_preload_ntt_kernels(tfhe_ctx *ctx);

// Device address of g_noalloc_scratch for the context's device (current when called).
// In host code the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress.  Also loads the kernels the entry point launches.  Not fatal for
// the context: on failure the entry point reports the recorded cause.
int tfhe_noalloc_prepare(tfhe_ctx *ctx) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        ctx->noalloc_scratch = nullptr;
        ctx->noalloc_err = std::string("scratch address lookup: ") + cudaGetErrorString(e);
        return TFHE_ECUDA;
    }
    int rc = tfhe_preload_gate_kernels(ctx);
    if (rc == TFHE_OK) rc = tfhe_preload_ntt_kernels(ctx);
    if (rc != TFHE_OK) {
        ctx->noalloc_scratch = nullptr;
        ctx->noalloc_err = "kernel preload: " + ctx->err;
        return rc;
    }
    ctx->noalloc_scratch = (uint32_t *)p;
    return TFHE_OK;
}

static size_t round256(size_t words) { return (words + 63) & ~(size_t)63; }

extern "C" int tfhe_gate_batch_noalloc(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in,
                                       const uint8_t *types, const int32_t *in_idx,
                                       uint32_t *out, int G, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    if (G < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch_noalloc: G < 0");
    if (G == 0) return TFHE_OK;
    if (!in || !types || !in_idx || !out || num_in < 1)
        return tfhe_set_error(ctx, TFHE_EINVAL, "gate_batch_noalloc: null pointer or num_in < 1");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "gate_batch_noalloc: no keys");
    const tfhe_params &p = ctx->p;
    const size_t bar_words = round256((size_t)G * (p.n + 1));
    const size_t need = bar_words + (size_t)G * 2 * p.N;
    if (need > kScratchWords) {
        const size_t per = (size_t)(p.n + 1) + 2 * (size_t)p.N;
        return tfhe_set_error(
            ctx, TFHE_EINVAL,
            "gate_batch_noalloc: batch needs " + std::to_string(need * 4) +
                " bytes of scratch, more than the fixed " + std::to_string(kScratchWords * 4) +
                " bytes; use at most about " + std::to_string(kScratchWords / per) +
                " gates per call with these parameters");
    }
    uint32_t *scratch = ctx->noalloc_scratch;  // resolved by tfhe_ctx_create
    if (!scratch)
        return tfhe_set_error(ctx, TFHE_ECUDA, "gate_batch_noalloc: scratch unavailable (" +
                                                   ctx->noalloc_err + ")");
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    uint32_t *bar = scratch;
    uint32_t *acc = scratch + bar_words;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = tfhe_launch_combine(ctx, in, num_in, types, in_idx, bar, G, st);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_blind_rotate_ntt(ctx, bar, acc, G, st);
    if (rc != TFHE_OK) return rc;
    return tfhe_launch_extract_keyswitch(ctx, acc, out, G, types, in_idx, num_in, st);
}
