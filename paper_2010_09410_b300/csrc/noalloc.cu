// noalloc.cu -- tfhe_gate_batch_noalloc: the NTT-form gate batch with its scratch in a
// fixed device array that the library owns from load time, for callers that must not
// allocate device memory while they run.
//
// The scratch is one file-scope __device__ array shared by every call on a device:
// the ModSwitched combinations u32[G][n+1] followed (at a 256-byte boundary) by the
// accumulators u32[G][2][N].  Every word a call reads from it was written earlier in
// the same call (the combination kernel writes all of bar, BlindRotate writes all of
// acc), so nothing needs clearing between calls; but two calls whose kernels overlap
// on the GPU (different streams, or different contexts on the same device) share the
// array and race.
#include <mutex>

#include "common.cuh"

int tfhe_launch_combine(tfhe_ctx *ctx, const uint32_t *in, int64_t num_in, const uint8_t *types,
                        const int32_t *in_idx, uint32_t *bar, int G, cudaStream_t st);
int tfhe_launch_extract_keyswitch(tfhe_ctx *ctx, const uint32_t *acc, uint32_t *out, int G,
                                  const uint8_t *types, const int32_t *idx, int64_t num_in,
                                  cudaStream_t st);

// 2 MiB of scratch per device (195 gates at n = 630, N = 1024).
static constexpr size_t kScratchWords = (size_t)1 << 19;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// Device address of g_noalloc_scratch per device.  In host code the array's name is
// only a host-side stand-in, so the address is looked up once per device (with that
// device current) and cached.
static constexpr int kMaxDevices = 128;
static std::mutex g_scratch_mu;
static uint32_t *g_scratch_addr[kMaxDevices];

static int scratch_address(tfhe_ctx *ctx, uint32_t **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const int dev = ctx->device;
    if (dev < 0 || dev >= kMaxDevices)
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "gate_batch_noalloc: device id too large");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return tfhe_set_error(ctx, TFHE_ECUDA,
                                  std::string("gate_batch_noalloc: scratch address lookup: ") +
                                      cudaGetErrorString(e));
        g_scratch_addr[dev] = (uint32_t *)p;
    }
    *out = g_scratch_addr[dev];
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
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    uint32_t *scratch = nullptr;
    int rc = scratch_address(ctx, &scratch);
    if (rc != TFHE_OK) return rc;
    uint32_t *bar = scratch;
    uint32_t *acc = scratch + bar_words;
    cudaStream_t st = (cudaStream_t)stream;
    rc = tfhe_launch_combine(ctx, in, num_in, types, in_idx, bar, G, st);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_blind_rotate_ntt(ctx, bar, acc, G, st);
    if (rc != TFHE_OK) return rc;
    return tfhe_launch_extract_keyswitch(ctx, acc, out, G, types, in_idx, num_in, st);
}
