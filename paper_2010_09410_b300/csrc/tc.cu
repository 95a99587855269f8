// tc.cu -- tensor-core form (placeholder until the tcgen05 engine lands).
#include "common.cuh"

int tfhe_tc_supported(const tfhe_ctx *) { return 0; }
int tfhe_blind_rotate_tc(tfhe_ctx *ctx, const uint32_t *, uint32_t *, int, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form not built");
}
int tfhe_cmux_tc(tfhe_ctx *ctx, const uint32_t *, const CmuxGeom &, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form not built");
}
int tfhe_ram_write_tc(tfhe_ctx *ctx, const uint32_t *, const uint32_t *, int, const uint32_t *,
                      uint32_t *, cudaStream_t) {
    return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form not built");
}
void tfhe_tc_free(tfhe_ctx *) {}
