// cmux.cu -- CMUX Memory (Section 8.2): the read unit's CMUX tree and the CMUX part
// of the write unit's write bars.
#include <algorithm>

#include "common.cuh"

// G - C_j for j < v (Remark, Section 8.2): the selector that encrypts 1 - a_j.
// G is the gadget TRGSW of 1: 2^{32 - (r+1) Bgbit} at coefficient 0 of the a column of
// row r < l and of the b column of row l + r, zero elsewhere.
__global__ void k_gadget_minus(const uint32_t *__restrict__ c, uint32_t *__restrict__ gmc,
                               int v, int l, int N, int Bgbit) {
    const size_t per = (size_t)2 * l * 2 * N;
    const size_t total = (size_t)v * per;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t w = e % per;
        const int row = (int)(w / (2 * (size_t)N));
        const int col = (int)((w / N) % 2);
        const int k = (int)(w % N);
        uint32_t g = 0;
        if (k == 0) {
            const int lev = (row < l ? row : row - l) + 1;
            if ((row < l && col == 0) || (row >= l && col == 1)) g = 1u << (32 - lev * Bgbit);
        }
        gmc[e] = g - c[e];
    }
}

static int check_common(tfhe_ctx *ctx, int v, int form) {
    if (v < 1 || v > 16) return tfhe_set_error(ctx, TFHE_EINVAL, "v must be in 1..16");
    if (form != TFHE_FORM_NTT && form != TFHE_FORM_TC && form != TFHE_FORM_NTT2)
        return tfhe_set_error(ctx, TFHE_EINVAL, "unknown form");
    if (form == TFHE_FORM_TC && !tfhe_tc_supported(ctx))
        return tfhe_set_error(ctx, TFHE_EUNSUPPORTED, "tensor-core form not supported here");
    return TFHE_OK;
}

extern "C" int tfhe_cmux_tree_read(tfhe_ctx *ctx, const uint32_t *addr_trgsw,
                                   const uint32_t *table, int v, uint32_t *out, int R, int form,
                                   void *stream) {
    if (!ctx) return TFHE_EINVAL;
    int rc = check_common(ctx, v, form);
    if (rc != TFHE_OK) return rc;
    if (R < 0) return tfhe_set_error(ctx, TFHE_EINVAL, "cmux_tree_read: R < 0");
    if (R == 0) return TFHE_OK;
    if (!addr_trgsw || !table || !out)
        return tfhe_set_error(ctx, TFHE_EINVAL, "cmux_tree_read: null pointer");
    if ((int64_t)R << (v - 1) > (int64_t)1 << 30)
        return tfhe_set_error(ctx, TFHE_EINVAL, "cmux_tree_read: R * 2^(v-1) too large");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const tfhe_params &p = ctx->p;
    const int64_t N2 = 2 * (int64_t)p.N;
    const size_t per = (size_t)2 * p.l * 2 * p.N;
    const int M0 = 1 << (v - 1);
    rc = tfhe_ensure_workspace(ctx, R * M0);
    if (rc != TFHE_OK) return rc;
    // tensor-core form: tree levels with at least one 128-CMUX tile per selector run on
    // the tensor cores, narrower levels (always the last ones) in the two-prime NTT form
    const bool tc = form == TFHE_FORM_TC;
    rc = tfhe_ensure_trgsw_ws(ctx, (size_t)R * v);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_sel_to_ntt(ctx, addr_trgsw, ctx->ws_trgsw_ntt, (size_t)R * v, st);
    if (rc != TFHE_OK) return rc;
    const uint64_t *sel_ntt = ctx->ws_trgsw_ntt;
    uint32_t *buf[2] = {ctx->ws_acc, ctx->ws_tmp};
    const uint32_t *in = table;
    int64_t in_ystride = 0;  // level 0 reads the shared table
    for (int j = 0; j < v; j++) {
        const int M = 1 << (v - 1 - j);
        uint32_t *o = (j == v - 1) ? out : buf[j & 1];
        CmuxGeom g{in + N2, in, o, 2 * N2, in_ystride, N2, (int64_t)M * N2, (int64_t)v,
                   M, R, (int64_t)R * M};
        if (tc && M >= TFHE_TC_TILE)
            rc = tfhe_cmux_tc(ctx, addr_trgsw + (size_t)j * per, g, st);
        else
            rc = tfhe_cmux_ntt(ctx, sel_ntt + (size_t)j * per, g, st);
        if (rc != TFHE_OK) return rc;
        in = o;
        in_ystride = (int64_t)M * N2;
    }
    return TFHE_OK;
}

extern "C" int tfhe_ram_write(tfhe_ctx *ctx, const uint32_t *addr_trgsw, int v,
                              const uint32_t *new_cell, uint32_t *cells, int form,
                              void *stream) {
    if (!ctx) return TFHE_EINVAL;
    int rc = check_common(ctx, v, form);
    if (rc != TFHE_OK) return rc;
    if (!addr_trgsw || !new_cell || !cells)
        return tfhe_set_error(ctx, TFHE_EINVAL, "ram_write: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const tfhe_params &p = ctx->p;
    const size_t per = (size_t)2 * p.l * 2 * p.N;
    if (ctx->ws_gmc_cap < v) {
        size_t cap = (size_t)ctx->ws_gmc_cap * per * 4;
        rc = tfhe_grow(ctx, (void **)&ctx->ws_gmc, &cap, (size_t)v * per * 4,
                       "ram_write: selector workspace");
        if (rc != TFHE_OK) {
            if (!ctx->ws_gmc) ctx->ws_gmc_cap = 0;
            return rc;
        }
        ctx->ws_gmc_cap = v;
    }
    k_gadget_minus<<<256, 256, 0, st>>>(addr_trgsw, ctx->ws_gmc, v, p.l, p.N, p.Bgbit);
    rc = tfhe_check_launch(ctx, "gadget_minus");
    if (rc != TFHE_OK) return rc;
    // every form runs the write bars in the two-prime NTT form: at step j a cell takes
    // C_j or G - C_j by bit j of its index, so cells sharing a selector are not contiguous
    rc = tfhe_ensure_trgsw_ws(ctx, (size_t)2 * v);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_sel_to_ntt(ctx, addr_trgsw, ctx->ws_trgsw_ntt, (size_t)v, st);
    if (rc != TFHE_OK) return rc;
    rc = tfhe_sel_to_ntt(ctx, ctx->ws_gmc, ctx->ws_trgsw_ntt + (size_t)v * per, (size_t)v, st);
    if (rc != TFHE_OK) return rc;
    return tfhe_ram_write_ntt(ctx, ctx->ws_trgsw_ntt, ctx->ws_trgsw_ntt + (size_t)v * per, v,
                              new_cell, cells, st);
}

// ---------------------------------------------------------------------------
// One RAM cycle (Section 8.2: read unit, control unit, write unit)
// ---------------------------------------------------------------------------

// idx3[b] = (flag, write bit b, read bit b) rows of the MUX input block.
__global__ void k_ram_mux_idx(int w, int32_t *idx3) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= w) return;
    idx3[3 * b] = 0;
    idx3[3 * b + 1] = 1 + b;
    idx3[3 * b + 2] = 1 + w + b;
}

extern "C" int tfhe_ram_cycle(tfhe_ctx *ctx, const uint32_t *addr_trgsw, int v, int w,
                              const uint32_t *flag, const uint32_t *wdata, uint32_t *cells,
                              uint32_t *rdata, int form, void *stream) {
    if (!ctx) return TFHE_EINVAL;
    int rc = check_common(ctx, v, form == -1 ? TFHE_FORM_NTT : form);
    if (rc != TFHE_OK) return rc;
    // form -1: each bootstrap batch takes the form chosen for its width
    int form_mux = form, form_refresh = form, lv = -1;
    if (form == -1) {
        tfhe_pick_form(ctx, 2 * (int64_t)w, &form_mux, &lv);
        tfhe_pick_form(ctx, (int64_t)w << v, &form_refresh, &lv);
    }
    if (w < 1 || ((int64_t)w << v) > (1 << 24))
        return tfhe_set_error(ctx, TFHE_EINVAL, "ram_cycle: w must be >= 1 and w * 2^v <= 2^24");
    if (!addr_trgsw || !flag || !wdata || !cells || !rdata)
        return tfhe_set_error(ctx, TFHE_EINVAL, "ram_cycle: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "ram_cycle: keys not set");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const tfhe_params &p = ctx->p;
    const size_t N2 = 2 * (size_t)p.N, w1 = (size_t)p.n + 1, per = (size_t)2 * p.l * N2;
    const int64_t cells_n = (int64_t)w << v;
    // scratch: read TRLWEs [w][2N] | controlled TRLWEs [w][2N] | MUX inputs [1+2w][n+1] |
    //          MUX indices [w][3] | lvl0 [w 2^v][n+1] | ModSwitched [w 2^v][n+1]
    const size_t o_rd = 0, o_ctl = o_rd + w * N2, o_min = o_ctl + w * N2,
                 o_idx = o_min + (1 + 2 * (size_t)w) * w1, o_l0 = o_idx + 3 * (size_t)w,
                 o_bar = o_l0 + (size_t)cells_n * w1, words = o_bar + (size_t)cells_n * w1;
    rc = tfhe_grow(ctx, (void **)&ctx->ws_ram, &ctx->ws_ram_cap, words * 4, "ram_cycle scratch");
    if (rc != TFHE_OK) return rc;
    uint32_t *S = ctx->ws_ram;
    uint32_t *min = S + o_min;
    int32_t *idx3 = (int32_t *)(S + o_idx);

    // selectors C_j and G - C_j in the NTT domain (the CMUX parts run in the NTT form)
    if (ctx->ws_gmc_cap < v) {
        size_t cap = (size_t)ctx->ws_gmc_cap * per * 4;
        rc = tfhe_grow(ctx, (void **)&ctx->ws_gmc, &cap, (size_t)v * per * 4, "ram_cycle selectors");
        if (rc != TFHE_OK) {
            if (!ctx->ws_gmc) ctx->ws_gmc_cap = 0;
            return rc;
        }
        ctx->ws_gmc_cap = v;
    }
    k_gadget_minus<<<256, 256, 0, st>>>(addr_trgsw, ctx->ws_gmc, v, p.l, p.N, p.Bgbit);
    rc = tfhe_check_launch(ctx, "gadget_minus");
    if (rc != TFHE_OK) return rc;
    rc = tfhe_ensure_trgsw_ws(ctx, (size_t)2 * v);
    if (rc != TFHE_OK) return rc;
    const uint64_t *c_ntt = ctx->ws_trgsw_ntt, *gmc_ntt = ctx->ws_trgsw_ntt + (size_t)v * per;
    rc = tfhe_sel_to_ntt(ctx, addr_trgsw, ctx->ws_trgsw_ntt, (size_t)v, st);
    if (rc == TFHE_OK)
        rc = tfhe_sel_to_ntt(ctx, ctx->ws_gmc, ctx->ws_trgsw_ntt + (size_t)v * per, (size_t)v, st);
    if (rc != TFHE_OK) return rc;

    // read unit: the w bit blocks' CMUX trees share the address (selector stride 0)
    rc = tfhe_ensure_workspace(ctx, (int)(w * ((int64_t)1 << (v - 1))));
    if (rc != TFHE_OK) return rc;
    {
        uint32_t *buf[2] = {ctx->ws_acc, ctx->ws_tmp};
        const uint32_t *in = cells;
        int64_t in_ystride = ((int64_t)1 << v) * (int64_t)N2;
        for (int j = 0; j < v && rc == TFHE_OK; j++) {
            const int M = 1 << (v - 1 - j);
            uint32_t *o = (j == v - 1) ? S + o_rd : buf[j & 1];
            CmuxGeom g{in + N2, in, o, 2 * (int64_t)N2, in_ystride, (int64_t)N2, (int64_t)M * (int64_t)N2,
                       0, M, w, (int64_t)w * M};
            rc = tfhe_cmux_ntt(ctx, c_ntt + (size_t)j * per, g, st);
            in = o;
            in_ystride = (int64_t)M * N2;
        }
        if (rc != TFHE_OK) return rc;
    }
    // control unit: read words to TLWE (returned), then MUX(flag, write bit, read bit)
    rc = tfhe_launch_extract_keyswitch(ctx, S + o_rd, rdata, w, nullptr, nullptr, 0, st);
    if (rc != TFHE_OK) return rc;
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(min, flag, w1 * 4, cudaMemcpyDeviceToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(min + w1, wdata, (size_t)w * w1 * 4, cudaMemcpyDeviceToDevice, st));
    TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(min + (1 + (size_t)w) * w1, rdata, (size_t)w * w1 * 4,
                                       cudaMemcpyDeviceToDevice, st));
    k_ram_mux_idx<<<(w + 127) / 128, 128, 0, st>>>(w, idx3);
    rc = tfhe_check_launch(ctx, "ram_mux_idx");
    if (rc == TFHE_OK) rc = tfhe_mux_batch_impl(ctx, min, 1 + 2 * (int64_t)w, idx3, S + o_ctl, w,
                                                form_mux, true, st);
    if (rc != TFHE_OK) return rc;
    // write unit: each block's write bar selects the controlled data at the address (one
    // launch over all w blocks) ...
    rc = tfhe_ram_write_ntt(ctx, c_ntt, gmc_ntt, v, S + o_ctl, cells, st, w, (int64_t)N2);
    if (rc != TFHE_OK) return rc;
    // ... and every cell is refreshed: SE, IKS, ModSwitch, BlindRotate back to a TRLWE
    rc = tfhe_launch_extract_keyswitch(ctx, cells, S + o_l0, (int)cells_n, nullptr, nullptr, 0, st);
    if (rc == TFHE_OK) rc = tfhe_launch_modswitch_rows(ctx, S + o_l0, S + o_bar, cells_n, st);
    if (rc == TFHE_OK)
        rc = tfhe_blind_rotate_form(ctx, S + o_bar, cells, (int)cells_n, form_refresh, st);
    return rc;
}

// ---------------------------------------------------------------------------
// ROM with vertical and horizontal packing (Section 8.3): N / w words of w bits per TRLWE
// ---------------------------------------------------------------------------

// out[o] = X^{-(base + (o % rep) * step)} in[o / rep] for `rows` output TRLWEs (both
// polynomials; 0 <= shift < N): coefficient c takes p[c + s], or -p[c + s - N] past N.
__global__ void k_rotate_rows(int N, int64_t rows, int rep, int base, int step,
                              const uint32_t *__restrict__ in, uint32_t *__restrict__ out) {
    const size_t total = (size_t)rows * 2 * N;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t o = e / (2 * N);
        const int w = (int)(e % (2 * N));
        const int poly = w / N, cidx = w % N;
        const int s = (base + (int)(o % rep) * step) % N;
        const uint32_t *src = in + ((o / rep) * 2 + poly) * (size_t)N;
        const int k = cidx + s;
        out[e] = k < N ? src[k] : 0u - src[k - N];
    }
}

extern "C" int tfhe_rom_read(tfhe_ctx *ctx, const uint32_t *addr_trgsw, const uint32_t *table,
                             int v, int w, uint32_t *out_trlwe, uint32_t *out_bits, int R,
                             void *stream) {
    if (!ctx) return TFHE_EINVAL;
    const tfhe_params &p = ctx->p;
    if (w < 1 || w > p.N || (w & (w - 1)))
        return tfhe_set_error(ctx, TFHE_EINVAL, "rom_read: w must be a power of two <= N");
    int lo = 0;
    while ((w << lo) < p.N) lo++;  // log2(N / w) address bits pick the word in a TRLWE
    if (v < lo || v - lo > 16)
        return tfhe_set_error(ctx, TFHE_EINVAL, "rom_read: need log2(N/w) <= v <= log2(N/w) + 16");
    if (R < 0 || (int64_t)R * w > (1 << 24))
        return tfhe_set_error(ctx, TFHE_EINVAL, "rom_read: R < 0 or R * w > 2^24");
    if (R == 0) return TFHE_OK;
    if (!addr_trgsw || !table || (!out_trlwe && !out_bits))
        return tfhe_set_error(ctx, TFHE_EINVAL, "rom_read: null pointer");
    if (!ctx->has_keys) return tfhe_set_error(ctx, TFHE_ENOKEYS, "rom_read: keys not set");
    cudaStream_t st = (cudaStream_t)stream;
    TFHE_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int hi = v - lo;
    const int64_t N2 = 2 * (int64_t)p.N;
    const size_t per = (size_t)2 * p.l * 2 * p.N;
    // selectors in the NTT domain, every read's v address bits
    int rc = tfhe_ensure_trgsw_ws(ctx, (size_t)R * v);
    if (rc == TFHE_OK) rc = tfhe_sel_to_ntt(ctx, addr_trgsw, ctx->ws_trgsw_ntt, (size_t)R * v, st);
    if (rc != TFHE_OK) return rc;
    const uint64_t *sel = ctx->ws_trgsw_ntt;
    // scratch: two accumulators and one rotated copy per read
    rc = tfhe_grow(ctx, (void **)&ctx->ws_ram, &ctx->ws_ram_cap, (size_t)3 * R * N2 * 4,
                   "rom_read scratch");
    if (rc != TFHE_OK) return rc;
    uint32_t *acc[2] = {ctx->ws_ram, ctx->ws_ram + (size_t)R * N2};
    uint32_t *rot = ctx->ws_ram + (size_t)2 * R * N2;
    rc = tfhe_ensure_workspace(ctx, std::max(R * w, hi > 0 ? R << (hi - 1) : 1));
    if (rc != TFHE_OK) return rc;
    // CMUX tree over the TRLWE-selecting bits lo .. v-1 (R7), into acc[0]
    if (hi == 0) {
        k_rotate_rows<<<1184, 256, 0, st>>>(p.N, R, R, 0, 0, table, acc[0]);  // broadcast row 0
        rc = tfhe_check_launch(ctx, "rotate_rows");
    } else {
        uint32_t *buf[2] = {ctx->ws_acc, ctx->ws_tmp};
        const uint32_t *in = table;
        int64_t in_ystride = 0;
        for (int j = 0; j < hi && rc == TFHE_OK; j++) {
            const int M = 1 << (hi - 1 - j);
            uint32_t *o = (j == hi - 1) ? acc[0] : buf[j & 1];
            CmuxGeom g{in + N2, in, o, 2 * N2, in_ystride, N2, (int64_t)M * N2, (int64_t)v,
                       M, R, (int64_t)R * M};
            rc = tfhe_cmux_ntt(ctx, sel + (size_t)(lo + j) * per, g, st);
            in = o;
            in_ystride = (int64_t)M * N2;
        }
    }
    if (rc != TFHE_OK) return rc;
    // blind rotation by the word bits: ACC <- CMUX(C_j, X^{-w 2^j} ACC, ACC)
    int cur = 0;
    for (int j = 0; j < lo && rc == TFHE_OK; j++) {
        k_rotate_rows<<<1184, 256, 0, st>>>(p.N, R, 1, (w << j) % p.N, 0, acc[cur], rot);
        rc = tfhe_check_launch(ctx, "rotate_rows");
        if (rc != TFHE_OK) break;
        CmuxGeom g{rot, acc[cur], acc[cur ^ 1], 0, N2, 0, N2, (int64_t)v, 1, R, (int64_t)R};
        rc = tfhe_cmux_ntt(ctx, sel + (size_t)j * per, g, st);
        cur ^= 1;
    }
    if (rc != TFHE_OK) return rc;
    if (out_trlwe)
        TFHE_CUDA_TRY(ctx, cudaMemcpyAsync(out_trlwe, acc[cur], (size_t)R * N2 * 4,
                                           cudaMemcpyDeviceToDevice, st));
    if (!out_bits) return TFHE_OK;
    // bit i: SE at coefficient i (X^{-i} then coefficient 0), then the identity key switch
    k_rotate_rows<<<1184, 256, 0, st>>>(p.N, (int64_t)R * w, w, 0, 1, acc[cur], ctx->ws_acc);
    rc = tfhe_check_launch(ctx, "rotate_rows");
    if (rc != TFHE_OK) return rc;
    return tfhe_launch_extract_keyswitch(ctx, ctx->ws_acc, out_bits, R * w, nullptr, nullptr, 0, st);
}
