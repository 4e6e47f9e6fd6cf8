// Sigma drivers: sigma_k = M z_k through the density-fitted sandwich
//   O_k = sum_P L^P Zt_k L^P,   sigma_(pq) = w (eps_p + eps_q) z_(pq) + O_k[p][q] / f_pq
// (Sec. "ppRPA Equation": <pq|rs> = sum_P L^P_pr L^P_qs turns A X + B Y and
// B^T X + C Y into the virtual and occupied diagonal blocks of O; Zt holds
// X on its virtual block and Y on its occupied block, with sqrt(2) on the
// singlet diagonal and antisymmetric for the triplet; f_pq = sqrt(2) on the
// singlet diagonal, else 1).
#include <algorithm>
#include <cstdlib>

#include "ctx.h"

namespace pprpa {

static int env_int(const char* name, int dflt);

int ws_get(pprpa_ctx* c, const std::string& name, size_t bytes, void** out) {
    DevBuf& b = c->ws[name];
    if (b.bytes < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(PPRPA_ERR_OOM, "workspace '" + name + "': cudaMalloc(" +
                                                std::to_string(bytes) + ") failed");
        }
        b.p = p;
        b.bytes = bytes;
    }
    *out = b.p;
    return PPRPA_OK;
}

int check_status(pprpa_ctx* c) {
    int st = 0;
    PP_CUDA(cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    if (st & DEV_TIMEOUT) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
        return set_error(PPRPA_ERR_TIMEOUT, "device-side wait expired in the tensor-core GEMM");
    }
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// FP64 form: blocked batched DGEMMs, P processed in chunks.
int sigma_f64(pprpa_ctx* c, int mult, int k, const double* d_z, double* d_sigma) {
    PairTable* pt;
    PP_TRY(ensure_pairs(c, mult, &pt));
    const int n = c->n(), no = c->no, nv = c->nv, naux = c->naux;
    const int64_t n2 = (int64_t)n * n;
    cudaStream_t st = c->stream;
    double *Zt, *O, *T;
    PP_TRY(ws_get(c, "f64_Zt", sizeof(double) * n2 * k, (void**)&Zt));
    PP_TRY(ws_get(c, "f64_O", sizeof(double) * n2 * k, (void**)&O));
    // chunk of P such that T = [pc][k][n][n] stays within the budget (default 4 GB)
    const int64_t per_p = sizeof(double) * n2 * k;
    const int64_t budget = (int64_t)env_int("PPRPA_F64_CHUNK_MB", 4096) << 20;
    int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, budget / per_p));
    PP_TRY(ws_get(c, "f64_T", per_p * pc, (void**)&T));
    PP_CUDA(cudaMemsetAsync(Zt, 0, sizeof(double) * n2 * k, st));
    PP_TRY(launch_unpack_f64(d_z, k, pt->N, pt->d_pp, pt->d_pq, n, mult, Zt, st));
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = std::min(pc, naux - P0);
        const double* L0 = c->d_L + (int64_t)P0 * n2;
        // stage 1: T[P][j] = L^P Zt_j  (virtual columns, then occupied columns)
        for (int blk = 0; blk < 2; ++blk) {
            const int off = blk == 0 ? no : 0;
            const int sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            Dgemm g;
            g.M = n; g.N = sz; g.K = sz;
            g.A = L0 + off; g.lda = n; g.sA1 = n2; g.sA2 = 0;
            g.B = Zt + (int64_t)off * n + off; g.ldb = n; g.sB1 = 0; g.sB2 = n2;
            g.C = T + off; g.ldc = n; g.sC1 = n2 * k; g.sC2 = n2;
            g.nb1 = np; g.nb2 = k;
            PP_TRY(dgemm(g, st));
        }
        // stage 2: O_j[blk] (+)= sum_P T[P][j][blk rows, :] L^P[:, blk]
        for (int blk = 0; blk < 2; ++blk) {
            const int off = blk == 0 ? no : 0;
            const int sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            Dgemm g;
            g.M = sz; g.N = sz; g.K = n;
            g.A = T + (int64_t)off * n; g.lda = n; g.sA1 = n2; g.sAr = n2 * k;
            g.B = L0 + off; g.ldb = n; g.sB1 = 0; g.sBr = n2;
            g.C = O + (int64_t)off * n + off; g.ldc = n; g.sC1 = n2;
            g.nb1 = k; g.nr = np;
            g.beta = P0 == 0 ? 0.0 : 1.0;
            PP_TRY(dgemm(g, st));
        }
    }
    PP_TRY(launch_pack_f64(O, d_z, k, pt->N, pt->nvv, pt->d_pp, pt->d_pq, n, c->d_eps, mult,
                           d_sigma, st));
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
int ensure_bf16(pprpa_ctx* c) {
    if (c->bf16_ready) return PPRPA_OK;
    c->pm = make_padmap(c->no, c->nv);
    const int64_t np = c->pm.n_pad;
    const size_t bytes = sizeof(__nv_bfloat16) * (size_t)c->naux * np * np;
    if (c->d_Lhi) cudaFree(c->d_Lhi);
    if (c->d_Llo) cudaFree(c->d_Llo);
    c->d_Lhi = c->d_Llo = nullptr;
    PP_CUDA(cudaMalloc(&c->d_Lhi, bytes));
    PP_CUDA(cudaMalloc(&c->d_Llo, bytes));
    PP_TRY(launch_quantize_bf16(c->d_L, c->naux, c->n(), c->pm, c->d_Lhi, c->d_Llo, c->stream));
    c->bf16_ready = true;
    return PPRPA_OK;
}

static std::vector<int2> triangle_tiles(int valid, int BN) {
    std::vector<int2> t;
    const int mt = (int)ceil_div(valid, 128), nt = (int)ceil_div(valid, BN);
    for (int mb = 0; mb < mt; ++mb)
        for (int nb = 0; nb < nt; ++nb) {
            const int col_max = std::min((nb + 1) * BN, valid) - 1;
            if (mb * 128 <= col_max) t.push_back(make_int2(mb, nb));
        }
    return t;
}

// N tile of the second stage: tensor-core efficiency needs wide tiles, so among the
// multiples of 16 in [64, 256] (or up to the block when it is narrower) take the one
// that pads the block least, the wider one on ties.  The autotuner may override it.
int stage2_bn(int valid) {
    const int lo = valid >= 64 ? 64 : 16;
    int best = 256, best_pad = INT32_MAX;
    for (int bn = 256; bn >= lo; bn -= 16) {
        const int pad = (int)(ceil_div(valid, bn) * bn) - valid;
        if (pad < best_pad) { best_pad = pad; best = bn; }
    }
    return best;
}

// Launch with optional event timing (pprpa_profile).
static int timed_launch(pprpa_ctx* c, int kind, double flops, const CUtensorMap& a_hi,
                        const CUtensorMap& a_lo, const CUtensorMap& b_hi, const CUtensorMap& b_lo,
                        const TcParams& p, int nterms) {
    ProfRec r;
    const bool rec = c->profile && c->prof.size() < 200000;
    if (rec) {
        r.kind = kind;
        r.flops = flops;
        PP_CUDA(cudaEventCreate(&r.a));
        PP_CUDA(cudaEventCreate(&r.b));
        PP_CUDA(cudaEventRecord(r.a, c->stream));
    }
    PP_TRY(tc_gemm_launch(a_hi, a_lo, b_hi, b_lo, p, nterms, c->num_sms, c->stream));
    if (rec) {
        PP_CUDA(cudaEventRecord(r.b, c->stream));
        c->prof.push_back(r);
    }
    return PPRPA_OK;
}

static int env_int(const char* name, int dflt) {
    const char* s = getenv(name);
    return s ? atoi(s) : dflt;
}

// Tensor-core form.  nterms = 1: BF16 operands; nterms = 3: BF16x3 split.
int sigma_tc(pprpa_ctx* c, int mult, int k, const double* d_z, double* d_sigma, int nterms) {
    PairTable* pt;
    PP_TRY(ensure_pairs(c, mult, &pt));
    PP_TRY(ensure_bf16(c));
    const PadMap pm = c->pm;
    const int no = c->no, nv = c->nv, naux = c->naux;
    const int64_t np = pm.n_pad;
    cudaStream_t st = c->stream;
    const bool split = nterms == 3;

    // B operands of stage 1: Xs [k][nv][nv_p], Ys [k][no][no_p]
    const int ldx = pm.nv_p, ldy = std::max(pm.no_p, 8);
    const size_t xs_bytes = sizeof(__nv_bfloat16) * (size_t)k * std::max(nv, 1) * ldx;
    const size_t ys_bytes = sizeof(__nv_bfloat16) * (size_t)k * std::max(no, 1) * ldy;
    __nv_bfloat16 *xs_hi, *xs_lo, *ys_hi, *ys_lo;
    PP_TRY(ws_get(c, "tc_xs_hi", xs_bytes, (void**)&xs_hi));
    PP_TRY(ws_get(c, "tc_xs_lo", xs_bytes, (void**)&xs_lo));
    PP_TRY(ws_get(c, "tc_ys_hi", ys_bytes, (void**)&ys_hi));
    PP_TRY(ws_get(c, "tc_ys_lo", ys_bytes, (void**)&ys_lo));
    PP_CUDA(cudaMemsetAsync(xs_hi, 0, xs_bytes, st));
    PP_CUDA(cudaMemsetAsync(ys_hi, 0, ys_bytes, st));
    if (split) {
        PP_CUDA(cudaMemsetAsync(xs_lo, 0, xs_bytes, st));
        PP_CUDA(cudaMemsetAsync(ys_lo, 0, ys_bytes, st));
    }
    PP_TRY(launch_unpack_bf16(d_z, k, pt->N, pt->nvv, pt->d_pp, pt->d_pq, pm, mult, xs_hi,
                              split ? xs_lo : nullptr, ldx, ys_hi, split ? ys_lo : nullptr, ldy,
                              st));
    // intermediate T [pc][n_pad][k][n_pad] (hi, lo) and output O [k][n_pad][n_pad] FP32
    const int64_t per_p = (int64_t)sizeof(__nv_bfloat16) * np * k * np;
    const int64_t budget = (int64_t)env_int("PPRPA_T_BUDGET_MB", 64 * 1024) << 20;
    int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, budget / (per_p * (split ? 2 : 1))));
    __nv_bfloat16 *t_hi, *t_lo = nullptr;
    {
        // T is zero-initialised once per allocation: padding columns are never written.
        DevBuf before = c->ws["tc_t_hi"];
        PP_TRY(ws_get(c, "tc_t_hi", per_p * pc, (void**)&t_hi));
        if (c->ws["tc_t_hi"].p != before.p) PP_CUDA(cudaMemsetAsync(t_hi, 0, c->ws["tc_t_hi"].bytes, st));
        if (split) {
            DevBuf b2 = c->ws["tc_t_lo"];
            PP_TRY(ws_get(c, "tc_t_lo", per_p * pc, (void**)&t_lo));
            if (c->ws["tc_t_lo"].p != b2.p) PP_CUDA(cudaMemsetAsync(t_lo, 0, c->ws["tc_t_lo"].bytes, st));
        }
    }
    float* O;
    const size_t o_bytes = sizeof(float) * (size_t)k * np * np;
    PP_TRY(ws_get(c, "tc_O", o_bytes, (void**)&O));
    PP_CUDA(cudaMemsetAsync(O, 0, o_bytes, st));

    const int BN1 = env_int("PPRPA_BN1", 256);
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int npc = std::min(pc, naux - P0);
        const __nv_bfloat16* Lh = c->d_Lhi + (int64_t)P0 * np * np;
        const __nv_bfloat16* Ll = c->d_Llo + (int64_t)P0 * np * np;
        // ---------------- stage 1 ----------------
        for (int blk = 0; blk < 2; ++blk) {
            const int sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
            const uint64_t adims[2] = {(uint64_t)np, (uint64_t)npc * np};
            const uint64_t astr[1] = {(uint64_t)np * 2};
            const uint32_t abox[2] = {64, 128};
            PP_TRY(make_tmap_bf16(&ta_hi, Lh, 2, adims, astr, abox));
            PP_TRY(make_tmap_bf16(&ta_lo, Ll, 2, adims, astr, abox));
            const int ld = blk == 0 ? ldx : ldy;
            const uint64_t bdims[2] = {(uint64_t)sz, (uint64_t)k * sz};
            const uint64_t bstr[1] = {(uint64_t)ld * 2};
            const int BN = std::min(BN1, (int)round_up(std::max(16, (int)std::min<int64_t>(256, (int64_t)k * sz)), 16));
            const uint32_t bbox[2] = {64, (uint32_t)BN};
            PP_TRY(make_tmap_bf16(&tb_hi, blk == 0 ? xs_hi : ys_hi, 2, bdims, bstr, bbox));
            PP_TRY(make_tmap_bf16(&tb_lo, blk == 0 ? xs_lo : ys_lo, 2, bdims, bstr, bbox));
            TcParams p;
            p.mode = 0;
            p.BN = BN;
            p.status = c->d_status;
            p.M_rows = (int64_t)npc * np;
            p.a_col_off = blk == 0 ? pm.no_p : 0;
            p.n_per_j = sz;
            p.n_total = k * sz;
            p.t_col_off = blk == 0 ? pm.no_p : 0;
            p.n_pad = (int)np;
            p.k_vec = k;
            p.t_hi = t_hi;
            p.t_lo = t_lo;
            p.kb_total = (int)ceil_div(sz, 64);
            p.tiles_n = (int)ceil_div(p.n_total, BN);
            const int64_t items = ceil_div(p.M_rows, 128) * p.tiles_n;
            if (items > INT32_MAX) return set_error(PPRPA_ERR_ARG, "sigma: too many stage-1 tiles");
            p.total_items = (int)items;
            const double fl = 2.0 * npc * (double)(no + nv) * (double)sz * sz * k;
            PP_TRY(timed_launch(c, split ? 2 : 0, fl, ta_hi, ta_lo, tb_hi, tb_lo, p, nterms));
        }
        // ---------------- stage 2 ----------------
        for (int blk = 0; blk < 2; ++blk) {
            const int sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            const int off = blk == 0 ? pm.no_p : 0;
            std::string key = std::string("bn2_") + std::to_string(sz);
            int BN = c->tuned_bn.count(key) ? c->tuned_bn[key] : stage2_bn(sz);
            const int forced = env_int("PPRPA_BN2", 0);
            if (forced) BN = forced;
            std::vector<int2> tiles = triangle_tiles(sz, BN);
            int2* d_tiles;
            PP_TRY(ws_get(c, "tc_tiles" + std::to_string(blk), sizeof(int2) * tiles.size(), (void**)&d_tiles));
            PP_CUDA(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(int2) * tiles.size(),
                                    cudaMemcpyHostToDevice, st));
            CUtensorMap ta_hi, ta_lo, tb_hi, tb_lo;
            const uint64_t adims[4] = {(uint64_t)np, (uint64_t)k, (uint64_t)np, (uint64_t)npc};
            const uint64_t astr[3] = {(uint64_t)np * 2, (uint64_t)k * np * 2, (uint64_t)np * k * np * 2};
            const uint32_t abox[4] = {64, 1, 128, 1};
            PP_TRY(make_tmap_bf16(&ta_hi, t_hi, 4, adims, astr, abox));
            PP_TRY(make_tmap_bf16(&ta_lo, split ? t_lo : t_hi, 4, adims, astr, abox));
            const uint64_t bdims[3] = {(uint64_t)np, (uint64_t)np, (uint64_t)npc};
            const uint64_t bstr[2] = {(uint64_t)np * 2, (uint64_t)np * np * 2};
            const uint32_t bbox[3] = {64, (uint32_t)BN, 1};
            PP_TRY(make_tmap_bf16(&tb_hi, Lh, 3, bdims, bstr, bbox));
            PP_TRY(make_tmap_bf16(&tb_lo, Ll, 3, bdims, bstr, bbox));
            TcParams p;
            p.mode = 1;
            p.BN = BN;
            p.status = c->d_status;
            p.tile_list = d_tiles;
            p.ntiles = (int)tiles.size();
            p.nbatch = k;
            p.kq_blocks = (int)ceil_div(np, 64);
            p.kb_total = npc * p.kq_blocks;
            // enough K slices for about four waves of work items; in the split form also
            // at most pcap auxiliary slices per accumulator, because the tensor-core FP32
            // accumulation loses accuracy over very long reductions (partial sums of the
            // slices are added in FP32 in L2)
            const int64_t base_items = (int64_t)p.ntiles * k;
            int64_t ns = ceil_div(4LL * c->num_sms, base_items);
            ns = std::max<int64_t>(1, std::min<int64_t>(ns, std::max(1, p.kb_total / 8)));
            const int pcap = env_int(split ? "PPRPA_S2_PCAP_SPLIT" : "PPRPA_S2_PCAP", split ? 2 : 128);
            if (pcap > 0) ns = std::max<int64_t>(ns, ceil_div(npc, pcap));
            // every K slice non-empty: recompute the count from the slice length
            const int64_t per = ceil_div(p.kb_total, ns);
            p.nsplit = (int)ceil_div(p.kb_total, per);
            p.row_off = off;
            p.col_off = off;
            p.m_valid = sz;
            p.n_valid = sz;
            p.n_pad = (int)np;
            p.O = O;
            p.total_items = (int)(base_items * p.nsplit);
            const double fl = 1.0 * npc * (double)(no + nv) * (double)sz * sz * k;
            PP_TRY(timed_launch(c, split ? 3 : 1, fl, ta_hi, ta_lo, tb_hi, tb_lo, p, nterms));
        }
    }
    PP_TRY(launch_pack_f32(O, d_z, k, pt->N, pt->nvv, pt->d_pp, pt->d_pq, pm, c->d_eps, mult,
                           d_sigma, st));
    return PPRPA_OK;
}

}  // namespace pprpa
