// Sigma drivers: sigma_k = M z_k through the density-fitted sandwich
//   O_k = sum_P L^P Zt_k L^P,   sigma_(pq) = w (eps_p + eps_q) z_(pq) + O_k[p][q] / f_pq
// (Sec. "ppRPA Equation": <pq|rs> = sum_P L^P_pr L^P_qs turns A X + B Y and
// B^T X + C Y into the virtual and occupied diagonal blocks of O; Zt holds
// X on its virtual block and Y on its occupied block, with sqrt(2) on the
// singlet diagonal and antisymmetric for the triplet; f_pq = sqrt(2) on the
// singlet diagonal, else 1).
#include <algorithm>
#include <cstdlib>

#include <cstring>

#include "ctx.h"

namespace pprpa {

static int env_int(const char* name, int dflt);

int ws_get(pprpa_ctx* c, const std::string& name, size_t bytes, void** out) {
    DevBuf& b = c->ws[name];
    if (b.bytes < bytes) {
        ++c->mem_epoch;
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
    PP_TRY(ctx_sync(c));
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
    ++c->mem_epoch;
    if (c->d_Lhi) cudaFree(c->d_Lhi);
    if (c->d_Llo) cudaFree(c->d_Llo);
    c->d_Lhi = c->d_Llo = nullptr;
    PP_CUDA(cudaMalloc(&c->d_Lhi, bytes));
    PP_CUDA(cudaMalloc(&c->d_Llo, bytes));
    PP_TRY(launch_quantize_bf16(c->d_L, c->naux, c->n(), c->pm, c->d_Lhi, c->d_Llo, c->stream));
    c->bf16_ready = true;
    return PPRPA_OK;
}

int ensure_fp8(pprpa_ctx* c) {
    if (c->fp8_ready) return PPRPA_OK;
    PP_TRY(ensure_bf16(c));
    const PadMap pm = c->pm;
    c->c_off8 = (int)round_up(c->no, 16);
    c->ncol8 = (int)round_up(c->c_off8 + c->nv, 16);
    ++c->mem_epoch;
    if (c->d_L8) cudaFree(c->d_L8);
    if (c->d_L8scale) cudaFree(c->d_L8scale);
    c->d_L8 = nullptr;
    c->d_L8scale = nullptr;
    PP_CUDA(cudaMalloc(&c->d_L8, (size_t)c->naux * pm.n_pad * c->ncol8));
    PP_CUDA(cudaMalloc(&c->d_L8scale, sizeof(float) * c->naux));
    PP_TRY(launch_quantize_fp8(c->d_L, c->naux, c->n(), pm, c->ncol8, c->c_off8, c->d_L8,
                               c->d_L8scale, c->stream));
    c->fp8_ready = true;
    return PPRPA_OK;
}

// Output tiles of the second stage over the upper triangle (row <= column) of a block of
// `valid` rows: each M tile of `mrows` rows starting at row r0 covers the columns [r0, valid)
// in near-equal widths, multiples of `wmul` and at most BN, so that only the diagonal corner
// and the rounding are computed beyond the triangle.  Entry: (M tile, first column, width).
static std::vector<int4> triangle_tiles(int valid, int BN, int mrows = 128, int wmul = 16) {
    std::vector<int4> t;
    const int mt = (int)ceil_div(valid, mrows);
    for (int mb = 0; mb < mt; ++mb) {
        const int r0 = mb * mrows, len = valid - r0;
        const int nch = (int)ceil_div(len, BN);
        const int w = std::min(BN, (int)round_up(ceil_div(len, nch), wmul));
        for (int n0 = r0; n0 < valid; n0 += w)
            t.push_back(make_int4(mb, n0, std::min(w, (int)round_up(valid - n0, wmul)), 0));
    }
    return t;
}

// Widest tile of the second stage.  The stage is bound by operand traffic from L2 (each
// output tile re-reads its A rows; B tiles are shared by a cluster), not by the MMAs, so
// among the multiples of 16 in [64, 256] (or up to the block when it is narrower) take the
// one that pads the block least, the wider one on ties; triangle_tiles then balances the
// widths within it.  The autotuner may override it.
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
                        const TcParams& p, int nterms, int cluster = 1, bool f8 = false,
                        bool pair = false, const CUtensorMap* t_hi = nullptr,
                        const CUtensorMap* t_lo = nullptr) {
    ProfRec r;
    const bool rec = c->profile && c->prof.size() < 200000;
    if (rec) {
        r.kind = kind;
        r.flops = flops;
        PP_CUDA(cudaEventCreate(&r.a));
        PP_CUDA(cudaEventCreate(&r.b));
        PP_CUDA(cudaEventRecord(r.a, c->stream));
    }
    if (cluster > 1)
        PP_TRY(tc_gemm_launch_cluster(a_hi, a_lo, b_hi, b_lo, p, nterms, cluster, c->num_sms, c->stream, f8,
                                      pair, t_hi, t_lo));
    else PP_TRY(tc_gemm_launch(a_hi, a_lo, b_hi, b_lo, p, nterms, c->num_sms, c->stream, f8, t_hi, t_lo));
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

// ---------------------------------------------------------------------------
// Tensor-core form.  nterms = 1: BF16 operands; nterms = 3: BF16x3 split.
//
// A sigma call is planned as a list of jobs, one per (stage, pair block, P chunk): each
// job carries its tensor maps and kernel parameters.  A single molecule runs its jobs
// one launch at a time; a batch of molecules runs all stage-1 jobs in one persistent
// launch and all stage-2 jobs in another.

struct TcPrepared {
    PairTable* pt = nullptr;
    PadMap pm;
    int k = 0, mult = 1, nterms = 1, pc = 0;
    int ldx = 0, ldy = 0;
    __nv_bfloat16 *xs_hi = nullptr, *xs_lo = nullptr, *ys_hi = nullptr, *ys_lo = nullptr;
    __nv_bfloat16 *t_hi = nullptr, *t_lo = nullptr;
    float* O = nullptr;
    const double* d_z = nullptr;
    // FP8 first stage
    bool f8 = false;
    int ld8x = 0, ld8y = 0;
    void *xs8 = nullptr, *ys8 = nullptr;
    float* zscale = nullptr;
};

struct TcJobHost {
    TcJob job;
    int kind = 0;        // profile row
    double flops = 0.0;  // algorithmic
    int cluster = 1;                     // clusters of this many CTAs sharing the B tile
    bool f8 = false;                     // E4M3 operands (stage 1 of the FP8 form)
    bool pair = false;                   // cluster of 2 as one tcgen05 CTA pair (M = 256)
    bool t_store = false;                // stage 1: T written by bulk tensor stores
    CUtensorMap t_hi_map, t_lo_map;      // T of this block: (column, vector, row), box 64 x 1 x 32
    CUtensorMap b_hi_half, b_lo_half;    // B boxes of BN / cluster rows for the cluster form
};

// Buffers (allocated on first use, sized for k vectors).
static int tc_alloc(pprpa_ctx* c, int mult, int k, const double* d_z, int nterms, TcPrepared& pr,
                    cudaStream_t st, bool f8 = false) {
    PP_TRY(ensure_pairs(c, mult, &pr.pt));
    // the BF16 / E4M3 copies of L are made on the context's stream; a batched launch on
    // another stream must not start before they are complete
    const bool fresh = !c->bf16_ready || (f8 && !c->fp8_ready);
    PP_TRY(ensure_bf16(c));
    pr.f8 = f8;
    if (f8) {
        PP_TRY(ensure_fp8(c));
        pr.ld8x = (int)round_up(std::max(c->nv, 1), 16);
        pr.ld8y = (int)round_up(std::max(c->no, 1), 16);
        PP_TRY(ws_get(c, "tc_xs8", (size_t)k * round_up(c->nv, 8) * pr.ld8x + 16, &pr.xs8));
        PP_TRY(ws_get(c, "tc_ys8", (size_t)k * round_up(std::max(c->no, 1), 8) * pr.ld8y + 16, &pr.ys8));
        PP_TRY(ws_get(c, "tc_zscale", sizeof(float) * k, (void**)&pr.zscale));
    }
    if (fresh && st != c->stream) PP_TRY(ctx_sync(c));
    pr.pm = c->pm;
    pr.k = k;
    pr.mult = mult;
    pr.nterms = nterms;
    pr.d_z = d_z;
    const PadMap pm = c->pm;
    const int64_t np = pm.n_pad;
    const bool split = nterms == 3;
    pr.ldx = std::max(pm.nv_p, 8);
    pr.ldy = std::max(pm.no_p, 8);
    const size_t xs_bytes = sizeof(__nv_bfloat16) * (size_t)k * pr.ldx * pr.ldx;
    const size_t ys_bytes = sizeof(__nv_bfloat16) * (size_t)k * pr.ldy * pr.ldy;
    PP_TRY(ws_get(c, "tc_xs_hi", xs_bytes, (void**)&pr.xs_hi));
    PP_TRY(ws_get(c, "tc_xs_lo", xs_bytes, (void**)&pr.xs_lo));
    PP_TRY(ws_get(c, "tc_ys_hi", ys_bytes, (void**)&pr.ys_hi));
    PP_TRY(ws_get(c, "tc_ys_lo", ys_bytes, (void**)&pr.ys_lo));
    // intermediate T [pc][n_pad][k][n_pad] (hi, lo) and output O [k][n_pad][n_pad] FP32
    const int64_t per_p = (int64_t)sizeof(__nv_bfloat16) * np * k * np;
    const int64_t budget = (int64_t)env_int("PPRPA_T_BUDGET_MB", 64 * 1024) << 20;
    pr.pc = (int)std::max<int64_t>(1, std::min<int64_t>(c->naux, budget / (per_p * (split ? 2 : 1))));
    {
        // T is zero-initialised once per allocation: padding columns only ever hold zeros
        DevBuf before = c->ws["tc_t_hi"];
        PP_TRY(ws_get(c, "tc_t_hi", per_p * pr.pc, (void**)&pr.t_hi));
        if (c->ws["tc_t_hi"].p != before.p) PP_CUDA(cudaMemsetAsync(pr.t_hi, 0, c->ws["tc_t_hi"].bytes, st));
        if (split) {
            DevBuf b2 = c->ws["tc_t_lo"];
            PP_TRY(ws_get(c, "tc_t_lo", per_p * pr.pc, (void**)&pr.t_lo));
            if (c->ws["tc_t_lo"].p != b2.p) PP_CUDA(cudaMemsetAsync(pr.t_lo, 0, c->ws["tc_t_lo"].bytes, st));
        }
    }
    const size_t o_bytes = sizeof(float) * (size_t)k * np * np;
    PP_TRY(ws_get(c, "tc_O", o_bytes, (void**)&pr.O));
    return PPRPA_OK;
}

// Device work before the GEMMs: the packed B operands of stage 1 and a zeroed O.
static int tc_device_prep(pprpa_ctx* c, const TcPrepared& pr, cudaStream_t st) {
    const bool split = pr.nterms == 3;
    if (pr.f8) {
        const size_t b8x = (size_t)pr.k * round_up(c->nv, 8) * pr.ld8x;
        const size_t b8y = (size_t)pr.k * round_up(std::max(c->no, 1), 8) * pr.ld8y;
        PP_CUDA(cudaMemsetAsync(pr.xs8, 0, b8x, st));
        PP_CUDA(cudaMemsetAsync(pr.ys8, 0, b8y, st));
        PP_TRY(launch_unpack_fp8(pr.d_z, pr.k, pr.pt->N, pr.pt->nvv, pr.pt->d_pp, pr.pt->d_pq,
                                 pr.pm, pr.mult, pr.zscale, pr.xs8, pr.ld8x, pr.ys8, pr.ld8y, st));
        const int64_t np = pr.pm.n_pad;
        PP_CUDA(cudaMemsetAsync(pr.O, 0, sizeof(float) * (size_t)pr.k * np * np, st));
        return PPRPA_OK;
    }
    const size_t xs_bytes = sizeof(__nv_bfloat16) * (size_t)pr.k * pr.ldx * pr.ldx;
    const size_t ys_bytes = sizeof(__nv_bfloat16) * (size_t)pr.k * pr.ldy * pr.ldy;
    PP_CUDA(cudaMemsetAsync(pr.xs_hi, 0, xs_bytes, st));
    PP_CUDA(cudaMemsetAsync(pr.ys_hi, 0, ys_bytes, st));
    if (split) {
        PP_CUDA(cudaMemsetAsync(pr.xs_lo, 0, xs_bytes, st));
        PP_CUDA(cudaMemsetAsync(pr.ys_lo, 0, ys_bytes, st));
    }
    PP_TRY(launch_unpack_bf16(pr.d_z, pr.k, pr.pt->N, pr.pt->nvv, pr.pt->d_pp, pr.pt->d_pq, pr.pm,
                              pr.mult, pr.xs_hi, split ? pr.xs_lo : nullptr, pr.ldx, pr.ys_hi,
                              split ? pr.ys_lo : nullptr, pr.ldy, st));
    const int64_t np = pr.pm.n_pad;
    PP_CUDA(cudaMemsetAsync(pr.O, 0, sizeof(float) * (size_t)pr.k * np * np, st));
    (void)c;
    return PPRPA_OK;
}

static int tc_prepare(pprpa_ctx* c, int mult, int k, const double* d_z, int nterms,
                      TcPrepared& pr, cudaStream_t st, bool f8 = false) {
    PP_TRY(tc_alloc(c, mult, k, d_z, nterms, pr, st, f8));
    return tc_device_prep(c, pr, st);
}

static std::string tune_key(int stage, int sz, int k) {
    return "s" + std::to_string(stage) + "_" + std::to_string(sz) + "_" + std::to_string(k);
}

// Tile width of a stage: forced by the environment, else the autotuned value, else the model.
static int tile_bn(pprpa_ctx* c, int stage, int sz, int k, int szp) {
    const int forced = env_int(stage == 1 ? "PPRPA_BN1" : "PPRPA_BN2", 0);
    if (forced) return forced;
    auto it = c->tuned_bn.find(tune_key(stage, sz, k));
    if (it != c->tuned_bn.end()) return it->second;
    if (stage == 1) return (int)round_up(std::max(16, (int)std::min<int64_t>(256, (int64_t)k * szp)), 16);
    return stage2_bn(sz);
}

// Jobs of one P chunk [P0, P0 + npc).
static int tc_jobs(pprpa_ctx* c, const TcPrepared& pr, int P0, int npc, std::vector<TcJobHost>& s1,
                   std::vector<TcJobHost>& s2, std::vector<std::vector<int4>>& tiles,
                   bool single_launch = true) {
    const PadMap pm = pr.pm;
    const int no = c->no, nv = c->nv, k = pr.k;
    const int64_t np = pm.n_pad;
    const bool split = pr.nterms == 3;
    const __nv_bfloat16* Lh = c->d_Lhi + (int64_t)P0 * np * np;
    const __nv_bfloat16* Ll = c->d_Llo + (int64_t)P0 * np * np;
    for (int blk = 0; blk < 2; ++blk) {  // stage 1: T = L Zt on the virtual / occupied columns
        const int sz = blk == 0 ? nv : no;
        if (sz == 0) continue;
        TcJobHost h;
        TcJob& j = h.job;
        const uint32_t bke = pr.f8 ? 128 : 64;   // elements per 128-byte K block
        const int szp = blk == 0 ? pm.nv_p : pm.no_p;  // rows per vector (8-aligned)
        const int BN = tile_bn(c, 1, sz, k, szp);
        const uint64_t bdims[2] = {(uint64_t)sz, (uint64_t)k * szp};
        const uint32_t bbox[2] = {bke, (uint32_t)BN};
        uint64_t bstr[1];
        if (pr.f8) {
            const uint8_t* L8 = (const uint8_t*)c->d_L8 + (int64_t)P0 * np * c->ncol8;
            const uint64_t adims[2] = {(uint64_t)c->ncol8, (uint64_t)npc * np};
            const uint64_t astr[1] = {(uint64_t)c->ncol8};
            const uint32_t abox[2] = {bke, 128};
            PP_TRY(make_tmap(&j.a_hi, L8, 2, adims, astr, abox, 1));
            j.a_lo = j.a_hi;
            bstr[0] = (uint64_t)(blk == 0 ? pr.ld8x : pr.ld8y);
            PP_TRY(make_tmap(&j.b_hi, blk == 0 ? pr.xs8 : pr.ys8, 2, bdims, bstr, bbox, 1));
            j.b_lo = j.b_hi;
        } else {
            const uint64_t adims[2] = {(uint64_t)np, (uint64_t)npc * np};
            const uint64_t astr[1] = {(uint64_t)np * 2};
            const uint32_t abox[2] = {64, 128};
            PP_TRY(make_tmap_bf16(&j.a_hi, Lh, 2, adims, astr, abox));
            PP_TRY(make_tmap_bf16(&j.a_lo, Ll, 2, adims, astr, abox));
            const int ld = blk == 0 ? pr.ldx : pr.ldy;
            bstr[0] = (uint64_t)ld * 2;
            PP_TRY(make_tmap_bf16(&j.b_hi, blk == 0 ? pr.xs_hi : pr.ys_hi, 2, bdims, bstr, bbox));
            PP_TRY(make_tmap_bf16(&j.b_lo, blk == 0 ? pr.xs_lo : pr.ys_lo, 2, bdims, bstr, bbox));
        }
        TcParams& p = j.p;
        p.mode = 0;
        p.BN = BN;
        p.status = c->d_status;
        p.M_rows = (int64_t)npc * np;
        p.a_col_off = blk == 0 ? (pr.f8 ? c->c_off8 : pm.no_p) : 0;
        if (pr.f8) {
            p.row_scale = c->d_L8scale + P0;
            p.col_scale = pr.zscale;
        }
        p.n_per_j = szp;
        p.n_total = k * szp;
        p.t_col_off = blk == 0 ? pm.no_p : 0;
        p.n_pad = (int)np;
        p.k_vec = k;
        p.t_hi = pr.t_hi;
        p.t_lo = pr.t_lo;
        p.kb_total = (int)ceil_div(sz, (int64_t)bke);
        p.tiles_n = (int)ceil_div(p.n_total, BN);
        const int64_t items = ceil_div(p.M_rows, 128) * p.tiles_n;
        if (items > INT32_MAX) return set_error(PPRPA_ERR_ARG, "sigma: too many stage-1 tiles");
        p.total_items = (int)items;
        h.kind = split ? 2 : 0;
        h.f8 = pr.f8;
        // T of this block as a 3-D tensor (column inside the block, vector, row R) for bulk
        // stores of 32 x 64 boxes; blocks narrower than one box keep per-thread stores.
        // Measured at the 50 + 600 active, naux 2700 case: faster for the FP8 form (stage 1
        // 1200 -> 1233 TF/s), not for BF16 (877 -> 859), so by default only for FP8.
        if (env_int("PPRPA_TSTORE", pr.f8 ? 1 : 0) && szp >= 64) {
            const uint64_t tdims[3] = {(uint64_t)szp, (uint64_t)k, (uint64_t)p.M_rows};
            const uint64_t tstr[2] = {(uint64_t)np * 2, (uint64_t)k * np * 2};
            const uint32_t tbox[3] = {64, 1, 32};
            PP_TRY(make_tmap_bf16(&h.t_hi_map, pr.t_hi + p.t_col_off, 3, tdims, tstr, tbox));
            PP_TRY(make_tmap_bf16(&h.t_lo_map, (split ? pr.t_lo : pr.t_hi) + p.t_col_off, 3, tdims, tstr, tbox));
            h.t_store = true;
        }
        h.flops = 2.0 * npc * (double)(no + nv) * (double)sz * sz * k;
        // clusters of CTAs share the B tile when there are enough M tiles to group: either a
        // tcgen05 CTA pair (each CTA holds half of B) or a multicast cluster (each holds all)
        int cl = env_int("PPRPA_CLUSTER", 4);
        while (cl > 1 && (BN % (16 * cl) != 0 || ceil_div(p.M_rows, 128) < cl)) cl /= 2;
        h.cluster = cl == 2 || cl == 4 ? cl : 1;
        if (single_launch && env_int("PPRPA_PAIR1", 0) && BN % 32 == 0 && ceil_div(p.M_rows, 128) >= 2) {
            h.cluster = 2;
            h.pair = true;
        }
        if (h.cluster > 1) {
            const uint32_t hbox[2] = {bke, (uint32_t)(BN / h.cluster)};
            if (pr.f8) {
                PP_TRY(make_tmap(&h.b_hi_half, blk == 0 ? pr.xs8 : pr.ys8, 2, bdims, bstr, hbox, 1));
                h.b_lo_half = h.b_hi_half;
            } else {
                PP_TRY(make_tmap_bf16(&h.b_hi_half, blk == 0 ? pr.xs_hi : pr.ys_hi, 2, bdims, bstr, hbox));
                PP_TRY(make_tmap_bf16(&h.b_lo_half, blk == 0 ? pr.xs_lo : pr.ys_lo, 2, bdims, bstr, hbox));
            }
        }
        s1.push_back(h);
    }
    for (int blk = 0; blk < 2; ++blk) {  // stage 2: O += T L on the upper triangle of a block
        const int sz = blk == 0 ? nv : no;
        if (sz == 0) continue;
        const int off = blk == 0 ? pm.no_p : 0;
        // stage 2 as tcgen05 CTA pairs: 256-row tiles, each CTA holding half of the L^P tile
        const bool pair2 = single_launch && env_int("PPRPA_PAIR2", 0) != 0;
        int BN = tile_bn(c, 2, sz, k, 0);
        if (pair2) BN = (int)std::min<int64_t>(256, round_up(BN, 32));
        tiles.push_back(pair2 ? triangle_tiles(sz, BN, 256, 32) : triangle_tiles(sz, BN));
        const std::vector<int4>& tl = tiles.back();
        TcJobHost h;
        TcJob& j = h.job;
        const uint64_t adims[4] = {(uint64_t)np, (uint64_t)k, (uint64_t)np, (uint64_t)npc};
        const uint64_t astr[3] = {(uint64_t)np * 2, (uint64_t)k * np * 2, (uint64_t)np * k * np * 2};
        const uint32_t abox[4] = {64, 1, 128, 1};
        PP_TRY(make_tmap_bf16(&j.a_hi, pr.t_hi, 4, adims, astr, abox));
        PP_TRY(make_tmap_bf16(&j.a_lo, split ? pr.t_lo : pr.t_hi, 4, adims, astr, abox));
        const uint64_t bdims[3] = {(uint64_t)np, (uint64_t)np, (uint64_t)npc};
        const uint64_t bstr[2] = {(uint64_t)np * 2, (uint64_t)np * np * 2};
        const uint32_t bbox[3] = {64, (uint32_t)BN, 1};
        PP_TRY(make_tmap_bf16(&j.b_hi, Lh, 3, bdims, bstr, bbox));
        PP_TRY(make_tmap_bf16(&j.b_lo, Ll, 3, bdims, bstr, bbox));
        TcParams& p = j.p;
        p.mode = 1;
        p.BN = BN;
        p.status = c->d_status;
        p.ntiles = (int)tl.size();
        p.nbatch = k;
        p.kq_blocks = (int)ceil_div(np, 64);
        p.kb_total = npc * p.kq_blocks;
        // enough K slices for about four waves of work items; in the split form also
        // at most pcap auxiliary slices per accumulator, because the tensor-core FP32
        // accumulation loses accuracy over very long reductions (partial sums of the
        // slices are added in FP32 in L2)
        const int64_t base_items = (int64_t)p.ntiles * k;
        const int64_t waves = std::max(1, env_int("PPRPA_S2_WAVES", 4));
        int64_t ns = ceil_div(waves * (pair2 ? c->num_sms / 2 : c->num_sms), base_items);
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
        p.O = pr.O;
        p.total_items = (int)(base_items * p.nsplit);
        // clusters over neighbouring vectors sharing the L^P tile (TMA multicast): 4 when it
        // divides k and BN / 4 is whole swizzle atoms, else 2
        int cl2 = env_int("PPRPA_CLUSTER2", -1);
        if (cl2 < 0) cl2 = (k % 4 == 0 && BN % 32 == 0) ? 4 : (k >= 2 ? 2 : 1);
        if (pair2) {
            cl2 = 2;
            h.pair = true;
        }
        if ((cl2 == 2 || cl2 == 4) && BN % 16 == 0 && BN % (8 * cl2) == 0 && (k >= 2 || pair2)) {
            h.cluster = cl2;
            const uint32_t hbox[3] = {64, (uint32_t)(BN / cl2), 1};
            PP_TRY(make_tmap_bf16(&h.b_hi_half, Lh, 3, bdims, bstr, hbox));
            PP_TRY(make_tmap_bf16(&h.b_lo_half, Ll, 3, bdims, bstr, hbox));
        }
        h.kind = split ? 3 : 1;
        h.flops = 1.0 * npc * (double)(no + nv) * (double)sz * sz * k;
        s2.push_back(h);
    }
    return PPRPA_OK;
}

int sigma_tc(pprpa_ctx* c, int mult, int k, const double* d_z, double* d_sigma, int nterms,
             bool f8) {
    cudaStream_t st = c->stream;
    TcPrepared pr;
    PP_TRY(tc_prepare(c, mult, k, d_z, nterms, pr, st, f8));
    for (int P0 = 0; P0 < c->naux; P0 += pr.pc) {
        const int npc = std::min(pr.pc, c->naux - P0);
        std::vector<TcJobHost> s1, s2;
        std::vector<std::vector<int4>> tiles;
        PP_TRY(tc_jobs(c, pr, P0, npc, s1, s2, tiles));
        for (auto& h : s1) {
            const CUtensorMap* th = h.t_store ? &h.t_hi_map : nullptr;
            const CUtensorMap* tl = h.t_store ? &h.t_lo_map : nullptr;
            if (h.cluster > 1)
                PP_TRY(timed_launch(c, h.kind, h.flops, h.job.a_hi, h.job.a_lo, h.b_hi_half,
                                    h.b_lo_half, h.job.p, nterms, h.cluster, h.f8, h.pair, th, tl));
            else
                PP_TRY(timed_launch(c, h.kind, h.flops, h.job.a_hi, h.job.a_lo, h.job.b_hi,
                                    h.job.b_lo, h.job.p, nterms, 1, h.f8, false, th, tl));
        }
        for (size_t b = 0; b < s2.size(); ++b) {
            TcJobHost& h = s2[b];
            int4* d_tiles;
            PP_TRY(ws_get(c, "tc_tiles" + std::to_string(b), sizeof(int4) * tiles[b].size(), (void**)&d_tiles));
            PP_CUDA(cudaMemcpyAsync(d_tiles, tiles[b].data(), sizeof(int4) * tiles[b].size(),
                                    cudaMemcpyHostToDevice, st));
            h.job.p.tile_list = d_tiles;
            if (h.cluster > 1)
                PP_TRY(timed_launch(c, h.kind, h.flops, h.job.a_hi, h.job.a_lo, h.b_hi_half,
                                    h.b_lo_half, h.job.p, nterms, h.cluster, false, h.pair));
            else
                PP_TRY(timed_launch(c, h.kind, h.flops, h.job.a_hi, h.job.a_lo, h.job.b_hi,
                                    h.job.b_lo, h.job.p, nterms));
        }
    }
    PP_TRY(launch_pack_f32(pr.O, d_z, k, pr.pt->N, pr.pt->nvv, pr.pt->d_pp, pr.pt->d_pq, pr.pm,
                           c->d_eps, mult, d_sigma, st));
    return PPRPA_OK;
}

// Work items of one job (the same decomposition the single launch decodes arithmetically).
static void append_items(const TcParams& p, int job, const std::vector<int4>* tiles,
                         std::vector<TcItem>& out) {
    if (p.mode == 0) {
        const int64_t mt = ceil_div(p.M_rows, 128);
        for (int64_t mb = 0; mb < mt; ++mb)
            for (int nb = 0; nb < p.tiles_n; ++nb)
                out.push_back(TcItem{job, (int)(mb * 128), nb * p.BN, 0, 0, p.kb_total, p.BN, 0});
    } else {
        const int per = (p.kb_total + p.nsplit - 1) / p.nsplit;
        for (int sp = 0; sp < p.nsplit; ++sp)
            for (int b = 0; b < p.nbatch; ++b)
                for (const int4& t : *tiles)
                    out.push_back(TcItem{job, t.x * 128, t.y, b, sp * per,
                                         std::min(p.kb_total, (sp + 1) * per), t.z, 0});
    }
}

// Batched sigma over molecules (each its own context, one device and stream).  The host
// part (buffers, tensor maps, work items, their upload) runs once per batch signature; the
// device part (operand packing, the two persistent GEMM launches, unpacking) is replayed
// as a CUDA graph while the signature is unchanged.
struct BatchPlan {
    std::vector<pprpa_ctx*> ctxs;
    std::vector<int> mults, ks;
    std::vector<const double*> z;
    std::vector<double*> sigma;
    std::vector<unsigned long long> epochs;  // each context's mem_epoch when the plan was built
    int nterms = 1;
    cudaStream_t st = nullptr;
    std::vector<TcPrepared> prs;
    TcJob *dj1 = nullptr, *dj2 = nullptr;
    TcItem *di1 = nullptr, *di2 = nullptr;
    int n1 = 0, n2 = 0, bn1 = 16, bn2 = 16;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
};

static void free_plan_graph(BatchPlan* bp) {
    if (bp->exec) cudaGraphExecDestroy(bp->exec);
    if (bp->graph) cudaGraphDestroy(bp->graph);
    bp->exec = nullptr;
    bp->graph = nullptr;
}

void destroy_batch_plan(void* plan) {
    BatchPlan* bp = (BatchPlan*)plan;
    if (!bp) return;
    free_plan_graph(bp);
    delete bp;
}

static int batch_exec(BatchPlan& bp, pprpa_ctx* owner) {
    for (size_t m = 0; m < bp.ctxs.size(); ++m) PP_TRY(tc_device_prep(bp.ctxs[m], bp.prs[m], bp.st));
    PP_TRY(tc_gemm_launch_batched(bp.dj1, bp.di1, bp.n1, bp.bn1, bp.nterms, owner->num_sms,
                                  owner->d_status, bp.st));
    PP_TRY(tc_gemm_launch_batched(bp.dj2, bp.di2, bp.n2, bp.bn2, bp.nterms, owner->num_sms,
                                  owner->d_status, bp.st));
    for (size_t m = 0; m < bp.ctxs.size(); ++m) {
        const TcPrepared& pr = bp.prs[m];
        PP_TRY(launch_pack_f32(pr.O, bp.z[m], pr.k, pr.pt->N, pr.pt->nvv, pr.pt->d_pp, pr.pt->d_pq,
                               pr.pm, bp.ctxs[m]->d_eps, pr.mult, bp.sigma[m], bp.st));
    }
    return PPRPA_OK;
}

static bool same_signature(const BatchPlan& bp, int nmol, pprpa_ctx* const* ctxs, const int* mults,
                           const int* ks, const double* const* z, double* const* sigma, int nterms,
                           cudaStream_t st) {
    if ((int)bp.ctxs.size() != nmol || bp.nterms != nterms || bp.st != st) return false;
    for (int m = 0; m < nmol; ++m)
        if (bp.ctxs[m] != ctxs[m] || bp.mults[m] != mults[m] || bp.ks[m] != ks[m] || bp.z[m] != z[m] ||
            bp.sigma[m] != sigma[m] || bp.epochs[m] != ctxs[m]->mem_epoch)
            return false;
    return true;
}

// All molecules' tiles in one persistent launch per stage (work-item lists, CUDA graph).
static int batch_persistent(int nmol, pprpa_ctx* const* ctxs, const int* mults, const int* ks,
                            const double* const* z, double* const* sigma, int nterms, cudaStream_t st,
                            pprpa_ctx* owner, bool use_graph) {
    void*& slot = nterms == 3 ? owner->batch_plan3 : owner->batch_plan;
    BatchPlan* bp = (BatchPlan*)slot;
    if (bp && use_graph && bp->exec && same_signature(*bp, nmol, ctxs, mults, ks, z, sigma, nterms, st)) {
        PP_CUDA(cudaGraphLaunch(bp->exec, st));
        count_launch(bp->graph_kernels);
        return PPRPA_OK;
    }
    destroy_batch_plan(bp);
    bp = new BatchPlan();
    slot = bp;
    bp->ctxs.assign(ctxs, ctxs + nmol);
    bp->mults.assign(mults, mults + nmol);
    bp->ks.assign(ks, ks + nmol);
    bp->z.assign(z, z + nmol);
    bp->sigma.assign(sigma, sigma + nmol);
    bp->nterms = nterms;
    bp->st = st;
    bp->prs.resize(nmol);
    std::vector<TcJobHost> s1, s2;
    std::vector<std::vector<int4>> tiles;
    std::vector<int> s2_tile_index;
    for (int m = 0; m < nmol; ++m) {
        pprpa_ctx* c = ctxs[m];
        PP_TRY(tc_alloc(c, mults[m], ks[m], z[m], nterms, bp->prs[m], st));
        if (bp->prs[m].pc < c->naux)
            return set_error(PPRPA_ERR_ARG, "sigma_batch: a molecule's intermediate exceeds the T budget");
        const size_t before = tiles.size(), s2_before = s2.size();
        PP_TRY(tc_jobs(c, bp->prs[m], 0, c->naux, s1, s2, tiles, false));
        for (size_t t = s2_before; t < s2.size(); ++t) s2_tile_index.push_back((int)(before + (t - s2_before)));
    }
    // The K slices of stage 2 were chosen per molecule (about four waves each); over a whole
    // batch that splits far finer than the GPU needs, so re-split for four waves in total.
    // The split form keeps its cap on auxiliary functions per accumulator.
    if (env_int("PPRPA_BATCH_RESPLIT", 1) && !s2.empty()) {
        int64_t base = 0;
        for (const TcJobHost& h : s2) base += (int64_t)h.job.p.ntiles * h.job.p.nbatch;
        const int64_t target = std::max<int64_t>(1, ceil_div(4LL * owner->num_sms, base));
        const int pcap = env_int(nterms == 3 ? "PPRPA_S2_PCAP_SPLIT" : "PPRPA_S2_PCAP", nterms == 3 ? 2 : 128);
        for (TcJobHost& h : s2) {
            TcParams& p = h.job.p;
            const int npc = p.kb_total / std::max(1, p.kq_blocks);
            int64_t ns = std::min<int64_t>(target, std::max(1, p.kb_total / 8));
            if (pcap > 0) ns = std::max<int64_t>(ns, ceil_div(npc, pcap));
            const int64_t per = ceil_div(p.kb_total, std::max<int64_t>(1, ns));
            p.nsplit = (int)ceil_div(p.kb_total, per);
            p.total_items = p.ntiles * p.nbatch * p.nsplit;
        }
    }
    std::vector<TcJob> j1, j2;
    std::vector<TcItem> i1, i2;
    for (size_t j = 0; j < s1.size(); ++j) {
        j1.push_back(s1[j].job);
        append_items(s1[j].job.p, (int)j, nullptr, i1);
        bp->bn1 = std::max(bp->bn1, s1[j].job.p.BN);
    }
    for (size_t j = 0; j < s2.size(); ++j) {
        j2.push_back(s2[j].job);
        append_items(s2[j].job.p, (int)j, &tiles[s2_tile_index[j]], i2);
        bp->bn2 = std::max(bp->bn2, s2[j].job.p.BN);
    }
    bp->n1 = (int)i1.size();
    bp->n2 = (int)i2.size();
    // each plan slot (BF16, BF16x3) keeps its job and item arrays in buffers of its own: a
    // graph of one slot is replayed after the other slot's plan has been rebuilt, so they
    // must not share (or reallocate) each other's arrays
    const std::string sfx = nterms == 3 ? "_x3" : "";
    PP_TRY(ws_get(owner, "batch_j1" + sfx, sizeof(TcJob) * std::max<size_t>(1, j1.size()), (void**)&bp->dj1));
    PP_TRY(ws_get(owner, "batch_j2" + sfx, sizeof(TcJob) * std::max<size_t>(1, j2.size()), (void**)&bp->dj2));
    PP_TRY(ws_get(owner, "batch_i1" + sfx, sizeof(TcItem) * std::max<size_t>(1, i1.size()), (void**)&bp->di1));
    PP_TRY(ws_get(owner, "batch_i2" + sfx, sizeof(TcItem) * std::max<size_t>(1, i2.size()), (void**)&bp->di2));
    // the uploads go through pinned staging of the owner: a copy from pageable memory is
    // staged by the driver at a few GB/s, and a solve rebuilds its plan nearly every round
    {
        const size_t b1 = sizeof(TcJob) * j1.size(), b2 = sizeof(TcItem) * i1.size();
        const size_t b3 = sizeof(TcJob) * j2.size(), b4 = sizeof(TcItem) * i2.size();
        void* hp;
        PP_TRY(host_stage(owner, b1 + b2 + b3 + b4 + 64, &hp, 1));
        char* h = static_cast<char*>(hp);
        if (b1) std::memcpy(h, j1.data(), b1);
        if (b2) std::memcpy(h + b1, i1.data(), b2);
        if (b3) std::memcpy(h + b1 + b2, j2.data(), b3);
        if (b4) std::memcpy(h + b1 + b2 + b3, i2.data(), b4);
        if (b1) PP_CUDA(cudaMemcpyAsync(bp->dj1, h, b1, cudaMemcpyHostToDevice, st));
        if (b2) PP_CUDA(cudaMemcpyAsync(bp->di1, h + b1, b2, cudaMemcpyHostToDevice, st));
        if (b3) PP_CUDA(cudaMemcpyAsync(bp->dj2, h + b1 + b2, b3, cudaMemcpyHostToDevice, st));
        if (b4) PP_CUDA(cudaMemcpyAsync(bp->di2, h + b1 + b2 + b3, b4, cudaMemcpyHostToDevice, st));
    }
    PP_CUDA(cudaStreamSynchronize(st));  // the staging is reused by the next plan
    // the pointers captured below are those of the contexts as they are now
    bp->epochs.resize(nmol);
    for (int m = 0; m < nmol; ++m) bp->epochs[m] = ctxs[m]->mem_epoch;
    if (!use_graph) return batch_exec(*bp, owner);
    const long long captured0 = pprpa_kernel_launches();
    PP_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = batch_exec(*bp, owner);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    count_launch(captured0 - pprpa_kernel_launches());  // captured launches have not run
    if (rc != PPRPA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return set_error(PPRPA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    bp->graph = g;
    PP_CUDA(cudaGraphInstantiate(&bp->exec, g, 0));
    size_t nnodes = 0;
    PP_CUDA(cudaGraphGetNodes(g, nullptr, &nnodes));
    std::vector<cudaGraphNode_t> nodes(nnodes);
    PP_CUDA(cudaGraphGetNodes(g, nodes.data(), &nnodes));
    int kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
    bp->graph_kernels = kernels;
    PP_CUDA(cudaGraphLaunch(bp->exec, st));
    count_launch(kernels);
    return PPRPA_OK;
}

// Autotuner: time the candidate tile widths of both stages on the context's own problem
// (one sigma of k vectors each) and keep the fastest.
// Batched sigma.  A molecule whose first stage alone fills the GPU many times over runs on its
// own clustered launches; the rest share the persistent launch.  Measured on 64 molecules with
// nvir 50..400 (8 vectors each): all in one persistent launch 345 TF/s, every molecule on its
// own 419, molecules with >= 4000 first-stage tiles on their own 435.  PPRPA_BATCH_SEQ_TILES
// sets that tile count (0: every molecule; a huge value: none).
int sigma_tc_batch(int nmol, pprpa_ctx* const* ctxs, const int* mults, const int* ks,
                   const double* const* z, double* const* sigma, int nterms, cudaStream_t st,
                   pprpa_ctx* owner, bool use_graph) {
    const int64_t thr = env_int("PPRPA_BATCH_SEQ_TILES", 26 * owner->num_sms);
    std::vector<pprpa_ctx*> sc;
    std::vector<int> sm, sk;
    std::vector<const double*> sz;
    std::vector<double*> ss;
    std::vector<int> own;
    for (int m = 0; m < nmol; ++m) {
        const pprpa_ctx* c = ctxs[m];
        const int64_t np = round_up(c->no, 8) + round_up(c->nv, 8);
        const int64_t tiles = ceil_div((int64_t)c->naux * np, 128) * ceil_div((int64_t)ks[m] * round_up(c->nv, 8), 256);
        if (tiles >= thr) {
            own.push_back(m);
        } else {
            sc.push_back(ctxs[m]); sm.push_back(mults[m]); sk.push_back(ks[m]);
            sz.push_back(z[m]); ss.push_back(sigma[m]);
        }
    }
    for (int m : own) {
        pprpa_ctx* c = ctxs[m];
        cudaStream_t keep = c->stream;
        c->stream = st;  // the batch runs on one stream
        const int rc = sigma_tc(c, mults[m], ks[m], z[m], sigma[m], nterms);
        c->stream = keep;
        PP_TRY(rc);
    }
    if (!sc.empty())
        PP_TRY(batch_persistent((int)sc.size(), sc.data(), sm.data(), sk.data(), sz.data(), ss.data(), nterms, st,
                                owner, use_graph));
    if (!own.empty()) {
        PP_CUDA(cudaStreamSynchronize(st));
        for (int m : own) PP_TRY(check_status(ctxs[m]));
    }
    return PPRPA_OK;
}

int autotune_tiles(pprpa_ctx* c, int mult, int k, int nterms, int* bn_out) {
    PairTable* pt;
    PP_TRY(ensure_pairs(c, mult, &pt));
    double *z, *sg;
    PP_TRY(ws_get(c, "tune_z", sizeof(double) * (size_t)k * pt->N, (void**)&z));
    PP_TRY(ws_get(c, "tune_s", sizeof(double) * (size_t)k * pt->N, (void**)&sg));
    PP_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)k * pt->N, c->stream));
    cudaEvent_t a, b;
    PP_CUDA(cudaEventCreate(&a));
    PP_CUDA(cudaEventCreate(&b));
    const int sizes[2] = {c->nv, c->no};
    int result[4] = {0, 0, 0, 0};
    for (int stage = 1; stage <= 2; ++stage) {
        for (int blk = 0; blk < 2; ++blk) {
            const int sz = sizes[blk];
            if (sz == 0) continue;
            std::vector<int> cand;
            const int szp = blk == 0 ? (int)round_up(c->nv, 8) : (int)round_up(c->no, 8);
            if (stage == 1) {
                for (int bn : {128, 192, 256}) cand.push_back(std::min(bn, (int)round_up((int64_t)k * szp, 16)));
            } else {
                cand.push_back(stage2_bn(sz));
                for (int bn : {128, 192, 256}) cand.push_back(std::min(bn, (int)round_up(sz, 16)));
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            const std::string key = tune_key(stage, sz, k);
            float best = 1e30f;
            int best_bn = cand[0];
            for (int bn : cand) {
                c->tuned_bn[key] = bn;
                PP_TRY(sigma_tc(c, mult, k, z, sg, nterms));  // warm
                PP_CUDA(cudaEventRecord(a, c->stream));
                PP_TRY(sigma_tc(c, mult, k, z, sg, nterms));
                PP_CUDA(cudaEventRecord(b, c->stream));
                PP_CUDA(cudaEventSynchronize(b));
                float ms = 0.f;
                PP_CUDA(cudaEventElapsedTime(&ms, a, b));
                if (ms < best) { best = ms; best_bn = bn; }
            }
            c->tuned_bn[key] = best_bn;
            result[(stage - 1) * 2 + blk] = best_bn;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (bn_out)
        for (int i = 0; i < 4; ++i) bn_out[i] = result[i];
    return check_status(c);
}

}  // namespace pprpa
