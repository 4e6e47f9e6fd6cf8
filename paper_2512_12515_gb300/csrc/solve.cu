// pprpa_solve: explicit-matrix full diagonalisation and the Davidson solver.
//
// Davidson (standard, for M z = omega W z, W = diag(I_nvv, -I_noo)):
//   guess    unit vectors at the lowest diagonal entries of the A block
//   sigma    Sg = M V for the new vectors (FP64, BF16 or BF16x3 split)
//   project  G = V Sg^T, S = V W V^T (FP64 dot products)
//   RR       shift-Cholesky + Jacobi on the GPU (one CTA), roots selected by
//            positive norm (Eq. xy_norm), lowest first
//   residual r_j = Sg^T c_j - omega_j W V^T c_j
//   correct  r_j / (D - omega_j w), two passes of classical Gram-Schmidt
//            against V, Cholesky-QR among the new vectors
//   restart  collapse to the current Ritz vectors when the subspace is full
// Mixed precision runs the same loop with BF16 sigma until the residuals
// reach the BF16 noise level, collapses to the Ritz vectors, recomputes
// their sigma with the BF16x3 split form and continues to conv_tol.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

#include "ctx.h"

namespace pprpa {

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    double total_ms = 0.0;
    cudaStream_t st;
    explicit Timer(cudaStream_t s, bool blocking = false) : st(s) {
        cudaEventCreate(&a);
        cudaEventCreateWithFlags(&b, blocking ? cudaEventBlockingSync : cudaEventDefault);
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    void start() { cudaEventRecord(a, st); }
    void stop() {
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        total_ms += ms;
    }
};

// C[i][j] (+)= alpha * sum_k A_i[k] B_j[k] for i < na, j < nb (rows of length K, stride lda/ldb).
// Always accumulates atomically; zero_first clears the na x nb block of C (ld ldc) first.
int dots(const double* A, int64_t lda, int na, const double* B, int64_t ldb, int nb, int K,
         double* C, int64_t ldc, double alpha, bool zero_first, cudaStream_t st) {
    if (na <= 0 || nb <= 0) return PPRPA_OK;
    Dgemm g;
    g.M = na; g.N = nb; g.K = K;
    g.A = A; g.lda = lda;
    g.B = B; g.ldb = ldb; g.transB = 1;
    g.C = C; g.ldc = ldc;
    g.alpha = alpha;
    if (K > 0 && dgemm_small(g)) {
        // a small product writes C (or adds to it) itself: no zeroing launch
        g.beta = zero_first ? 0.0 : 1.0;
        return dgemm(g, st);
    }
    if (zero_first)
        PP_CUDA(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * nb, na, st));
    if (K <= 0) return PPRPA_OK;
    g.splitk = std::max(2, auto_splitk(na, nb, K, 1));
    return dgemm(g, st);
}

// Out[j] = alpha * sum_i coef[j][i] X[i] + beta * Out[j]   (nc x m) x (m x N)
int combine(const double* coef, int ldc_, int nc, int m, const double* X, int64_t N, double* Out,
            double alpha, double beta, cudaStream_t st) {
    if (nc <= 0) return PPRPA_OK;
    Dgemm g;
    g.M = nc; g.N = (int)N; g.K = m;
    g.A = coef; g.lda = ldc_;
    g.B = X; g.ldb = N;
    g.C = Out; g.ldc = N;
    g.alpha = alpha; g.beta = beta;
    return dgemm(g, st);
}

void fix_phase(double* z, int N) {
    int imax = 0;
    double vmax = -1.0;
    for (int i = 0; i < N; ++i)
        if (std::fabs(z[i]) > vmax) { vmax = std::fabs(z[i]); imax = i; }
    if (N > 0 && z[imax] < 0.0)
        for (int i = 0; i < N; ++i) z[i] = -z[i];
}

int write_outputs(pprpa_ctx* c, PairTable* pt, int nroots, const double* d_Z, const double* h_omega,
                  double* omega, double* X, double* Y) {
    const int N = pt->N;
    std::vector<double> Z((size_t)nroots * N);
    PP_CUDA(cudaMemcpyAsync(Z.data(), d_Z, sizeof(double) * Z.size(), cudaMemcpyDeviceToHost, c->stream));
    PP_TRY(ctx_sync(c));
    for (int j = 0; j < nroots; ++j) {
        fix_phase(Z.data() + (size_t)j * N, N);
        if (omega) omega[j] = h_omega[j];
        if (X) std::copy(Z.begin() + (size_t)j * N, Z.begin() + (size_t)j * N + pt->nvv, X + (size_t)j * pt->nvv);
        if (Y && pt->noo)
            std::copy(Z.begin() + (size_t)j * N + pt->nvv, Z.begin() + (size_t)(j + 1) * N, Y + (size_t)j * pt->noo);
    }
    // keep the eigenvectors for gradients
    if (c->d_lastZ) cudaFree(c->d_lastZ);
    c->d_lastZ = nullptr;
    PP_CUDA(cudaMalloc(&c->d_lastZ, sizeof(double) * Z.size()));
    PP_CUDA(cudaMemcpyAsync(c->d_lastZ, Z.data(), sizeof(double) * Z.size(), cudaMemcpyHostToDevice, c->stream));
    PP_TRY(ctx_sync(c));
    c->last_nroots = nroots;
    c->last_N = N;
    return PPRPA_OK;
}

// Shift candidates between the highest two-electron removal estimate `lo`
// and the lowest addition estimate `hi`, best guess first.
std::vector<double> shift_candidates(double lo, double hi, double prev, bool have_prev) {
    std::vector<double> m;
    if (have_prev) m.push_back(prev);
    if (hi > lo) {
        const double fr[] = {0.5, 0.25, 0.75, 0.1, 0.9, 0.4, 0.6, 0.02, 0.98};
        for (double f : fr) m.push_back(lo + f * (hi - lo));
    } else {
        const double d = std::max(1e-3, std::fabs(hi - lo));
        for (int t = 1; t <= 8; ++t) m.push_back(hi - d * t);
    }
    return m;
}

int env_int(const char* name, int dflt) {
    const char* s = getenv(name);
    return s ? atoi(s) : dflt;
}
double env_dbl(const char* name, double dflt) {
    const char* s = getenv(name);
    return s ? atof(s) : dflt;
}

}  // namespace

// ---------------------------------------------------------------------------
// Explicit ppRPA matrix: the (pr|qs) = sum_P L^P_pr L^P_qs table as one
// (n^2 x n^2) FP64 product of the fitted integrals, then the spin-adapted
// elements of Sec. "ppRPA Equation" gathered from it.
static int build_explicit(pprpa_ctx* c, PairTable* pt, int mult, double* eri, double* M) {
    const int64_t n2 = (int64_t)c->n() * c->n();
    Dgemm g;
    g.M = (int)n2; g.N = (int)n2; g.K = c->naux;
    g.A = c->d_L; g.lda = n2; g.transA = 1;
    g.B = c->d_L; g.ldb = n2;
    g.C = eri; g.ldc = n2;
    PP_TRY(dgemm(g, c->stream));
    return launch_build_matrix(eri, c->n(), pt->d_pp, pt->d_pq, pt->N, pt->nvv, c->d_eps, mult, M,
                               c->stream);
}

static int solve_full(pprpa_ctx* c, const pprpa_options* o, PairTable* pt, double* omega, double* X,
                      double* Y, double* ec, pprpa_info* info) {
    const int N = pt->N, nvv = pt->nvv, n = c->n();
    cudaStream_t st = c->stream;
    if (N > 1024) return set_error(PPRPA_ERR_ARG, "full diagonalisation is limited to N <= 1024 pairs; use Davidson");
    Timer tt(st, c->blocking_sync);
    tt.start();
    const int64_t n2 = (int64_t)n * n;
    double *eri, *M, *W, *work, *om, *coef, *rinfo, *D, *dwork, *mus, *dec;
    PP_TRY(ws_get(c, "full_eri", sizeof(double) * n2 * n2, (void**)&eri));
    PP_TRY(ws_get(c, "full_M", sizeof(double) * (size_t)N * N, (void**)&M));
    PP_TRY(ws_get(c, "full_W", sizeof(double) * (size_t)N * N, (void**)&W));
    PP_TRY(ws_get(c, "full_work", sizeof(double) * (4 * (size_t)N * N + 8 * (size_t)N), (void**)&work));
    PP_TRY(ws_get(c, "full_om", sizeof(double) * N, (void**)&om));
    PP_TRY(ws_get(c, "full_coef", sizeof(double) * (size_t)N * N, (void**)&coef));
    PP_TRY(ws_get(c, "full_info", sizeof(double) * 8, (void**)&rinfo));
    PP_TRY(ws_get(c, "full_D", sizeof(double) * N, (void**)&D));
    PP_TRY(ws_get(c, "full_dwork", sizeof(double) * (size_t)c->naux * n, (void**)&dwork));
    PP_TRY(ws_get(c, "full_mus", sizeof(double) * 32, (void**)&mus));
    PP_TRY(ws_get(c, "full_ec", sizeof(double), (void**)&dec));
    // pp channel: the lowest roots of positive norm of (M, W).  hh channel: the highest roots
    // of negative norm, i.e. the lowest roots of positive norm of (M, -W) with omega = -mu.
    const bool hh = o->channel == PPRPA_CHANNEL_HH;
    const double ws = hh ? -1.0 : 1.0;
    const int noo = pt->noo;
    const int npos = hh ? noo : nvv;  // roots of positive norm in the solved pencil
    if (o->mult == PPRPA_AB) PP_TRY(build_ab(c, pt, M));
    else PP_TRY(build_explicit(c, pt, o->mult, eri, M));
    PP_TRY(launch_metric_matrix(W, N, nvv, st, ws));
    if (o->mult == PPRPA_AB) PP_TRY(diag_ab(c, pt, D));
    else PP_TRY(launch_diag(c->d_L, c->naux, n, c->d_eps, pt->d_pp, pt->d_pq, nvv, N, o->mult, D, dwork, st));
    std::vector<double> hD(N);
    PP_CUDA(cudaMemcpyAsync(hD.data(), D, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    PP_TRY(ctx_sync(c));
    // gap edges of the solved pencil from the diagonal: its positive-norm block (vv, or oo
    // for hh) starts near min D there, its negative-norm block ends near max(-D)
    double hi = 1e300, lo = -1e300;
    for (int i = 0; i < N; ++i) {
        if ((i < nvv) != hh) hi = std::min(hi, hD[i]);
        else lo = std::max(lo, -hD[i]);
    }
    if (npos == N) lo = hi - 1.0;
    // wide scan: the diagonal only estimates the gap edges
    std::vector<double> cand = shift_candidates(lo, hi, 0.0, false);
    for (int t = 1; t <= 6; ++t) {
        cand.push_back(lo - 0.25 * t);
        cand.push_back(hi + 0.25 * t);
    }
    cand.resize(std::min<size_t>(cand.size(), 32));
    PP_CUDA(cudaMemcpyAsync(mus, cand.data(), sizeof(double) * cand.size(), cudaMemcpyHostToDevice, st));
    RRArgs a;
    a.G = M; a.S = W; a.ld = N; a.m = N;
    a.mus = mus; a.nmu = (int)cand.size();
    a.nwant = o->nroots; a.nkeep = npos;
    a.work = work; a.omega = om; a.coef = coef; a.info = rinfo;
    PP_TRY(launch_rayleigh_ritz(a, st));
    double hinfo[8];
    PP_CUDA(cudaMemcpyAsync(hinfo, rinfo, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
    PP_TRY(ctx_sync(c));
    if ((int)hinfo[0] == DEV_NOTPD)
        return set_error(PPRPA_ERR_UNSTABLE, "full: no shift makes M - mu W positive definite");
    if ((int)hinfo[2] != npos)
        return set_error(PPRPA_ERR_UNSTABLE, "full: root count by norm differs from the pair count");
    std::vector<double> h_om(npos);
    PP_CUDA(cudaMemcpyAsync(h_om.data(), om, sizeof(double) * npos, cudaMemcpyDeviceToHost, st));
    if (ec) {
        // E_c = sum Omega^{+2e} - Tr A (pp), or -sum Omega^{-2e} - Tr C = sum mu - Tr C (hh)
        // (Eq. correlation_energy); both need every root of the channel, which FULL has
        if (hh) PP_TRY(launch_ec_sum(om, noo, D + nvv, noo, dec, st));
        else PP_TRY(launch_ec_sum(om, nvv, D, nvv, dec, st));
        PP_CUDA(cudaMemcpyAsync(ec, dec, sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    PP_TRY(ctx_sync(c));
    if (hh)
        for (double& v : h_om) v = -v;  // omega of the removal roots, highest first
    PP_TRY(write_outputs(c, pt, o->nroots, coef, h_om.data(), omega, X, Y));
    c->last_all_roots = o->nroots == npos;
    c->last_channel = o->channel;
    tt.stop();
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->converged = 1;
        info->nconv = o->nroots;
        info->n_real = npos;
        info->mu = hinfo[1];
        info->t_total_ms = tt.total_ms;
    }
    c->last_mult = o->mult;
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
static int solve_davidson(pprpa_ctx* c, const pprpa_options* o, PairTable* pt, double* omega,
                          double* X, double* Y, double* ec, pprpa_info* info, SigmaHook* hook) {
    const int N = pt->N, nvv = pt->nvv, noo = pt->noo;
    const int nroots = o->nroots;
    cudaStream_t st = c->stream;
    // hh channel: solve (M, -W) for its lowest positive-norm roots mu (omega = -mu); every
    // use of the metric below carries its sign ws, and the blocks of positive and negative
    // norm trade places
    const bool hh = o->channel == PPRPA_CHANNEL_HH;
    const double ws = hh ? -1.0 : 1.0;
    const int pos0 = hh ? nvv : 0, npos_blk = hh ? noo : nvv;  // positive-norm block
    const int nguess = std::min(npos_blk, std::max(2 * nroots, nroots + 8));
    // subspace cap and thick-restart size: unstable problems (complex pairs near the
    // targets) need a restart that keeps many Ritz vectors, so both are generous
    // automatic cap: the largest subspace whose Rayleigh-Ritz matrices stay in shared memory
    int m_max = o->max_subspace > 0 ? o->max_subspace : 112;
    m_max = std::min(m_max, 128);
    m_max = std::min(m_max, N);
    if (m_max < nguess + 1 && N > nguess) m_max = std::min(N, nguess + 1);
    int nkeep = std::max(nguess, std::max(4 * nroots, 40));
    nkeep = std::min(nkeep, std::max(1, m_max - std::max(nroots, 8)));
    // automatic cap on the definite (shift-Cholesky) path: restart at 72, the range of the
    // clustered Rayleigh-Ritz kernel, while one sigma vector costs less than about one
    // Rayleigh-Ritz call beyond it (PPRPA_SOFT_CAP_FLOPS, default 5e11 flop: a few ms of FP64
    // work on one SM against a sigma vector of that size); the general path keeps the full cap
    const double fsig = 3.0 * c->naux * c->n() * ((double)c->nv * c->nv + (double)c->no * c->no);
    const double cap_flops = env_dbl("PPRPA_SOFT_CAP_FLOPS", 5e11);
    const int m_soft = (o->max_subspace > 0 || fsig >= cap_flops) ? m_max
                                                                    : std::min(m_max, std::max(72, nkeep + nroots));
    const int max_new = nroots;
    Timer t_all(st, c->blocking_sync), t_sig(st, c->blocking_sync);
    t_all.start();

    double *V, *Sg, *G, *S, *D, *dwork, *R, *Zr, *SZ, *Dn, *Dn2, *H, *rwork, *om, *coef, *rinfo,
        *mus, *nrm, *Gm, *Tm, *cwork, *dom;
    int *keep, *sel, *idx;
    PP_TRY(ws_get(c, "dv_V", sizeof(double) * (size_t)m_max * N, (void**)&V));
    PP_TRY(ws_get(c, "dv_Sg", sizeof(double) * (size_t)m_max * N, (void**)&Sg));
    PP_TRY(ws_get(c, "dv_G", sizeof(double) * m_max * m_max, (void**)&G));
    double* Go;
    PP_TRY(ws_get(c, "dv_Go", sizeof(double) * m_max * m_max, (void**)&Go));
    PP_TRY(ws_get(c, "dv_S", sizeof(double) * m_max * m_max, (void**)&S));
    PP_TRY(ws_get(c, "dv_D", sizeof(double) * N, (void**)&D));
    PP_TRY(ws_get(c, "dv_dwork", sizeof(double) * (size_t)c->naux * c->n(), (void**)&dwork));
    PP_TRY(ws_get(c, "dv_R", sizeof(double) * (size_t)nroots * N, (void**)&R));
    PP_TRY(ws_get(c, "dv_Zr", sizeof(double) * (size_t)m_max * N, (void**)&Zr));
    PP_TRY(ws_get(c, "dv_SZ", sizeof(double) * (size_t)m_max * N, (void**)&SZ));
    const int nbuf = std::max(max_new, std::max(nkeep, nroots));
    PP_TRY(ws_get(c, "dv_Dn", sizeof(double) * (size_t)nbuf * N, (void**)&Dn));
    PP_TRY(ws_get(c, "dv_Dn2", sizeof(double) * (size_t)nbuf * N, (void**)&Dn2));
    PP_TRY(ws_get(c, "dv_H", sizeof(double) * m_max * m_max, (void**)&H));
    PP_TRY(ws_get(c, "dv_rwork", sizeof(double) * (4 * (size_t)m_max * m_max + 8 * (size_t)m_max), (void**)&rwork));
    PP_TRY(ws_get(c, "dv_om", sizeof(double) * m_max, (void**)&om));
    PP_TRY(ws_get(c, "dv_coef", sizeof(double) * m_max * m_max, (void**)&coef));
    PP_TRY(ws_get(c, "dv_info", sizeof(double) * 8, (void**)&rinfo));
    PP_TRY(ws_get(c, "dv_mus", sizeof(double) * 32, (void**)&mus));
    PP_TRY(ws_get(c, "dv_nrm", sizeof(double) * m_max, (void**)&nrm));
    PP_TRY(ws_get(c, "dv_Gm", sizeof(double) * m_max * m_max, (void**)&Gm));
    PP_TRY(ws_get(c, "dv_Tm", sizeof(double) * m_max * m_max, (void**)&Tm));
    PP_TRY(ws_get(c, "dv_cwork", sizeof(double) * (m_max * m_max + m_max), (void**)&cwork));
    PP_TRY(ws_get(c, "dv_keep", sizeof(int) * m_max, (void**)&keep));
    PP_TRY(ws_get(c, "dv_sel", sizeof(int) * m_max, (void**)&sel));
    PP_TRY(ws_get(c, "dv_idx", sizeof(int) * m_max, (void**)&idx));
    PP_TRY(ws_get(c, "dv_dom", sizeof(double) * m_max, (void**)&dom));
    // pinned staging of the per-iteration readbacks and uploads (one wait per decision point):
    // RR info (8), Ritz values (m_max), residual norms (m_max), norms before / after the
    // orthogonalisation (nbuf each), shifts (32), then ints: selected roots (nbuf), the keep
    // flags of the two Cholesky-QR passes (2 nbuf) and the row lists of the two gathers (2 nbuf)
    void* hst;
    PP_TRY(host_stage(c, sizeof(double) * (8 + 2 * (size_t)m_max + 2 * (size_t)nbuf + 32) +
                             sizeof(int) * 5 * (size_t)nbuf, &hst));
    double* hs_info = static_cast<double*>(hst);
    double* hs_om = hs_info + 8;
    double* hs_nrm = hs_om + m_max;
    double* hs_nb = hs_nrm + m_max;
    double* hs_na = hs_nb + nbuf;
    double* hs_mus = hs_na + nbuf;
    int* hs_sel = reinterpret_cast<int*>(hs_mus + 32);
    int* hs_keep = hs_sel + nbuf;
    int* hs_live = hs_keep + 2 * nbuf;  // rows kept by the orthogonalisation, then by Cholesky-QR
    int* hs_kept = hs_live + nbuf;

    // a3: diagonal, then the initial guess
    if (o->mult == PPRPA_AB) PP_TRY(diag_ab(c, pt, D));
    else PP_TRY(launch_diag(c->d_L, c->naux, c->n(), c->d_eps, pt->d_pp, pt->d_pq, nvv, N, o->mult, D, dwork, st));
    std::vector<double> hD(N);
    PP_CUDA(cudaMemcpyAsync(hD.data(), D, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    PP_TRY(ctx_sync(c));
    std::vector<int> order(npos_blk);
    std::iota(order.begin(), order.end(), pos0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hD[a] < hD[b]; });
    // lowest positive-norm estimate, highest negative-norm estimate
    double dv_min = hD[order[0]], oo_max = -1e300;
    for (int i = 0; i < N; ++i)
        if ((i < pos0) || (i >= pos0 + npos_blk)) oo_max = std::max(oo_max, -hD[i]);
    PP_CUDA(cudaMemsetAsync(V, 0, sizeof(double) * (size_t)nguess * N, st));
    PP_CUDA(cudaMemcpyAsync(idx, order.data(), sizeof(int) * nguess, cudaMemcpyHostToDevice, st));
    PP_TRY(launch_scatter_unit(V, N, idx, nguess, st));

    // stages: 0 FP64 throughout; 1 BF16 (or 3 FP8) until the low-precision noise level,
    // then 2 BF16x3 to conv_tol
    const bool mixed = o->precision == PPRPA_PREC_BF16 || o->precision == PPRPA_PREC_FP8;
    int stage = o->precision == PPRPA_PREC_FP8 ? 3 : (mixed ? 1 : 0);
    // residual level at which the low-precision stage hands over: about the sigma noise of
    // its operands (BF16 unit roundoff 2^-8, E4M3 2^-4)
    const double tol1 = env_dbl("PPRPA_STAGE1_TOL",
                                std::max(o->conv_tol * 10.0,
                                         o->precision == PPRPA_PREC_FP8 ? 8e-2 : 1e-2));
    auto run_sigma = [&](int k, const double* z, double* out) -> int {
        t_sig.start();
        int rc;
        if (o->mult == PPRPA_AB) rc = sigma_ab_f64(c, k, z, out);
        else if (stage == 0) rc = sigma_f64(c, o->mult, k, z, out);
        else if (stage == 3) rc = sigma_tc(c, o->mult, k, z, out, 1, true);
        else if (hook) rc = hook->sigma(c, o->mult, k, z, out, stage == 1 ? 1 : 3);
        else rc = sigma_tc(c, o->mult, k, z, out, stage == 1 ? 1 : 3);
        t_sig.stop();
        if (rc != PPRPA_OK) return rc;
        if (stage != 0 && !(hook && (stage == 1 || stage == 2))) PP_TRY(check_status(c));
        if (info) {
            info->n_sigma += k;
            info->sigma_flops += (double)k * 3.0 * c->naux * c->n() *
                                 ((double)c->nv * c->nv + (double)c->no * c->no);
        }
        return PPRPA_OK;
    };
    auto project_block = [&](int m0, int m) -> int {
        const int kn = m - m0;
        // Gp = V Sg^T over the positive-norm pairs and Gn over the others (virtual and
        // occupied pairs, swapped for hh), blocks [0:m, m0:m] and [m0:m, 0:m0]:
        // V^T M V = Gp + Gn and V^T (ws W) M V = Gp - Gn.
        double* Gv = hh ? Go : G;  // virtual-pair part
        double* Gq = hh ? G : Go;  // occupied-pair part
        PP_TRY(dots(V, N, m, Sg + (size_t)m0 * N, N, kn, nvv, Gv + m0, m_max, 1.0, true, st));
        PP_TRY(dots(V + (size_t)m0 * N, N, kn, Sg, N, m0, nvv, Gv + (size_t)m0 * m_max, m_max, 1.0, true, st));
        PP_TRY(dots(V + nvv, N, m, Sg + (size_t)m0 * N + nvv, N, kn, noo, Gq + m0, m_max, 1.0, true, st));
        PP_TRY(dots(V + (size_t)m0 * N + nvv, N, kn, Sg + nvv, N, m0, noo, Gq + (size_t)m0 * m_max, m_max, 1.0,
                    true, st));
        // S[0:m, m0:m] = V (ws W) V^T (virtual pairs ws, occupied pairs -ws)
        PP_TRY(dots(V, N, m, V + (size_t)m0 * N, N, kn, nvv, S + m0, m_max, ws, true, st));
        PP_TRY(dots(V + nvv, N, m, V + (size_t)m0 * N + nvv, N, kn, noo, S + m0, m_max, -ws, false, st));
        return PPRPA_OK;
    };
    // collapse the basis onto the first nk Ritz vectors (coef rows), orthonormalised
    auto collapse = [&](int nk, int m, bool resigma) -> int {
        PP_TRY(dots(coef, m, nk, coef, m, nk, m, Gm, nk, 1.0, true, st));
        PP_TRY(launch_cholqr_small(Gm, nk, 1e-14, Tm, keep, cwork, st));
        PP_TRY(combine(Tm, nk, nk, nk, coef, m, H, 1.0, 0.0, st));  // H = T coef (nk x m)
        PP_TRY(combine(H, m, nk, m, V, N, Dn2, 1.0, 0.0, st));
        PP_CUDA(cudaMemcpyAsync(V, Dn2, sizeof(double) * (size_t)nk * N, cudaMemcpyDeviceToDevice, st));
        if (resigma) {
            PP_TRY(run_sigma(nk, V, Sg));
        } else {
            PP_TRY(combine(H, m, nk, m, Sg, N, Dn2, 1.0, 0.0, st));
            PP_CUDA(cudaMemcpyAsync(Sg, Dn2, sizeof(double) * (size_t)nk * N, cudaMemcpyDeviceToDevice, st));
        }
        return project_block(0, nk);
    };

    int m = nguess;
    PP_TRY(run_sigma(nguess, V, Sg));
    PP_TRY(project_block(0, m));
    double mu_prev = 0.0;
    bool have_mu = false;
    bool general = false;
    double max_imag_below = 0.0;
    double lo_est = oo_max, hi_est = dv_min;
    if (noo == 0) lo_est = dv_min - 1.0;
    std::vector<double> h_om(m_max), h_nrm(nroots), best_hist;
    int rc_final = PPRPA_ERR_NOCONV;
    int it = 0, stage1_iters = 0;
    // iterations of persistent complex pairs below the targets without a tenfold residual drop
    // after which the solve reports the problem as unstable (PPRPA_UNSTABLE_WINDOW)
    const int unstable_win = std::max(1, env_int("PPRPA_UNSTABLE_WINDOW", 40));
    std::vector<int> cplx_hist;
    std::vector<double> gen_hist;
    double hinfo[8] = {0};
    for (it = 1; it <= o->max_iter; ++it) {
        // ---- Rayleigh-Ritz: shifted symmetric reduction while the pencil is definite,
        //      general (non-symmetric) projection once it is not ----
        const int nk_req = std::max(nkeep, nroots);
        int npos = 0;
        if (!general) {
            std::vector<double> cand = shift_candidates(lo_est, hi_est, mu_prev, have_mu);
            for (int t = 1; t <= 4 && cand.size() < 32; ++t) {
                cand.push_back(lo_est - 0.5 * t);
                cand.push_back(hi_est - 0.05 * t);
            }
            cand.resize(std::min<size_t>(cand.size(), 32));
            std::copy(cand.begin(), cand.end(), hs_mus);
            PP_CUDA(cudaMemcpyAsync(mus, hs_mus, sizeof(double) * cand.size(), cudaMemcpyHostToDevice, st));
            RRArgs a;
            a.G = G; a.Go = Go; a.S = S; a.ld = m_max; a.m = m;
            a.mus = mus; a.nmu = (int)cand.size();
            a.nwant = nroots; a.nkeep = nk_req;
            a.work = rwork; a.omega = om; a.coef = coef; a.info = rinfo;
            PP_TRY(launch_rayleigh_ritz(a, st));
            // status and Ritz values in one wait (the values are used only when the call succeeded)
            PP_CUDA(cudaMemcpyAsync(hs_info, rinfo, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
            PP_CUDA(cudaMemcpyAsync(hs_om, om, sizeof(double) * std::min(nk_req, m), cudaMemcpyDeviceToHost, st));
            PP_TRY(ctx_sync(c));
            std::copy(hs_info, hs_info + 6, hinfo);
            if ((int)hinfo[0] == DEV_NOTPD) {
                if (o->require_definite) {
                    if (info) {
                        info->iters = it;
                        info->n_real = 0;  // no iterate is returned
                    }
                    return set_error(PPRPA_ERR_UNSTABLE, "Davidson: the subspace pencil has no definite shift");
                }
                if (m > 128) return set_error(PPRPA_ERR_UNSTABLE, "Davidson: no definite shift and subspace > 128");
                general = true;
                if (env_int("PPRPA_LOG", 0)) fprintf(stderr, "[pprpa] no definite shift: general Rayleigh-Ritz\n");
            } else {
                npos = (int)hinfo[2];
                mu_prev = hinfo[1];
                have_mu = true;
                hi_est = hinfo[3];
                if (hinfo[4] > -1e299) lo_est = hinfo[4];
            }
        }
        if (general) {
            RRGenArgs g;
            g.Gv = G; g.Go = Go; g.S = S; g.ld = m_max; g.m = m;
            g.nwant = nroots; g.nkeep = nk_req;
            g.work = rwork; g.omega = om; g.coef = coef; g.info = rinfo;
            PP_TRY(launch_rr_general(g, st));
            PP_CUDA(cudaMemcpyAsync(hs_info, rinfo, sizeof(double) * 8, cudaMemcpyDeviceToHost, st));
            PP_CUDA(cudaMemcpyAsync(hs_om, om, sizeof(double) * std::min(nk_req, m), cudaMemcpyDeviceToHost, st));
            PP_TRY(ctx_sync(c));
            std::copy(hs_info, hs_info + 8, hinfo);
            if ((int)hinfo[0] == DEV_NOTPD)
                return set_error(PPRPA_ERR_UNSTABLE, "Davidson: subspace eigenvalue iteration failed");
            npos = (int)hinfo[2];
        }
        if (npos < 1)
            return set_error(PPRPA_ERR_UNSTABLE, "Davidson: the subspace holds no real addition root");
        const int ntg = std::min(npos, nroots);  // targets this iteration
        std::copy(hs_om, hs_om + std::min(npos, nk_req), h_om.begin());
        const int nk_avail = std::min(npos, nk_req);
        // complex Ritz values below the highest target: complex roots among the lowest
        if (general) max_imag_below = (hinfo[6] < h_om[ntg - 1]) ? hinfo[7] : 0.0;
        // ---- Ritz vectors and residuals of the targets ----
        PP_TRY(combine(coef, m, ntg, m, V, N, Zr, 1.0, 0.0, st));
        PP_TRY(combine(coef, m, ntg, m, Sg, N, SZ, 1.0, 0.0, st));
        PP_CUDA(cudaMemsetAsync(nrm, 0, sizeof(double) * ntg, st));
        PP_TRY(launch_residual(SZ, Zr, om, ntg, N, nvv, R, nrm, st, ws));
        PP_CUDA(cudaMemcpyAsync(hs_nrm, nrm, sizeof(double) * ntg, cudaMemcpyDeviceToHost, st));
        PP_TRY(ctx_sync(c));
        std::copy(hs_nrm, hs_nrm + ntg, h_nrm.begin());
        double rmax = 0.0;
        std::vector<int> todo;
        for (int j = 0; j < ntg; ++j) {
            h_nrm[j] = std::sqrt(h_nrm[j]);
            rmax = std::max(rmax, h_nrm[j]);
            if (!(h_nrm[j] <= o->conv_tol)) todo.push_back(j);
        }
        if (ntg < nroots) rmax = std::max(rmax, 1e300);  // not enough real roots yet
        if (env_int("PPRPA_LOG", 0))
            fprintf(stderr, "[pprpa] it %d stage %d m %d mu %.6f omega0 %.10f max|r| %.3e sweeps %d\n", it, stage,
                    m, mu_prev, h_om[0], rmax, general ? -1 : (int)hinfo[5]);
        if (info) {
            info->max_resid = rmax;
            info->nconv = ntg - (int)todo.size();
            info->n_real = npos;
            info->max_imag = max_imag_below;
        }
        if (general) {
            // complex Ritz pairs below the highest target in at least half of the last
            // unstable_win iterations while the residual has not dropped tenfold over them: the
            // lowest roots are interleaved with complex pairs (no definite shift), where a
            // Davidson iteration on the real Ritz values does not settle
            gen_hist.push_back(rmax);
            cplx_hist.push_back(max_imag_below > 0.0 ? 1 : 0);
            const int nh = (int)gen_hist.size();
            if (nh >= unstable_win) {
                int with_cplx = 0;
                for (int t = nh - unstable_win; t < nh; ++t) with_cplx += cplx_hist[t];
                const double then = gen_hist[nh - unstable_win];
                const double best = *std::min_element(gen_hist.end() - unstable_win, gen_hist.end());
                if (2 * with_cplx >= unstable_win && best > 0.1 * then) {
                    rc_final = PPRPA_ERR_UNSTABLE;
                    break;
                }
            }
        }
        if (stage == 1 || stage == 3) {
            ++stage1_iters;
            best_hist.push_back(rmax);
            bool stalled = false;
            if (best_hist.size() >= 4) {
                const double prev = best_hist[best_hist.size() - 4];
                stalled = rmax > 0.5 * prev;
            }
            if (rmax <= tol1 || stalled || stage1_iters >= o->max_iter / 2) {
                stage = 2;
                PP_TRY(collapse(nk_avail, m, true));
                m = nk_avail;
                continue;
            }
        }
        if (todo.empty() && ntg == nroots) {
            rc_final = PPRPA_OK;
            break;
        }
        if (todo.empty()) {
            // every current target converged but the subspace has too few real roots:
            // expand along all targets
            for (int j = 0; j < ntg; ++j) todo.push_back(j);
        }
        if (it == o->max_iter) break;
        // ---- correction vectors ----
        const int kn = (int)todo.size();
        std::copy(todo.begin(), todo.end(), hs_sel);
        PP_CUDA(cudaMemcpyAsync(sel, hs_sel, sizeof(int) * kn, cudaMemcpyHostToDevice, st));
        PP_TRY(launch_correction(R, D, om, sel, kn, N, nvv, Dn, st, ws));
        if (m + kn > (general ? m_max : m_soft)) {
            PP_TRY(collapse(nk_avail, m, false));
            m = nk_avail;
        }
        // ---- orthogonalise against V (two passes of classical Gram-Schmidt) ----
        PP_TRY(launch_row_norms2(Dn, kn, N, nrm, st));
        PP_CUDA(cudaMemcpyAsync(hs_nb, nrm, sizeof(double) * kn, cudaMemcpyDeviceToHost, st));
        for (int pass = 0; pass < 2; ++pass) {
            PP_TRY(dots(V, N, m, Dn, N, kn, N, H, kn, 1.0, true, st));  // H = V Dn^T (m x kn)
            Dgemm g;  // Dn -= H^T V
            g.M = kn; g.N = N; g.K = m;
            g.A = H; g.lda = kn; g.transA = 1;
            g.B = V; g.ldb = N;
            g.C = Dn; g.ldc = N;
            g.alpha = -1.0; g.beta = 1.0;
            PP_TRY(dgemm(g, st));
        }
        PP_TRY(launch_row_norms2(Dn, kn, N, nrm, st));
        PP_CUDA(cudaMemcpyAsync(hs_na, nrm, sizeof(double) * kn, cudaMemcpyDeviceToHost, st));
        PP_TRY(ctx_sync(c));
        std::vector<int> live;
        for (int t = 0; t < kn; ++t)
            if (hs_na[t] > 1e-20 * std::max(hs_nb[t], 1e-300)) live.push_back(t);
        if (live.empty()) break;  // stagnation: no new directions
        // compact live rows into Dn2 (one gather; the device row list reuses sel, whose last
        // reader, the correction kernel, precedes it on the stream)
        int kl = (int)live.size();
        std::copy(live.begin(), live.end(), hs_live);
        PP_CUDA(cudaMemcpyAsync(sel, hs_live, sizeof(int) * kl, cudaMemcpyHostToDevice, st));
        PP_TRY(launch_gather_rows(Dn2, Dn, sel, kl, N, st));
        // ---- Cholesky-QR twice among the new vectors ----
        // (the second pass does not depend on the first one's flags: both are read in one wait;
        // the copy of the first pass's flags is queued before the second pass overwrites them)
        for (int pass = 0; pass < 2; ++pass) {
            PP_TRY(dots(Dn2, N, kl, Dn2, N, kl, N, Gm, kl, 1.0, true, st));
            PP_TRY(launch_cholqr_small(Gm, kl, 1e-12, Tm, keep, cwork, st));
            PP_TRY(combine(Tm, kl, kl, kl, Dn2, N, Dn, 1.0, 0.0, st));
            PP_CUDA(cudaMemcpyAsync(Dn2, Dn, sizeof(double) * (size_t)kl * N, cudaMemcpyDeviceToDevice, st));
            PP_CUDA(cudaMemcpyAsync(hs_keep + pass * nbuf, keep, sizeof(int) * kl, cudaMemcpyDeviceToHost, st));
        }
        PP_TRY(ctx_sync(c));
        std::vector<int> hkeep(kl);
        for (int t = 0; t < kl; ++t) hkeep[t] = hs_keep[t] & hs_keep[nbuf + t];
        int added = 0;
        for (int t = 0; t < kl; ++t)
            if (hkeep[t]) hs_kept[added++] = t;
        if (added == 0) break;
        PP_CUDA(cudaMemcpyAsync(sel, hs_kept, sizeof(int) * added, cudaMemcpyHostToDevice, st));
        PP_TRY(launch_gather_rows(V + (size_t)m * N, Dn2, sel, added, N, st));
        PP_TRY(run_sigma(added, V + (size_t)m * N, Sg + (size_t)m * N));
        PP_TRY(project_block(m, m + added));
        m += added;
    }
    if (ec && rc_final == PPRPA_OK && nroots == npos_blk) {
        // every root of the channel converged: E_c = sum Omega^{+2e} - Tr A (pp), or
        // sum mu - Tr C = -sum Omega^{-2e} - Tr C (hh) (Eq. correlation_energy), summed in FP64
        // on the device from the Ritz values (om, the targets first) and the diagonal
        double* dec;
        PP_TRY(ws_get(c, "dv_ec", sizeof(double), (void**)&dec));
        if (hh) PP_TRY(launch_ec_sum(om, nroots, D + nvv, noo, dec, st));
        else PP_TRY(launch_ec_sum(om, nroots, D, nvv, dec, st));
        PP_CUDA(cudaMemcpyAsync(ec, dec, sizeof(double), cudaMemcpyDeviceToHost, st));
        PP_TRY(ctx_sync(c));
    }
    if (hh)
        for (int j = 0; j < nroots; ++j) h_om[j] = -h_om[j];  // omega of the removal roots
    PP_TRY(write_outputs(c, pt, nroots, Zr, h_om.data(), omega, X, Y));
    c->last_all_roots = rc_final == PPRPA_OK && nroots == npos_blk;
    c->last_channel = o->channel;
    t_all.stop();
    if (info) {
        info->iters = std::min(it, o->max_iter);
        info->iters_stage1 = stage1_iters;
        info->converged = rc_final == PPRPA_OK;
        info->mu = general ? 0.0 : mu_prev;
        info->t_sigma_ms = t_sig.total_ms;
        info->t_total_ms = t_all.total_ms;
    }
    c->last_mult = o->mult;
    if (rc_final == PPRPA_ERR_UNSTABLE)
        return set_error(PPRPA_ERR_UNSTABLE,
                         "Davidson: complex Ritz pairs among the lowest roots persist and the residual "
                         "stagnates (no definite shift); outputs hold the last iterate");
    if (rc_final != PPRPA_OK) return set_error(PPRPA_ERR_NOCONV, "Davidson: max_iter reached");
    return PPRPA_OK;
}

}  // namespace pprpa

using namespace pprpa;

extern "C" int pprpa_solve(pprpa_ctx* c, const pprpa_options* o, double* omega, double* X, double* Y,
                           double* ec, pprpa_info* info) {
    return solve_checked(c, o, omega, X, Y, ec, info, nullptr);
}

int pprpa::solve_checked(pprpa_ctx* c, const pprpa_options* o, double* omega, double* X, double* Y,
                         double* ec, pprpa_info* info, SigmaHook* hook) {
    if (!c || !o) return set_error(PPRPA_ERR_ARG, "solve: null argument");
    PP_CUDA(cudaSetDevice(c->device));
    if (!c->have_L) return set_error(PPRPA_ERR_STATE, "solve: integrals not set");
    if (o->mult != 1 && o->mult != 3 && o->mult != PPRPA_AB)
        return set_error(PPRPA_ERR_ARG, "solve: mult must be 1, 3 or PPRPA_AB");
    if (o->mult == PPRPA_AB && o->method == PPRPA_METHOD_DAVIDSON && o->precision != PPRPA_PREC_FP64)
        return set_error(PPRPA_ERR_UNSUPPORTED, "solve: the alpha-beta subspace runs in FP64 only");
    if (o->channel != PPRPA_CHANNEL_PP && o->channel != PPRPA_CHANNEL_HH)
        return set_error(PPRPA_ERR_ARG, "solve: channel must be PPRPA_CHANNEL_PP or PPRPA_CHANNEL_HH");
    if (o->method != PPRPA_METHOD_FULL && o->method != PPRPA_METHOD_DAVIDSON)
        return set_error(PPRPA_ERR_ARG, "solve: unknown method");
    if (o->precision != PPRPA_PREC_FP64 && o->precision != PPRPA_PREC_BF16 &&
        o->precision != PPRPA_PREC_FP8)
        return set_error(PPRPA_ERR_ARG, "solve: unknown precision");
    PairTable* pt;
    PP_TRY(ensure_pairs(c, o->mult, &pt));
    const int nmax = o->channel == PPRPA_CHANNEL_HH ? pt->noo : pt->nvv;
    if (o->nroots < 1 || o->nroots > nmax)
        return set_error(PPRPA_ERR_ARG, "solve: nroots out of range (1..nvv for pp, 1..noo for hh)");
    if (info) std::memset(info, 0, sizeof(*info));
    if (o->method == PPRPA_METHOD_FULL) return solve_full(c, o, pt, omega, X, Y, ec, info);
    if (!(o->conv_tol > 0.0) || o->max_iter < 1) return set_error(PPRPA_ERR_ARG, "solve: bad tolerance / max_iter");
    if (ec) *ec = NAN;
    return solve_davidson(c, o, pt, omega, X, Y, o->want_ec ? ec : nullptr, info, hook);
}

extern "C" int pprpa_build_matrix(pprpa_ctx* c, int mult, double* Mout, int where) {
    if (!c || !Mout) return set_error(PPRPA_ERR_ARG, "build_matrix: null argument");
    PP_CUDA(cudaSetDevice(c->device));
    if (!c->have_L) return set_error(PPRPA_ERR_STATE, "build_matrix: integrals not set");
    PairTable* pt;
    PP_TRY(ensure_pairs(c, mult, &pt));
    const int64_t n2 = (int64_t)c->n() * c->n();
    const size_t mbytes = sizeof(double) * (size_t)pt->N * pt->N;
    double *eri, *M;
    if (where == PPRPA_DEVICE) M = Mout;
    else PP_TRY(ws_get(c, "bm_M", mbytes, (void**)&M));
    if (mult == PPRPA_AB) {
        PP_TRY(build_ab(c, pt, M));
    } else {
        PP_TRY(ws_get(c, "bm_eri", sizeof(double) * n2 * n2, (void**)&eri));
        PP_TRY(build_explicit(c, pt, mult, eri, M));
    }
    if (where != PPRPA_DEVICE)
        PP_CUDA(cudaMemcpyAsync(Mout, M, mbytes, cudaMemcpyDeviceToHost, c->stream));
    PP_TRY(ctx_sync(c));
    return PPRPA_OK;
}
