// pprpa_analyze: the analysis outputs of one root of the last solve.
//
// Sec. "Natural Transition Orbital": with the addition (removal) eigenvector viewed as the
// upper-triangular matrix X (nv x nv) or Y (no x no) over the pair list, the NTOs are its
// singular value decomposition X = C^p1 sqrt(lambda^p) C^p2^T (Eq. nto_pp, nto_hh for Y).
// They are formed here from the symmetric eigenproblem X X^T = C^p1 lambda^p C^p1^T (one-CTA
// Jacobi), weights descending, with C^p2 = X^T C^p1 / sqrt(lambda^p).
// Sec. "Density Matrix": D^2e has the virtual block X X^T + X^T X and the occupied block
// -(Y Y^T + Y^T Y), zero occupied-virtual blocks.
// Alpha-beta roots: X (alpha virtuals x beta virtuals) and Y (alpha x beta occupied) are full
// rectangles; the two orbital slots of a pair are told apart by spin, so D^2e is
// diag(D^alpha, D^beta) with D^alpha = (X X^T, -Y Y^T) and D^beta = (X^T X, -Y^T Y), and
// C^p2 = X^T C^p1 / sqrt(lambda^p) runs over beta virtuals.
#include "ctx.h"

namespace pprpa {
namespace {

// z (one root, pair order: virtual pairs then occupied pairs) -> X (nva x nvb) and Y
// (noa x nob), zeroed by the caller: the upper triangles of square matrices for a restricted
// multiplicity (nva = nvb, noa = nob), full rectangles for the alpha-beta subspace.
__global__ void triangular_kernel(const double* __restrict__ z, int N, int nvv, const int* __restrict__ pp,
                                  const int* __restrict__ pq, int noa, int nob, int nvb,
                                  double* __restrict__ X, double* __restrict__ Y) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        if (I < nvv) X[(int64_t)(pp[I] - noa) * nvb + (pq[I] - nob)] = z[I];
        else Y[(int64_t)pp[I] * nob + pq[I]] = z[I];
    }
}

// Eigenpairs of X X^T (eigenvalues on the diagonal of H, vectors in the columns of U) ->
// weights descending (clamped at 0) and C1 with the largest-magnitude entry of each column
// positive.  One CTA; thread i handles eigenpair i.
__global__ void nto_order_kernel(const double* __restrict__ H, const double* __restrict__ U, int m,
                                 double* __restrict__ lam, double* __restrict__ C1) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double li = H[(int64_t)i * m + i];
        int rank = 0;
        for (int j = 0; j < m; ++j) {
            const double lj = H[(int64_t)j * m + j];
            if (lj > li || (lj == li && j < i)) ++rank;
        }
        int arg = 0;
        double best = -1.0;
        for (int r = 0; r < m; ++r) {
            const double a = fabs(U[(int64_t)r * m + i]);
            if (a > best) { best = a; arg = r; }
        }
        const double sg = U[(int64_t)arg * m + i] < 0.0 ? -1.0 : 1.0;
        lam[rank] = li > 0.0 ? li : 0.0;
        for (int r = 0; r < m; ++r) C1[(int64_t)r * m + rank] = sg * U[(int64_t)r * m + i];
    }
}

// C2[:, k] = (T^T C1)[:, k] / sqrt(lam_k), or zero when lam_k is negligible (C2: m2 x m).
__global__ void nto_scale_kernel(double* __restrict__ C2, const double* __restrict__ lam, int m, int m2) {
    const double lmax = lam[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m2; t += gridDim.x * blockDim.x) {
        const int k = t % m;
        const double l = lam[k];
        C2[t] = (l > 1e-28 * lmax && l > 0.0) ? C2[t] / sqrt(l) : 0.0;
    }
}

int to_caller(pprpa_ctx* c, double* dst, const double* src, size_t count, int where) {
    if (!dst || count == 0) return PPRPA_OK;
    PP_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                            where == PPRPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    return PPRPA_OK;
}

// NTOs of one block T (m x m2, device): lam[m], C1 [m][m] and C2 [m2][m] (device).
int ntos_of(pprpa_ctx* c, const double* T, int m, int m2, double* lam, double* C1, double* C2, double* H,
            double* U, double* work, int* iwork) {
    if (m == 0) return PPRPA_OK;
    cudaStream_t st = c->stream;
    Dgemm g;  // H = T T^T
    g.M = m; g.N = m; g.K = m2;
    g.A = T; g.lda = m2;
    g.B = T; g.ldb = m2; g.transB = 1;
    g.C = H; g.ldc = m;
    PP_TRY(dgemm(g, st));
    PP_TRY(launch_sym_eig(H, U, m, 1, (int64_t)m * m, work, iwork, st));
    nto_order_kernel<<<1, 1024, 0, st>>>(H, U, m, lam, C1);
    PP_CHECK_LAUNCH();
    if (m2 == 0) return PPRPA_OK;
    Dgemm g2;  // C2 = T^T C1
    g2.M = m2; g2.N = m; g2.K = m;
    g2.A = T; g2.lda = m2; g2.transA = 1;
    g2.B = C1; g2.ldb = m;
    g2.C = C2; g2.ldc = m;
    PP_TRY(dgemm(g2, st));
    nto_scale_kernel<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)m * m2, 256), 1024), 256, 0, st>>>(C2, lam, m, m2);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace
}  // namespace pprpa

using namespace pprpa;

extern "C" int pprpa_analyze(pprpa_ctx* c, int root, double* D2e, double* lam_p, double* lam_h,
                             double* Cp1, double* Cp2, double* Ch1, double* Ch2, int where) {
    if (!c) return set_error(PPRPA_ERR_ARG, "analyze: null context");
    PP_CUDA(cudaSetDevice(c->device));
    if (where != PPRPA_HOST && where != PPRPA_DEVICE) return set_error(PPRPA_ERR_ARG, "analyze: bad `where`");
    if (c->last_nroots == 0 || !c->d_lastZ) return set_error(PPRPA_ERR_STATE, "analyze: no solve to analyse");
    if (root < 0 || root >= c->last_nroots) return set_error(PPRPA_ERR_ARG, "analyze: root index out of range");
    const bool ab = c->last_mult == PPRPA_AB;
    PairTable* pt;
    if (ab) PP_TRY(ensure_pairs_ab(c, &pt));
    else PP_TRY(ensure_pairs(c, c->last_mult, &pt));
    if (pt->N != c->last_N) return set_error(PPRPA_ERR_STATE, "analyze: the pair space changed since the solve");
    // X is nva x nvb and Y noa x nob: square triangles (restricted) or rectangles (alpha-beta)
    const int noa = c->no, nva = c->nv, nob = ab ? c->nob : c->no, nvb = ab ? c->nvb : c->nv;
    const int na = c->n(), nd = ab ? na + c->nb() : na;  // D2e is nd x nd
    const bool want_p = lam_p || Cp1 || Cp2, want_h = lam_h || Ch1 || Ch2;
    if ((want_p && nva > 1024) || (want_h && noa > 1024))
        return set_error(PPRPA_ERR_ARG, "analyze: NTOs are limited to 1024 orbitals per block");
    cudaStream_t st = c->stream;
    const double* z = c->d_lastZ + (size_t)root * pt->N;
    const int mmax = std::max(std::max(noa, nva), std::max(nob, nvb));
    const size_t mm = (size_t)mmax * mmax;
    double *X, *Y, *D, *H, *U, *lam, *C1, *C2, *work;
    int* iwork;
    PP_TRY(ws_get(c, "an_X", sizeof(double) * std::max<size_t>(1, (size_t)nva * nvb), (void**)&X));
    PP_TRY(ws_get(c, "an_Y", sizeof(double) * std::max<size_t>(1, (size_t)noa * nob), (void**)&Y));
    PP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)nva * nvb, st));
    PP_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)noa * nob, st));
    triangular_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pt->N, 256), 1024)), 256, 0, st>>>(
        z, pt->N, pt->nvv, pt->d_pp, pt->d_pq, noa, nob, nvb, X, Y);
    PP_CHECK_LAUNCH();
    if (D2e) {
        PP_TRY(ws_get(c, "an_D", sizeof(double) * (size_t)nd * nd, (void**)&D));
        PP_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)nd * nd, st));
        // restricted: virtual block X X^T + X^T X, occupied -(Y Y^T + Y^T Y);
        // alpha-beta: D^alpha = (X X^T, -Y Y^T), D^beta = (X^T X, -Y^T Y) on the diagonal of D2e
        for (int blk = 0; blk < 2; ++blk) {
            const double* T = blk == 0 ? X : Y;
            const int m1 = blk == 0 ? nva : noa, m2 = blk == 0 ? nvb : nob;
            const double a = blk == 0 ? 1.0 : -1.0;
            for (int t = 0; t < 2; ++t) {  // t = 0: T T^T (alpha side), t = 1: T^T T (beta side)
                const int m = t == 0 ? m1 : m2, k = t == 0 ? m2 : m1;
                if (m == 0) continue;
                const int off = ab ? (t == 0 ? (blk == 0 ? noa : 0) : na + (blk == 0 ? nob : 0)) : (blk == 0 ? noa : 0);
                Dgemm g;
                g.M = m; g.N = m; g.K = k;
                g.A = T; g.lda = m2; g.transA = t;
                g.B = T; g.ldb = m2; g.transB = 1 - t;
                g.C = D + (size_t)off * nd + off; g.ldc = nd;
                g.alpha = a;
                g.beta = (!ab && t == 1) ? 1.0 : 0.0;
                PP_TRY(dgemm(g, st));
            }
        }
        PP_TRY(to_caller(c, D2e, D, (size_t)nd * nd, where));
    }
    if (want_p || want_h) {
        PP_TRY(ws_get(c, "an_H", sizeof(double) * mm, (void**)&H));
        PP_TRY(ws_get(c, "an_U", sizeof(double) * mm, (void**)&U));
        PP_TRY(ws_get(c, "an_C1", sizeof(double) * mm, (void**)&C1));
        PP_TRY(ws_get(c, "an_C2", sizeof(double) * mm, (void**)&C2));
        PP_TRY(ws_get(c, "an_lam", sizeof(double) * mmax, (void**)&lam));
        PP_TRY(ws_get(c, "an_work", sizeof(double) * 8192, (void**)&work));
        PP_TRY(ws_get(c, "an_iwork", sizeof(int) * 1024, (void**)&iwork));
        for (int blk = 0; blk < 2; ++blk) {
            const bool want = blk == 0 ? want_p : want_h;
            const int m = blk == 0 ? nva : noa, m2 = blk == 0 ? nvb : nob;
            if (!want || m == 0) continue;
            PP_TRY(ntos_of(c, blk == 0 ? X : Y, m, m2, lam, C1, C2, H, U, work, iwork));
            PP_TRY(to_caller(c, blk == 0 ? lam_p : lam_h, lam, m, where));
            PP_TRY(to_caller(c, blk == 0 ? Cp1 : Ch1, C1, (size_t)m * m, where));
            PP_TRY(to_caller(c, blk == 0 ? Cp2 : Ch2, C2, (size_t)m2 * m, where));
            PP_CUDA(cudaStreamSynchronize(st));  // the buffers are reused by the next block
        }
    }
    PP_CUDA(cudaStreamSynchronize(st));
    return PPRPA_OK;
}
