// pprpa_analyze: the analysis outputs of one root of the last solve.
//
// Sec. "Natural Transition Orbital": with the addition (removal) eigenvector viewed as the
// upper-triangular matrix X (nv x nv) or Y (no x no) over the pair list, the NTOs are its
// singular value decomposition X = C^p1 sqrt(lambda^p) C^p2^T (Eq. nto_pp, nto_hh for Y).
// They are formed here from the symmetric eigenproblem X X^T = C^p1 lambda^p C^p1^T (one-CTA
// Jacobi), weights descending, with C^p2 = X^T C^p1 / sqrt(lambda^p).
// Sec. "Density Matrix": D^2e has the virtual block X X^T + X^T X and the occupied block
// -(Y Y^T + Y^T Y), zero occupied-virtual blocks.
#include "ctx.h"

namespace pprpa {
namespace {

// z (one root, pair order: virtual pairs then occupied pairs) -> triangular X and Y (zeroed
// by the caller).
__global__ void triangular_kernel(const double* __restrict__ z, int N, int nvv, const int* __restrict__ pp,
                                  const int* __restrict__ pq, int no, int nv, double* __restrict__ X,
                                  double* __restrict__ Y) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        if (I < nvv) X[(int64_t)(pp[I] - no) * nv + (pq[I] - no)] = z[I];
        else Y[(int64_t)pp[I] * no + pq[I]] = z[I];
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

// C2[:, k] = (X^T C1)[:, k] / sqrt(lam_k), or zero when lam_k is negligible.
__global__ void nto_scale_kernel(double* __restrict__ C2, const double* __restrict__ lam, int m) {
    const double lmax = lam[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
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

// NTOs of one triangular matrix T (m x m, device): lam[m], C1 and C2 [m][m] (device).
int ntos_of(pprpa_ctx* c, const double* T, int m, double* lam, double* C1, double* C2, double* H,
            double* U, double* work, int* iwork) {
    if (m == 0) return PPRPA_OK;
    cudaStream_t st = c->stream;
    Dgemm g;  // H = T T^T
    g.M = m; g.N = m; g.K = m;
    g.A = T; g.lda = m;
    g.B = T; g.ldb = m; g.transB = 1;
    g.C = H; g.ldc = m;
    PP_TRY(dgemm(g, st));
    PP_TRY(launch_sym_eig(H, U, m, 1, (int64_t)m * m, work, iwork, st));
    nto_order_kernel<<<1, 1024, 0, st>>>(H, U, m, lam, C1);
    PP_CHECK_LAUNCH();
    Dgemm g2;  // C2 = T^T C1
    g2.M = m; g2.N = m; g2.K = m;
    g2.A = T; g2.lda = m; g2.transA = 1;
    g2.B = C1; g2.ldb = m;
    g2.C = C2; g2.ldc = m;
    PP_TRY(dgemm(g2, st));
    nto_scale_kernel<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)m * m, 256), 1024), 256, 0, st>>>(C2, lam, m);
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
    if (c->last_mult == PPRPA_AB)
        return set_error(PPRPA_ERR_UNSUPPORTED, "analyze: the alpha-beta subspace is not built here");
    PairTable* pt;
    PP_TRY(ensure_pairs(c, c->last_mult, &pt));
    const int no = c->no, nv = c->nv, n = c->n();
    const bool want_p = lam_p || Cp1 || Cp2, want_h = lam_h || Ch1 || Ch2;
    if ((want_p && nv > 1024) || (want_h && no > 1024))
        return set_error(PPRPA_ERR_ARG, "analyze: NTOs are limited to 1024 orbitals per block");
    cudaStream_t st = c->stream;
    const double* z = c->d_lastZ + (size_t)root * pt->N;
    const int mmax = std::max(no, nv);
    const size_t mm = (size_t)mmax * mmax;
    double *X, *Y, *D, *H, *U, *lam, *C1, *C2, *work;
    int* iwork;
    PP_TRY(ws_get(c, "an_X", sizeof(double) * std::max<size_t>(1, (size_t)nv * nv), (void**)&X));
    PP_TRY(ws_get(c, "an_Y", sizeof(double) * std::max<size_t>(1, (size_t)no * no), (void**)&Y));
    PP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * (size_t)nv * nv, st));
    PP_CUDA(cudaMemsetAsync(Y, 0, sizeof(double) * (size_t)no * no, st));
    triangular_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(pt->N, 256), 1024)), 256, 0, st>>>(
        z, pt->N, pt->nvv, pt->d_pp, pt->d_pq, no, nv, X, Y);
    PP_CHECK_LAUNCH();
    if (D2e) {
        PP_TRY(ws_get(c, "an_D", sizeof(double) * (size_t)n * n, (void**)&D));
        PP_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n * n, st));
        for (int blk = 0; blk < 2; ++blk) {  // virtual block X X^T + X^T X, occupied -(Y Y^T + Y^T Y)
            const int m = blk == 0 ? nv : no, off = blk == 0 ? no : 0;
            if (m == 0) continue;
            const double* T = blk == 0 ? X : Y;
            const double a = blk == 0 ? 1.0 : -1.0;
            for (int t = 0; t < 2; ++t) {
                Dgemm g;
                g.M = m; g.N = m; g.K = m;
                g.A = T; g.lda = m; g.transA = t;
                g.B = T; g.ldb = m; g.transB = 1 - t;
                g.C = D + (size_t)off * n + off; g.ldc = n;
                g.alpha = a;
                g.beta = t == 0 ? 0.0 : 1.0;
                PP_TRY(dgemm(g, st));
            }
        }
        PP_TRY(to_caller(c, D2e, D, (size_t)n * n, where));
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
            const int m = blk == 0 ? nv : no;
            if (!want || m == 0) continue;
            PP_TRY(ntos_of(c, blk == 0 ? X : Y, m, lam, C1, C2, H, U, work, iwork));
            PP_TRY(to_caller(c, blk == 0 ? lam_p : lam_h, lam, m, where));
            PP_TRY(to_caller(c, blk == 0 ? Cp1 : Ch1, C1, (size_t)m * m, where));
            PP_TRY(to_caller(c, blk == 0 ? Cp2 : Ch2, C2, (size_t)m * m, where));
            PP_CUDA(cudaStreamSynchronize(st));  // the buffers are reused by the next block
        }
    }
    PP_CUDA(cudaStreamSynchronize(st));
    return PPRPA_OK;
}
