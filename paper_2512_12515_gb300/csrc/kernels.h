// Internal launchers of the ppRPA GB300 library (not part of the C ABI).
#pragma once
#include "common.cuh"

namespace pprpa {

// ---------------------------------------------------------------------------
// FP64 GEMM:  C[i1,i2] = alpha * sum_r op(A[i1,i2,r]) * op(B[i1,i2,r]) + beta * C[i1,i2]
// Row-major.  A(m,k) = transA ? A[k*lda + m] : A[m*lda + k];
//             B(k,n) = transB ? B[n*ldb + k] : B[k*ldb + n].
// Operand pointer for batch (i1, i2) and reduction index r:
//   base + i1*s1 + i2*s2 + r*sr.
// splitk > 1 divides K over extra blocks that atomically add alpha*partial
// into C; the caller must have applied beta (e.g. zeroed C) beforehand.
struct Dgemm {
    int M = 0, N = 0, K = 0;
    const double* A = nullptr;
    int64_t lda = 0, sA1 = 0, sA2 = 0, sAr = 0;
    int transA = 0;
    const double* B = nullptr;
    int64_t ldb = 0, sB1 = 0, sB2 = 0, sBr = 0;
    int transB = 0;
    double* C = nullptr;
    int64_t ldc = 0, sC1 = 0, sC2 = 0;
    int nb1 = 1, nb2 = 1, nr = 1;
    double alpha = 1.0, beta = 0.0;
    int splitk = 1;
    int rsplit = 1;  // set by dgemm(): CTAs sharing the reduction over r (atomic accumulation)
};
int dgemm(const Dgemm& g, cudaStream_t st);
// True when dgemm() gives g to the small-product kernels (one unbatched small product).
bool dgemm_small(const Dgemm& g);
// Picks a split-K factor for a GEMM whose output has few tiles.
int auto_splitk(int M, int N, int K, int batches);

// ---------------------------------------------------------------------------
// Elementwise / reduction kernels (FP64 unless noted).
// X[P][s][t] *= w[s] w[t] over naux slices of n x n.
int launch_scale_slots(double* X, int naux, int n, const double* w, cudaStream_t st);
// dst[m][orb[s]] += src[m][s]: dst nbasis x nmo, src nbasis x n.
int launch_scatter_add_cols(double* dst, int nmo, const double* src, int nbasis, int n, const int* orb,
                            cudaStream_t st);
int launch_extract_active(const double* Lfull, int naux, int nmo, const int* orb, int n,
                          double* Lact, cudaStream_t st);
int launch_diag(const double* L, int naux, int n, const double* eps, const int* pp,
                const int* pq, int nvv, int N, int mult, double* D, double* work,
                cudaStream_t st);
int launch_unpack_f64(const double* z, int k, int N, const int* pp, const int* pq, int n,
                      int mult, double* Zt, cudaStream_t st);
int launch_pack_f64(const double* O, const double* z, int k, int N, int nvv, const int* pp,
                    const int* pq, int n, const double* eps, int mult, double* sigma,
                    cudaStream_t st);

// Padded BF16 layout of L used by the tensor-core sigma:
//   rows/cols: occupied p -> p, virtual a -> no_p + a; n_pad = no_p + nv_p.
struct PadMap {
    int no = 0, nv = 0, no_p = 0, nv_p = 0, n_pad = 0;
    __host__ __device__ int map(int p) const { return p < no ? p : no_p + (p - no); }
};
PadMap make_padmap(int no, int nv);
int launch_quantize_bf16(const double* L, int naux, int n, PadMap pm, __nv_bfloat16* hi,
                         __nv_bfloat16* lo, cudaStream_t st);
// z (k x N) -> B operands of the first sandwich stage, bf16 hi[/lo]:
//   Xs[j][c][d] = Zt_j[no_p+d][no_p+c] (virtual block, c < nv_p rows per vector, ld = ldx),
//   Ys[j][c][d] = Zt_j[d][c]            (occupied block, c < no_p rows per vector, ld = ldy).
int launch_unpack_bf16(const double* z, int k, int N, int nvv, const int* pp, const int* pq,
                       PadMap pm, int mult, __nv_bfloat16* xs_hi, __nv_bfloat16* xs_lo,
                       int ldx, __nv_bfloat16* ys_hi, __nv_bfloat16* ys_lo, int ldy,
                       cudaStream_t st);
int launch_quantize_fp8(const double* L, int naux, int n, PadMap pm, int ncol8, int c_off8,
                        void* L8, float* scale, cudaStream_t st);
int launch_unpack_fp8(const double* z, int k, int N, int nvv, const int* pp, const int* pq,
                      PadMap pm, int mult, float* zscale, void* xs, int ldx, void* ys, int ldy,
                      cudaStream_t st);
int launch_pack_f32(const float* O, const double* z, int k, int N, int nvv, const int* pp,
                    const int* pq, PadMap pm, const double* eps, int mult, double* sigma,
                    cudaStream_t st);

// Davidson vector kernels.
int launch_residual(const double* SZ, const double* Zr, const double* omega, int k, int N,
                    int nvv, double* R, double* norms2, cudaStream_t st, double wsign = 1.0);
int launch_correction(const double* R, const double* D, const double* omega, const int* sel,
                      int kn, int N, int nvv, double* out, cudaStream_t st, double wsign = 1.0);
// out[j] = ||X_j||^2 for the k rows of X (k x N); out need not be zeroed
int launch_row_norms2(const double* X, int k, int N, double* out, cudaStream_t st);
// dst row t = src row idx[t] (rows of N doubles, idx on the device), t < n
int launch_gather_rows(double* dst, const double* src, const int* idx, int n, int64_t N, cudaStream_t st);
int launch_scatter_unit(double* V, int ld, const int* idx, int k, cudaStream_t st);
int launch_build_matrix(const double* eri, int n, const int* pp, const int* pq, int N,
                        int nvv, const double* eps, int mult, double* M, cudaStream_t st);
int launch_ec_sum(const double* omega, int nw, const double* D, int nvv, double* out,
                  cudaStream_t st);
// W = diag(wsign I_nvv, -wsign I_noo); wsign = -1 gives the metric of the removal channel
int launch_metric_matrix(double* W, int N, int nvv, cudaStream_t st, double wsign = 1.0);
// Subtracts the derivative of the A-block (blk = 0) or C-block (blk = 1) trace from dL
// (naux slices) and deps; either may be null.
int launch_trace_block_grad(const double* L, int naux, int n, int no, int mult, int blk,
                            double* dL, double* deps, cudaStream_t st);
// X[r][:] *= f[r] (f on the device) for k rows of length len.
int launch_scale_rows(double* X, int k, int64_t len, const double* f, cudaStream_t st);
int launch_grad_eps(const double* z, int N, int nvv, const int* pp, const int* pq, int n,
                    double s, double* deps, cudaStream_t st);

// ---------------------------------------------------------------------------
// One-CTA dense FP64 linear algebra (Rayleigh-Ritz, block orthonormalisation).
struct RRArgs {
    const double* G = nullptr;   // m x m (ld): V^T M V restricted to virtual pairs (or all of M)
    const double* Go = nullptr;  // optional m x m (ld): occupied-pair part; G + Go is symmetrised
    const double* S = nullptr;  // m x m (ld), upper block valid
    int ld = 0, m = 0;
    const double* mus = nullptr;  // device: candidate shifts
    int nmu = 0;
    int nwant = 0;    // targets (lowest positive-norm roots)
    int nkeep = 0;    // Ritz vectors returned (>= nwant)
    double* work = nullptr;  // >= 4*m*m + 8*m doubles
    int eig = 0;             // set by the launcher: 0 Jacobi (fused update), 1 Jacobi, 2 Householder + QR
    int pad = 1;             // set by the launcher: odd leading dimension of H and U in shared memory
    int prof = 0;            // set by the launcher: print the phase clocks of each call (PPRPA_RR_PROF)
    double tol32 = 1e-10;    // set by the launcher: FP32 stage stops at off^2 <= tol32 total^2
    double* omega = nullptr;   // nkeep
    double* coef = nullptr;    // nkeep x m (row j = coefficients of Ritz vector j)
    double* info = nullptr;    // [0]=status, [1]=mu used, [2]=npos, [3]=omega_min_pp,
                               // [4]=omega_max_hh, [5]=sweeps
};
int launch_rayleigh_ritz(const RRArgs& a, cudaStream_t st);

// General Rayleigh-Ritz for an indefinite pencil: G c = theta S c with G = Gv + Go = V^T M V,
// solved as X = S^-1 G; keeps the lowest real roots of positive norm c^T S c, normalised to
// c^T S c = 1.
struct RRGenArgs {
    const double* Gv = nullptr;  // m x m (ld): rows V (virtual-pair part) . M V
    const double* Go = nullptr;  // m x m (ld): occupied-pair part
    const double* S = nullptr;   // m x m (ld), upper triangle valid
    int ld = 0, m = 0;
    int nwant = 0, nkeep = 0;
    double imag_tol = 1e-9;   // |Im theta| <= imag_tol * max|theta| counts as real
    double norm_tol = 1e-8;   // |c^T S c| below this (for |c| = 1) is not classified
    double* work = nullptr;   // >= 3*m*m + m doubles
    double* omega = nullptr;  // nkeep
    double* coef = nullptr;   // nkeep x m
    double* info = nullptr;   // [0] status, [2] kept, [3] lowest kept, [4] highest negative-norm
                              // seen, [5] real count, [6] lowest complex real part, [7] max |Im|
};
int launch_rr_general(const RRGenArgs& a, cudaStream_t st);

// Block orthonormalisation of k rows: given Gram Gm (k x k), returns T (k x k) with
// T * X orthonormal rows; rows whose residual pivot is below tol are zeroed and flagged
// keep[j] = 0.
// Symmetric eigendecomposition (one CTA per m x m matrix, m <= 1024): eigenvalues on the
// diagonal of H, eigenvectors as the columns of U.  work: batch*8192 doubles, iwork: batch*1024.
int launch_sym_eig(double* H, double* U, int m, int batch, int64_t stride, double* work, int* iwork,
                   cudaStream_t st);
int launch_cholqr_small(const double* Gm, int k, double tol, double* T, int* keep,
                        double* work, cudaStream_t st);

}  // namespace pprpa
