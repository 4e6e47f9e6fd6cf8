// General (non-symmetric) Rayleigh-Ritz for the Davidson subspace, one CTA, FP64.
//
// When no shift makes the projected pencil (G, S) definite (the ppRPA problem
// is unstable: two-electron addition and removal roots interleave or form
// complex pairs), the subspace problem G c = theta S c (G = V^T M V,
// S = V^T W V, V orthonormal) is solved as a standard eigenproblem of
// X = S^-1 G:
//   1. LU factorisation of S with partial pivoting, X = S^-1 G.
//   2. Householder reduction X = Q Hh Q^T (Hh upper Hessenberg), Q kept.
//   3. Eigenvalues of Hh by the Francis double-shift QR iteration
//      (implicit bulge chase with 3x3 reflectors, deflation on small
//      subdiagonals, exceptional shifts), following the textbook
//      formulation (Golub & Van Loan, "Matrix Computations", Sec. 7.5).  The
//      exceptional shift is the published one of the Handbook's hqr procedure
//      (Martin, Peters & Wilkinson, "The QR algorithm for real Hessenberg
//      matrices", Numer. Math. 14 (1970), Wilkinson & Reinsch, Handbook for
//      Automatic Computation II/14; EISPACK HQR).
//   4. Real eigenvalues in ascending order; for each, inverse iteration on
//      the Hessenberg form (O(m^2) LU with partial pivoting), c = Q x.
//   5. Roots of positive norm c^T S c (two-electron addition, Eq. xy_norm)
//      are kept, lowest first, normalised to c^T S c = 1.
#include "kernels.h"

namespace pprpa {

constexpr int RG_THREADS = 256;
constexpr int RG_MAX = 128;

__device__ __forceinline__ double dsign(double a, double b) { return b >= 0.0 ? fabs(a) : -fabs(a); }

// Apply the 3-vector Householder reflector I - 2 v v^T / (v^T v) to rows r0..r0+nr-1
// (columns c0..c1) and columns r0..r0+nr-1 (rows q0..q1) of A (ld), warp-parallel.
__device__ void reflect_rows(double* A, int ld, int r0, int nr, const double* v, double beta,
                             int c0, int c1, int lane) {
    for (int j = c0 + lane; j <= c1; j += 32) {
        double s = 0.0;
        for (int t = 0; t < nr; ++t) s += v[t] * A[(r0 + t) * ld + j];
        s *= beta;
        for (int t = 0; t < nr; ++t) A[(r0 + t) * ld + j] -= s * v[t];
    }
}
__device__ void reflect_cols(double* A, int ld, int r0, int nr, const double* v, double beta,
                             int q0, int q1, int lane) {
    for (int i = q0 + lane; i <= q1; i += 32) {
        double s = 0.0;
        for (int t = 0; t < nr; ++t) s += A[i * ld + r0 + t] * v[t];
        s *= beta;
        for (int t = 0; t < nr; ++t) A[i * ld + r0 + t] -= s * v[t];
    }
}

// Eigenvalues of the upper Hessenberg matrix A (n x n, ld), destroyed.  Warp 0 only.
// Returns false if an eigenvalue failed to converge.
__device__ bool francis_eigs(double* A, int ld, int n, double* wr, double* wi, int lane) {
    double anorm = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = (i > 0 ? i - 1 : 0); j < n; ++j) anorm += fabs(A[i * ld + j]);
    if (anorm == 0.0) anorm = 1.0;
    int hi = n - 1;
    int iter = 0;
    double exc = 0.0;  // accumulated exceptional shift
    __shared__ double v[3];
    while (hi >= 0) {
        // deflation: find the start lo of the unreduced block ending at hi
        int lo = hi;
        while (lo > 0) {
            double s = fabs(A[(lo - 1) * ld + lo - 1]) + fabs(A[lo * ld + lo]);
            if (s == 0.0) s = anorm;
            if (fabs(A[lo * ld + lo - 1]) <= 2.2e-16 * s) {
                if (lane == 0) A[lo * ld + lo - 1] = 0.0;
                __syncwarp();
                break;
            }
            --lo;
        }
        if (lo == hi) {  // 1x1 block
            if (lane == 0) { wr[hi] = A[hi * ld + hi] + exc; wi[hi] = 0.0; }
            __syncwarp();
            --hi;
            iter = 0;
            continue;
        }
        if (lo == hi - 1) {  // 2x2 block: eigenvalues from the characteristic quadratic
            if (lane == 0) {
                const double a = A[lo * ld + lo], b = A[lo * ld + hi];
                const double c = A[hi * ld + lo], d = A[hi * ld + hi];
                const double p = 0.5 * (a - d);
                const double disc = p * p + b * c;
                const double mid = 0.5 * (a + d);
                if (disc >= 0.0) {
                    // larger-magnitude root first, the other from the determinant
                    const double r = sqrt(disc);
                    const double l1 = mid + dsign(r, mid);
                    const double l2 = (l1 != 0.0) ? (a * d - b * c) / l1 : mid - dsign(r, mid);
                    wr[lo] = l1 + exc;
                    wr[hi] = l2 + exc;
                    wi[lo] = wi[hi] = 0.0;
                } else {
                    const double r = sqrt(-disc);
                    wr[lo] = wr[hi] = mid + exc;
                    wi[lo] = r;
                    wi[hi] = -r;
                }
            }
            __syncwarp();
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++iter > 60) return false;
        // shifts: eigenvalues of the trailing 2x2 block (sum s, product t), or, every 10
        // iterations without deflation, the exceptional shift of the Handbook's hqr (shift
        // the diagonal by h22, then sum 1.5 w and product w^2 with w the two trailing
        // subdiagonal magnitudes)
        double s, t;
        const double h11 = A[(hi - 1) * ld + hi - 1], h12 = A[(hi - 1) * ld + hi];
        const double h21 = A[hi * ld + hi - 1], h22 = A[hi * ld + hi];
        if (iter % 10 == 0) {
            const double x = h22;
            exc += x;
            if (lane == 0)  // every row not yet deflated carries the accumulated shift
                for (int i = 0; i <= hi; ++i) A[i * ld + i] -= x;
            __syncwarp();
            const double w = fabs(A[hi * ld + hi - 1]) + fabs(A[(hi - 1) * ld + hi - 2]);
            s = 1.5 * w;
            t = w * w;
        } else {
            s = h11 + h22;
            t = h11 * h22 - h12 * h21;
        }
        // first column of (H - s1)(H - s2) restricted to rows lo..lo+2
        const double a00 = A[lo * ld + lo], a01 = A[lo * ld + lo + 1];
        const double a10 = A[(lo + 1) * ld + lo], a11 = A[(lo + 1) * ld + lo + 1];
        const double a21 = A[(lo + 2) * ld + lo + 1];
        double x = a00 * a00 + a01 * a10 - s * a00 + t;
        double y = a10 * (a00 + a11 - s);
        double z = a10 * a21;
        for (int k = lo; k <= hi - 2; ++k) {
            // reflector mapping (x, y, z) to a multiple of e1
            const double nr = sqrt(x * x + y * y + z * z);
            if (nr != 0.0) {
                const double alpha = -dsign(nr, x);
                if (lane == 0) { v[0] = x - alpha; v[1] = y; v[2] = z; }
                __syncwarp();
                const double vtv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                if (vtv > 0.0) {
                    const double beta = 2.0 / vtv;
                    const int c0 = k > lo ? k - 1 : lo;
                    reflect_rows(A, ld, k, 3, v, beta, c0, hi, lane);
                    __syncwarp();
                    const int q1 = min(k + 3, hi);
                    reflect_cols(A, ld, k, 3, v, beta, lo, q1, lane);
                    __syncwarp();
                }
            }
            x = A[(k + 1) * ld + k];
            y = A[(k + 2) * ld + k];
            z = (k < hi - 2) ? A[(k + 3) * ld + k] : 0.0;
        }
        // final 2-vector reflector on rows/cols hi-1, hi
        {
            const double nr = sqrt(x * x + y * y);
            if (nr != 0.0) {
                const double alpha = -dsign(nr, x);
                if (lane == 0) { v[0] = x - alpha; v[1] = y; }
                __syncwarp();
                const double vtv = v[0] * v[0] + v[1] * v[1];
                if (vtv > 0.0) {
                    const double beta = 2.0 / vtv;
                    reflect_rows(A, ld, hi - 1, 2, v, beta, hi - 2, hi, lane);
                    __syncwarp();
                    reflect_cols(A, ld, hi - 1, 2, v, beta, lo, hi, lane);
                    __syncwarp();
                }
            }
        }
        // clean the entries the chase leaves below the subdiagonal
        if (lane == 0)
            for (int i = lo + 2; i <= hi; ++i) {
                A[i * ld + i - 2] = 0.0;
                if (i > lo + 2) A[i * ld + i - 3] = 0.0;
            }
        __syncwarp();
    }
    return true;
}

__global__ void __launch_bounds__(RG_THREADS, 1) rr_general_kernel(RRGenArgs a) {
    extern __shared__ double sm[];
    const int m = a.m, ld = a.ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    double* A = sm;                 // m x m working matrix (Hessenberg, then QR)
    double* vh = sm + m * m;        // Householder vector
    double* wr = vh + m;
    double* wi = wr + m;
    double* xv = wi + m;            // inverse-iteration vector
    double* Q = a.work;             // m x m
    double* Hh = a.work + m * m;    // saved Hessenberg form
    double* LU = a.work + 2 * m * m;
    double* cv = a.work + 3 * m * m;  // m
    __shared__ double red[RG_THREADS / 32 + 2];
    __shared__ int order_sh[RG_MAX];
    __shared__ int nreal_sh, ok_sh;

    // S (symmetric, upper triangle valid) -> LU with partial pivoting in LU; X = S^-1 G
    double gs = 0.0;
    for (int i = 0; i < m; ++i) gs = fmax(gs, fabs(a.Gv[i * ld + i] + a.Go[i * ld + i]));
    const double th_max = 1e3 * (gs + 1.0);  // larger |theta| come from a near-singular S
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        LU[t] = (i <= j) ? a.S[i * ld + j] : a.S[j * ld + i];
        A[t] = 0.5 * (a.Gv[i * ld + j] + a.Go[i * ld + j] + a.Gv[j * ld + i] + a.Go[j * ld + i]);
        Q[t] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (tid == 0) {
            int piv = j;
            double best = fabs(LU[j * m + j]);
            for (int i = j + 1; i < m; ++i)
                if (fabs(LU[i * m + j]) > best) { best = fabs(LU[i * m + j]); piv = i; }
            order_sh[j] = piv;
            if (best == 0.0) LU[piv * m + j] = 1e-300;
        }
        __syncthreads();
        const int piv = order_sh[j];
        if (piv != j) {
            for (int c = tid; c < m; c += nt) {
                double t1 = LU[j * m + c]; LU[j * m + c] = LU[piv * m + c]; LU[piv * m + c] = t1;
                double t2 = A[j * m + c]; A[j * m + c] = A[piv * m + c]; A[piv * m + c] = t2;
            }
        }
        __syncthreads();
        const double d = LU[j * m + j];
        for (int i = j + 1 + tid; i < m; i += nt) LU[i * m + j] /= d;
        __syncthreads();
        const int r = m - j - 1;
        for (int t = tid; t < r * r; t += nt) {
            const int i = j + 1 + t / r, c = j + 1 + t % r;
            LU[i * m + c] -= LU[i * m + j] * LU[j * m + c];
        }
        __syncthreads();
    }
    // solve column by column: A <- U^-1 L^-1 A
    for (int c = tid; c < m; c += nt) {
        for (int i = 1; i < m; ++i) {
            double v = A[i * m + c];
            for (int k = 0; k < i; ++k) v -= LU[i * m + k] * A[k * m + c];
            A[i * m + c] = v;
        }
        for (int i = m - 1; i >= 0; --i) {
            double v = A[i * m + c];
            for (int k = i + 1; k < m; ++k) v -= LU[i * m + k] * A[k * m + c];
            A[i * m + c] = v / LU[i * m + i];
        }
    }
    __syncthreads();
    // 2. Householder reduction to Hessenberg form, accumulating Q (X = Q Hh Q^T)
    for (int k = 0; k + 2 < m; ++k) {
        const int len = m - k - 1;
        if (tid == 0) {
            double nrm = 0.0;
            for (int i = 0; i < len; ++i) nrm += A[(k + 1 + i) * m + k] * A[(k + 1 + i) * m + k];
            nrm = sqrt(nrm);
            const double x0 = A[(k + 1) * m + k];
            const double alpha = -dsign(nrm, x0);
            for (int i = 0; i < len; ++i) vh[i] = A[(k + 1 + i) * m + k];
            vh[0] = x0 - alpha;
            double vtv = 0.0;
            for (int i = 0; i < len; ++i) vtv += vh[i] * vh[i];
            red[0] = (nrm == 0.0 || vtv == 0.0) ? 0.0 : 2.0 / vtv;
        }
        __syncthreads();
        const double beta = red[0];
        if (beta != 0.0) {
            // left: rows k+1.., columns k..m-1
            for (int j = k + tid; j < m; j += nt) {
                double s = 0.0;
                for (int i = 0; i < len; ++i) s += vh[i] * A[(k + 1 + i) * m + j];
                s *= beta;
                for (int i = 0; i < len; ++i) A[(k + 1 + i) * m + j] -= s * vh[i];
            }
            __syncthreads();
            // right: all rows, columns k+1..; and Q <- Q P
            for (int r = tid; r < 2 * m; r += nt) {
                double* M_ = r < m ? A : Q;
                const int i = r < m ? r : r - m;
                double s = 0.0;
                for (int j = 0; j < len; ++j) s += M_[i * m + k + 1 + j] * vh[j];
                s *= beta;
                for (int j = 0; j < len; ++j) M_[i * m + k + 1 + j] -= s * vh[j];
            }
        }
        __syncthreads();
        for (int i = k + 2 + tid; i < m; i += nt) A[i * m + k] = 0.0;
        __syncthreads();
    }
    for (int t = tid; t < m * m; t += nt) Hh[t] = A[t];
    if (tid == 0) ok_sh = 1;
    __syncthreads();
    // 3. eigenvalues (warp 0)
    if (warp == 0) {
        const bool ok = francis_eigs(A, m, m, wr, wi, lane);
        if (lane == 0) ok_sh = ok ? 1 : 0;
    }
    __syncthreads();
    if (!ok_sh) {
        if (tid == 0) a.info[0] = DEV_NOTPD;
        return;
    }
    // scale for the realness test (finite part of the spectrum)
    double sc = 0.0;
    for (int i = 0; i < m; ++i)
        if (fabs(wr[i]) <= th_max) sc = fmax(sc, fabs(wr[i]) + fabs(wi[i]));
    sc = fmax(sc, 1e-300);
    // 3. real eigenvalues in ascending order
    if (tid == 0) {
        int nr = 0;
        for (int i = 0; i < m; ++i)
            if (fabs(wi[i]) <= a.imag_tol * sc && fabs(wr[i]) <= th_max) order_sh[nr++] = i;
        for (int i = 1; i < nr; ++i) {  // insertion sort by real part
            const int v = order_sh[i];
            int j = i - 1;
            while (j >= 0 && wr[order_sh[j]] > wr[v]) { order_sh[j + 1] = order_sh[j]; --j; }
            order_sh[j + 1] = v;
        }
        nreal_sh = nr;
    }
    __syncthreads();
    const int nreal = nreal_sh;
    int found = 0;
    double om_min = 1e300, om_hh = -1e300, lowest_cplx = 1e300, max_im = 0.0;
    for (int i = 0; i < m; ++i)
        if (fabs(wi[i]) > a.imag_tol * sc && fabs(wr[i]) <= th_max) {
            lowest_cplx = fmin(lowest_cplx, wr[i]);
            max_im = fmax(max_im, fabs(wi[i]));
        }
    for (int r = 0; r < nreal && found < a.nkeep; ++r) {
        const double th = wr[order_sh[r]];
        // 4. inverse iteration on (Hh - th') x = x_prev, th' nudged off the eigenvalue
        if (tid == 0) {
            const double thp = th + 1e-12 * sc;
            for (int t = 0; t < m; ++t) xv[t] = 1.0 / sqrt((double)m) * (1.0 + 0.01 * (t % 7));
            for (int sweep = 0; sweep < 3; ++sweep) {
                // LU of the Hessenberg matrix with row pivoting between neighbours
                for (int t = 0; t < m * m; ++t) LU[t] = Hh[t];
                for (int t = 0; t < m; ++t) LU[t * m + t] -= thp;
                for (int j = 0; j < m - 1; ++j) {
                    if (fabs(LU[(j + 1) * m + j]) > fabs(LU[j * m + j])) {
                        for (int c = j; c < m; ++c) {
                            const double tmp = LU[j * m + c];
                            LU[j * m + c] = LU[(j + 1) * m + c];
                            LU[(j + 1) * m + c] = tmp;
                        }
                        const double tx = xv[j];
                        xv[j] = xv[j + 1];
                        xv[j + 1] = tx;
                    }
                    double piv = LU[j * m + j];
                    if (piv == 0.0) piv = LU[j * m + j] = 1e-300;
                    const double f = LU[(j + 1) * m + j] / piv;
                    if (f != 0.0) {
                        for (int c = j; c < m; ++c) LU[(j + 1) * m + c] -= f * LU[j * m + c];
                        xv[j + 1] -= f * xv[j];
                    }
                }
                if (LU[(m - 1) * m + m - 1] == 0.0) LU[(m - 1) * m + m - 1] = 1e-300;
                for (int i = m - 1; i >= 0; --i) {
                    double v = xv[i];
                    for (int c = i + 1; c < m; ++c) v -= LU[i * m + c] * xv[c];
                    xv[i] = v / LU[i * m + i];
                }
                double nrm = 0.0;
                for (int t = 0; t < m; ++t) nrm += xv[t] * xv[t];
                nrm = sqrt(nrm);
                for (int t = 0; t < m; ++t) xv[t] /= nrm;
            }
        }
        __syncthreads();
        // c = Q x
        for (int i = tid; i < m; i += nt) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += Q[i * m + j] * xv[j];
            cv[i] = s;
        }
        __syncthreads();
        // norm c^T S c (S symmetric, upper triangle valid)
        double part = 0.0;
        for (int i = tid; i < m; i += nt) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += ((i <= j) ? a.S[i * ld + j] : a.S[j * ld + i]) * cv[j];
            part += cv[i] * s;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        double nrmW = 0.0;
        for (int w = 0; w < nt / 32; ++w) nrmW += red[w];
        __syncthreads();
        if (nrmW > a.norm_tol) {
            const double f = 1.0 / sqrt(nrmW);
            for (int i = tid; i < m; i += nt) a.coef[(size_t)found * m + i] = cv[i] * f;
            if (tid == 0) a.omega[found] = th;
            om_min = fmin(om_min, th);
            ++found;
        } else if (nrmW < -a.norm_tol) {
            om_hh = fmax(om_hh, th);
        }
        __syncthreads();
    }
    if (tid == 0) {
        a.info[0] = (found >= a.nwant) ? DEV_OK : DEV_FEWROOTS;
        a.info[1] = 0.0;
        a.info[2] = found;
        a.info[3] = om_min;
        a.info[4] = om_hh;
        a.info[5] = nreal;
        a.info[6] = lowest_cplx;
        a.info[7] = max_im;
    }
}

int launch_rr_general(const RRGenArgs& a, cudaStream_t st) {
    if (a.m <= 0 || a.m > RG_MAX) return set_error(PPRPA_ERR_ARG, "rr_general: size must be 1..128");
    const size_t smem = sizeof(double) * ((size_t)a.m * a.m + 4 * a.m);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rr_general_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * (RG_MAX * RG_MAX + 4 * RG_MAX)));
        attr = true;
    }
    rr_general_kernel<<<1, RG_THREADS, smem, st>>>(a);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa
