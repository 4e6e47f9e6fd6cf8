// One-CTA dense FP64 linear algebra for the Davidson subspace.
//
// Rayleigh-Ritz for the generalised problem G c = omega S c (G = V^T M V,
// S = V^T W V): with a shift mu that makes G - mu S positive definite,
// G - mu S = Lc Lc^T (Cholesky) turns it into the symmetric problem
// H u = kappa u, H = Lc^-1 S Lc^-T, omega = mu + 1/kappa, c = Lc^-T u.
// The sign of kappa is the sign of the norm c^T S c (two-electron addition
// roots have kappa > 0), and the lowest addition roots have the largest
// kappa.  H is diagonalised with the parallel cyclic Jacobi method.
#include "kernels.h"

namespace pprpa {

constexpr int RR_THREADS = 1024;
// Subspace matrices up to 112 x 112 keep H and U in shared memory (2 x 98 KB plus ~13 KB of
// static shared memory, within the 227 KB a CTA may use); larger ones work in global memory,
// where the Jacobi sweeps are several times slower.
constexpr int RR_SMEM_MAX = 112;

// In-place Cholesky of the lower triangle of K (m x m, ld).  Returns false on a
// pivot <= rel_tol * scale.  All threads of the block must call it.
__device__ bool block_cholesky(double* K, int m, int ld, double rel_tol, double scale,
                               int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < m; ++j) {
        __syncthreads();
        if (tid == 0) {
            const double d = K[j * ld + j];
            if (!(d > rel_tol * scale)) *flag = 1;
            else K[j * ld + j] = sqrt(d);
        }
        __syncthreads();
        if (*flag) return false;
        const double piv = K[j * ld + j];
        for (int i = j + 1 + tid; i < m; i += nt) K[i * ld + j] /= piv;
        __syncthreads();
        const int r = m - j - 1;
        const int64_t cnt = (int64_t)r * r;
        for (int64_t t = tid; t < cnt; t += nt) {
            const int i = j + 1 + (int)(t / r);
            const int l = j + 1 + (int)(t % r);
            if (l <= i) K[i * ld + l] -= K[i * ld + j] * K[l * ld + j];
        }
    }
    __syncthreads();
    return true;
}

// Parallel cyclic Jacobi on symmetric H (m x m, ld); U (m x m, ld) receives the
// eigenvectors as columns.  Returns the number of sweeps.
__device__ int block_jacobi(double* H, double* U, int m, int ld, double* rot, int* pairs,
                            double* red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        U[i * ld + j] = (i == j) ? 1.0 : 0.0;
    }
    const int me = (m + 1) & ~1;  // even number of players (a dummy when m is odd)
    const int half = me / 2;
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
        // convergence: off-diagonal vs total Frobenius norm
        __syncthreads();
        double off = 0.0, tot = 0.0;
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            const double h = H[i * ld + j];
            tot += h * h;
            if (i != j) off += h * h;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) { red[2 * (tid >> 5)] = off; red[2 * (tid >> 5) + 1] = tot; }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < nt / 32; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
            red[64] = a;
            red[65] = b;
        }
        __syncthreads();
        if (!(red[64] > 1e-30 * red[65]) || me < 2) break;
        for (int s = 0; s < me - 1; ++s) {
            // pair i: fixed player me-1 vs s, others (s+i, s-i) mod (me-1)
            for (int i = tid; i < half; i += nt) {
                int p, q;
                if (i == 0) { p = me - 1; q = s; }
                else { p = (s + i) % (me - 1); q = (s - i + (me - 1)) % (me - 1); }
                if (p > q) { const int x = p; p = q; q = x; }
                pairs[2 * i] = p;
                pairs[2 * i + 1] = q;
                double c = 1.0, sn = 0.0;
                if (q < m) {
                    const double apq = H[p * ld + q];
                    const double app = H[p * ld + p], aqq = H[q * ld + q];
                    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        sn = tt * c;
                    }
                }
                rot[2 * i] = c;
                rot[2 * i + 1] = sn;
            }
            __syncthreads();
            // rows: H <- J^T H
            for (int t = tid; t < half * m; t += nt) {
                const int i = t / m, col = t % m;
                const int p = pairs[2 * i], q = pairs[2 * i + 1];
                if (q >= m) continue;
                const double c = rot[2 * i], sn = rot[2 * i + 1];
                const double hp = H[p * ld + col], hq = H[q * ld + col];
                H[p * ld + col] = c * hp - sn * hq;
                H[q * ld + col] = sn * hp + c * hq;
            }
            __syncthreads();
            // columns: H <- H J, U <- U J
            for (int t = tid; t < half * m; t += nt) {
                const int i = t / m, row = t % m;
                const int p = pairs[2 * i], q = pairs[2 * i + 1];
                if (q >= m) continue;
                const double c = rot[2 * i], sn = rot[2 * i + 1];
                const double hp = H[row * ld + p], hq = H[row * ld + q];
                H[row * ld + p] = c * hp - sn * hq;
                H[row * ld + q] = sn * hp + c * hq;
                const double up = U[row * ld + p], uq = U[row * ld + q];
                U[row * ld + p] = c * up - sn * uq;
                U[row * ld + q] = sn * up + c * uq;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return sweep;
}

__global__ void __launch_bounds__(RR_THREADS, 1) rayleigh_ritz_kernel(RRArgs a) {
    extern __shared__ double sm[];
    __shared__ double rot[2 * 512 + 2];
    __shared__ int pairs[2 * 512 + 2];
    __shared__ double red[2 * 32 + 4];
    __shared__ int flag;
    __shared__ int npos_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = a.m, ld = a.ld;
    const int lw = m;  // leading dimension of work matrices
    const bool in_smem = m <= RR_SMEM_MAX;
    double* Kc = a.work;                          // Cholesky factor (global)
    double* H = in_smem ? sm : a.work + (size_t)m * m;
    double* U = in_smem ? sm + (size_t)m * m : a.work + 2 * (size_t)m * m;
    double* X = a.work + 3 * (size_t)m * m;       // triangular-solve scratch
    int* rank = (int*)(a.work + 4 * (size_t)m * m);

    if (tid == 0) a.info[0] = DEV_NOTPD;
    // scale for the pivot test
    double sc = 0.0;
    for (int i = tid; i < m; i += nt)
        sc = fmax(sc, fabs(a.G[i * ld + i] + (a.Go ? a.Go[i * ld + i] : 0.0)) + fabs(a.S[i * ld + i]));
    for (int o = 16; o > 0; o >>= 1) sc = fmax(sc, __shfl_xor_sync(0xffffffffu, sc, o));
    if ((tid & 31) == 0) red[tid >> 5] = sc;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nt / 32; ++w) s = fmax(s, red[w]);
        red[64] = s;
    }
    __syncthreads();
    const double scale = red[64] > 0.0 ? red[64] : 1.0;

    int used = -1;
    double mu = 0.0;
    for (int c = 0; c < a.nmu && used < 0; ++c) {
        mu = a.mus[c];
        // K = sym(G) - mu S (S symmetric: read the upper triangle)
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            double g = 0.5 * (a.G[i * ld + j] + a.G[j * ld + i]);
            if (a.Go) g += 0.5 * (a.Go[i * ld + j] + a.Go[j * ld + i]);
            const double s = (i <= j) ? a.S[i * ld + j] : a.S[j * ld + i];
            Kc[i * lw + j] = g - mu * s;
        }
        if (tid == 0) flag = 0;
        __syncthreads();
        if (block_cholesky(Kc, m, lw, 1e-13, scale, &flag)) used = c;
        __syncthreads();
    }
    if (used < 0) {
        if (tid == 0) { a.info[0] = DEV_NOTPD; a.info[1] = mu; }
        return;
    }
    // X = Lc^-1 S (column per thread), then H = Lc^-1 X^T
    for (int col = tid; col < m; col += nt) {
        for (int i = 0; i < m; ++i) {
            double v = (i <= col) ? a.S[i * ld + col] : a.S[col * ld + i];
            for (int l = 0; l < i; ++l) v -= Kc[i * lw + l] * X[l * lw + col];
            X[i * lw + col] = v / Kc[i * lw + i];
        }
    }
    __syncthreads();
    for (int col = tid; col < m; col += nt) {
        for (int i = 0; i < m; ++i) {
            double v = X[col * lw + i];
            for (int l = 0; l < i; ++l) v -= Kc[i * lw + l] * H[l * lw + col];
            H[i * lw + col] = v / Kc[i * lw + i];
        }
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        if (i < j) {
            const double v = 0.5 * (H[i * lw + j] + H[j * lw + i]);
            H[i * lw + j] = v;
            H[j * lw + i] = v;
        }
    }
    const int sweeps = block_jacobi(H, U, m, lw, rot, pairs, red);
    // rank the positive kappas (descending) -> targets
    if (tid == 0) npos_sh = 0;
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
        const double ki = H[i * lw + i];
        int r = -1;
        if (ki > 0.0) {
            r = 0;
            for (int j = 0; j < m; ++j) {
                const double kj = H[j * lw + j];
                if (kj > 0.0 && (kj > ki || (kj == ki && j < i))) ++r;
            }
            atomicAdd(&npos_sh, 1);
        }
        rank[i] = r;
    }
    __syncthreads();
    const int npos = npos_sh;
    const int nk = min(a.nkeep, npos);
    // Ritz coefficients c_j = Lc^-T u_j / sqrt(kappa_j) for the kept roots
    for (int i = tid; i < m; i += nt) {
        const int r = rank[i];
        if (r < 0 || r >= nk) continue;
        const double kap = H[i * lw + i];
        double* c = a.coef + (size_t)r * m;
        for (int row = m - 1; row >= 0; --row) {
            double v = U[row * lw + i];
            for (int l = row + 1; l < m; ++l) v -= Kc[l * lw + row] * c[l];
            c[row] = v / Kc[row * lw + row];
        }
        const double f = 1.0 / sqrt(kap);
        for (int row = 0; row < m; ++row) c[row] *= f;
        a.omega[r] = mu + 1.0 / kap;
    }
    __syncthreads();
    if (tid == 0) {
        double kmin = 0.0, kmax = 0.0;
        for (int i = 0; i < m; ++i) {
            const double k = H[i * lw + i];
            if (k < kmin) kmin = k;
            if (k > kmax) kmax = k;
        }
        a.info[0] = (npos >= a.nwant) ? DEV_OK : DEV_FEWROOTS;
        a.info[1] = mu;
        a.info[2] = npos;
        a.info[3] = kmax > 0.0 ? mu + 1.0 / kmax : 1e300;
        a.info[4] = kmin < 0.0 ? mu + 1.0 / kmin : -1e300;
        a.info[5] = sweeps;
    }
}

int launch_rayleigh_ritz(const RRArgs& a, cudaStream_t st) {
    if (a.m <= 0 || a.m > 1024) return set_error(PPRPA_ERR_ARG, "rayleigh_ritz: size must be 1..1024");
    const size_t smem = a.m <= RR_SMEM_MAX ? 2 * sizeof(double) * a.m * a.m : 0;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(rayleigh_ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             2 * sizeof(double) * RR_SMEM_MAX * RR_SMEM_MAX);
        attr_set = true;
    }
    rayleigh_ritz_kernel<<<1, RR_THREADS, smem, st>>>(a);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// Block orthonormalisation helper (Cholesky QR with dropping).
__global__ void cholqr_small_kernel(const double* __restrict__ Gm, int k, double tol,
                                    double* __restrict__ T, int* __restrict__ keep,
                                    double* __restrict__ work) {
    // single thread: k is small (<= 64)
    if (threadIdx.x != 0) return;
    double* Lc = work;            // k x k
    double* s = work + k * k;     // k
    for (int i = 0; i < k; ++i) {
        const double d = Gm[i * k + i];
        s[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
        keep[i] = d > 0.0 ? 1 : 0;
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Lc[i * k + j] = (j <= i) ? Gm[i * k + j] * s[i] * s[j] : 0.0;
    for (int j = 0; j < k; ++j) {
        double d = Lc[j * k + j];
        for (int l = 0; l < j; ++l) d -= Lc[j * k + l] * Lc[j * k + l];
        if (!keep[j] || !(d > tol)) {
            keep[j] = 0;
            for (int l = 0; l < j; ++l) Lc[j * k + l] = 0.0;
            Lc[j * k + j] = 1.0;
            for (int i = j + 1; i < k; ++i) Lc[i * k + j] = 0.0;
            continue;
        }
        const double piv = sqrt(d);
        Lc[j * k + j] = piv;
        for (int i = j + 1; i < k; ++i) {
            double v = Lc[i * k + j];
            for (int l = 0; l < j; ++l) v -= Lc[i * k + l] * Lc[j * k + l];
            Lc[i * k + j] = v / piv;
        }
    }
    // T = Lc^-1 diag(s); dropped rows zero
    for (int col = 0; col < k; ++col) {
        for (int i = 0; i < k; ++i) {
            double v = (i == col) ? 1.0 : 0.0;
            for (int l = 0; l < i; ++l) v -= Lc[i * k + l] * T[l * k + col];
            T[i * k + col] = v / Lc[i * k + i];
        }
    }
    for (int i = 0; i < k; ++i)
        for (int col = 0; col < k; ++col)
            T[i * k + col] = keep[i] ? T[i * k + col] * s[col] : 0.0;
}

int launch_cholqr_small(const double* Gm, int k, double tol, double* T, int* keep, double* work,
                        cudaStream_t st) {
    if (k <= 0) return PPRPA_OK;
    if (k > 256) return set_error(PPRPA_ERR_ARG, "cholqr_small: block too large");
    cholqr_small_kernel<<<1, 32, 0, st>>>(Gm, k, tol, T, keep, work);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Symmetric eigendecomposition of `batch` matrices H (m x m each, row-major, `stride` doubles
// apart) by the one-CTA parallel Jacobi above, one CTA per matrix: H is overwritten (the
// eigenvalues end on its diagonal) and U receives the eigenvectors as columns.
// work: batch x 1152 doubles, iwork: batch x 1024 ints (m <= 1024).
__global__ void __launch_bounds__(1024, 1) sym_eig_kernel(double* H, double* U, int m, int64_t stride,
                                                          double* work, int* iwork) {
    const int b = blockIdx.x;
    double* rot = work + (int64_t)b * 1152;
    block_jacobi(H + b * stride, U + b * stride, m, m, rot, iwork + (int64_t)b * 1024, rot + 1024);
}

int launch_sym_eig(double* H, double* U, int m, int batch, int64_t stride, double* work, int* iwork,
                   cudaStream_t st) {
    if (m <= 0 || batch <= 0) return PPRPA_OK;
    if (m > 1024) return set_error(PPRPA_ERR_ARG, "sym_eig: order above 1024");
    sym_eig_kernel<<<batch, 1024, 0, st>>>(H, U, m, stride, work, iwork);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa
