// One-CTA dense FP64 linear algebra for the Davidson subspace.
//
// Rayleigh-Ritz for the generalised problem G c = omega S c (G = V^T M V,
// S = V^T W V): with a shift mu that makes G - mu S positive definite,
// G - mu S = Lc Lc^T (Cholesky) turns it into the symmetric problem
// H u = kappa u, H = Lc^-1 S Lc^-T, omega = mu + 1/kappa, c = Lc^-T u.
// The sign of kappa is the sign of the norm c^T S c (two-electron addition
// roots have kappa > 0), and the lowest addition roots have the largest
// kappa.  H is diagonalised with the parallel cyclic Jacobi method.
#include <cooperative_groups.h>

#include "kernels.h"

namespace pprpa {

constexpr int RR_THREADS = 1024;
// Subspace matrices up to 112 x 112 keep H and U in shared memory (2 x 98 KB plus ~13 KB of
// static shared memory, within the 227 KB a CTA may use); larger ones work in global memory,
// where the Jacobi sweeps are several times slower.
constexpr int RR_SMEM_MAX = 112;

__host__ __device__ inline int rr_ld(int m, int pad) { return pad ? (m | 1) : m; }

// Sums over the CTA of per-thread values, returned to every thread.  The partial sums of the
// warps are added by a shuffle tree on warp 0: a serial chain of dependent FP64 additions on
// one thread costs thousands of cycles on this GPU.  red: >= 99 doubles (partials at 0..95,
// results at 96..98).
__device__ void block_sum3(double& a, double& b, double& c, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    __syncthreads();
    if (lane == 0) {
        red[w] = a;
        red[32 + w] = b;
        red[64 + w] = c;
    }
    __syncthreads();
    if (w == 0) {
        double x = lane < nw ? red[lane] : 0.0, y = lane < nw ? red[32 + lane] : 0.0, z = lane < nw ? red[64 + lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            red[96] = x;
            red[97] = y;
            red[98] = z;
        }
    }
    __syncthreads();
    a = red[96];
    b = red[97];
    c = red[98];
}

__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
    double c = 0.0;
    block_sum3(a, b, c, red);
}

// Maximum over the CTA of a per-thread value (same tree; red as above).
__device__ double block_max(double v, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        double x = lane < nw ? red[lane] : -1e300;
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
        if (lane == 0) red[96] = x;
    }
    __syncthreads();
    return red[96];
}


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
        block_sum2(off, tot, red);
        if (!(off > 1e-30 * tot) || me < 2) break;
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

__device__ inline double jsqrt(double x) { return sqrt(x); }
__device__ inline float jsqrt(float x) { return sqrtf(x); }
__device__ inline double jabs(double x) { return fabs(x); }
__device__ inline float jabs(float x) { return fabsf(x); }
__device__ inline double jrsqrt(double x) { return rsqrt(x); }
__device__ inline float jrsqrt(float x) { return rsqrtf(x); }

// The same parallel cyclic Jacobi with H <- J^T H J done in one pass over the 2 x 2 blocks of
// the pairing: block (a, b), a <= b, gets the row rotation of pair a and the column rotation of
// pair b, and is written to both triangles.  Distinct blocks touch disjoint entries, so the
// update is in place; U <- U J runs in the same pass.  Two thirds of the FP64 operations and
// two barriers per round instead of three.  T = float serves the first pass of the mixed
// solver below.  Sweeps stop once off-diagonal^2 <= tol2 * total^2 (Frobenius); rotations
// with |h_pq| <= skip * sqrt|h_pp h_qq| are skipped.
template <typename T>
__device__ int jacobi_sym_t(T* H, T* U, int m, int ld, T* rot, int* pairs, double* red, double tol2,
                            T skip, T tiny, int max_sweeps = 40, bool stop_on_stall = false) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        U[i * ld + j] = (i == j) ? T(1) : T(0);
    }
    const int me = (m + 1) & ~1;
    const int half = me / 2;
    const int nblk = half * (half + 1) / 2;
    int sweep = 0;
    double prev_off = 0.0;
    for (; sweep < max_sweeps; ++sweep) {
        __syncthreads();
        T off = 0, tot = 0;
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            const T h = H[i * ld + j];
            tot += h * h;
            if (i != j) off += h * h;
        }
        double offd = off, totd = tot;
        block_sum2(offd, totd, red);
        if (!(offd > tol2 * totd) || me < 2) break;
        // rounding floor of a low precision: quadratic convergence has stopped
        if (stop_on_stall && sweep >= 2 && offd > 0.25 * prev_off) break;
        prev_off = offd;
        for (int s = 0; s < me - 1; ++s) {
            for (int i = tid; i < half; i += nt) {
                int p, q;
                if (i == 0) { p = me - 1; q = s; }
                else { p = (s + i) % (me - 1); q = (s - i + (me - 1)) % (me - 1); }
                if (p > q) { const int x = p; p = q; q = x; }
                pairs[2 * i] = p;
                pairs[2 * i + 1] = q;
                T c = 1, sn = 0;
                if (q < m) {
                    const T apq = H[p * ld + q];
                    const T app = H[p * ld + p], aqq = H[q * ld + q];
                    if (jabs(apq) > tiny && jabs(apq) > skip * jsqrt(jabs(app * aqq))) {
                        // tan of the smaller annihilating angle, t = sgn(d) 2 h_pq / (|d| + sqrt(d^2 + 4 h_pq^2))
                        // with d = h_qq - h_pp: one division, one square root and one reciprocal root
                        const T d = aqq - app, a2 = T(2) * apq;
                        const T tt = (d >= T(0) ? a2 : -a2) / (jabs(d) + jsqrt(d * d + a2 * a2));
                        c = jrsqrt(T(1) + tt * tt);
                        sn = tt * c;
                    }
                }
                rot[2 * i] = c;
                rot[2 * i + 1] = sn;
            }
            __syncthreads();
            // H: blocks (a, b), a <= b, in triangular order t = b (b + 1) / 2 + a
            for (int t = tid; t < nblk; t += nt) {
                int b = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                while (b * (b + 1) / 2 > t) --b;
                while ((b + 1) * (b + 2) / 2 <= t) ++b;
                const int aa = t - b * (b + 1) / 2;
                const int pa = pairs[2 * aa], qa = pairs[2 * aa + 1];
                const int pb = pairs[2 * b], qb = pairs[2 * b + 1];
                const bool va = qa < m, vb = qb < m;  // q = m marks the dummy player (odd m)
                const T ca = rot[2 * aa], sa = rot[2 * aa + 1];
                const T cb = rot[2 * b], sb = rot[2 * b + 1];
                const T h00 = H[pa * ld + pb];
                const T h01 = vb ? H[pa * ld + qb] : T(0);
                const T h10 = va ? H[qa * ld + pb] : T(0);
                const T h11 = (va && vb) ? H[qa * ld + qb] : T(0);
                // rows: (p, q) <- (c h_p - s h_q, s h_p + c h_q)
                const T r00 = ca * h00 - sa * h10, r01 = ca * h01 - sa * h11;
                const T r10 = sa * h00 + ca * h10, r11 = sa * h01 + ca * h11;
                // columns, the same rotation form
                const T o00 = cb * r00 - sb * r01, o01 = sb * r00 + cb * r01;
                const T o10 = cb * r10 - sb * r11, o11 = sb * r10 + cb * r11;
                if (aa == b) {
                    const T od = T(0.5) * (o01 + o10);
                    H[pa * ld + pa] = o00;
                    if (va) {
                        H[pa * ld + qa] = od;
                        H[qa * ld + pa] = od;
                        H[qa * ld + qa] = o11;
                    }
                } else {
                    H[pa * ld + pb] = o00;
                    H[pb * ld + pa] = o00;
                    if (vb) { H[pa * ld + qb] = o01; H[qb * ld + pa] = o01; }
                    if (va) { H[qa * ld + pb] = o10; H[pb * ld + qa] = o10; }
                    if (va && vb) { H[qa * ld + qb] = o11; H[qb * ld + qa] = o11; }
                }
            }
            // U <- U J (one thread per row and pair; consecutive threads take consecutive rows)
            for (int t = tid; t < half * m; t += nt) {
                const int i = t / m, row = t % m;
                const int p = pairs[2 * i], q = pairs[2 * i + 1];
                if (q >= m) continue;
                const T c = rot[2 * i], sn = rot[2 * i + 1];
                const T up = U[row * ld + p], uq = U[row * ld + q];
                U[row * ld + p] = c * up - sn * uq;
                U[row * ld + q] = sn * up + c * uq;
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return sweep;
}

__device__ int block_jacobi_sym(double* H, double* U, int m, int ld, double* rot, int* pairs,
                                double* red, double tol2 = 1e-30) {
    return jacobi_sym_t<double>(H, U, m, ld, rot, pairs, red, tol2, 1e-18, 1e-300);
}

// C (m x m, ldc) = op(A) B with op(A) = A or A^T; A (lda), B (ldb) row-major.  One thread per
// output element; the FP64 pipe, not latency, bounds it with a full CTA of threads.
__device__ void block_gemm(double* C, int ldc, const double* A, int lda, bool transA, const double* B,
                           int ldb, int m) {
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int i = t / m, j = t % m;
        double acc = 0.0;
        if (transA)
            for (int k = 0; k < m; ++k) acc = fma(A[k * lda + i], B[k * ldb + j], acc);
        else
            for (int k = 0; k < m; ++k) acc = fma(A[i * lda + k], B[k * ldb + j], acc);
        C[i * ldc + j] = acc;
    }
}

// Mixed-precision symmetric eigensolver, same contract as block_jacobi (H in, eigenvalues on
// its diagonal; eigenvectors as the columns of U; both m x m with leading dimension ld).
//  1. Jacobi in FP32 on a float copy of H (stored in U's space): rotations on the FP32 pipe,
//     which has many times the FP64 rate, to an off-diagonal norm near FP32 rounding.
//  2. Its eigenvector matrix G is orthonormalised in FP64 by two Newton-Schulz steps
//     G <- G (3 I - G^T G) / 2 (quadratic: FP32-level 1e-6 -> 1e-12 -> rounding).
//  3. H' = G^T H G in FP64 is diagonal up to FP32-level terms; FP64 Jacobi sweeps finish it
//     (quadratic convergence: one or two sweeps) and U = G U'.
// G and T are m x m FP64 scratch (leading dimension m) outside H and U.  Returns
// 100 * FP32 sweeps + FP64 sweeps (+ 10 * the reason a refinement fell back to them), or
// 100 * FP32 sweeps + 50 + refinement steps.
// One step of the iterative refinement of a symmetric eigendecomposition by Ogita and Aishima
// ("Iterative refinement for symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math.
// 35, 2018), in FP64: for approximate eigenvectors G (columns, m x m, leading dimension m) of
// the symmetric H (ld),
//   R = I - G^T G,  S = G^T H G,  lam_i = S_ii / (1 - R_ii),
//   E_ii = R_ii / 2,  E_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i)  (i != j),
//   G <- G (I + E),
// which squares the error of eigenpairs whose eigenvalues are well separated relative to their
// coupling.  Returns false, with G unchanged, when some pair is coupled by more than 1 % of
// its gap (the refinement cannot separate it) or the start is too far off; otherwise lam holds the refined eigenvalues, G the refined vectors and
// *corr the Frobenius norm of E; *flag says why it returned false (1 close eigenvalues, 2 a start
// too far off).  T (m x m, ld m) and W (m x ld) are scratch; H is untouched.
__device__ bool oa_refine(const double* H, int ld, double* G, double* T, double* W, int m, double* lam,
                          double* red, double* corr, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    block_gemm(T, m, H, ld, false, G, m, m);  // T = H G
    __syncthreads();
    // W = S = G^T (H G) and T = R = I - G^T G afterwards, upper triangles mirrored
    for (int t = tid; t < m * (m + 1) / 2; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], T[k * m + j], acc);
        W[i * ld + j] = acc;
        W[j * ld + i] = acc;
    }
    __syncthreads();
    for (int t = tid; t < m * (m + 1) / 2; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], G[k * m + j], acc);
        const double r = (i == j ? 1.0 : 0.0) - acc;
        T[i * m + j] = r;
        T[j * m + i] = r;
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt) lam[i] = W[i * ld + i] / (1.0 - T[i * m + i]);
    __syncthreads();
    double ns = 0.0, nh = 0.0, nr = 0.0;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        const double sij = W[i * ld + j] - (i == j ? lam[i] : 0.0);
        ns += sij * sij;
        nh += H[i * ld + j] * H[i * ld + j];
        nr += T[t] * T[t];
    }
    block_sum3(ns, nh, nr, red);
    if (tid == 0) *flag = (sqrt(nr) > 1e-3 || sqrt(ns) > 1e-3 * sqrt(nh)) ? 2 : 0;
    __syncthreads();
    // pairs the first-order step cannot separate: a coupling |S_ij + lam_j R_ij| above 1 % of
    // the gap (the step's error is the square of that ratio), or eigenvalues equal to rounding.
    // This per-pair form of the method's separation condition keeps well-resolved pairs of
    // close eigenvalues, which the norm bound delta would reject together with the rest.
    const double tiny = 1e-13 * sqrt(nh);
    for (int t = tid; t < m * m && !*flag; t += nt) {
        const int i = t / m, j = t % m;
        if (i >= j) continue;
        const double gap = fabs(lam[j] - lam[i]);
        const double cpl = fmax(fabs(W[i * ld + j] + lam[j] * T[i * m + j]), fabs(W[i * ld + j] + lam[i] * T[i * m + j]));
        if (gap <= tiny || cpl > 0.01 * gap) *flag = 1;
    }
    __syncthreads();
    if (*flag) return false;
    // E in place of S in W
    double ne = 0.0;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        const double e = (i == j) ? 0.5 * T[t] : (W[i * ld + j] + lam[j] * T[i * m + j]) / (lam[j] - lam[i]);
        W[i * ld + j] = e;
        ne += e * e;
    }
    double z0 = 0.0, z1 = 0.0;
    block_sum3(ne, z0, z1, red);
    // T = G (I + E), then G = T
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        double acc = G[t];
        for (int k = 0; k < m; ++k) acc = fma(G[i * m + k], W[k * ld + j], acc);
        T[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) G[t] = T[t];
    __syncthreads();
    *corr = sqrt(ne);
    return true;
}

__device__ int block_mixed_eig(double* H, double* U, int m, int ld, double* G, double* T, double* rot,
                               int* pairs, double* red, double tol32, bool refine_oa, long long* pclk = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    float* H32 = reinterpret_cast<float*>(U);  // two m x ld float matrices fill U's doubles
    float* U32 = H32 + (size_t)m * ld;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        H32[i * ld + j] = (float)H[i * ld + j];
    }
    const int s32 = jacobi_sym_t<float>(H32, U32, m, ld, reinterpret_cast<float*>(rot), pairs, red, tol32,
                                        1e-9f, 1e-30f, 16, true);
    if (pclk && tid == 0) *pclk = clock64();
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        G[t] = (double)U32[i * ld + j];
    }
    __syncthreads();
    int fallback = 0;  // why the refinement fell back: 1 close eigenvalues, 2 poor start, 3 slow
    if (refine_oa) {
        // FP64 refinement by matrix products (about 3 m^3 FP64 FMAs a step instead of the
        // ~10 m^3 of the orthonormalisation and Jacobi sweeps below); falls back to them when
        // eigenvalues are too close for it
        __shared__ int oa_flag;
        double* lam = rot;  // the rotation buffer is free until a fallback Jacobi needs it
        // a step squares the error; from the FP32 floor (~1e-7) one step reaches FP64 rounding,
        // and a correction below 1e-6 leaves an error near its square
        double corr = 1.0;
        bool ok = true;
        int steps = 0;
        while (steps < 2 && ok && corr > 1e-6) {
            ok = oa_refine(H, ld, G, T, U, m, lam, red, &corr, &oa_flag);
            ++steps;
        }
        if (ok && corr <= 1e-6) {
            for (int t = tid; t < m * m; t += nt) {
                const int i = t / m, j = t % m;
                U[i * ld + j] = G[t];
                H[i * ld + j] = (i == j) ? lam[i] : 0.0;
            }
            __syncthreads();
            return 100 * s32 + 50 + steps;
        }
        // refined only in part: G is still a good start for the path below
        fallback = ok ? 3 : oa_flag;
    }
    for (int ns = 0; ns < 2; ++ns) {
        block_gemm(T, m, G, m, true, G, m, m);  // T = G^T G
        __syncthreads();
        for (int t = tid; t < m * m; t += nt) T[t] = (t / m == t % m ? 1.5 : 0.0) - 0.5 * T[t];
        __syncthreads();
        block_gemm(U, ld, G, m, false, T, m, m);  // U = G (3 I - G^T G) / 2
        __syncthreads();
        for (int t = tid; t < m * m; t += nt) G[t] = U[(t / m) * ld + t % m];
        __syncthreads();
    }
    block_gemm(T, m, H, ld, false, G, m, m);  // T = H G
    __syncthreads();
    // H' = G^T T, upper triangle mirrored (t = j (j + 1) / 2 + i, i <= j)
    for (int t = tid; t < m * (m + 1) / 2; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], T[k * m + j], acc);
        H[i * ld + j] = acc;
        H[j * ld + i] = acc;
    }
    __syncthreads();
    // off-diagonal <= 1e-13 of the total (Frobenius): the eigenvalues are then exact to
    // rounding (their error is second order) and the eigenvectors to about 1e-13 / gap
    const int s64 = block_jacobi_sym(H, U, m, ld, rot, pairs, red, 1e-26);
    block_gemm(T, m, G, m, false, U, ld, m);  // eigenvectors G U'
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) U[(t / m) * ld + t % m] = T[t];
    __syncthreads();
    return 100 * s32 + 10 * fallback + s64;
}

// Symmetric eigendecomposition by Householder reduction to tridiagonal form followed by the
// implicit symmetric QR iteration with Wilkinson shifts (Golub and Van Loan, Matrix
// Computations, Secs. 8.3.1 and 8.3.3).  FP64 arithmetic is scarce on this GPU, and this needs
// a few times fewer operations than cyclic Jacobi sweeps, and O(m) CTA barriers: each QR step's
// chain of rotations is formed by one thread and then applied to the rows of U in parallel.
// Same contract as block_jacobi: H (m x m, ld, symmetric) is overwritten with its eigenvalues on
// the diagonal (the rest is scratch), U (m x m, ld) receives the eigenvectors as columns.
// vec: >= 6m doubles of scratch.  Returns the number of QR steps.
__device__ int block_tridiag_eig(double* H, double* U, int m, int ld, double* vec) {
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ double red_s[33];
    __shared__ int lh_s[3];
    double* d = vec;              // diagonal of T
    double* e = vec + m;          // e[k] = T[k][k+1]
    double* beta = vec + 2 * m;   // Householder scalars
    double* cs = vec + 3 * m;     // rotation chain of one QR step
    double* sn = vec + 4 * m;
    double* pw = vec + 5 * m;     // p, then w, of one Householder step
    auto block_sum = [&](double x) -> double {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        __syncthreads();
        if ((tid & 31) == 0) red_s[tid >> 5] = x;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nt / 32; ++w) t += red_s[w];
            red_s[32] = t;
        }
        __syncthreads();
        return red_s[32];
    };
    // ---- Householder: column k below the subdiagonal is reflected onto e_{k+1} ----
    for (int k = 0; k + 2 < m; ++k) {
        const int r0 = k + 1, r = m - r0;  // trailing block rows/columns r0 .. m-1
        double x2 = 0.0;
        for (int i = tid; i < r; i += nt) x2 += H[(r0 + i) * ld + k] * H[(r0 + i) * ld + k];
        x2 = block_sum(x2);
        const double x0 = H[r0 * ld + k];
        if (x2 <= 1e-300) {  // nothing to eliminate
            if (tid == 0) { beta[k] = 0.0; e[k] = x0; d[k] = H[k * ld + k]; }
            __syncthreads();
            continue;
        }
        const double alpha = x0 >= 0.0 ? -sqrt(x2) : sqrt(x2);
        const double bt = x2 - x0 * alpha;  // v^T v / 2 with v = x - alpha e_1
        __syncthreads();
        if (tid == 0) {
            H[r0 * ld + k] = x0 - alpha;  // v stays in the column (v_i = x_i for i > 0)
            beta[k] = bt;
            e[k] = alpha;
            d[k] = H[k * ld + k];
        }
        __syncthreads();
        // p = A22 v / beta; A22 is symmetric, so thread i walks column i (coalesced)
        for (int i = tid; i < r; i += nt) {
            double acc = 0.0;
            for (int j = 0; j < r; ++j) acc = fma(H[(r0 + j) * ld + r0 + i], H[(r0 + j) * ld + k], acc);
            pw[i] = acc / bt;
        }
        __syncthreads();
        double vp = 0.0;
        for (int i = tid; i < r; i += nt) vp += H[(r0 + i) * ld + k] * pw[i];
        vp = block_sum(vp);
        const double kk = vp / (2.0 * bt);
        for (int i = tid; i < r; i += nt) pw[i] -= kk * H[(r0 + i) * ld + k];  // w = p - K v
        __syncthreads();
        // A22 -= v w^T + w v^T
        for (int t = tid; t < r * r; t += nt) {
            const int i = t / r, j = t % r;
            const double vi = H[(r0 + i) * ld + k], vj = H[(r0 + j) * ld + k];
            H[(r0 + i) * ld + r0 + j] -= vi * pw[j] + pw[i] * vj;
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (m >= 2) {
            d[m - 2] = H[(m - 2) * ld + m - 2];
            e[m - 2] = H[(m - 1) * ld + m - 2];
            beta[m - 2] = 0.0;
        }
        d[m - 1] = H[(m - 1) * ld + m - 1];
        e[m - 1] = 0.0;
    }
    // ---- Q = H_0 H_1 ... H_{m-3}, built from the right on the identity ----
    for (int t = tid; t < m * m; t += nt) U[(t / m) * ld + t % m] = (t / m == t % m) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = m - 3; k >= 0; --k) {
        const double bt = beta[k];
        if (bt == 0.0) continue;
        const int r0 = k + 1, r = m - r0;
        // rows r0.. of U: U -= v (v^T U) / beta, columns r0.. (the others are still identity)
        for (int j = tid; j < r; j += nt) {
            double acc = 0.0;
            for (int i = 0; i < r; ++i) acc = fma(H[(r0 + i) * ld + k], U[(r0 + i) * ld + r0 + j], acc);
            pw[j] = acc / bt;
        }
        __syncthreads();
        for (int t = tid; t < r * r; t += nt) {
            const int i = t / r, j = t % r;
            U[(r0 + i) * ld + r0 + j] -= H[(r0 + i) * ld + k] * pw[j];
        }
        __syncthreads();
    }
    // U now holds Q.  The rotations below act on pairs of columns of Q; they are applied to
    // the rows of Q^T instead, so that the threads (one per row of Q) touch consecutive words.
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        if (i < j) {
            const double x = U[i * ld + j];
            U[i * ld + j] = U[j * ld + i];
            U[j * ld + i] = x;
        }
    }
    __syncthreads();
    // ---- implicit QR steps with Wilkinson shifts on the unreduced trailing block ----
    int steps = 0;
    const int max_steps = 40 * m + 40;
    for (;;) {
        if (tid == 0) {
            int h = lh_s[1] = -1;
            // deflate from the bottom: the largest h whose e[h-1] is not negligible
            for (h = m - 1; h > 0; --h) {
                if (fabs(e[h - 1]) <= 2.2e-16 * (fabs(d[h - 1]) + fabs(d[h])) + 1e-300) e[h - 1] = 0.0;
                else break;
            }
            int l = h;
            while (l > 0 && fabs(e[l - 1]) > 2.2e-16 * (fabs(d[l - 1]) + fabs(d[l])) + 1e-300) --l;
            if (l > 0) e[l - 1] = 0.0;
            lh_s[0] = l;
            lh_s[1] = h;
            if (h > 0 && steps < max_steps) {
                // Wilkinson shift from the trailing 2 x 2
                const double a = d[h - 1], b = e[h - 1], c = d[h];
                const double dl = 0.5 * (a - c);
                const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * hypot(dl, b);
                const double mu = den != 0.0 ? c - b * b / den : c;
                double x = d[l] - mu, z = e[l];
                for (int k = l; k < h; ++k) {
                    const double r2 = fma(x, x, z * z);  // |x|, |z| are far from overflow here
                    const double inv = r2 > 0.0 ? rsqrt(r2) : 0.0;
                    const double rr = r2 * inv;
                    const double cc = r2 > 0.0 ? x * inv : 1.0, ss = z * inv;
                    if (k > l) e[k - 1] = rr;
                    const double dk = d[k], ek = e[k], dk1 = d[k + 1];
                    d[k] = cc * cc * dk + 2.0 * cc * ss * ek + ss * ss * dk1;
                    d[k + 1] = ss * ss * dk - 2.0 * cc * ss * ek + cc * cc * dk1;
                    e[k] = cc * ss * (dk1 - dk) + (cc * cc - ss * ss) * ek;
                    if (k + 1 < h) {
                        z = ss * e[k + 1];
                        e[k + 1] = cc * e[k + 1];
                        x = e[k];
                    }
                    cs[k] = cc;
                    sn[k] = ss;
                }
            }
        }
        __syncthreads();
        const int l = lh_s[0], h = lh_s[1];
        if (h <= 0 || steps >= max_steps) break;
        // Q <- Q G_l ... G_{h-1}: each thread applies the whole chain to its row of Q, stored
        // as column `row` of Q^T
        for (int row = tid; row < m; row += nt) {
            double uk = U[l * ld + row];
            for (int k = l; k < h; ++k) {
                const double c = cs[k], s = sn[k], uk1 = U[(k + 1) * ld + row];
                U[k * ld + row] = c * uk + s * uk1;
                uk = -s * uk + c * uk1;
            }
            U[h * ld + row] = uk;
        }
        ++steps;
        __syncthreads();
    }
    for (int t = tid; t < m * m; t += nt) {  // Q^T back to Q: eigenvectors as columns
        const int i = t / m, j = t % m;
        if (i < j) {
            const double x = U[i * ld + j];
            U[i * ld + j] = U[j * ld + i];
            U[j * ld + i] = x;
        }
    }
    for (int i = tid; i < m; i += nt) H[i * ld + i] = d[i];
    __syncthreads();
    return steps;
}

__global__ void __launch_bounds__(RR_THREADS, 1) rayleigh_ritz_kernel(RRArgs a) {
    extern __shared__ double sm[];
    __shared__ double rot[2 * 512 + 2];
    __shared__ int pairs[2 * 512 + 2];
    __shared__ double red[104];
    __shared__ int flag;
    __shared__ int npos_sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int m = a.m, ld = a.ld;
    const int lw = m;  // leading dimension of the global work matrices
    const bool in_smem = m <= RR_SMEM_MAX;
    // H and U in shared memory get an odd leading dimension: column-wise walks (one thread per
    // row) then fall on distinct banks
    const int lh = in_smem ? rr_ld(m, a.pad) : m;
    double* Kc = a.work;                          // Cholesky factor (global)
    double* H = in_smem ? sm : a.work + (size_t)m * m;
    double* U = in_smem ? sm + (size_t)m * lh : a.work + 2 * (size_t)m * m;
    double* X = a.work + 3 * (size_t)m * m;       // triangular-solve scratch
    int* rank = (int*)(a.work + 4 * (size_t)m * m);

    __shared__ long long clk[6];  // phase clocks of thread 0 (PPRPA_RR_PROF)
    __shared__ long long clk6;    // end of the FP32 stage of the mixed eigensolver
    if (tid == 0) clk[0] = clock64();
    if (tid == 0) a.info[0] = DEV_NOTPD;
    // scale for the pivot test
    double sc = 0.0;
    for (int i = tid; i < m; i += nt)
        sc = fmax(sc, fabs(a.G[i * ld + i] + (a.Go ? a.Go[i * ld + i] : 0.0)) + fabs(a.S[i * ld + i]));
    sc = block_max(sc, red);
    const double scale = sc > 0.0 ? sc : 1.0;

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
    if (tid == 0) clk[1] = clock64();
    // reciprocal pivots (after the eigensolver's scratch at 4 m^2 + m .. 4 m^2 + 7 m)
    double* rdiag = a.work + 4 * (size_t)m * m + 7 * (size_t)m;
    for (int i = tid; i < m; i += nt) rdiag[i] = 1.0 / Kc[i * lw + i];
    __syncthreads();
    // X = Lc^-1 S (column per thread), then H = Lc^-1 X^T.  Four partial sums per row keep
    // four independent FMA chains in flight (the FP64 latency would otherwise bound a row).
    for (int col = tid; col < m; col += nt) {
        for (int i = 0; i < m; ++i) {
            double v0 = (i <= col) ? a.S[i * ld + col] : a.S[col * ld + i], v1 = 0.0, v2 = 0.0, v3 = 0.0;
            const double* kr = Kc + (size_t)i * lw;
            int l = 0;
            for (; l + 4 <= i; l += 4) {
                v0 = fma(-kr[l], X[l * lw + col], v0);
                v1 = fma(-kr[l + 1], X[(l + 1) * lw + col], v1);
                v2 = fma(-kr[l + 2], X[(l + 2) * lw + col], v2);
                v3 = fma(-kr[l + 3], X[(l + 3) * lw + col], v3);
            }
            for (; l < i; ++l) v0 = fma(-kr[l], X[l * lw + col], v0);
            X[i * lw + col] = ((v0 + v1) + (v2 + v3)) * rdiag[i];
        }
    }
    __syncthreads();
    for (int col = tid; col < m; col += nt) {
        for (int i = 0; i < m; ++i) {
            double v0 = X[col * lw + i], v1 = 0.0, v2 = 0.0, v3 = 0.0;
            const double* kr = Kc + (size_t)i * lw;
            int l = 0;
            for (; l + 4 <= i; l += 4) {
                v0 = fma(-kr[l], H[l * lh + col], v0);
                v1 = fma(-kr[l + 1], H[(l + 1) * lh + col], v1);
                v2 = fma(-kr[l + 2], H[(l + 2) * lh + col], v2);
                v3 = fma(-kr[l + 3], H[(l + 3) * lh + col], v3);
            }
            for (; l < i; ++l) v0 = fma(-kr[l], H[l * lh + col], v0);
            H[i * lh + col] = ((v0 + v1) + (v2 + v3)) * rdiag[i];
        }
    }
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        if (i < j) {
            const double v = 0.5 * (H[i * lh + j] + H[j * lh + i]);
            H[i * lh + j] = v;
            H[j * lh + i] = v;
        }
    }
    __syncthreads();
    if (tid == 0) clk6 = clk[2] = clock64();
    const int sweeps = ((a.eig == 3 || a.eig == 4) && in_smem)
                           ? block_mixed_eig(H, U, m, lh, a.work + (size_t)m * m, a.work + 2 * (size_t)m * m, rot,
                                             pairs, red, a.tol32, a.eig == 4, &clk6)
                       : (a.eig == 0 || a.eig == 3) ? block_jacobi_sym(H, U, m, lh, rot, pairs, red)
                       : a.eig == 1                 ? block_jacobi(H, U, m, lh, rot, pairs, red)
                                    : block_tridiag_eig(H, U, m, lh,
                                                        6 * m <= 2 * 512 + 2 ? rot : a.work + 4 * (size_t)m * m + m);
    if (tid == 0) clk[3] = clock64();
    // rank the positive kappas (descending) -> targets
    if (tid == 0) npos_sh = 0;
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
        const double ki = H[i * lh + i];
        int r = -1;
        if (ki > 0.0) {
            r = 0;
            for (int j = 0; j < m; ++j) {
                const double kj = H[j * lh + j];
                if (kj > 0.0 && (kj > ki || (kj == ki && j < i))) ++r;
            }
            atomicAdd(&npos_sh, 1);
        }
        rank[i] = r;
    }
    __syncthreads();
    const int npos = npos_sh;
    const int nk = min(a.nkeep, npos);
    if (tid == 0) clk[4] = clock64();
    // Ritz coefficients c_j = Lc^-T u_j / sqrt(kappa_j) for the kept roots
    for (int i = tid; i < m; i += nt) {
        const int r = rank[i];
        if (r < 0 || r >= nk) continue;
        const double kap = H[i * lh + i];
        double* c = a.coef + (size_t)r * m;
        for (int row = m - 1; row >= 0; --row) {
            double v0 = U[row * lh + i], v1 = 0.0, v2 = 0.0, v3 = 0.0;
            int l = row + 1;
            for (; l + 4 <= m; l += 4) {
                v0 = fma(-Kc[l * lw + row], c[l], v0);
                v1 = fma(-Kc[(l + 1) * lw + row], c[l + 1], v1);
                v2 = fma(-Kc[(l + 2) * lw + row], c[l + 2], v2);
                v3 = fma(-Kc[(l + 3) * lw + row], c[l + 3], v3);
            }
            for (; l < m; ++l) v0 = fma(-Kc[l * lw + row], c[l], v0);
            c[row] = ((v0 + v1) + (v2 + v3)) * rdiag[row];
        }
        const double f = 1.0 / sqrt(kap);
        for (int row = 0; row < m; ++row) c[row] *= f;
        a.omega[r] = mu + 1.0 / kap;
    }
    __syncthreads();
    if (tid == 0) {
        double kmin = 0.0, kmax = 0.0;
        for (int i = 0; i < m; ++i) {
            const double k = H[i * lh + i];
            if (k < kmin) kmin = k;
            if (k > kmax) kmax = k;
        }
        a.info[0] = (npos >= a.nwant) ? DEV_OK : DEV_FEWROOTS;
        a.info[1] = mu;
        a.info[2] = npos;
        a.info[3] = kmax > 0.0 ? mu + 1.0 / kmax : 1e300;
        a.info[4] = kmin < 0.0 ? mu + 1.0 / kmin : -1e300;
        a.info[5] = sweeps;
        if (a.prof) {
            clk[5] = clock64();
            printf("[rr] m %d sweeps %d cycles: factor %lld solves %lld eig %lld (fp32 %lld) rank %lld ritz %lld\n", m,
                   sweeps, clk[1] - clk[0], clk[2] - clk[1], clk[3] - clk[2], clk6 - clk[2], clk[4] - clk[3],
                   clk[5] - clk[4]);
        }
    }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz on a cluster of CTAs (m <= RRC_MAX, eigensolver 4).
//
// GB300 runs FP64 at about two FMAs per clock per SM, so the O(m^3) FP64 products of the
// one-CTA kernel above (the triangular solves of the reduction, the Ogita-Aishima
// refinement) are bound by a single SM's FP64 pipe.  Here RRC_SIZE CTAs of one thread-block
// cluster each hold a full copy of the state in shared memory and run the same control flow
// on it.  The serial steps (the shifted Cholesky, the FP32 Jacobi rotations of H, the
// reductions and tests) run on every CTA alike and give bit-identical results, since every
// CTA executes the same instructions on the same data; each FP64 product and each
// triangular solve is split over the CTAs (rows, or columns), and every CTA stores its slice
// into the copies of all CTAs through distributed shared memory, a cluster barrier then
// publishing it.  A buffer that other CTAs write is never read across such a barrier: every
// broadcast phase starts after a barrier that follows the last local read of its target.
// In the FP32 Jacobi each CTA applies the rotations to its own slice of the rows of U.
constexpr int RRC_SIZE = 8;   // CTAs per cluster (the portable maximum)
constexpr int RRC_MAX = 72;   // largest subspace of the clustered form (its five m x m buffers fit)

namespace cg = cooperative_groups;

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }

// v stored at the address p (a shared-memory buffer) in every CTA of the cluster
__device__ __forceinline__ void cl_bcast(double* p, double v) {
    cg::cluster_group cl = cg::this_cluster();
#pragma unroll
    for (int r = 0; r < RRC_SIZE; ++r) *cl.map_shared_rank(p, r) = v;
}

// packed lower triangle: element (i, j), j <= i
__device__ __forceinline__ int lp(int i, int j) { return i * (i + 1) / 2 + j; }

// In-place Cholesky of the packed lower triangle K (m x m); false on a pivot <= rel_tol * scale.
// Right-looking.  The pivot takes one reciprocal square root (r = d rsqrt(d)), and the trailing
// update walks the lower triangle of the trailing block as one flat index, so that the FP64
// pipe (the scarce unit here) sees no idle lanes.
__device__ bool chol_packed(double* K, int m, double rel_tol, double scale, int* flag, double* rpiv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < m; ++j) {
        __syncthreads();
        if (tid == 0) {
            const double d = K[lp(j, j)];
            if (!(d > rel_tol * scale)) *flag = 1;
            else {
                const double ri = rsqrt(d);
                K[lp(j, j)] = d * ri;
                *rpiv = ri;
            }
        }
        __syncthreads();
        if (*flag) return false;
        const double ri = *rpiv;
        for (int i = j + 1 + tid; i < m; i += nt) K[lp(i, j)] *= ri;
        __syncthreads();
        const int r = m - j - 1;
        for (int t = tid; t < r * (r + 1) / 2; t += nt) {
            int a = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while (a * (a + 1) / 2 > t) --a;
            while ((a + 1) * (a + 2) / 2 <= t) ++a;
            const int i = j + 1 + a, l = j + 1 + t - a * (a + 1) / 2;  // j < l <= i
            K[lp(i, l)] = fma(-K[lp(i, j)], K[lp(l, j)], K[lp(i, l)]);
        }
    }
    __syncthreads();
    return true;
}

// Triangular solves of a warp with the unit lower factor Ls = L D^-1 (packed, diagonal
// unused): L x = b is Ls y = b with x = D^-1 y, and L^T c = u is Ls^T c = D^-1 u.  Column-
// oriented substitution: element i is final once the elements before it have updated it; the
// lane holding it broadcasts it and it updates the ones after it.  Three elements per lane
// (m <= 96); a block of 32 elements with none left to update skips the step.
// warp_lsolve_unit: Ls y = b, element r = m - 1 - (lane + 32 k) in x_k (the partial block
// holds the first rows and drops out first).
__device__ __forceinline__ void warp_lsolve_unit(const double* Ls, int m, double& x0, double& x1, double& x2) {
    const int lane = threadIdx.x & 31;
    const int r0 = m - 1 - lane, r1 = r0 - 32, r2 = r0 - 64;
    for (int i = 0; i < m - 1; ++i) {
        const int idx = m - 1 - i, k = idx >> 5, src = idx & 31;
        const double yi = __shfl_sync(0xffffffffu, k == 0 ? x0 : (k == 1 ? x1 : x2), src);
        if (r0 > i) x0 = fma(-Ls[lp(r0, i)], yi, x0);
        if (m - 33 > i && r1 > i) x1 = fma(-Ls[lp(r1, i)], yi, x1);
        if (m - 65 > i && r2 > i) x2 = fma(-Ls[lp(r2, i)], yi, x2);
    }
}

// warp_usolve_unit: Ls^T c = v, element r = lane + 32 k in x_k.
__device__ __forceinline__ void warp_usolve_unit(const double* Ls, int m, double& x0, double& x1, double& x2) {
    const int lane = threadIdx.x & 31;
    const int r0 = lane, r1 = lane + 32, r2 = lane + 64;
    for (int i = m - 1; i > 0; --i) {
        const int k = i >> 5, src = i & 31;
        const double ci = __shfl_sync(0xffffffffu, k == 0 ? x0 : (k == 1 ? x1 : x2), src);
        if (r0 < i) x0 = fma(-Ls[lp(i, r0)], ci, x0);
        if (i > 32 && r1 < i) x1 = fma(-Ls[lp(i, r1)], ci, x1);
        if (i > 64 && r2 < i) x2 = fma(-Ls[lp(i, r2)], ci, x2);
    }
}

// FP32 parallel cyclic Jacobi with the pairing, rotations, fused 2 x 2 block update and
// stopping rules of jacobi_sym_t, for the clustered kernel.  The round is latency-bound (a few
// warps, each a chain of dependent shared-memory accesses), so each thread keeps its work item
// for the whole solve in registers: block (a, b), a <= b, of the pairing, or one (pair, row) of
// the rows [u0, u1) of U that this CTA updates (rows of U evolve independently); the pairs of
// a round are computed, not loaded.  rot holds the (c, s) of each pair of the current round.
__device__ __forceinline__ void jac_pair(int s, int i, int me, int& p, int& q) {
    if (i == 0) { p = me - 1; q = s; }
    else {
        p = s + i;
        if (p >= me - 1) p -= me - 1;
        q = s - i;
        if (q < 0) q += me - 1;
    }
    if (p > q) { const int x = p; p = q; q = x; }
}

// work item t of a round: block (x, y) = (a, b), a <= b, for t < nblk (triangular order
// t = b (b + 1) / 2 + a), else pair x and row y of U
__device__ __forceinline__ void jac_item(int t, int nblk, int nu, int u0, int& x, int& y) {
    if (t < nblk) {
        int b = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (b * (b + 1) / 2 > t) --b;
        while ((b + 1) * (b + 2) / 2 <= t) ++b;
        x = t - b * (b + 1) / 2;
        y = b;
    } else {
        const int tu = t - nblk;
        x = tu / nu;
        y = u0 + tu - x * nu;
    }
}

__device__ __noinline__ int jacobi32_cl(float* H, float* U, int m, int ld, int u0, int u1, float2* rot,
                                        double* red, double tol2, int max_sweeps) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nu = u1 - u0;
    for (int t = tid; t < nu * m; t += nt) {
        const int i = u0 + t / m, j = t % m;
        U[i * ld + j] = (i == j) ? 1.0f : 0.0f;
    }
    const int me = (m + 1) & ~1;
    const int half = me / 2;
    const int nblk = half * (half + 1) / 2;
    const int nwork = nblk + half * nu;
    // this thread's first work item, decoded once
    int x0 = 0, y0 = 0;
    if (tid < nwork) jac_item(tid, nblk, nu, u0, x0, y0);
    int sweep = 0;
    double prev_off = 0.0;
    for (; sweep < max_sweeps; ++sweep) {
        __syncthreads();
        float off = 0.0f, tot = 0.0f;
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            const float h = H[i * ld + j];
            tot += h * h;
            if (i != j) off += h * h;
        }
        double offd = off, totd = tot;
        block_sum2(offd, totd, red);
        if (!(offd > tol2 * totd) || me < 2) break;
        if (sweep >= 2 && offd > 0.25 * prev_off) break;  // FP32 rounding floor reached
        prev_off = offd;
        for (int s = 0; s < me - 1; ++s) {
            for (int i = tid; i < half; i += nt) {
                int p, q;
                jac_pair(s, i, me, p, q);
                float c = 1.0f, sn = 0.0f;
                if (q < m) {
                    const float apq = H[p * ld + q], app = H[p * ld + p], aqq = H[q * ld + q];
                    if (fabsf(apq) > 1e-30f && apq * apq > 1e-18f * fabsf(app * aqq)) {
                        // the hardware reciprocal square root and division (a few ulp): a
                        // rotation stays orthogonal to that order whatever its angle, and the
                        // FP64 refinement takes the FP32 result from there
                        const float d = aqq - app, a2 = 2.0f * apq;
                        const float h2 = fmaf(d, d, a2 * a2);
                        const float tt = __fdividef(d >= 0.0f ? a2 : -a2, fabsf(d) + h2 * rsqrtf(h2));
                        c = rsqrtf(fmaf(tt, tt, 1.0f));
                        sn = tt * c;
                    }
                }
                rot[i] = make_float2(c, sn);
            }
            __syncthreads();
            for (int t = tid; t < nwork; t += nt) {
                int x, y;
                if (t == tid) { x = x0; y = y0; }
                else jac_item(t, nblk, nu, u0, x, y);
                if (t >= nblk) {
                    // U <- U J on this CTA's row y, pair x
                    int p, q;
                    jac_pair(s, x, me, p, q);
                    if (q >= m) continue;
                    const float2 r = rot[x];
                    const float up = U[y * ld + p], uq = U[y * ld + q];
                    U[y * ld + p] = r.x * up - r.y * uq;
                    U[y * ld + q] = r.y * up + r.x * uq;
                    continue;
                }
                const int aa = x, b = y;
                int pa, qa, pb, qb;
                jac_pair(s, aa, me, pa, qa);
                jac_pair(s, b, me, pb, qb);
                const bool va = qa < m, vb = qb < m;  // q = m marks the dummy player (odd m)
                const float2 ra = rot[aa], rb = rot[b];
                const float h00 = H[pa * ld + pb];
                const float h01 = vb ? H[pa * ld + qb] : 0.0f;
                const float h10 = va ? H[qa * ld + pb] : 0.0f;
                const float h11 = (va && vb) ? H[qa * ld + qb] : 0.0f;
                const float r00 = ra.x * h00 - ra.y * h10, r01 = ra.x * h01 - ra.y * h11;
                const float r10 = ra.y * h00 + ra.x * h10, r11 = ra.y * h01 + ra.x * h11;
                const float o00 = rb.x * r00 - rb.y * r01, o01 = rb.y * r00 + rb.x * r01;
                const float o10 = rb.x * r10 - rb.y * r11, o11 = rb.y * r10 + rb.x * r11;
                if (aa == b) {
                    const float od = 0.5f * (o01 + o10);
                    H[pa * ld + pa] = o00;
                    if (va) {
                        H[pa * ld + qa] = od;
                        H[qa * ld + pa] = od;
                        H[qa * ld + qa] = o11;
                    }
                } else {
                    H[pa * ld + pb] = o00;
                    H[pb * ld + pa] = o00;
                    if (vb) { H[pa * ld + qb] = o01; H[qb * ld + pa] = o01; }
                    if (va) { H[qa * ld + pb] = o10; H[pb * ld + qa] = o10; }
                    if (va && vb) { H[qa * ld + qb] = o11; H[qb * ld + qa] = o11; }
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();
    return sweep;
}

// One Ogita-Aishima step (same arithmetic as oa_refine above) with every O(m^3) product and
// every O(m^2) step split over the cluster: T = H G and G (I + E) by rows, S = G^T T and
// R = I - G^T G by upper-triangle entries, the separation test and E by entries; each slice
// is stored into every CTA, and each CTA stores its partial sums (of S, R and E squared) and
// its test result into slot `rank` of every CTA, which all add in the same order.  G (m x m)
// and T swap roles on success (*G then holds the refined vectors); W (m x ld) is scratch and
// holds E off its diagonal at the end, dE (m) the diagonal; nh = ||H||_F^2; flags has
// RRC_SIZE + 1 entries, the last one the reason of a failed step.  Entered and left just
// after a cluster barrier.
__device__ __noinline__ bool oa_refine_cl(const double* H, int ld, double*& G, double*& T, double* W, int m, double* lam,
                             double nh, double* red, double (*part)[RRC_SIZE], int* flags, double* dE,
                             double* scal, double* corr, long long* pc) {
    const int tid = threadIdx.x, nt = blockDim.x;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int i0 = rank * m / RRC_SIZE, i1 = (rank + 1) * m / RRC_SIZE;
    const int ntri = m * (m + 1) / 2;
    const int t0 = (int)((long long)rank * ntri / RRC_SIZE), t1 = (int)((long long)(rank + 1) * ntri / RRC_SIZE);
    const int e0 = rank * m * m / RRC_SIZE, e1 = (rank + 1) * m * m / RRC_SIZE;
    // T = H G, rows [i0, i1)
    for (int t = tid; t < (i1 - i0) * m; t += nt) {
        const int i = i0 + t / m, j = t % m;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(H[i * ld + k], G[k * m + j], acc);
        cl_bcast(&T[i * m + j], acc);
    }
    cl_sync();
    if (tid == 0) pc[0] = clock64();
    // W = S = G^T T, upper-triangle entries [t0, t1), mirrored; partial sum of the squares of
    // its off-diagonal entries
    double so = 0.0, z = 0.0, z2 = 0.0;
    for (int t = t0 + tid; t < t1; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], T[k * m + j], acc);
        cl_bcast(&W[i * ld + j], acc);
        if (i != j) {
            cl_bcast(&W[j * ld + i], acc);
            so = fma(2.0 * acc, acc, so);
        }
    }
    block_sum3(so, z, z2, red);
    if (tid == 0) cl_bcast(&part[0][rank], so);
    cl_sync();
    if (tid == 0) pc[1] = clock64();
    // T = R = I - G^T G, same split (every CTA has finished reading T above)
    double sr = 0.0;
    z = z2 = 0.0;
    for (int t = t0 + tid; t < t1; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], G[k * m + j], acc);
        const double r = (i == j ? 1.0 : 0.0) - acc;
        cl_bcast(&T[i * m + j], r);
        if (i != j) cl_bcast(&T[j * m + i], r);
        sr = fma(i != j ? 2.0 * r : r, r, sr);
    }
    block_sum3(sr, z, z2, red);
    if (tid == 0) cl_bcast(&part[1][rank], sr);
    cl_sync();
    if (tid == 0) pc[2] = clock64();
    // lam and the diagonal of E (0.5 R_ii) kept aside: the E stores below leave the diagonal
    // of W (S_ii) alone, and T (R) is not written before the next barrier
    for (int i = tid; i < m; i += nt) {
        lam[i] = W[i * ld + i] / (1.0 - T[i * m + i]);
        dE[i] = 0.5 * T[i * m + i];
    }
    __syncthreads();
    // scalars once, by warp 0 (FP64 work repeated on every thread costs the FP64 pipe):
    // ||S - diag(lam)||^2 = off-diagonal part + diagonal terms, ||R||^2, the test on a poor
    // start, and the rounding-level gap
    if (tid < 32) {
        double d2 = 0.0;
        for (int i = tid; i < m; i += 32) {
            const double d = W[i * ld + i] - lam[i];
            d2 = fma(d, d, d2);
        }
        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        if (tid == 0) {
            double ns = d2, nr = 0.0;
            for (int r = 0; r < RRC_SIZE; ++r) { ns += part[0][r]; nr += part[1][r]; }
            scal[0] = (sqrt(nr) > 1e-3 || sqrt(ns) > 1e-3 * sqrt(nh)) ? 2.0 : 0.0;
            scal[1] = 1e-13 * sqrt(nh);
        }
    }
    __syncthreads();
    const int poor = (int)scal[0];
    const double tiny = scal[1];
    // separation test and E on the off-diagonal entries [e0, e1): a pair coupled by more than
    // 1 % of its gap, or eigenvalues equal to rounding, cannot be separated by the step
    int bad = 0;
    double ne = 0.0;
    z = z2 = 0.0;
    for (int t = e0 + tid; t < e1; t += nt) {
        const int i = t / m, j = t % m;
        double e = dE[i];
        if (i != j) {
            const double g = lam[j] - lam[i];
            const double sij = W[i * ld + j];
            const double cpl = fmax(fabs(sij + lam[j] * T[i * m + j]), fabs(sij + lam[i] * T[i * m + j]));
            if (fabs(g) <= tiny || cpl > 0.01 * fabs(g)) bad = 1;
            // 1 / gap: FP32 reciprocal and one Newton step (relative error ~1e-14; E is a
            // correction of FP32 size, so its own relative accuracy need not be FP64's)
            double rg = (double)__frcp_rn((float)g);
            rg = rg * fma(-g, rg, 2.0);
            e = (sij + lam[j] * T[i * m + j]) * rg;
            if (!bad) cl_bcast(&W[i * ld + j], e);  // the owner of (i, j) alone reads S_ij
        }
        ne = fma(e, e, ne);
    }
    bad = __syncthreads_or(bad);
    block_sum3(ne, z, z2, red);
    if (tid == 0) {
        cl_bcast(&part[2][rank], ne);
        for (int r = 0; r < RRC_SIZE; ++r) *cl.map_shared_rank(&flags[rank], r) = poor ? poor : bad;
    }
    cl_sync();
    if (tid == 0) pc[3] = clock64();
    if (tid == 0) {
        int f = 0;
        double x = 0.0;
        for (int r = 0; r < RRC_SIZE; ++r) {
            f = max(f, flags[r]);
            x += part[2][r];
        }
        flags[RRC_SIZE] = f;  // why a step fails: 1 close eigenvalues, 2 a start too far off
        scal[0] = sqrt(x);
    }
    __syncthreads();
    if (flags[RRC_SIZE]) return false;  // the same on every CTA: no barrier is skipped by one CTA alone
    const double ne_sqrt = scal[0];
    // T = G (I + E), rows [i0, i1) (the diagonal of E from dE: W_jj still holds S_jj)
    for (int t = tid; t < (i1 - i0) * m; t += nt) {
        const int i = i0 + t / m, j = t % m;
        const double gij = G[i * m + j];
        double acc = fma(gij, dE[j] - W[j * ld + j], gij);
        for (int k = 0; k < m; ++k) acc = fma(G[i * m + k], W[k * ld + j], acc);
        cl_bcast(&T[i * m + j], acc);
    }
    cl_sync();
    if (tid == 0) pc[4] = clock64();
    double* x = G;
    G = T;
    T = x;
    *corr = ne_sqrt;
    return true;
}

// Clustered form of block_mixed_eig (same contract and return code).  G and T are m x m
// shared-memory buffers at the same offsets in every CTA.
__device__ int mixed_eig_cl(double* H, double* U, int m, int ld, double* G, double* T, double* rot, int* pq,
                            double* red, double tol32, long long* pclk) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rank = (int)cg::this_cluster().block_rank();
    const int u0 = rank * m / RRC_SIZE, u1 = (rank + 1) * m / RRC_SIZE;
    float* H32 = reinterpret_cast<float*>(U);  // two m x ld float matrices fill U's doubles
    float* U32 = H32 + (size_t)m * ld;
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        H32[i * ld + j] = (float)H[i * ld + j];
    }
    const int s32 = jacobi32_cl(H32, U32, m, ld, u0, u1, reinterpret_cast<float2*>(rot), red, tol32, 16);
    if (tid == 0) pclk[0] = clock64();
    // G = the FP32 eigenvectors: this CTA's rows, stored into every CTA
    for (int t = tid; t < (u1 - u0) * m; t += nt) {
        const int i = u0 + t / m, j = t % m;
        cl_bcast(&G[i * m + j], (double)U32[i * ld + j]);
    }
    cl_sync();
    if (tid == 0) pclk[1] = clock64();
    double* lam = rot;  // free once the FP32 stage is done
    __shared__ double part[3][RRC_SIZE];
    __shared__ int flags[RRC_SIZE + 1];
    __shared__ double dE[RRC_MAX];
    __shared__ double scal[2];
    double nh = 0.0, z0 = 0.0, z1 = 0.0;
    for (int t = tid; t < m * m; t += nt) {
        const double h = H[(t / m) * ld + t % m];
        nh = fma(h, h, nh);
    }
    block_sum3(nh, z0, z1, red);
    double corr = 1.0;
    bool ok = true;
    int steps = 0;
    while (steps < 2 && ok && corr > 1e-6) {
        ok = oa_refine_cl(H, ld, G, T, U, m, lam, nh, red, part, flags, dE, scal, &corr, pclk + 4 + 5 * steps);
        ++steps;
        if (tid == 0) pclk[1 + steps] = clock64();
    }
    if (ok && corr <= 1e-6) {
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            U[i * ld + j] = G[t];
            H[i * ld + j] = (i == j) ? lam[i] : 0.0;
        }
        __syncthreads();
        return 100 * s32 + 50 + steps;
    }
    // fallback (close eigenvalues): the one-CTA path on every CTA alike, from the current G
    const int fallback = ok ? 3 : flags[RRC_SIZE];
    for (int ns = 0; ns < 2; ++ns) {
        block_gemm(T, m, G, m, true, G, m, m);
        __syncthreads();
        for (int t = tid; t < m * m; t += nt) T[t] = (t / m == t % m ? 1.5 : 0.0) - 0.5 * T[t];
        __syncthreads();
        block_gemm(U, ld, G, m, false, T, m, m);
        __syncthreads();
        for (int t = tid; t < m * m; t += nt) G[t] = U[(t / m) * ld + t % m];
        __syncthreads();
    }
    block_gemm(T, m, H, ld, false, G, m, m);
    __syncthreads();
    for (int t = tid; t < m * (m + 1) / 2; t += nt) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        const int i = t - j * (j + 1) / 2;
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(G[k * m + i], T[k * m + j], acc);
        H[i * ld + j] = acc;
        H[j * ld + i] = acc;
    }
    __syncthreads();
    const int s64 = block_jacobi_sym(H, U, m, ld, rot, pq, red, 1e-26);
    block_gemm(T, m, G, m, false, U, ld, m);
    __syncthreads();
    for (int t = tid; t < m * m; t += nt) U[(t / m) * ld + t % m] = T[t];
    __syncthreads();
    return 100 * s32 + 10 * fallback + s64;
}

__global__ void __cluster_dims__(RRC_SIZE, 1, 1) __launch_bounds__(RR_THREADS, 1) rr_cluster_kernel(RRArgs a) {
    extern __shared__ double sm[];
    __shared__ double rot[2 * 64 + 2];
    __shared__ int pq[2 * 64 + 2];
    __shared__ double red[104];
    __shared__ int inv[RRC_MAX];
    __shared__ int flag, npos_sh;
    __shared__ double rpiv;
    __shared__ long long clk[20];  // phase clocks of thread 0 of CTA 0 (PPRPA_RR_PROF)
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, w = tid >> 5, nw = nt >> 5;
    const int rank = (int)cg::this_cluster().block_rank();
    const int m = a.m, ld = a.ld;
    const int lh = rr_ld(m, a.pad);
    double* H = sm;
    double* U = H + (size_t)m * lh;
    double* G = U + (size_t)m * lh;
    double* T = G + (size_t)m * m;
    double* Kc = T + (size_t)m * m;  // packed lower triangle of the Cholesky factor
    double* rd = Kc + (size_t)m * (m + 1) / 2;
    cl_sync();  // every CTA of the cluster runs before any store into its shared memory
    if (tid == 0) clk[0] = clock64();
    if (rank == 0 && tid == 0) a.info[0] = DEV_NOTPD;
    double sc = 0.0;
    for (int i = tid; i < m; i += nt)
        sc = fmax(sc, fabs(a.G[i * ld + i] + (a.Go ? a.Go[i * ld + i] : 0.0)) + fabs(a.S[i * ld + i]));
    sc = block_max(sc, red);
    const double scale = sc > 0.0 ? sc : 1.0;
    int used = -1;
    double mu = 0.0;
    for (int c = 0; c < a.nmu && used < 0; ++c) {
        mu = a.mus[c];
        // K = sym(G) - mu S, lower triangle (S: upper triangle valid)
        for (int t = tid; t < m * m; t += nt) {
            const int i = t / m, j = t % m;
            if (j > i) continue;
            double g = 0.5 * (a.G[i * ld + j] + a.G[j * ld + i]);
            if (a.Go) g += 0.5 * (a.Go[i * ld + j] + a.Go[j * ld + i]);
            Kc[lp(i, j)] = g - mu * a.S[j * ld + i];
        }
        if (tid == 0) flag = 0;
        __syncthreads();
        if (chol_packed(Kc, m, 1e-13, scale, &flag, &rpiv)) used = c;
        __syncthreads();
    }
    if (used < 0) {
        if (rank == 0 && tid == 0) { a.info[0] = DEV_NOTPD; a.info[1] = mu; }
        cl_sync();
        return;
    }
    if (tid == 0) clk[1] = clock64();
    for (int i = tid; i < m; i += nt) rd[i] = 1.0 / Kc[lp(i, i)];
    __syncthreads();
    // Lc = Ls D: columns scaled to a unit diagonal
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        if (j < i) Kc[lp(i, j)] *= rd[j];
    }
    __syncthreads();
    // X = Lc^-1 S into G: a warp per column, the columns dealt over the cluster
    for (int col = rank + RRC_SIZE * w; col < m; col += RRC_SIZE * nw) {
        double x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = m - 1 - lane - 32 * k;
            x[k] = r >= 0 ? (r <= col ? a.S[r * ld + col] : a.S[col * ld + r]) : 0.0;
        }
        warp_lsolve_unit(Kc, m, x[0], x[1], x[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = m - 1 - lane - 32 * k;
            if (r >= 0) cl_bcast(&G[r * m + col], x[k] * rd[r]);
        }
    }
    cl_sync();
    // H = Lc^-1 X^T
    for (int col = rank + RRC_SIZE * w; col < m; col += RRC_SIZE * nw) {
        double x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = m - 1 - lane - 32 * k;
            x[k] = r >= 0 ? G[col * m + r] : 0.0;
        }
        warp_lsolve_unit(Kc, m, x[0], x[1], x[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = m - 1 - lane - 32 * k;
            if (r >= 0) cl_bcast(&H[r * lh + col], x[k] * rd[r]);
        }
    }
    cl_sync();
    for (int t = tid; t < m * m; t += nt) {
        const int i = t / m, j = t % m;
        if (i < j) {
            const double v = 0.5 * (H[i * lh + j] + H[j * lh + i]);
            H[i * lh + j] = v;
            H[j * lh + i] = v;
        }
    }
    __syncthreads();
    if (tid == 0) clk[2] = clock64();
    if (tid == 0) clk[6] = clk[7] = clk[8] = clk[9] = clk[2];
    const int sweeps = mixed_eig_cl(H, U, m, lh, G, T, rot, pq, red, a.tol32, clk + 6);
    if (tid == 0) clk[3] = clock64();
    // rank the positive kappas (descending) -> targets
    if (tid == 0) npos_sh = 0;
    __syncthreads();
    for (int i = tid; i < m; i += nt) {
        const double ki = H[i * lh + i];
        if (ki > 0.0) {
            int r = 0;
            for (int j = 0; j < m; ++j) {
                const double kj = H[j * lh + j];
                if (kj > 0.0 && (kj > ki || (kj == ki && j < i))) ++r;
            }
            inv[r] = i;
            atomicAdd(&npos_sh, 1);
        }
    }
    __syncthreads();
    const int npos = npos_sh;
    const int nk = min(a.nkeep, npos);
    if (tid == 0) clk[4] = clock64();
    // Ritz coefficients c = Lc^-T u / sqrt(kappa): a warp per kept root, dealt over the cluster
    for (int slot = rank + RRC_SIZE * w; slot < nk; slot += RRC_SIZE * nw) {
        const int i = inv[slot];
        const double kap = H[i * lh + i];
        double x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = lane + 32 * k;
            x[k] = r < m ? U[r * lh + i] * rd[r] : 0.0;
        }
        warp_usolve_unit(Kc, m, x[0], x[1], x[2]);
        const double f = 1.0 / sqrt(kap);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int r = lane + 32 * k;
            if (r < m) a.coef[(size_t)slot * m + r] = x[k] * f;
        }
        if (lane == 0) a.omega[slot] = mu + 1.0 / kap;
    }
    if (rank == 0 && tid == 0) {
        double kmin = 0.0, kmax = 0.0;
        for (int i = 0; i < m; ++i) {
            const double k = H[i * lh + i];
            if (k < kmin) kmin = k;
            if (k > kmax) kmax = k;
        }
        a.info[0] = (npos >= a.nwant) ? DEV_OK : DEV_FEWROOTS;
        a.info[1] = mu;
        a.info[2] = npos;
        a.info[3] = kmax > 0.0 ? mu + 1.0 / kmax : 1e300;
        a.info[4] = kmin < 0.0 ? mu + 1.0 / kmin : -1e300;
        a.info[5] = sweeps;
        if (a.prof) {
            clk[5] = clock64();
            printf("[rr-cl] m %d sweeps %d cycles: factor %lld solves %lld eig %lld (fp32 %lld to-G %lld oa %lld %lld) "
                   "rank %lld ritz %lld\n",
                   m, sweeps, clk[1] - clk[0], clk[2] - clk[1], clk[3] - clk[2], clk[6] - clk[2], clk[7] - clk[6],
                   clk[8] - clk[7], clk[9] - clk[8], clk[4] - clk[3], clk[5] - clk[4]);
            printf("[rr-cl] oa step 1: HG %lld S %lld R %lld E %lld G(I+E) %lld\n", clk[10] - clk[7], clk[11] - clk[10],
                   clk[12] - clk[11], clk[13] - clk[12], clk[14] - clk[13]);
        }
    }
    cl_sync();  // no CTA leaves while a store into it could still be in flight
}

// Eigensolver of the one-CTA kernels (PPRPA_EIG): 4 (default) FP32 Jacobi refined in FP64 by
// Ogita-Aishima steps where H and U fit in shared memory, with the path of 3 as its fallback;
// 3 mixed FP32 / FP64 Jacobi (Newton-Schulz orthonormalisation, FP64 Jacobi sweeps); 0 FP64
// Jacobi with the fused symmetric update (also the default beyond shared memory); 1 FP64 Jacobi
// with separate row and column passes; 2 Householder + implicit QR.
static int eig_method() {
    const char* v = getenv("PPRPA_EIG");
    return v ? atoi(v) : 4;
}

// Odd leading dimension of the shared-memory matrices unless PPRPA_RR_PAD=0.
static int rr_pad() {
    const char* v = getenv("PPRPA_RR_PAD");
    return v ? atoi(v) : 1;
}

int launch_rayleigh_ritz(const RRArgs& ain, cudaStream_t st) {
    RRArgs a = ain;
    a.eig = eig_method();
    if (a.m <= 0 || a.m > 1024) return set_error(PPRPA_ERR_ARG, "rayleigh_ritz: size must be 1..1024");
    a.pad = rr_pad();
    const char* tv = getenv("PPRPA_RR_TOL32");
    // the FP64 refinement by Ogita-Aishima steps separates only eigenvalues farther apart than
    // about twice the off-diagonal left by the FP32 stage: run that stage to its rounding floor
    // (it stops on stalling) before refining, or to 1e-5 of the norm before FP64 Jacobi
    a.tol32 = tv ? atof(tv) : (a.eig == 4 ? 1e-14 : 1e-10);
    const char* pv = getenv("PPRPA_RR_PROF");
    a.prof = pv ? atoi(pv) : 0;
    const char* cv = getenv("PPRPA_RR_CLUSTER");
    if (a.eig == 4 && a.m <= RRC_MAX && (cv ? atoi(cv) : 1) != 0) {
        // clustered form: H, U (odd leading dimension), G, T, the packed Cholesky factor and its
        // reciprocal pivots in each CTA's shared memory
        const auto bytes = [&](int m) {
            const int lh = rr_ld(m, a.pad);
            return sizeof(double) * ((size_t)2 * m * lh + (size_t)2 * m * m + (size_t)m * (m + 1) / 2 + m);
        };
        cudaFuncSetAttribute(rr_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes(RRC_MAX));
        rr_cluster_kernel<<<RRC_SIZE, RR_THREADS, bytes(a.m), st>>>(a);
        // a cluster that cannot be placed is a launch error, not a sticky one: the one-CTA
        // kernel below takes the call instead
        if (cudaGetLastError() == cudaSuccess) return PPRPA_OK;
    }
    const size_t smem = a.m <= RR_SMEM_MAX ? 2 * sizeof(double) * a.m * rr_ld(a.m, a.pad) : 0;
    // per device and cheap: set on every launch (several host threads may launch at once)
    cudaFuncSetAttribute(rayleigh_ritz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * sizeof(double) * RR_SMEM_MAX * (RR_SMEM_MAX + 1));
    rayleigh_ritz_kernel<<<1, RR_THREADS, smem, st>>>(a);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// Block orthonormalisation helper (Cholesky QR with dropping).
__global__ void __launch_bounds__(256) cholqr_small_kernel(const double* __restrict__ Gm, int k, double tol,
                                                           double* __restrict__ T, int* __restrict__ keep,
                                                           double* __restrict__ work) {
    // One CTA; every serial chain is O(k): the right-looking Cholesky takes k steps of parallel
    // column scaling and trailing updates, the inverse one column per thread.
    const int tid = threadIdx.x, nt = blockDim.x;
    double* Lc = work;            // k x k
    double* s = work + k * k;     // k
    __shared__ int drop_sh;
    for (int i = tid; i < k; i += nt) {
        const double d = Gm[i * k + i];
        s[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
        keep[i] = d > 0.0 ? 1 : 0;
    }
    __syncthreads();
    for (int t = tid; t < k * k; t += nt) {
        const int i = t / k, j = t % k;
        Lc[t] = (j <= i) ? Gm[t] * s[i] * s[j] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            const double d = Lc[j * k + j];  // the trailing updates of columns < j are applied
            drop_sh = (!keep[j] || !(d > tol)) ? 1 : 0;
            if (drop_sh) keep[j] = 0;
            else Lc[j * k + j] = sqrt(d);
        }
        __syncthreads();
        if (drop_sh) {  // dependent direction: row and column j become those of the identity
            for (int l = tid; l < k; l += nt) {
                if (l < j) Lc[j * k + l] = 0.0;
                if (l > j) Lc[l * k + j] = 0.0;
            }
            if (tid == 0) Lc[j * k + j] = 1.0;
            __syncthreads();
            continue;
        }
        const double piv = Lc[j * k + j];
        for (int i = j + 1 + tid; i < k; i += nt) Lc[i * k + j] /= piv;
        __syncthreads();
        const int r = k - j - 1;
        for (int t = tid; t < r * r; t += nt) {
            const int i = j + 1 + t / r, l = j + 1 + t % r;
            if (l <= i) Lc[i * k + l] -= Lc[i * k + j] * Lc[l * k + j];
        }
        __syncthreads();
    }
    // T = Lc^-1 diag(s), one column per thread; dropped rows zero
    for (int col = tid; col < k; col += nt) {
        for (int i = 0; i < k; ++i) {
            double v = (i == col) ? 1.0 : 0.0;
            for (int l = col; l < i; ++l) v -= Lc[i * k + l] * T[l * k + col];  // T[l][col] = 0 for l < col
            T[i * k + col] = (i < col) ? 0.0 : v / Lc[i * k + i];
        }
    }
    __syncthreads();
    for (int t = tid; t < k * k; t += nt) {
        const int i = t / k, col = t % k;
        T[t] = keep[i] ? T[t] * s[col] : 0.0;
    }
}

int launch_cholqr_small(const double* Gm, int k, double tol, double* T, int* keep, double* work,
                        cudaStream_t st) {
    if (k <= 0) return PPRPA_OK;
    if (k > 256) return set_error(PPRPA_ERR_ARG, "cholqr_small: block too large");
    cholqr_small_kernel<<<1, 256, 0, st>>>(Gm, k, tol, T, keep, work);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Symmetric eigendecomposition of `batch` matrices H (m x m each, row-major, `stride` doubles
// apart) by the one-CTA parallel Jacobi above, one CTA per matrix: H is overwritten (the
// eigenvalues end on its diagonal) and U receives the eigenvectors as columns.
// work: batch x 8192 doubles, iwork: batch x 1024 ints (m <= 1024).
__global__ void __launch_bounds__(1024, 1) sym_eig_kernel(double* H, double* U, int m, int64_t stride,
                                                          double* work, int* iwork, int eig) {
    const int b = blockIdx.x;
    double* w = work + (int64_t)b * 8192;
    if (eig == 0 || eig == 3 || eig == 4) block_jacobi_sym(H + b * stride, U + b * stride, m, m, w, iwork + (int64_t)b * 1024, w + 1024);
    else if (eig == 1) block_jacobi(H + b * stride, U + b * stride, m, m, w, iwork + (int64_t)b * 1024, w + 1024);
    else block_tridiag_eig(H + b * stride, U + b * stride, m, m, w);
}

int launch_sym_eig(double* H, double* U, int m, int batch, int64_t stride, double* work, int* iwork,
                   cudaStream_t st) {
    if (m <= 0 || batch <= 0) return PPRPA_OK;
    if (m > 1024) return set_error(PPRPA_ERR_ARG, "sym_eig: order above 1024");
    sym_eig_kernel<<<batch, 1024, 0, st>>>(H, U, m, stride, work, iwork, eig_method());
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa
