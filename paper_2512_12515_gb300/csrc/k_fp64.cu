// FP64 kernels: tiled GEMM and the HBM-bound elementwise steps of the ppRPA path.
//
// GB300 has a small FP64 pipe, so these kernels aim at keeping it busy with
// simple register tiling; everything here is either latency-bound (small
// shapes) or HBM-bound (pair packing, diagonal, residuals).
#include <cuda_fp8.h>

#include "kernels.h"

namespace pprpa {

// ---------------------------------------------------------------------------
// FP64 GEMM, 64x64 tile, 16-deep k slab, 256 threads, 4x4 outputs per thread.
constexpr int DG_BM = 64, DG_BN = 64, DG_BK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(Dgemm g) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int n0 = blockIdx.x * DG_BN, m0 = blockIdx.y * DG_BM;
    // blockIdx.z = ((batch * rsplit) + rslice) * splitk + kslice
    const int z = blockIdx.z;
    const int split = z % g.splitk;
    const int rs = (z / g.splitk) % g.rsplit;
    const int b = z / (g.splitk * g.rsplit);
    const int i2 = b % g.nb2, i1 = b / g.nb2;
    const double* A0 = g.A + i1 * g.sA1 + i2 * g.sA2;
    const double* B0 = g.B + i1 * g.sB1 + i2 * g.sB2;
    double* C = g.C + i1 * g.sC1 + i2 * g.sC2;
    int kchunk = (g.K + g.splitk - 1) / g.splitk;
    kchunk = (kchunk + DG_BK - 1) / DG_BK * DG_BK;
    const int kbeg = split * kchunk;
    const int kend = min(g.K, kbeg + kchunk);

    __shared__ double As[DG_BK][DG_BM + 1];
    __shared__ double Bs[DG_BK][DG_BN + 1];
    const int imax = min(4, (g.M - m0 + 15) / 16), jmax = min(4, (g.N - n0 + 15) / 16);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    // this CTA's slice of the reduction over batches r (all of them unless rsplit > 1)
    const int rper = (g.nr + g.rsplit - 1) / g.rsplit;
    const int r0 = rs * rper, r1 = min(g.nr, r0 + rper);
    for (int r = r0; r < r1; ++r) {
        const double* A = A0 + r * g.sAr;
        const double* B = B0 + r * g.sBr;
        for (int k0 = kbeg; k0 < kend; k0 += DG_BK) {
            for (int i = tid; i < DG_BM * DG_BK; i += 256) {
                int mm, kk;
                if (!g.transA) { mm = i / DG_BK; kk = i % DG_BK; }
                else { kk = i / DG_BM; mm = i % DG_BM; }
                const int64_t gm = m0 + mm, gk = k0 + kk;
                double v = 0.0;
                if (gm < g.M && gk < kend) v = g.transA ? A[gk * g.lda + gm] : A[gm * g.lda + gk];
                As[kk][mm] = v;
            }
            for (int i = tid; i < DG_BN * DG_BK; i += 256) {
                int nn, kk;
                if (!g.transB) { kk = i / DG_BN; nn = i % DG_BN; }
                else { nn = i / DG_BK; kk = i % DG_BK; }
                const int64_t gn = n0 + nn, gk = k0 + kk;
                double v = 0.0;
                if (gn < g.N && gk < kend) v = g.transB ? B[gn * g.ldb + gk] : B[gk * g.ldb + gn];
                Bs[kk][nn] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < DG_BK; ++kk) {
                double a[4], bb[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
                // 16-row / 16-column groups wholly outside C are skipped (uniform over the
                // CTA): an FP64 FMA is expensive here, and small outputs fill a fraction of a tile
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= imax) break;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j >= jmax) break;
                        acc[i][j] = fma(a[i], bb[j], acc[i][j]);
                    }
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t gm = m0 + ty + 16 * i;
        if (gm >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gn = n0 + tx + 16 * j;
            if (gn >= g.N) continue;
            double* c = C + gm * g.ldc + gn;
            if (g.splitk > 1 || g.rsplit > 1) {
                atomicAdd(c, g.alpha * acc[i][j]);
            } else {
                double v = g.alpha * acc[i][j];
                if (g.beta != 0.0) v += g.beta * (*c);
                *c = v;
            }
        }
    }
}

// Small FP64 products: few outputs and a moderate K, like the Davidson projections and
// combinations of a small problem.  FP64 runs at about two FMAs per clock per SM here, so a
// product of a few hundred thousand FMAs on the handful of CTAs its 64 x 64 tiles give takes
// tens of microseconds; these two kernels spread it over the GPU, without atomics.
// C = alpha A B^T + beta C, A (M x K, lda), B (N x K, ldb): a warp per output, lanes over K.
__global__ void __launch_bounds__(256) small_abt_kernel(Dgemm g) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)g.M * g.N;
    for (int64_t o = w; o < total; o += nw) {
        const int64_t i = o / g.N, j = o % g.N;
        const double* a = g.A + i * g.lda;
        const double* b = g.B + j * g.ldb;
        double sa[4] = {0.0, 0.0, 0.0, 0.0};
        int k = lane;
        for (; k + 96 < g.K; k += 128) {
            const double a0 = a[k], a1 = a[k + 32], a2 = a[k + 64], a3 = a[k + 96];
            const double b0 = b[k], b1 = b[k + 32], b2 = b[k + 64], b3 = b[k + 96];
            sa[0] = fma(a0, b0, sa[0]);
            sa[1] = fma(a1, b1, sa[1]);
            sa[2] = fma(a2, b2, sa[2]);
            sa[3] = fma(a3, b3, sa[3]);
        }
        for (; k < g.K; k += 32) sa[0] = fma(a[k], b[k], sa[0]);
        double acc = (sa[0] + sa[1]) + (sa[2] + sa[3]);
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            double* c = g.C + i * g.ldc + j;
            *c = g.beta == 0.0 ? g.alpha * acc : fma(g.beta, *c, g.alpha * acc);
        }
    }
}

// C = alpha op(A) B + beta C, op(A) (M x K) = A[i lda + k] or (transA) A[k lda + i], B (K x N,
// ldb): a warp per row of C and 32 consecutive columns, a lane per column.
__global__ void __launch_bounds__(256) small_ab_kernel(Dgemm g) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nch = (g.N + 31) / 32;
    const int64_t total = (int64_t)g.M * nch;
    const int64_t as = g.transA ? g.lda : 1, ai = g.transA ? 1 : g.lda;  // strides of op(A) over k, i
    for (int64_t o = w; o < total; o += nw) {
        const int64_t i = o / nch, n = (o % nch) * 32 + lane;
        const bool on = n < g.N;
        const double* a = g.A + i * ai;
        const double* b = g.B + n;
        // eight rows of B in flight per step: the loop is bound by the latency of these loads
        double sa[4] = {0.0, 0.0, 0.0, 0.0};
        int k = 0;
        if (on) {
            for (; k + 7 < g.K; k += 8) {
                double av[8], bv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    av[u] = a[(k + u) * as];
                    bv[u] = b[(int64_t)(k + u) * g.ldb];
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) sa[u & 3] = fma(av[u], bv[u], sa[u & 3]);
            }
            for (; k < g.K; ++k) sa[0] = fma(a[k * as], b[(int64_t)k * g.ldb], sa[0]);
            double* c = g.C + i * g.ldc + n;
            const double acc = (sa[0] + sa[1]) + (sa[2] + sa[3]);
            *c = g.beta == 0.0 ? g.alpha * acc : fma(g.beta, *c, g.alpha * acc);
        }
    }
}

int auto_splitk(int M, int N, int K, int batches) {
    const int64_t tiles = ceil_div(M, DG_BM) * ceil_div(N, DG_BN) * (int64_t)batches;
    const int64_t target = 4 * 152;
    if (tiles >= target) return 1;
    int64_t s = ceil_div(target, tiles);
    const int64_t kmax = ceil_div(K, DG_BK);  // at least one k-slab per split
    if (s > kmax) s = kmax;
    if (s > 1024) s = 1024;
    return s < 1 ? 1 : (int)s;
}

// C = beta * C over every output element of g (before the atomic accumulation of a launch
// whose reduction over batches is split).
__global__ void dgemm_scale_c_kernel(Dgemm g) {
    const int64_t per = (int64_t)g.M * g.N;
    const int64_t total = per * g.nb1 * g.nb2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / per, e = t % per;
        const int i1 = (int)(b / g.nb2), i2 = (int)(b % g.nb2);
        double* c = g.C + i1 * g.sC1 + i2 * g.sC2 + (e / g.N) * g.ldc + (e % g.N);
        *c = g.beta == 0.0 ? 0.0 : g.beta * *c;
    }
}

bool dgemm_small(const Dgemm& g) {
    const int64_t outs = (int64_t)g.M * g.N;
    return g.M > 0 && g.N > 0 && g.nr == 1 && g.nb1 == 1 && g.nb2 == 1 && g.K > 0 && g.K <= 8192 &&
           outs <= 65536 && outs * g.K <= ((int64_t)1 << 26) && !(g.transA && g.transB);
}

int dgemm(const Dgemm& gin, cudaStream_t st) {
    Dgemm g = gin;
    if (g.M <= 0 || g.N <= 0) return PPRPA_OK;
    // a single small product (at most 64 Ki outputs, K <= 8192, 2^26 FMAs) goes to the
    // small-product kernels; a split-K request of the caller means C += alpha op(A) op(B)
    const int64_t outs = (int64_t)g.M * g.N;
    if (dgemm_small(g)) {
        if (g.splitk > 1) g.beta = 1.0;
        g.splitk = 1;
        // warps per block: as few as spread the warps over every SM (each SM's FP64 pipe is
        // the scarce unit), at most 8
        const int64_t warps = g.transB ? outs : g.M * ceil_div(g.N, 32);
        const int wpb = (int)std::min<int64_t>(8, std::max<int64_t>(1, ceil_div(warps, 152)));
        const unsigned blocks = (unsigned)std::min<int64_t>(ceil_div(warps, wpb), 152 * 16);
        if (g.transB) small_abt_kernel<<<blocks, 32 * wpb, 0, st>>>(g);
        else small_ab_kernel<<<blocks, 32 * wpb, 0, st>>>(g);
        PP_CHECK_LAUNCH();
        return PPRPA_OK;
    }
    // FP64 arithmetic is scarce on this GPU: a launch with few output tiles and a long
    // reduction over batches (sum_r A_r B_r) spreads that reduction over CTAs, which then add
    // their partial sums atomically into C after C has been scaled by beta
    g.rsplit = 1;
    bool split = false;
    const int64_t tiles = ceil_div(g.N, DG_BN) * ceil_div(g.M, DG_BM) * (int64_t)g.nb1 * g.nb2;
    if (g.nr > 1 && g.splitk == 1) {
        if (tiles < 2 * 152) g.rsplit = (int)std::min<int64_t>(g.nr, ceil_div(2 * 152, tiles));
        split = g.rsplit > 1;
    } else if (g.nr == 1 && g.splitk == 1 && tiles < 152 && g.K >= 4 * DG_BK) {
        // the same for a single long product: its K range is split instead
        g.splitk = auto_splitk(g.M, g.N, g.K, g.nb1 * g.nb2);
        split = g.splitk > 1;
    }
    if (split) {
        const int64_t total = (int64_t)g.M * g.N * g.nb1 * g.nb2;
        dgemm_scale_c_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 8), 256, 0, st>>>(g);
        PP_CHECK_LAUNCH();
    }
    if (g.K <= 0 || g.nr <= 0) {
        // C = beta * C
        if (g.splitk > 1) return PPRPA_OK;
    }
    if (ceil_div(g.M, DG_BM) > 65535) return set_error(PPRPA_ERR_ARG, "dgemm: M too large");
    // the grid's z dimension (at most 65535) covers batches x K slices x reduction slices:
    // launch the batches in as many pieces as that needs
    const int64_t per_b = (int64_t)g.splitk * g.rsplit;
    if (per_b > 65535) return set_error(PPRPA_ERR_ARG, "dgemm: too many K / reduction slices");
    const int c2 = (int)std::min<int64_t>(g.nb2, 65535 / per_b);
    for (int b2 = 0; b2 < g.nb2; b2 += c2) {
        const int n2c = std::min(c2, g.nb2 - b2);
        const int c1 = (int)std::max<int64_t>(1, std::min<int64_t>(g.nb1, 65535 / (per_b * n2c)));
        for (int b1 = 0; b1 < g.nb1; b1 += c1) {
            Dgemm p = g;
            p.nb1 = std::min(c1, g.nb1 - b1);
            p.nb2 = n2c;
            p.A = g.A + b1 * g.sA1 + b2 * g.sA2;
            p.B = g.B + b1 * g.sB1 + b2 * g.sB2;
            p.C = g.C + b1 * g.sC1 + b2 * g.sC2;
            const int64_t zb = (int64_t)p.nb1 * p.nb2 * per_b;
            dim3 grid((unsigned)ceil_div(g.N, DG_BN), (unsigned)ceil_div(g.M, DG_BM), (unsigned)zb);
            dgemm_kernel<<<grid, 256, 0, st>>>(p);
            PP_CHECK_LAUNCH();
        }
    }
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
__global__ void extract_active_kernel(const double* __restrict__ Lfull, int naux, int nmo,
                                      const int* __restrict__ orb, int n,
                                      double* __restrict__ Lact) {
    const int64_t total = (int64_t)naux * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = t % n;
        const int p = (t / n) % n;
        const int64_t P = t / ((int64_t)n * n);
        Lact[t] = Lfull[(P * nmo + orb[p]) * nmo + orb[q]];
    }
}

int launch_extract_active(const double* Lfull, int naux, int nmo, const int* orb, int n,
                          double* Lact, cudaStream_t st) {
    const int64_t total = (int64_t)naux * n * n;
    if (!total) return PPRPA_OK;
    extract_active_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0,
                            st>>>(Lfull, naux, nmo, orb, n, Lact);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// Diagonal of M (singlet: ((pp|qq) + (pq|pq)) / (1 + d_pq); triplet: (pp|qq) - (pq|pq)).
__global__ void ldiag_kernel(const double* __restrict__ L, int naux, int n, double* __restrict__ Ld) {
    const int64_t total = (int64_t)naux * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int p = t % n;
        const int64_t P = t / n;
        Ld[t] = L[(P * n + p) * n + p];
    }
}

__global__ void diag_kernel(const double* __restrict__ L, const double* __restrict__ Ld, int naux,
                            int n, const double* __restrict__ eps, const int* __restrict__ pp,
                            const int* __restrict__ pq, int nvv, int N, int mult,
                            double* __restrict__ D) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= N) return;
    const int p = pp[I], q = pq[I];
    double J = 0.0, K = 0.0;
    for (int P = 0; P < naux; ++P) {
        const double lpq = L[((int64_t)P * n + p) * n + q];
        J = fma(Ld[(int64_t)P * n + p], Ld[(int64_t)P * n + q], J);
        K = fma(lpq, lpq, K);
    }
    const double w = I < nvv ? 1.0 : -1.0;
    double two_e;
    if (mult == 1) two_e = (J + K) / (p == q ? 2.0 : 1.0);
    else two_e = J - K;
    D[I] = w * (eps[p] + eps[q]) + two_e;
}

int launch_diag(const double* L, int naux, int n, const double* eps, const int* pp,
                const int* pq, int nvv, int N, int mult, double* D, double* work,
                cudaStream_t st) {
    if (N <= 0) return PPRPA_OK;
    const int64_t tot = (int64_t)naux * n;
    ldiag_kernel<<<(unsigned)std::min<int64_t>(ceil_div(tot, 256), 4096), 256, 0, st>>>(L, naux, n, work);
    PP_CHECK_LAUNCH();
    diag_kernel<<<(unsigned)ceil_div(N, 128), 128, 0, st>>>(L, work, naux, n, eps, pp, pq, nvv, N,
                                                           mult, D);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// Pair packing (FP64 sigma path).  Zt must be zeroed by the caller.
__global__ void unpack_f64_kernel(const double* __restrict__ z, int k, int N,
                                  const int* __restrict__ pp, const int* __restrict__ pq, int n,
                                  int mult, double* __restrict__ Zt) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const int p = pp[I], q = pq[I];
        const double v = z[t];
        double* Z = Zt + j * (int64_t)n * n;
        if (mult == 1) {
            if (p == q) Z[(int64_t)p * n + p] = 1.4142135623730951 * v;
            else { Z[(int64_t)p * n + q] = v; Z[(int64_t)q * n + p] = v; }
        } else {
            Z[(int64_t)p * n + q] = v;
            Z[(int64_t)q * n + p] = -v;
        }
    }
}

int launch_unpack_f64(const double* z, int k, int N, const int* pp, const int* pq, int n,
                      int mult, double* Zt, cudaStream_t st) {
    const int64_t total = (int64_t)k * N;
    if (!total) return PPRPA_OK;
    unpack_f64_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(
        z, k, N, pp, pq, n, mult, Zt);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

__global__ void pack_f64_kernel(const double* __restrict__ O, const double* __restrict__ z, int k,
                                int N, int nvv, const int* __restrict__ pp,
                                const int* __restrict__ pq, int n, const double* __restrict__ eps,
                                int mult, double* __restrict__ sigma) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const int p = pp[I], q = pq[I];
        double o = O[j * (int64_t)n * n + (int64_t)p * n + q];
        if (mult == 1 && p == q) o *= 0.7071067811865476;
        const double w = I < nvv ? 1.0 : -1.0;
        sigma[t] = fma(w * (eps[p] + eps[q]), z[t], o);
    }
}

int launch_pack_f64(const double* O, const double* z, int k, int N, int nvv, const int* pp,
                    const int* pq, int n, const double* eps, int mult, double* sigma,
                    cudaStream_t st) {
    const int64_t total = (int64_t)k * N;
    if (!total) return PPRPA_OK;
    pack_f64_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(
        O, z, k, N, nvv, pp, pq, n, eps, mult, sigma);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// BF16 layouts for the tensor-core sigma.
PadMap make_padmap(int no, int nv) {
    PadMap m;
    m.no = no;
    m.nv = nv;
    m.no_p = (int)round_up(no, 8);
    m.nv_p = (int)round_up(nv, 8);
    m.n_pad = m.no_p + m.nv_p;
    return m;
}

__device__ __forceinline__ int pad_to_orb(const PadMap& pm, int r) {
    if (r < pm.no) return r;
    if (r >= pm.no_p && r < pm.no_p + pm.nv) return pm.no + (r - pm.no_p);
    return -1;
}

__global__ void quantize_bf16_kernel(const double* __restrict__ L, int naux, int n, PadMap pm,
                                     __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const int64_t np = pm.n_pad;
    const int64_t total = (int64_t)naux * np * np;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = t % np;
        const int r = (t / np) % np;
        const int64_t P = t / (np * np);
        const int p = pad_to_orb(pm, r), q = pad_to_orb(pm, c);
        double x = 0.0;
        if (p >= 0 && q >= 0) x = L[(P * n + p) * n + q];
        const __nv_bfloat16 h = __double2bfloat16(x);
        hi[t] = h;
        if (lo) lo[t] = __double2bfloat16(x - (double)__bfloat162float(h));
    }
}

int launch_quantize_bf16(const double* L, int naux, int n, PadMap pm, __nv_bfloat16* hi,
                         __nv_bfloat16* lo, cudaStream_t st) {
    const int64_t total = (int64_t)naux * pm.n_pad * pm.n_pad;
    if (!total) return PPRPA_OK;
    quantize_bf16_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 64), 256, 0,
                           st>>>(L, naux, n, pm, hi, lo);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Writes the transposed pair matrix Zt^T of each vector into the B operand stacks.
// The caller zeroes the stacks (padding and the triplet diagonal stay zero).
__global__ void unpack_bf16_kernel(const double* __restrict__ z, int k, int N, int nvv,
                                   const int* __restrict__ pp, const int* __restrict__ pq,
                                   PadMap pm, int mult, __nv_bfloat16* __restrict__ xs_hi,
                                   __nv_bfloat16* __restrict__ xs_lo, int ldx,
                                   __nv_bfloat16* __restrict__ ys_hi,
                                   __nv_bfloat16* __restrict__ ys_lo, int ldy) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const double v = z[t];
        int p = pp[I], q = pq[I];
        __nv_bfloat16 *hi, *lo;
        int64_t rows, ld;
        // each vector owns a block of rows padded to a multiple of 8 (nv_p / no_p); the
        // padding rows stay zero
        if (I < nvv) { p -= pm.no; q -= pm.no; hi = xs_hi; lo = xs_lo; rows = pm.nv_p; ld = ldx; }
        else { hi = ys_hi; lo = ys_lo; rows = pm.no_p; ld = ldy; }
        const int64_t base = j * rows * ld;
        // Zt[p][q] (p <= q) and Zt[q][p]; stack entry [c][d] = Zt[d][c].
        double zpq, zqp;
        if (mult == 1) {
            zpq = (p == q) ? 1.4142135623730951 * v : v;
            zqp = zpq;
        } else {
            zpq = v;
            zqp = -v;
        }
        const int64_t e1 = base + (int64_t)q * ld + p;  // [c=q][d=p] = Zt[p][q]
        const int64_t e2 = base + (int64_t)p * ld + q;  // [c=p][d=q] = Zt[q][p]
        __nv_bfloat16 h1 = __double2bfloat16(zpq);
        hi[e1] = h1;
        if (lo) lo[e1] = __double2bfloat16(zpq - (double)__bfloat162float(h1));
        if (p != q) {
            __nv_bfloat16 h2 = __double2bfloat16(zqp);
            hi[e2] = h2;
            if (lo) lo[e2] = __double2bfloat16(zqp - (double)__bfloat162float(h2));
        }
    }
}

int launch_unpack_bf16(const double* z, int k, int N, int nvv, const int* pp, const int* pq,
                       PadMap pm, int mult, __nv_bfloat16* xs_hi, __nv_bfloat16* xs_lo, int ldx,
                       __nv_bfloat16* ys_hi, __nv_bfloat16* ys_lo, int ldy, cudaStream_t st) {
    const int64_t total = (int64_t)k * N;
    if (!total) return PPRPA_OK;
    unpack_bf16_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(
        z, k, N, nvv, pp, pq, pm, mult, xs_hi, xs_lo, ldx, ys_hi, ys_lo, ldy);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

__global__ void pack_f32_kernel(const float* __restrict__ O, const double* __restrict__ z, int k,
                                int N, int nvv, const int* __restrict__ pp,
                                const int* __restrict__ pq, PadMap pm,
                                const double* __restrict__ eps, int mult,
                                double* __restrict__ sigma) {
    const int64_t total = (int64_t)k * N;
    const int64_t np = pm.n_pad;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const int p = pp[I], q = pq[I];
        double o = (double)O[j * np * np + (int64_t)pm.map(p) * np + pm.map(q)];
        if (mult == 1 && p == q) o *= 0.7071067811865476;
        const double w = I < nvv ? 1.0 : -1.0;
        sigma[t] = fma(w * (eps[p] + eps[q]), z[t], o);
    }
}

int launch_pack_f32(const float* O, const double* z, int k, int N, int nvv, const int* pp,
                    const int* pq, PadMap pm, const double* eps, int mult, double* sigma,
                    cudaStream_t st) {
    const int64_t total = (int64_t)k * N;
    if (!total) return PPRPA_OK;
    pack_f32_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(
        O, z, k, N, nvv, pp, pq, pm, eps, mult, sigma);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// ---------------------------------------------------------------------------
// Davidson vector kernels.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// R = SZ - omega * W * Zr; norms2[j] += ||R_j||^2 (norms2 zeroed by the caller).
__global__ void residual_kernel(const double* __restrict__ SZ, const double* __restrict__ Zr,
                                const double* __restrict__ omega, int N, int nvv, double wsign,
                                double* __restrict__ R, double* __restrict__ norms2) {
    __shared__ double sh[32];
    const int j = blockIdx.y;
    const double om = omega[j];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = (int64_t)j * N + i;
        const double w = i < nvv ? wsign : -wsign;
        const double r = SZ[t] - om * w * Zr[t];
        R[t] = r;
        acc = fma(r, r, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(norms2 + j, acc);
}

int launch_residual(const double* SZ, const double* Zr, const double* omega, int k, int N,
                    int nvv, double* R, double* norms2, cudaStream_t st, double wsign) {
    if (!k || !N) return PPRPA_OK;
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(N, 256), 256), k);
    residual_kernel<<<grid, 256, 0, st>>>(SZ, Zr, omega, N, nvv, wsign, R, norms2);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Diagonal preconditioner: out_t = R_sel[t] / (D - omega_sel[t] * w), |denominator| >= 1e-4.
__global__ void correction_kernel(const double* __restrict__ R, const double* __restrict__ D,
                                  const double* __restrict__ omega, const int* __restrict__ sel,
                                  int N, int nvv, double wsign, double* __restrict__ out) {
    const int t = blockIdx.y;
    const int j = sel[t];
    const double om = omega[j];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = i < nvv ? wsign : -wsign;
        double den = D[i] - om * w;
        if (fabs(den) < 1e-4) den = den < 0.0 ? -1e-4 : 1e-4;
        out[(int64_t)t * N + i] = R[(int64_t)j * N + i] / den;
    }
}

int launch_correction(const double* R, const double* D, const double* omega, const int* sel,
                      int kn, int N, int nvv, double* out, cudaStream_t st, double wsign) {
    if (!kn || !N) return PPRPA_OK;
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(N, 256), 256), kn);
    correction_kernel<<<grid, 256, 0, st>>>(R, D, omega, sel, N, nvv, wsign, out);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

__global__ void row_norms2_kernel(const double* __restrict__ X, int N, double* __restrict__ out) {
    __shared__ double sh[32];
    const int j = blockIdx.y;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[(int64_t)j * N + i];
        acc = fma(x, x, acc);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) atomicAdd(out + j, acc);
}

// out[j] = ||X_j||^2 written by one block per row (no prior zeroing)
__global__ void row_norms2_set_kernel(const double* __restrict__ X, int N, double* __restrict__ out) {
    __shared__ double sh[32];
    const int j = blockIdx.x;
    double a0 = 0.0, a1 = 0.0;
    int64_t i = threadIdx.x;
    for (; i + blockDim.x < N; i += 2 * (int64_t)blockDim.x) {
        const double x0 = X[(int64_t)j * N + i], x1 = X[(int64_t)j * N + i + blockDim.x];
        a0 = fma(x0, x0, a0);
        a1 = fma(x1, x1, a1);
    }
    if (i < N) {
        const double x = X[(int64_t)j * N + i];
        a0 = fma(x, x, a0);
    }
    const double acc = block_sum(a0 + a1, sh);
    if (threadIdx.x == 0) out[j] = acc;
}

int launch_row_norms2(const double* X, int k, int N, double* out, cudaStream_t st) {
    if (!k) return PPRPA_OK;
    if (N <= 65536) {
        // a block per row writes its norm: one launch, no zeroing of out
        row_norms2_set_kernel<<<k, 256, 0, st>>>(X, N, out);
        PP_CHECK_LAUNCH();
        return PPRPA_OK;
    }
    PP_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * k, st));
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(N, 256), 256), k);
    row_norms2_kernel<<<grid, 256, 0, st>>>(X, N, out);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// dst row t = src row idx[t] (rows of N doubles), t < n
__global__ void gather_rows_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                   const int* __restrict__ idx, int n, int64_t N) {
    const int t = blockIdx.y;
    if (t >= n) return;
    const double* s = src + (int64_t)idx[t] * N;
    double* d = dst + (int64_t)t * N;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = s[i];
}

int launch_gather_rows(double* dst, const double* src, const int* idx, int n, int64_t N, cudaStream_t st) {
    if (n <= 0 || N <= 0) return PPRPA_OK;
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(N, 256), 64), (unsigned)n);
    gather_rows_kernel<<<grid, 256, 0, st>>>(dst, src, idx, n, N);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

__global__ void scatter_unit_kernel(double* V, int ld, const int* idx, int k) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) V[(int64_t)t * ld + idx[t]] = 1.0;
}

int launch_scatter_unit(double* V, int ld, const int* idx, int k, cudaStream_t st) {
    if (!k) return PPRPA_OK;
    scatter_unit_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>(V, ld, idx, k);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Explicit ppRPA matrix from the dense (pr|qs) table: eri[(p*n+r)*n*n + (q*n+s)].
__global__ void build_matrix_kernel(const double* __restrict__ eri, int n,
                                    const int* __restrict__ pp, const int* __restrict__ pq, int N,
                                    int nvv, const double* __restrict__ eps, int mult,
                                    double* __restrict__ M) {
    const int64_t total = (int64_t)N * N;
    const int64_t n2 = (int64_t)n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int J = t % N;
        const int I = t / N;
        const int p = pp[I], q = pq[I], r = pp[J], s = pq[J];
        const double direct = eri[((int64_t)p * n + r) * n2 + (int64_t)q * n + s];  // <pq|rs>
        const double exch = eri[((int64_t)p * n + s) * n2 + (int64_t)q * n + r];    // <pq|sr>
        double v;
        if (mult == 1) {
            const double f = ((p == q) ? 0.7071067811865476 : 1.0) * ((r == s) ? 0.7071067811865476 : 1.0);
            v = f * (direct + exch);
        } else {
            v = direct - exch;
        }
        if (I == J) v += (I < nvv ? 1.0 : -1.0) * (eps[p] + eps[q]);
        M[t] = v;
    }
}

int launch_build_matrix(const double* eri, int n, const int* pp, const int* pq, int N, int nvv,
                        const double* eps, int mult, double* M, cudaStream_t st) {
    const int64_t total = (int64_t)N * N;
    if (!total) return PPRPA_OK;
    build_matrix_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 64), 256, 0, st>>>(
        eri, n, pp, pq, N, nvv, eps, mult, M);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// d omega / d eps_p = s * sum_I w_I z_I^2 (d_{p,p_I} + d_{p,q_I}).  deps zeroed by the caller.
__global__ void grad_eps_kernel(const double* __restrict__ z, int N, int nvv,
                                const int* __restrict__ pp, const int* __restrict__ pq, double s,
                                double* __restrict__ deps) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= N) return;
    const double w = I < nvv ? 1.0 : -1.0;
    const double v = s * w * z[I] * z[I];
    atomicAdd(deps + pp[I], v);
    atomicAdd(deps + pq[I], v);
}

int launch_grad_eps(const double* z, int N, int nvv, const int* pp, const int* pq, int n,
                    double s, double* deps, cudaStream_t st) {
    (void)n;
    if (!N) return PPRPA_OK;
    grad_eps_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(z, N, nvv, pp, pq, s, deps);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa

namespace pprpa {

// out[0] = sum_{i < nw} omega_i - sum_{I < nvv} D_I  (one block, FP64).
__global__ void ec_sum_kernel(const double* __restrict__ omega, int nw, const double* __restrict__ D,
                              int nvv, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) acc += omega[i];
    for (int i = threadIdx.x; i < nvv; i += blockDim.x) acc -= D[i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] = acc;
}

int launch_ec_sum(const double* omega, int nw, const double* D, int nvv, double* out,
                  cudaStream_t st) {
    ec_sum_kernel<<<1, 1024, 0, st>>>(omega, nw, D, nvv, out);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

__global__ void set_diag_kernel(double* M, int N, int nvv, double wsign) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) M[(int64_t)i * N + i] = i < nvv ? wsign : -wsign;
}

int launch_metric_matrix(double* W, int N, int nvv, cudaStream_t st, double wsign) {
    PP_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * (size_t)N * N, st));
    set_diag_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(W, N, nvv, wsign);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa

namespace pprpa {

// Derivatives of the two-electron part of Tr A (Sec. "ppRPA Equation"), subtracted from the
// sum of root gradients to give d E_c (Eq. correlation_energy).  With
// Two-electron part of the trace of the A block (blk = 0, virtual pairs) or of the C block
// (blk = 1, occupied pairs); with tr L^P over the block's orbitals,
//   Tr_2e = 1/2 sum_P [(tr L^P)^2 +- sum_{xy} (L^P_xy)^2]   (+ singlet, - triplet),
//   d Tr_2e / d L^P_xy = d_xy tr L^P +- L^P_xy  for x, y in the block, 0 otherwise.
// The orbital-energy part: d Tr A / d eps_a = nv +- 1 (virtual a), d Tr C / d eps_i =
// -(no +- 1) (occupied i).  The kernels subtract these derivatives from dL / deps.
__global__ void trace_block_grad_kernel(const double* __restrict__ L, int n, int x0, int x1,
                                        int mult, double* __restrict__ dL) {
    __shared__ double sh[32];
    const int64_t P = blockIdx.x;
    const double* Lp = L + P * (int64_t)n * n;
    double* dp = dL + P * (int64_t)n * n;
    double tr = 0.0;
    for (int a = x0 + threadIdx.x; a < x1; a += blockDim.x) tr += Lp[(int64_t)a * n + a];
    tr = block_sum(tr, sh);
    __shared__ double trb;
    if (threadIdx.x == 0) trb = tr;
    __syncthreads();
    const double sg = mult == 1 ? 1.0 : -1.0;
    const int nb = x1 - x0;
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int x = x0 + t / nb, y = x0 + t % nb;
        const int64_t o = (int64_t)x * n + y;
        dp[o] -= (x == y ? trb : 0.0) + sg * Lp[o];
    }
}

__global__ void trace_block_eps_kernel(int x0, int x1, double d, double* deps) {
    const int p = x0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (p < x1) deps[p] -= d;
}

int launch_trace_block_grad(const double* L, int naux, int n, int no, int mult, int blk,
                            double* dL, double* deps, cudaStream_t st) {
    const int x0 = blk == 0 ? no : 0, x1 = blk == 0 ? n : no;
    if (x1 <= x0) return PPRPA_OK;
    if (dL && naux > 0) {
        trace_block_grad_kernel<<<naux, 256, 0, st>>>(L, n, x0, x1, mult, dL);
        PP_CHECK_LAUNCH();
    }
    if (deps) {
        const double nb = (double)(x1 - x0), sg = mult == 1 ? 1.0 : -1.0;
        const double d = blk == 0 ? nb + sg : -(nb + sg);
        trace_block_eps_kernel<<<(unsigned)ceil_div(x1 - x0, 128), 128, 0, st>>>(x0, x1, d, deps);
        PP_CHECK_LAUNCH();
    }
    return PPRPA_OK;
}

// X[r][i] *= f[r] for k rows of length len.
__global__ void scale_rows_kernel(double* __restrict__ X, int k, int64_t len, const double* __restrict__ f) {
    const int64_t total = (int64_t)k * len;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x)
        X[t] *= f[t / len];
}

int launch_scale_rows(double* X, int k, int64_t len, const double* f, cudaStream_t st) {
    const int64_t total = (int64_t)k * len;
    if (total <= 0) return PPRPA_OK;
    scale_rows_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(X, k, len, f);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa

namespace pprpa {

// ---------------------------------------------------------------------------
// FP8 (E4M3) operands of the first sandwich stage.
// L8[P][r][c8]: rows as the BF16 padded layout; columns occupied at [0, no), virtual at
// [c_off8, c_off8 + nv) with c_off8 a multiple of 16 (so every TMA box starts 16-byte
// aligned); scale[P] = max|L^P| / 448, L8 = e4m3(L / scale).
__global__ void quantize_fp8_kernel(const double* __restrict__ L, int n, PadMap pm, int ncol8,
                                    int c_off8, __nv_fp8_e4m3* __restrict__ L8,
                                    float* __restrict__ scale) {
    __shared__ double sh[32];
    __shared__ double inv_sh;
    const int64_t P = blockIdx.x;
    const double* Lp = L + P * (int64_t)n * n;
    double m = 0.0;
    for (int64_t t = threadIdx.x; t < (int64_t)n * n; t += blockDim.x) m = fmax(m, fabs(Lp[t]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, sh[w]);
        const double sc = a > 0.0 ? a / 448.0 : 1.0;
        scale[P] = (float)sc;
        inv_sh = 1.0 / (double)(float)sc;
    }
    __syncthreads();
    const double inv = inv_sh;
    const int np = pm.n_pad;
    __nv_fp8_e4m3* out = L8 + P * (int64_t)np * ncol8;
    for (int64_t t = threadIdx.x; t < (int64_t)np * ncol8; t += blockDim.x) {
        const int r = (int)(t / ncol8), c8 = (int)(t % ncol8);
        const int p = r < pm.no ? r : ((r >= pm.no_p && r < pm.no_p + pm.nv) ? pm.no + r - pm.no_p : -1);
        const int q = c8 < pm.no ? c8 : ((c8 >= c_off8 && c8 < c_off8 + pm.nv) ? pm.no + c8 - c_off8 : -1);
        const double x = (p >= 0 && q >= 0) ? Lp[(int64_t)p * n + q] * inv : 0.0;
        out[t] = __nv_fp8_e4m3((float)x);
    }
}

int launch_quantize_fp8(const double* L, int naux, int n, PadMap pm, int ncol8, int c_off8,
                        void* L8, float* scale, cudaStream_t st) {
    if (naux <= 0) return PPRPA_OK;
    quantize_fp8_kernel<<<naux, 256, 0, st>>>(L, n, pm, ncol8, c_off8, (__nv_fp8_e4m3*)L8, scale);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// zscale[j] = max over the packed pair matrix of vector j (sqrt(2) on singlet diagonals) / 448.
__global__ void zscale_kernel(const double* __restrict__ z, int N, const int* __restrict__ pp,
                              const int* __restrict__ pq, int mult, float* __restrict__ zscale) {
    __shared__ double sh[32];
    const int64_t j = blockIdx.x;
    double m = 0.0;
    for (int I = threadIdx.x; I < N; I += blockDim.x) {
        double v = fabs(z[j * N + I]);
        if (mult == 1 && pp[I] == pq[I]) v *= 1.4142135623730951;
        m = fmax(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a = fmax(a, sh[w]);
        zscale[j] = a > 0.0 ? (float)(a / 448.0) : 1.0f;
    }
}

// Same stacks as unpack_bf16 (Xs[j][c][d] = Zt_j[d][c], nv_p / no_p rows per vector) in E4M3,
// each vector divided by its scale.  The caller zeroes the stacks.
__global__ void unpack_fp8_kernel(const double* __restrict__ z, int k, int N, int nvv,
                                  const int* __restrict__ pp, const int* __restrict__ pq,
                                  PadMap pm, int mult, const float* __restrict__ zscale,
                                  __nv_fp8_e4m3* __restrict__ xs, int ldx,
                                  __nv_fp8_e4m3* __restrict__ ys, int ldy) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const double inv = 1.0 / (double)zscale[j];
        const double v = z[t] * inv;
        int p = pp[I], q = pq[I];
        __nv_fp8_e4m3* st;
        int64_t rows, ld;
        if (I < nvv) { p -= pm.no; q -= pm.no; st = xs; rows = pm.nv_p; ld = ldx; }
        else { st = ys; rows = pm.no_p; ld = ldy; }
        const int64_t base = j * rows * ld;
        double zpq, zqp;
        if (mult == 1) { zpq = (p == q) ? 1.4142135623730951 * v : v; zqp = zpq; }
        else { zpq = v; zqp = -v; }
        st[base + (int64_t)q * ld + p] = __nv_fp8_e4m3((float)zpq);
        if (p != q) st[base + (int64_t)p * ld + q] = __nv_fp8_e4m3((float)zqp);
    }
}

int launch_unpack_fp8(const double* z, int k, int N, int nvv, const int* pp, const int* pq,
                      PadMap pm, int mult, float* zscale, void* xs, int ldx, void* ys, int ldy,
                      cudaStream_t st) {
    if (!k || !N) return PPRPA_OK;
    zscale_kernel<<<k, 256, 0, st>>>(z, N, pp, pq, mult, zscale);
    PP_CHECK_LAUNCH();
    const int64_t total = (int64_t)k * N;
    unpack_fp8_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 16), 256, 0, st>>>(
        z, k, N, nvv, pp, pq, pm, mult, zscale, (__nv_fp8_e4m3*)xs, ldx, (__nv_fp8_e4m3*)ys, ldy);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Fractional occupations: X[P][s][t] *= w[s] w[t] (slot weights sqrt(n) / sqrt(1 - n)).
__global__ void scale_slots_kernel(double* __restrict__ X, int naux, int n, const double* __restrict__ w) {
    const int64_t total = (int64_t)naux * n * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = t % n, p = (t / n) % n;
        X[t] *= w[p] * w[q];
    }
}

int launch_scale_slots(double* X, int naux, int n, const double* w, cudaStream_t st) {
    const int64_t total = (int64_t)naux * n * n;
    if (!total) return PPRPA_OK;
    scale_slots_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 32), 256, 0, st>>>(X, naux, n, w);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// dst[m][orb[s]] += src[m][s] (an orbital may own several slots).
__global__ void scatter_add_cols_kernel(double* __restrict__ dst, int nmo, const double* __restrict__ src,
                                        int nbasis, int n, const int* __restrict__ orb) {
    const int64_t total = (int64_t)nbasis * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int s = t % n;
        const int64_t m = t / n;
        atomicAdd(dst + m * nmo + orb[s], src[t]);
    }
}

int launch_scatter_add_cols(double* dst, int nmo, const double* src, int nbasis, int n, const int* orb,
                            cudaStream_t st) {
    const int64_t total = (int64_t)nbasis * n;
    if (!total) return PPRPA_OK;
    scatter_add_cols_kernel<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 8), 256, 0, st>>>(
        dst, nmo, src, nbasis, n, orb);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

}  // namespace pprpa
