// The (alpha alpha; beta beta) subspace of spin-unrestricted ppRPA (Sec. "Implementation
// Details": the spin-unrestricted matrix is built and diagonalised in three subspaces).
//
// The context's own active orbitals and integrals are the alpha set; pprpa_set_beta adds the
// beta set (its own active space, orbital energies and MO-space fitting integrals).  The
// same-spin subspaces are the restricted triplet formulas of one spin (pairs a < b with
// <ab|cd> - <ab|dc>), i.e. a context per spin solved with PPRPA_TRIPLET.  The alpha-beta
// pairs are every (alpha virtual a, beta virtual b) and every (alpha occupied i, beta
// occupied j); opposite spins have no exchange, so with (pr|qs) = sum_P L^{aP}_pr L^{bP}_qs
//   A_{ab,cd} = d_ac d_bd (eps_a + eps_b) + (ac|bd), B_{ab,kl} = (ak|bl),
//   C_{ij,kl} = -d_ik d_jl (eps_i + eps_j) + (ik|jl),
// and the matrix-vector product is the rectangular sandwich O = sum_P L^{aP} Zt L^{bP} with
// Zt (n_alpha x n_beta) holding X on its virtual block and Y on its occupied block.
#include "ctx.h"

namespace pprpa {
namespace {

// D_I = w (eps_a[p] + eps_b[q]) + sum_P L^a_pp L^b_qq, w = +1 on virtual pairs, -1 on occupied.
__global__ void diag_ab_kernel(const double* __restrict__ La, int na, const double* __restrict__ Lb, int nb,
                               int naux, const double* __restrict__ ea, const double* __restrict__ eb,
                               const int* __restrict__ pp, const int* __restrict__ pq, int nvv, int N,
                               double* __restrict__ D) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        const int p = pp[I], q = pq[I];
        double v = 0.0;
        for (int P = 0; P < naux; ++P)
            v = fma(La[((int64_t)P * na + p) * na + p], Lb[((int64_t)P * nb + q) * nb + q], v);
        const double w = I < nvv ? 1.0 : -1.0;
        D[I] = w * (ea[p] + eb[q]) + v;
    }
}

// Zt_j[p][q] = z_j[I] for pair I = (p, q) (the caller zeroes Zt).
__global__ void unpack_ab_kernel(const double* __restrict__ z, int k, int N, const int* __restrict__ pp,
                                 const int* __restrict__ pq, int na, int nb, double* __restrict__ Zt) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        Zt[(j * na + pp[I]) * nb + pq[I]] = z[t];
    }
}

// sigma_j[I] = w (eps_a[p] + eps_b[q]) z_j[I] + O_j[p][q].
__global__ void pack_ab_kernel(const double* __restrict__ O, const double* __restrict__ z, int k, int N,
                               int nvv, const int* __restrict__ pp, const int* __restrict__ pq, int na,
                               int nb, const double* __restrict__ ea, const double* __restrict__ eb,
                               double* __restrict__ sigma) {
    const int64_t total = (int64_t)k * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = t % N;
        const int64_t j = t / N;
        const int p = pp[I], q = pq[I];
        const double w = I < nvv ? 1.0 : -1.0;
        sigma[t] = fma(w * (ea[p] + eb[q]), z[t], O[(j * na + p) * nb + q]);
    }
}

// M[I][J] = sum_P L^a_{p_I p_J} L^b_{q_I q_J} + d_IJ w_I (eps_a[p_I] + eps_b[q_I]).
__global__ void build_ab_kernel(const double* __restrict__ La, int na, const double* __restrict__ Lb, int nb,
                                int naux, const double* __restrict__ ea, const double* __restrict__ eb,
                                const int* __restrict__ pp, const int* __restrict__ pq, int nvv, int N,
                                double* __restrict__ M) {
    const int64_t total = (int64_t)N * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(t / N), J = (int)(t % N);
        const int p = pp[I], q = pq[I], r = pp[J], s = pq[J];
        double v = 0.0;
        for (int P = 0; P < naux; ++P)
            v = fma(La[((int64_t)P * na + p) * na + r], Lb[((int64_t)P * nb + q) * nb + s], v);
        if (I == J) v += (I < nvv ? 1.0 : -1.0) * (ea[p] + eb[q]);
        M[t] = v;
    }
}

// d omega / d eps of one alpha-beta pair vector z (Sec. Analytic Gradient): pair I = (p, q)
// adds w_I s z_I^2 to alpha orbital p and to beta orbital q (w = +1 virtual, -1 occupied).
__global__ void grad_eps_ab_kernel(const double* __restrict__ z, int N, int nvv, const int* __restrict__ pp,
                                   const int* __restrict__ pq, double s, double* __restrict__ da,
                                   double* __restrict__ db) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < N; I += gridDim.x * blockDim.x) {
        const double v = (I < nvv ? s : -s) * z[I] * z[I];
        if (da) atomicAdd(&da[pp[I]], v);
        if (db) atomicAdd(&db[pq[I]], v);
    }
}

unsigned grid_for(int64_t total) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 152 * 16)); }

}  // namespace

int ensure_pairs_ab(pprpa_ctx* c, PairTable** out) {
    if (!c->have_Lb) return set_error(PPRPA_ERR_STATE, "alpha-beta subspace: call pprpa_set_beta first");
    PairTable& t = c->pairs[2];
    if (!t.ready) {
        t.pp.clear();
        t.pq.clear();
        const int noa = c->no, nva = c->nv, nob = c->nob, nvb = c->nvb;
        for (int a = 0; a < nva; ++a)
            for (int b = 0; b < nvb; ++b) {
                t.pp.push_back(noa + a);
                t.pq.push_back(nob + b);
            }
        t.nvv = (int)t.pp.size();
        for (int i = 0; i < noa; ++i)
            for (int j = 0; j < nob; ++j) {
                t.pp.push_back(i);
                t.pq.push_back(j);
            }
        t.N = (int)t.pp.size();
        t.noo = t.N - t.nvv;
        if (t.d_pp) cudaFree(t.d_pp);
        if (t.d_pq) cudaFree(t.d_pq);
        t.d_pp = t.d_pq = nullptr;
        if (t.N > 0) {
            PP_CUDA(cudaMalloc(&t.d_pp, sizeof(int) * t.N));
            PP_CUDA(cudaMalloc(&t.d_pq, sizeof(int) * t.N));
            PP_CUDA(cudaMemcpyAsync(t.d_pp, t.pp.data(), sizeof(int) * t.N, cudaMemcpyHostToDevice, c->stream));
            PP_CUDA(cudaMemcpyAsync(t.d_pq, t.pq.data(), sizeof(int) * t.N, cudaMemcpyHostToDevice, c->stream));
            PP_CUDA(cudaStreamSynchronize(c->stream));
        }
        t.ready = true;
    }
    *out = &t;
    return PPRPA_OK;
}

int diag_ab(pprpa_ctx* c, PairTable* t, double* D) {
    if (!t->N) return PPRPA_OK;
    diag_ab_kernel<<<grid_for(t->N), 256, 0, c->stream>>>(c->d_L, c->n(), c->d_Lb, c->nb(), c->naux, c->d_eps,
                                                          c->d_epsb, t->d_pp, t->d_pq, t->nvv, t->N, D);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

int build_ab(pprpa_ctx* c, PairTable* t, double* M) {
    if (!t->N) return PPRPA_OK;
    build_ab_kernel<<<grid_for((int64_t)t->N * t->N), 256, 0, c->stream>>>(
        c->d_L, c->n(), c->d_Lb, c->nb(), c->naux, c->d_eps, c->d_epsb, t->d_pp, t->d_pq, t->nvv, t->N, M);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// FP64 alpha-beta sigma: blocked batched DGEMMs, P processed in chunks.
int sigma_ab_f64(pprpa_ctx* c, int k, const double* d_z, double* d_sigma) {
    PairTable* t;
    PP_TRY(ensure_pairs_ab(c, &t));
    const int na = c->n(), nb = c->nb(), noa = c->no, nva = c->nv, nob = c->nob, nvb = c->nvb;
    const int naux = c->naux;
    const int64_t na2 = (int64_t)na * na, nb2 = (int64_t)nb * nb, nab = (int64_t)na * nb;
    cudaStream_t st = c->stream;
    double *Zt, *O, *T;
    PP_TRY(ws_get(c, "ab_Zt", sizeof(double) * nab * k, (void**)&Zt));
    PP_TRY(ws_get(c, "ab_O", sizeof(double) * nab * k, (void**)&O));
    const int64_t per_p = sizeof(double) * nab * k;
    const int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (4LL << 30) / per_p));
    PP_TRY(ws_get(c, "ab_T", per_p * pc, (void**)&T));
    PP_CUDA(cudaMemsetAsync(Zt, 0, sizeof(double) * nab * k, st));
    unpack_ab_kernel<<<grid_for((int64_t)k * t->N), 256, 0, st>>>(d_z, k, t->N, t->d_pp, t->d_pq, na, nb, Zt);
    PP_CHECK_LAUNCH();
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = std::min(pc, naux - P0);
        const double* La0 = c->d_L + (int64_t)P0 * na2;
        const double* Lb0 = c->d_Lb + (int64_t)P0 * nb2;
        // T[P][j] = L^a Zt_j (na x nb): beta-virtual columns from the virtual block of Zt,
        // beta-occupied columns from its occupied block
        for (int blk = 0; blk < 2; ++blk) {
            const int ka = blk == 0 ? nva : noa, offa = blk == 0 ? noa : 0;
            const int kb = blk == 0 ? nvb : nob, offb = blk == 0 ? nob : 0;
            if (ka == 0 || kb == 0) continue;
            Dgemm g;
            g.M = na; g.N = kb; g.K = ka;
            g.A = La0 + offa; g.lda = na; g.sA1 = na2;
            g.B = Zt + (int64_t)offa * nb + offb; g.ldb = nb; g.sB2 = nab;
            g.C = T + offb; g.ldc = nb; g.sC1 = nab * k; g.sC2 = nab;
            g.nb1 = np; g.nb2 = k;
            PP_TRY(dgemm(g, st));
        }
        // O_j[blk] (+)= sum_P T[P][j][alpha rows of blk, :] L^b[:, beta columns of blk]
        for (int blk = 0; blk < 2; ++blk) {
            const int ma = blk == 0 ? nva : noa, offa = blk == 0 ? noa : 0;
            const int mb = blk == 0 ? nvb : nob, offb = blk == 0 ? nob : 0;
            if (ma == 0 || mb == 0) continue;
            Dgemm g;
            g.M = ma; g.N = mb; g.K = nb;
            g.A = T + (int64_t)offa * nb; g.lda = nb; g.sA1 = nab; g.sAr = nab * k;
            g.B = Lb0 + offb; g.ldb = nb; g.sBr = nb2;
            g.C = O + (int64_t)offa * nb + offb; g.ldc = nb; g.sC1 = nab;
            g.nb1 = k; g.nr = np;
            g.beta = P0 == 0 ? 0.0 : 1.0;
            PP_TRY(dgemm(g, st));
        }
    }
    pack_ab_kernel<<<grid_for((int64_t)k * t->N), 256, 0, st>>>(O, d_z, k, t->N, t->nvv, t->d_pp, t->d_pq, na, nb,
                                                               c->d_eps, c->d_epsb, d_sigma);
    PP_CHECK_LAUNCH();
    return PPRPA_OK;
}

// Hellmann-Feynman gradient of one alpha-beta root (Sec. Analytic Gradient): with Zt the
// na x nb matrix of z and s = z^T W z,
//   d omega / d L^{alpha P} = s Zt L^{beta P} Zt^T,  d omega / d L^{beta P} = s Zt^T L^{alpha P} Zt,
// two batched FP64 GEMMs each per chunk of P.
int grad_ab(pprpa_ctx* c, const double* z, double s, double* dLa, double* dLb, double* dea, double* deb,
            int where) {
    PairTable* t;
    PP_TRY(ensure_pairs_ab(c, &t));
    const int na = c->n(), nb = c->nb(), naux = c->naux;
    const int64_t na2 = (int64_t)na * na, nb2 = (int64_t)nb * nb, nab = (int64_t)na * nb;
    cudaStream_t st = c->stream;
    const cudaMemcpyKind kind = where == PPRPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dea || deb) {
        double* d;
        PP_TRY(ws_get(c, "gab_eps", sizeof(double) * (na + nb), (void**)&d));
        PP_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (na + nb), st));
        if (t->N) {
            grad_eps_ab_kernel<<<grid_for(t->N), 256, 0, st>>>(z, t->N, t->nvv, t->d_pp, t->d_pq, s, d, d + na);
            PP_CHECK_LAUNCH();
        }
        if (dea) PP_CUDA(cudaMemcpyAsync(dea, d, sizeof(double) * na, kind, st));
        if (deb) PP_CUDA(cudaMemcpyAsync(deb, d + na, sizeof(double) * nb, kind, st));
    }
    if (dLa || dLb) {
        double *Zt, *T, *out = nullptr;
        PP_TRY(ws_get(c, "gab_Zt", sizeof(double) * nab, (void**)&Zt));
        PP_CUDA(cudaMemsetAsync(Zt, 0, sizeof(double) * nab, st));
        if (t->N) {
            unpack_ab_kernel<<<grid_for(t->N), 256, 0, st>>>(z, 1, t->N, t->d_pp, t->d_pq, na, nb, Zt);
            PP_CHECK_LAUNCH();
        }
        const int64_t per_p = std::max(na2, std::max(nb2, nab));
        const int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (1LL << 30) / (8 * per_p)));
        PP_TRY(ws_get(c, "gab_T", sizeof(double) * nab * pc, (void**)&T));
        if (where == PPRPA_HOST) PP_TRY(ws_get(c, "gab_out", sizeof(double) * per_p * pc, (void**)&out));
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = std::min(pc, naux - P0);
            if (dLa) {
                Dgemm g1;  // T^P = L^{beta P} Zt^T (nb x na)
                g1.M = nb; g1.N = na; g1.K = nb;
                g1.A = c->d_Lb + (size_t)P0 * nb2; g1.lda = nb; g1.sA1 = nb2;
                g1.B = Zt; g1.ldb = nb; g1.transB = 1;
                g1.C = T; g1.ldc = na; g1.sC1 = nab;
                g1.nb1 = np;
                PP_TRY(dgemm(g1, st));
                Dgemm g2;  // d L^{alpha P} = s Zt T^P (na x na)
                g2.M = na; g2.N = na; g2.K = nb;
                g2.A = Zt; g2.lda = nb;
                g2.B = T; g2.ldb = na; g2.sB1 = nab;
                g2.C = where == PPRPA_DEVICE ? dLa + (size_t)P0 * na2 : out; g2.ldc = na; g2.sC1 = na2;
                g2.nb1 = np;
                g2.alpha = s;
                PP_TRY(dgemm(g2, st));
                if (where == PPRPA_HOST) {
                    PP_CUDA(cudaMemcpyAsync(dLa + (size_t)P0 * na2, out, sizeof(double) * na2 * np,
                                            cudaMemcpyDeviceToHost, st));
                    PP_CUDA(cudaStreamSynchronize(st));
                }
            }
            if (dLb) {
                Dgemm g1;  // T^P = L^{alpha P} Zt (na x nb)
                g1.M = na; g1.N = nb; g1.K = na;
                g1.A = c->d_L + (size_t)P0 * na2; g1.lda = na; g1.sA1 = na2;
                g1.B = Zt; g1.ldb = nb;
                g1.C = T; g1.ldc = nb; g1.sC1 = nab;
                g1.nb1 = np;
                PP_TRY(dgemm(g1, st));
                Dgemm g2;  // d L^{beta P} = s Zt^T T^P (nb x nb)
                g2.M = nb; g2.N = nb; g2.K = na;
                g2.A = Zt; g2.lda = nb; g2.transA = 1;
                g2.B = T; g2.ldb = nb; g2.sB1 = nab;
                g2.C = where == PPRPA_DEVICE ? dLb + (size_t)P0 * nb2 : out; g2.ldc = nb; g2.sC1 = nb2;
                g2.nb1 = np;
                g2.alpha = s;
                PP_TRY(dgemm(g2, st));
                if (where == PPRPA_HOST) {
                    PP_CUDA(cudaMemcpyAsync(dLb + (size_t)P0 * nb2, out, sizeof(double) * nb2 * np,
                                            cudaMemcpyDeviceToHost, st));
                    PP_CUDA(cudaStreamSynchronize(st));
                }
            }
        }
    }
    PP_CUDA(cudaStreamSynchronize(st));
    return PPRPA_OK;
}

}  // namespace pprpa

using namespace pprpa;

extern "C" int pprpa_grad_ab(pprpa_ctx* c, int root, double* dLa, double* dLb, double* deps_a, double* deps_b,
                             int where) {
    if (!c) return set_error(PPRPA_ERR_ARG, "grad_ab: null context");
    PP_CUDA(cudaSetDevice(c->device));
    if (where != PPRPA_HOST && where != PPRPA_DEVICE) return set_error(PPRPA_ERR_ARG, "grad_ab: bad `where`");
    if (!c->have_L || !c->have_Lb) return set_error(PPRPA_ERR_STATE, "grad_ab: set the alpha and beta integrals first");
    if (c->last_nroots == 0 || !c->d_lastZ || c->last_mult != PPRPA_AB)
        return set_error(PPRPA_ERR_STATE, "grad_ab: no alpha-beta solve to differentiate");
    if (root < 0 || root >= c->last_nroots) return set_error(PPRPA_ERR_ARG, "grad_ab: root index out of range");
    PairTable* t;
    PP_TRY(ensure_pairs_ab(c, &t));
    if (t->N != c->last_N) return set_error(PPRPA_ERR_STATE, "grad_ab: the pair space changed since the solve");
    // addition roots have z^T W z = +1, removal roots (hh channel) -1
    const double s = c->last_channel == PPRPA_CHANNEL_HH ? -1.0 : 1.0;
    return grad_ab(c, c->d_lastZ + (size_t)root * c->last_N, s, dLa, dLb, deps_a, deps_b, where);
}

extern "C" int pprpa_set_beta(pprpa_ctx* c, int nocc_b, int nvir_b, int naux, const double* eps_b,
                              const double* L_b, int where) {
    if (!c) return set_error(PPRPA_ERR_ARG, "set_beta: null context");
    PP_CUDA(cudaSetDevice(c->device));
    if (!c->have_L) return set_error(PPRPA_ERR_STATE, "set_beta: set the alpha integrals first");
    if (nocc_b < 0 || nvir_b < 0 || nocc_b + nvir_b == 0 || !eps_b || !L_b ||
        (where != PPRPA_HOST && where != PPRPA_DEVICE))
        return set_error(PPRPA_ERR_ARG, "set_beta: bad arguments");
    if (naux != c->naux) return set_error(PPRPA_ERR_ARG, "set_beta: naux differs from the alpha integrals");
    const int nb = nocc_b + nvir_b;
    for (int p = 0; where == PPRPA_HOST && p < nb; ++p)
        if (!std::isfinite(eps_b[p])) return set_error(PPRPA_ERR_ARG, "set_beta: non-finite energy");
    if (c->d_Lb) cudaFree(c->d_Lb);
    if (c->d_epsb) cudaFree(c->d_epsb);
    c->d_Lb = c->d_epsb = nullptr;
    c->have_Lb = false;
    const cudaMemcpyKind kind = where == PPRPA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    PP_CUDA(cudaMalloc(&c->d_Lb, sizeof(double) * (size_t)naux * nb * nb));
    PP_CUDA(cudaMalloc(&c->d_epsb, sizeof(double) * nb));
    PP_CUDA(cudaMemcpyAsync(c->d_Lb, L_b, sizeof(double) * (size_t)naux * nb * nb, kind, c->stream));
    PP_CUDA(cudaMemcpyAsync(c->d_epsb, eps_b, sizeof(double) * nb, kind, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    c->nob = nocc_b;
    c->nvb = nvir_b;
    c->pairs[2].ready = false;
    c->have_Lb = true;
    if (c->last_mult == PPRPA_AB) {  // a stored alpha-beta solve no longer matches the pair table
        if (c->d_lastZ) cudaFree(c->d_lastZ);
        c->d_lastZ = nullptr;
        c->last_nroots = 0;
    }
    return PPRPA_OK;
}
