// C ABI entry points: context, inputs (with the AO->MO transform), kernels, gradient.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "ctx.h"

namespace pprpa {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

int set_error(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

void count_launch(long long n) { g_launches += n; }

int ctx_sync(pprpa_ctx* c) {
    if (!c->blocking_sync) {
        PP_CUDA(cudaStreamSynchronize(c->stream));
        return PPRPA_OK;
    }
    if (!c->sync_ev) PP_CUDA(cudaEventCreateWithFlags(&c->sync_ev, cudaEventBlockingSync | cudaEventDisableTiming));
    PP_CUDA(cudaEventRecord(c->sync_ev, c->stream));
    PP_CUDA(cudaEventSynchronize(c->sync_ev));
    return PPRPA_OK;
}

int host_stage(pprpa_ctx* c, size_t bytes, void** out, int slot) {
    if (c->hstage_bytes[slot] < bytes) {
        if (c->hstage[slot]) {
            PP_CUDA(cudaDeviceSynchronize());  // no copy from or into the old buffer is still queued
            PP_CUDA(cudaFreeHost(c->hstage[slot]));
            c->hstage[slot] = nullptr;
            c->hstage_bytes[slot] = 0;
        }
        PP_CUDA(cudaMallocHost(&c->hstage[slot], bytes));
        c->hstage_bytes[slot] = bytes;
    }
    *out = c->hstage[slot];
    return PPRPA_OK;
}

static int check_ctx(pprpa_ctx* c) {
    if (!c) return set_error(PPRPA_ERR_ARG, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return set_error(PPRPA_ERR_CUDA, cudaGetErrorString(e));
    return PPRPA_OK;
}

static int need_L(pprpa_ctx* c) {
    if (!c->have_L) return set_error(PPRPA_ERR_STATE, "integrals not set (call pprpa_set_ao or pprpa_set_mo)");
    return PPRPA_OK;
}

int ensure_pairs(pprpa_ctx* c, int mult, PairTable** out) {
    if (mult == PPRPA_AB) return ensure_pairs_ab(c, out);
    if (mult != 1 && mult != 3) return set_error(PPRPA_ERR_ARG, "mult must be 1, 3 or PPRPA_AB");
    PairTable& t = c->pairs[mult == 1 ? 0 : 1];
    if (!t.ready) {
        t.pp.clear();
        t.pq.clear();
        const int no = c->no, nv = c->nv;
        for (int a = 0; a < nv; ++a)
            for (int b = (mult == 1 ? a : a + 1); b < nv; ++b) {
                t.pp.push_back(no + a);
                t.pq.push_back(no + b);
            }
        t.nvv = (int)t.pp.size();
        for (int i = 0; i < no; ++i)
            for (int j = (mult == 1 ? i : i + 1); j < no; ++j) {
                t.pp.push_back(i);
                t.pq.push_back(j);
            }
        t.N = (int)t.pp.size();
        t.noo = t.N - t.nvv;
        ++c->mem_epoch;
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

static void reset_integrals(pprpa_ctx* c) {
    ++c->mem_epoch;
    if (c->d_L) cudaFree(c->d_L);
    if (c->d_Lhi) cudaFree(c->d_Lhi);
    if (c->d_Llo) cudaFree(c->d_Llo);
    if (c->d_lastZ) cudaFree(c->d_lastZ);
    if (c->d_L8) cudaFree(c->d_L8);
    if (c->d_L8scale) cudaFree(c->d_L8scale);
    c->d_L8 = nullptr;
    c->d_L8scale = nullptr;
    c->fp8_ready = false;
    c->d_L = nullptr;
    c->d_Lhi = c->d_Llo = nullptr;
    c->d_lastZ = nullptr;
    c->bf16_ready = false;
    c->have_L = false;
    c->last_nroots = 0;
    for (auto& t : c->pairs) t.ready = false;
}

// Slot energies, weights and MO indices on the device.
static int upload_eps(pprpa_ctx* c) {
    const int n = c->n();
    ++c->mem_epoch;
    if (c->d_eps) cudaFree(c->d_eps);
    if (c->d_slot_w) cudaFree(c->d_slot_w);
    if (c->d_slot_orb) cudaFree(c->d_slot_orb);
    c->d_eps = c->d_slot_w = nullptr;
    c->d_slot_orb = nullptr;
    if (n == 0) return PPRPA_OK;
    std::vector<double> e(n), w(n);
    std::vector<int> o(n);
    for (int s = 0; s < n; ++s) {
        o[s] = c->orb(s);
        e[s] = c->eps[o[s]];
        w[s] = c->slot_w(s);
    }
    PP_CUDA(cudaMalloc(&c->d_eps, sizeof(double) * n));
    PP_CUDA(cudaMemcpy(c->d_eps, e.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    PP_CUDA(cudaMalloc(&c->d_slot_w, sizeof(double) * n));
    PP_CUDA(cudaMemcpy(c->d_slot_w, w.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    PP_CUDA(cudaMalloc(&c->d_slot_orb, sizeof(int) * n));
    PP_CUDA(cudaMemcpy(c->d_slot_orb, o.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    return PPRPA_OK;
}

// Active columns of C (nbasis x nmo, row-major) in slot order -> d_Cact (nbasis x n).
static int gather_slot_columns(pprpa_ctx* c, const double* C, int nbasis, int where, double* d_Cact) {
    const int n = c->n(), nmo = c->nmo;
    cudaStream_t st = c->stream;
    if (where == PPRPA_HOST) {
        std::vector<double> ca((size_t)nbasis * n);
        for (int m = 0; m < nbasis; ++m)
            for (int s = 0; s < n; ++s) ca[(size_t)m * n + s] = C[(size_t)m * nmo + c->orb(s)];
        PP_CUDA(cudaMemcpyAsync(d_Cact, ca.data(), sizeof(double) * ca.size(), cudaMemcpyHostToDevice, st));
        PP_CUDA(cudaStreamSynchronize(st));
    } else {
        // hole slots and particle slots are each a contiguous range of MO columns
        if (c->no)
            PP_CUDA(cudaMemcpy2DAsync(d_Cact, sizeof(double) * n, C + c->orb(0), sizeof(double) * nmo,
                                      sizeof(double) * c->no, nbasis, cudaMemcpyDeviceToDevice, st));
        if (c->nv)
            PP_CUDA(cudaMemcpy2DAsync(d_Cact + c->no, sizeof(double) * n, C + c->orb(c->no),
                                      sizeof(double) * nmo, sizeof(double) * c->nv, nbasis,
                                      cudaMemcpyDeviceToDevice, st));
    }
    return PPRPA_OK;
}

}  // namespace pprpa

using namespace pprpa;

extern "C" {

const char* pprpa_strerror(int code) {
    switch (code) {
        case PPRPA_OK: return "ok";
        case PPRPA_ERR_ARG: return "invalid argument";
        case PPRPA_ERR_CUDA: return "CUDA error";
        case PPRPA_ERR_OOM: return "out of device memory";
        case PPRPA_ERR_NOCONV: return "Davidson did not converge";
        case PPRPA_ERR_UNSTABLE: return "no positive-definite shift (unstable ppRPA problem)";
        case PPRPA_ERR_TIMEOUT: return "device-side wait timed out";
        case PPRPA_ERR_STATE: return "required input not set";
        case PPRPA_ERR_UNSUPPORTED: return "GPU is not sm_103 (GB300)";
        default: return "unknown error";
    }
}

const char* pprpa_last_error(void) { return g_last_error.c_str(); }

long long pprpa_kernel_launches(void) { return g_launches.load(); }

int pprpa_create(pprpa_ctx** out, int device, void* cuda_stream) {
    if (!out) return set_error(PPRPA_ERR_ARG, "null out pointer");
    *out = nullptr;
    int ndev = 0;
    PP_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return set_error(PPRPA_ERR_ARG, "bad device index");
    PP_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    PP_CUDA(cudaGetDeviceProperties(&prop, device));
    if (!(prop.major == 10 && prop.minor == 3))
        return set_error(PPRPA_ERR_UNSUPPORTED, std::string("device is sm_") + std::to_string(prop.major) +
                                                    std::to_string(prop.minor) + ", need sm_103");
    pprpa_ctx* c = new pprpa_ctx();
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete c; return set_error(PPRPA_ERR_CUDA, cudaGetErrorString(e)); }
        c->own_stream = true;
    }
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess) {
        pprpa_destroy(c);
        return set_error(PPRPA_ERR_OOM, "status word");
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    *out = c;
    return PPRPA_OK;
}

void pprpa_destroy(pprpa_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    reset_integrals(c);
    if (c->d_eps) cudaFree(c->d_eps);
    if (c->d_slot_w) cudaFree(c->d_slot_w);
    if (c->d_slot_orb) cudaFree(c->d_slot_orb);
    if (c->d_Lb) cudaFree(c->d_Lb);
    if (c->d_epsb) cudaFree(c->d_epsb);
    for (auto& t : c->pairs) {
        if (t.d_pp) cudaFree(t.d_pp);
        if (t.d_pq) cudaFree(t.d_pq);
    }
    for (auto& kv : c->ws)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto& r : c->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    destroy_batch_plan(c->batch_plan);
    destroy_batch_plan(c->batch_plan3);
    if (c->sync_ev) cudaEventDestroy(c->sync_ev);
    for (void* h : c->hstage)
        if (h) cudaFreeHost(h);
    if (c->d_status) cudaFree(c->d_status);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int pprpa_set_orbitals(pprpa_ctx* c, int nmo, const double* occ, const double* eps) {
    PP_TRY(check_ctx(c));
    if (nmo <= 0 || !occ || !eps) return set_error(PPRPA_ERR_ARG, "set_orbitals: bad arguments");
    int nocc = 0, nfull = 0;
    for (int i = 0; i < nmo; ++i) {
        if (!(occ[i] >= 0.0 && occ[i] <= 1.0))
            return set_error(PPRPA_ERR_ARG, "set_orbitals: occupations must lie in [0, 1]");
        if (i > 0 && occ[i] > occ[i - 1])
            return set_error(PPRPA_ERR_ARG, "set_orbitals: occupations must be non-increasing");
        if (occ[i] > 0.0) ++nocc;
        if (occ[i] == 1.0) ++nfull;
        if (!std::isfinite(eps[i])) return set_error(PPRPA_ERR_ARG, "set_orbitals: non-finite energy");
        if (i > 0 && eps[i] < eps[i - 1]) return set_error(PPRPA_ERR_ARG, "set_orbitals: energies must be ascending");
    }
    reset_integrals(c);
    c->nmo = nmo;
    c->nocc = nocc;
    c->nfull = nfull;
    c->occ.assign(occ, occ + nmo);
    c->eps.assign(eps, eps + nmo);
    c->no = nocc;
    c->nv = nmo - nfull;
    return upload_eps(c);
}

int pprpa_set_active(pprpa_ctx* c, int nocc_act, int nvir_act) {
    PP_TRY(check_ctx(c));
    if (c->nmo == 0) return set_error(PPRPA_ERR_STATE, "set_active: call set_orbitals first");
    if (nocc_act < 0 || nvir_act < 0 || nocc_act > c->nocc || nvir_act > c->nmo - c->nfull)
        return set_error(PPRPA_ERR_ARG, "set_active: active space larger than the orbital space");
    if (nocc_act + nvir_act == 0) return set_error(PPRPA_ERR_ARG, "set_active: empty active space");
    if (c->have_L) return set_error(PPRPA_ERR_STATE, "set_active must precede set_ao / set_mo");
    c->no = nocc_act;
    c->nv = nvir_act;
    for (auto& t : c->pairs) t.ready = false;
    return upload_eps(c);
}

int pprpa_set_ao(pprpa_ctx* c, int nbasis, int naux, const double* C, const double* ao3c, int where) {
    PP_TRY(check_ctx(c));
    if (c->nmo == 0) return set_error(PPRPA_ERR_STATE, "set_ao: call set_orbitals first");
    if (nbasis <= 0 || naux <= 0 || !C || !ao3c || (where != PPRPA_HOST && where != PPRPA_DEVICE))
        return set_error(PPRPA_ERR_ARG, "set_ao: bad arguments");
    if (c->have_L) reset_integrals(c);
    const int n = c->n();
    cudaStream_t st = c->stream;
    // active columns of C (nbasis x n, slot order) on the device
    double* d_Cact;
    PP_TRY(ws_get(c, "ao_Cact", sizeof(double) * nbasis * n, (void**)&d_Cact));
    PP_TRY(gather_slot_columns(c, C, nbasis, where, d_Cact));
    const int64_t nb2 = (int64_t)nbasis * nbasis;
    PP_CUDA(cudaMalloc(&c->d_L, sizeof(double) * (size_t)naux * n * n));
    c->naux = naux;
    // chunk of P: AO slices (host input) plus the half-transformed H = AO^P C_act
    const int64_t per_p = sizeof(double) * (nb2 + (int64_t)nbasis * n);
    const int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (2LL << 30) / per_p));
    double *d_ao = nullptr, *d_H;
    if (where == PPRPA_HOST) PP_TRY(ws_get(c, "ao_slab", sizeof(double) * nb2 * pc, (void**)&d_ao));
    PP_TRY(ws_get(c, "ao_H", sizeof(double) * (size_t)nbasis * n * pc, (void**)&d_H));
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = std::min(pc, naux - P0);
        const double* src;
        if (where == PPRPA_HOST) {
            PP_CUDA(cudaMemcpyAsync(d_ao, ao3c + (size_t)P0 * nb2, sizeof(double) * nb2 * np,
                                    cudaMemcpyHostToDevice, st));
            src = d_ao;
        } else {
            src = ao3c + (size_t)P0 * nb2;
        }
        // H^P = (P|mu nu) C_act   (nbasis x n)
        Dgemm g1;
        g1.M = nbasis; g1.N = n; g1.K = nbasis;
        g1.A = src; g1.lda = nbasis; g1.sA1 = nb2;
        g1.B = d_Cact; g1.ldb = n;
        g1.C = d_H; g1.ldc = n; g1.sC1 = (int64_t)nbasis * n;
        g1.nb1 = np;
        PP_TRY(dgemm(g1, st));
        // L^P = C_act^T H^P   (n x n)
        Dgemm g2;
        g2.M = n; g2.N = n; g2.K = nbasis;
        g2.A = d_Cact; g2.lda = n; g2.transA = 1;
        g2.B = d_H; g2.ldb = n; g2.sB1 = (int64_t)nbasis * n;
        g2.C = c->d_L + (size_t)P0 * n * n; g2.ldc = n; g2.sC1 = (int64_t)n * n;
        g2.nb1 = np;
        PP_TRY(dgemm(g2, st));
        if (where == PPRPA_HOST) PP_CUDA(cudaStreamSynchronize(st));
    }
    // fractional occupations: L~^P_st = w_s w_t L^P_st
    if (c->weighted()) PP_TRY(launch_scale_slots(c->d_L, naux, n, c->d_slot_w, st));
    PP_CUDA(cudaStreamSynchronize(st));
    c->have_L = true;
    return PPRPA_OK;
}

int pprpa_grad_ao(pprpa_ctx* c, int nbasis, int naux, const double* C, const double* ao3c,
                  const double* dL, double* dAO, double* dC, int where) {
    PP_TRY(check_ctx(c));
    if (c->nmo == 0) return set_error(PPRPA_ERR_STATE, "grad_ao: call set_orbitals first");
    if (nbasis <= 0 || naux <= 0 || !C || !dL || (where != PPRPA_HOST && where != PPRPA_DEVICE))
        return set_error(PPRPA_ERR_ARG, "grad_ao: bad arguments");
    if (dC && !ao3c) return set_error(PPRPA_ERR_ARG, "grad_ao: dC needs the AO integrals");
    if (!dAO && !dC) return PPRPA_OK;
    const int n = c->n(), nmo = c->nmo;
    cudaStream_t st = c->stream;
    const bool host = where == PPRPA_HOST;
    const bool weighted = c->weighted();
    const int64_t nb2 = (int64_t)nbasis * nbasis, nbn = (int64_t)nbasis * n, n2 = (int64_t)n * n;
    // active columns of C (nbasis x n, slot order)
    double* d_Cact;
    PP_TRY(ws_get(c, "gao_Cact", sizeof(double) * nbn, (void**)&d_Cact));
    PP_TRY(gather_slot_columns(c, C, nbasis, where, d_Cact));
    // chunk of P: dL slices, AO slices and the outputs staged on the device for host arguments,
    // the half-transformed products always
    const int64_t per_p = sizeof(double) * (nbn + (host || weighted ? n2 : 0) +
                                            (host ? (dAO ? nb2 : 0) + (dC ? nb2 : 0) : 0));
    const int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (2LL << 30) / per_p));
    double *d_T, *d_dL = nullptr, *d_ao = nullptr, *d_out = nullptr, *d_dCact = nullptr;
    PP_TRY(ws_get(c, "gao_T", sizeof(double) * nbn * pc, (void**)&d_T));
    if (host || weighted) PP_TRY(ws_get(c, "gao_dL", sizeof(double) * n2 * pc, (void**)&d_dL));
    if (host && dC) PP_TRY(ws_get(c, "gao_ao", sizeof(double) * nb2 * pc, (void**)&d_ao));
    if (host && dAO) PP_TRY(ws_get(c, "gao_out", sizeof(double) * nb2 * pc, (void**)&d_out));
    if (dC) PP_TRY(ws_get(c, "gao_dCact", sizeof(double) * nbn, (void**)&d_dCact));
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = std::min(pc, naux - P0);
        const double* g;
        if (host || weighted) {
            PP_CUDA(cudaMemcpyAsync(d_dL, dL + (size_t)P0 * n2, sizeof(double) * n2 * np,
                                    host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
            // the slots carry weights: L~_st = w_s w_t C_s^T (P|..) C_t
            if (weighted) PP_TRY(launch_scale_slots(d_dL, np, n, c->d_slot_w, st));
            g = d_dL;
        } else {
            g = dL + (size_t)P0 * n2;
        }
        if (dAO) {
            // d/d(P|mu nu) = C_act dL^P C_act^T
            Dgemm g1;  // T^P = C_act dL^P  (nbasis x n)
            g1.M = nbasis; g1.N = n; g1.K = n;
            g1.A = d_Cact; g1.lda = n;
            g1.B = g; g1.ldb = n; g1.sB1 = n2;
            g1.C = d_T; g1.ldc = n; g1.sC1 = nbn;
            g1.nb1 = np;
            PP_TRY(dgemm(g1, st));
            Dgemm g2;  // out^P = T^P C_act^T  (nbasis x nbasis)
            g2.M = nbasis; g2.N = nbasis; g2.K = n;
            g2.A = d_T; g2.lda = n; g2.sA1 = nbn;
            g2.B = d_Cact; g2.ldb = n; g2.transB = 1;
            g2.C = host ? d_out : dAO + (size_t)P0 * nb2; g2.ldc = nbasis; g2.sC1 = nb2;
            g2.nb1 = np;
            PP_TRY(dgemm(g2, st));
            if (host)
                PP_CUDA(cudaMemcpyAsync(dAO + (size_t)P0 * nb2, d_out, sizeof(double) * nb2 * np,
                                        cudaMemcpyDeviceToHost, st));
        }
        if (dC) {
            const double* src;
            if (host) {
                PP_CUDA(cudaMemcpyAsync(d_ao, ao3c + (size_t)P0 * nb2, sizeof(double) * nb2 * np,
                                        cudaMemcpyHostToDevice, st));
                src = d_ao;
            } else {
                src = ao3c + (size_t)P0 * nb2;
            }
            Dgemm g1;  // H^P = (P|mu nu) C_act  (nbasis x n)
            g1.M = nbasis; g1.N = n; g1.K = nbasis;
            g1.A = src; g1.lda = nbasis; g1.sA1 = nb2;
            g1.B = d_Cact; g1.ldb = n;
            g1.C = d_T; g1.ldc = n; g1.sC1 = nbn;
            g1.nb1 = np;
            PP_TRY(dgemm(g1, st));
            // d/dC_act (+)= sum_P H^P (dL^P)^T + H^P dL^P  (the AO slices are symmetric)
            for (int t = 0; t < 2; ++t) {
                Dgemm g3;
                g3.M = nbasis; g3.N = n; g3.K = n;
                g3.A = d_T; g3.lda = n; g3.sAr = nbn;
                g3.B = g; g3.ldb = n; g3.sBr = n2; g3.transB = t == 0 ? 1 : 0;
                g3.C = d_dCact; g3.ldc = n;
                g3.nr = np;
                g3.beta = (P0 == 0 && t == 0) ? 0.0 : 1.0;
                PP_TRY(dgemm(g3, st));
            }
        }
        if (host) PP_CUDA(cudaStreamSynchronize(st));
    }
    if (dC) {
        // slot columns back to MO columns, summed where an orbital is both a hole and a
        // particle slot
        if (host) {
            std::vector<double> da((size_t)nbn);
            PP_CUDA(cudaMemcpyAsync(da.data(), d_dCact, sizeof(double) * nbn, cudaMemcpyDeviceToHost, st));
            PP_CUDA(cudaStreamSynchronize(st));
            std::fill(dC, dC + (size_t)nbasis * nmo, 0.0);
            for (int m = 0; m < nbasis; ++m)
                for (int s = 0; s < n; ++s) dC[(size_t)m * nmo + c->orb(s)] += da[(size_t)m * n + s];
        } else {
            PP_CUDA(cudaMemsetAsync(dC, 0, sizeof(double) * (size_t)nbasis * nmo, st));
            PP_TRY(launch_scatter_add_cols(dC, nmo, d_dCact, nbasis, n, c->d_slot_orb, st));
        }
    }
    PP_CUDA(cudaStreamSynchronize(st));
    return PPRPA_OK;
}

int pprpa_set_mo(pprpa_ctx* c, int naux, const double* L, int where) {
    PP_TRY(check_ctx(c));
    if (c->nmo == 0) return set_error(PPRPA_ERR_STATE, "set_mo: call set_orbitals first");
    if (naux <= 0 || !L || (where != PPRPA_HOST && where != PPRPA_DEVICE))
        return set_error(PPRPA_ERR_ARG, "set_mo: bad arguments");
    if (c->have_L) reset_integrals(c);
    const int n = c->n(), nmo = c->nmo;
    cudaStream_t st = c->stream;
    const int* d_orb = c->d_slot_orb;  // MO index of every slot
    PP_CUDA(cudaMalloc(&c->d_L, sizeof(double) * (size_t)naux * n * n));
    c->naux = naux;
    const int64_t nm2 = (int64_t)nmo * nmo;
    if (where == PPRPA_DEVICE) {
        PP_TRY(launch_extract_active(L, naux, nmo, d_orb, n, c->d_L, st));
    } else {
        const int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (1LL << 30) / (8 * nm2)));
        double* d_slab;
        PP_TRY(ws_get(c, "mo_slab", sizeof(double) * nm2 * pc, (void**)&d_slab));
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = std::min(pc, naux - P0);
            PP_CUDA(cudaMemcpyAsync(d_slab, L + (size_t)P0 * nm2, sizeof(double) * nm2 * np,
                                    cudaMemcpyHostToDevice, st));
            PP_TRY(launch_extract_active(d_slab, np, nmo, d_orb, n, c->d_L + (size_t)P0 * n * n, st));
            PP_CUDA(cudaStreamSynchronize(st));
        }
    }
    // fractional occupations: L~^P_st = w_s w_t L^P_st
    if (c->weighted()) PP_TRY(launch_scale_slots(c->d_L, naux, n, c->d_slot_w, st));
    PP_CUDA(cudaStreamSynchronize(st));
    c->have_L = true;
    return PPRPA_OK;
}

int pprpa_get_L(pprpa_ctx* c, double* out, int where) {
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if (!out) return set_error(PPRPA_ERR_ARG, "get_L: null output");
    const size_t bytes = sizeof(double) * (size_t)c->naux * c->n() * c->n();
    PP_CUDA(cudaMemcpyAsync(out, c->d_L, bytes,
                            where == PPRPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return PPRPA_OK;
}

int pprpa_dims(pprpa_ctx* c, int mult, int* n, int* naux, int* nvv, int* noo) {
    PP_TRY(check_ctx(c));
    if (c->nmo == 0) return set_error(PPRPA_ERR_STATE, "dims: call set_orbitals first");
    PairTable* t;
    PP_TRY(ensure_pairs(c, mult, &t));
    if (n) *n = c->n();
    if (naux) *naux = c->naux;
    if (nvv) *nvv = t->nvv;
    if (noo) *noo = t->noo;
    return PPRPA_OK;
}

int pprpa_diag(pprpa_ctx* c, int mult, double* out, int where) {
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if (!out) return set_error(PPRPA_ERR_ARG, "diag: null output");
    PairTable* t;
    PP_TRY(ensure_pairs(c, mult, &t));
    double *D, *work;
    PP_TRY(ws_get(c, "diag_D", sizeof(double) * std::max(t->N, 1), (void**)&D));
    PP_TRY(ws_get(c, "diag_work", sizeof(double) * (size_t)c->naux * c->n(), (void**)&work));
    if (mult == PPRPA_AB) PP_TRY(diag_ab(c, t, D));
    else PP_TRY(launch_diag(c->d_L, c->naux, c->n(), c->d_eps, t->d_pp, t->d_pq, t->nvv, t->N, mult, D,
                            work, c->stream));
    PP_CUDA(cudaMemcpyAsync(out, D, sizeof(double) * t->N,
                            where == PPRPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return PPRPA_OK;
}

int pprpa_sigma(pprpa_ctx* c, int mult, int precision, int k, const double* z, double* sigma,
                int where) {
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if (k < 0 || (k > 0 && (!z || !sigma))) return set_error(PPRPA_ERR_ARG, "sigma: bad arguments");
    if (k == 0) return PPRPA_OK;
    PairTable* t;
    PP_TRY(ensure_pairs(c, mult, &t));
    const size_t bytes = sizeof(double) * (size_t)k * t->N;
    const double* dz = z;
    double* ds = sigma;
    if (where == PPRPA_HOST) {
        double *bz, *bs;
        PP_TRY(ws_get(c, "sig_z", bytes, (void**)&bz));
        PP_TRY(ws_get(c, "sig_s", bytes, (void**)&bs));
        PP_CUDA(cudaMemcpyAsync(bz, z, bytes, cudaMemcpyHostToDevice, c->stream));
        dz = bz;
        ds = bs;
    }
    int rc;
    if (mult == PPRPA_AB) {
        if (precision != PPRPA_PREC_FP64)
            return set_error(PPRPA_ERR_UNSUPPORTED, "sigma: the alpha-beta subspace runs in FP64 only");
        rc = sigma_ab_f64(c, k, dz, ds);
    } else if (precision == PPRPA_PREC_FP64) rc = sigma_f64(c, mult, k, dz, ds);
    else if (precision == PPRPA_PREC_BF16) rc = sigma_tc(c, mult, k, dz, ds, 1);
    else if (precision == PPRPA_PREC_BF16 + 16) rc = sigma_tc(c, mult, k, dz, ds, 3);
    else if (precision == PPRPA_PREC_FP8) rc = sigma_tc(c, mult, k, dz, ds, 1, true);
    else return set_error(PPRPA_ERR_ARG, "sigma: unknown precision");
    if (rc != PPRPA_OK) return rc;
    if (precision != PPRPA_PREC_FP64) PP_TRY(check_status(c));
    if (where == PPRPA_HOST)
        PP_CUDA(cudaMemcpyAsync(sigma, ds, bytes, cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return PPRPA_OK;
}

}  // extern "C"

namespace pprpa {
// Weighted Hellmann-Feynman gradient (Sec. "Analytic Gradient") of nr pair vectors Z (device,
// nr x N, row r = z_r):
//   G = sum_r f_r z_r^T (dM / d theta) z_r  [- d Tr A (trace_blk 0) or - d Tr C (trace_blk 1)]
// with respect to every entry of L^P (dL[naux][n][n]) and to eps (deps[n]); f on the host.
// Per root, z^T (dM / d L^P) z = 1/2 (Zt L^P Zt^T + Zt^T L^P Zt) = t Zt L^P Zt, t = +1
// singlet (Zt symmetric), -1 triplet (Zt antisymmetric).  The roots go through batched FP64
// GEMMs, T[P][r] = L^P Zt_r for a slice of P and a chunk of roots, then
// dL^P (+)= sum_r (t f_r Zt_r) T[P][r] as one GEMM reducing over the roots.
static int grad_weighted(pprpa_ctx* c, int mult, const double* Z, int nr, const double* f,
                         int trace_blk, double* dL, double* deps, int where) {
    PairTable* t;
    PP_TRY(ensure_pairs(c, mult, &t));
    const int n = c->n(), naux = c->naux, N = t->N;
    const int64_t n2 = (int64_t)n * n;
    cudaStream_t st = c->stream;
    const cudaMemcpyKind kind = where == PPRPA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (deps) {
        double* d;
        PP_TRY(ws_get(c, "grad_eps", sizeof(double) * n, (void**)&d));
        PP_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n, st));
        for (int r = 0; r < nr; ++r)
            if (f[r] != 0.0)
                PP_TRY(launch_grad_eps(Z + (size_t)r * N, N, t->nvv, t->d_pp, t->d_pq, n, f[r], d, st));
        if (trace_blk >= 0) PP_TRY(launch_trace_block_grad(c->d_L, 0, n, c->no, mult, trace_blk, nullptr, d, st));
        PP_CUDA(cudaMemcpyAsync(deps, d, sizeof(double) * n, kind, st));
    }
    if (dL) {
        // roots per chunk: their packed pair matrices (plain and weighted) within 1 GiB
        const int rc = (int)std::max<int64_t>(1, std::min<int64_t>(nr, (1LL << 30) / (16 * n2)));
        // auxiliary slices per pass: T within 1 GiB and the batched launch within its grid
        int pc = (int)std::max<int64_t>(1, std::min<int64_t>(naux, (1LL << 30) / (8 * n2 * rc)));
        pc = std::min(pc, std::max(1, 65535 / rc));
        double *Zt, *Zw, *T, *out, *fd;
        PP_TRY(ws_get(c, "grad_Zt", sizeof(double) * n2 * rc, (void**)&Zt));
        PP_TRY(ws_get(c, "grad_Zw", sizeof(double) * n2 * rc, (void**)&Zw));
        PP_TRY(ws_get(c, "grad_T", sizeof(double) * n2 * rc * pc, (void**)&T));
        PP_TRY(ws_get(c, "grad_f", sizeof(double) * nr, (void**)&fd));
        std::vector<double> tf(f, f + nr);
        for (double& v : tf) v *= mult == 1 ? 1.0 : -1.0;
        PP_CUDA(cudaMemcpyAsync(fd, tf.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st));
        if (where == PPRPA_DEVICE) out = dL;
        else PP_TRY(ws_get(c, "grad_dL", sizeof(double) * n2 * pc, (void**)&out));
        auto unpack_chunk = [&](int r0, int kr) -> int {
            PP_CUDA(cudaMemsetAsync(Zt, 0, sizeof(double) * n2 * kr, st));
            PP_TRY(launch_unpack_f64(Z + (size_t)r0 * N, kr, N, t->d_pp, t->d_pq, n, mult, Zt, st));
            PP_CUDA(cudaMemcpyAsync(Zw, Zt, sizeof(double) * n2 * kr, cudaMemcpyDeviceToDevice, st));
            return launch_scale_rows(Zw, kr, n2, fd + r0, st);
        };
        if (nr <= rc) PP_TRY(unpack_chunk(0, nr));
        for (int P0 = 0; P0 < naux; P0 += pc) {
            const int np = std::min(pc, naux - P0);
            double* dst = where == PPRPA_DEVICE ? out + (size_t)P0 * n2 : out;
            for (int r0 = 0; r0 < nr; r0 += rc) {
                const int kr = std::min(rc, nr - r0);
                if (nr > rc) PP_TRY(unpack_chunk(r0, kr));
                Dgemm g1;  // T[p][r] = L^P Zt_r
                g1.M = n; g1.N = n; g1.K = n;
                g1.A = c->d_L + (size_t)P0 * n2; g1.lda = n; g1.sA1 = n2;
                g1.B = Zt; g1.ldb = n; g1.sB2 = n2;
                g1.C = T; g1.ldc = n; g1.sC1 = n2 * kr; g1.sC2 = n2;
                g1.nb1 = np; g1.nb2 = kr;
                PP_TRY(dgemm(g1, st));
                Dgemm g2;  // dL^P (+)= sum_r (t f_r Zt_r) T[p][r]
                g2.M = n; g2.N = n; g2.K = n;
                g2.A = Zw; g2.lda = n; g2.sAr = n2;
                g2.B = T; g2.ldb = n; g2.sB1 = n2 * kr; g2.sBr = n2;
                g2.C = dst; g2.ldc = n; g2.sC1 = n2;
                g2.nb1 = np; g2.nr = kr;
                g2.beta = r0 == 0 ? 0.0 : 1.0;
                PP_TRY(dgemm(g2, st));
            }
            if (trace_blk >= 0)
                PP_TRY(launch_trace_block_grad(c->d_L + (size_t)P0 * n2, np, n, c->no, mult, trace_blk, dst,
                                               nullptr, st));
            if (where == PPRPA_HOST) {
                PP_CUDA(cudaMemcpyAsync(dL + (size_t)P0 * n2, out, sizeof(double) * n2 * np,
                                        cudaMemcpyDeviceToHost, st));
                PP_CUDA(cudaStreamSynchronize(st));
            }
        }
    }
    PP_CUDA(cudaStreamSynchronize(st));
    return PPRPA_OK;
}

// Checks that the last solve can be differentiated; returns its pair table.
static int last_solve_pairs(pprpa_ctx* c, const char* who, PairTable** out) {
    if (c && c->last_nroots && c->last_mult == PPRPA_AB)
        return set_error(PPRPA_ERR_UNSUPPORTED,
                         std::string(who) + ": roots of the alpha-beta subspace take pprpa_grad_ab");
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if (c->last_nroots == 0 || !c->d_lastZ) return set_error(PPRPA_ERR_STATE, std::string(who) + ": no solve to differentiate");
    PP_TRY(ensure_pairs(c, c->last_mult, out));
    if ((*out)->N != c->last_N)
        return set_error(PPRPA_ERR_STATE, std::string(who) + ": the pair space changed since the solve");
    return PPRPA_OK;
}
}  // namespace pprpa

extern "C" {

int pprpa_grad(pprpa_ctx* c, int root, double* dL, double* deps, int where) {
    PairTable* t;
    PP_TRY(last_solve_pairs(c, "grad", &t));
    if (root < 0 || root >= c->last_nroots) return set_error(PPRPA_ERR_ARG, "grad: root index out of range");
    // addition roots have z^T W z = +1, removal roots (hh channel) -1
    const double s = c->last_channel == PPRPA_CHANNEL_HH ? -1.0 : 1.0;
    return grad_weighted(c, c->last_mult, c->d_lastZ + (size_t)root * t->N, 1, &s, -1, dL, deps, where);
}

int pprpa_grad_sum(pprpa_ctx* c, int nw, const double* w, double* dL, double* deps, int where) {
    PairTable* t;
    PP_TRY(last_solve_pairs(c, "grad_sum", &t));
    if (nw < 1 || nw > c->last_nroots || !w) return set_error(PPRPA_ERR_ARG, "grad_sum: need 1 <= nw <= roots of the last solve");
    const double s = c->last_channel == PPRPA_CHANNEL_HH ? -1.0 : 1.0;
    std::vector<double> f(w, w + nw);
    for (double& v : f) {
        if (!std::isfinite(v)) return set_error(PPRPA_ERR_ARG, "grad_sum: non-finite weight");
        v *= s;
    }
    return grad_weighted(c, c->last_mult, c->d_lastZ, nw, f.data(), -1, dL, deps, where);
}

int pprpa_grad_ec(pprpa_ctx* c, double* dL, double* deps, int where) {
    PairTable* t;
    PP_TRY(last_solve_pairs(c, "grad_ec", &t));
    if (!c->last_all_roots)
        return set_error(PPRPA_ERR_STATE,
                         "grad_ec: needs every root of one channel (nroots = nvv for pp, nroots = noo for hh)");
    // pp: E_c = sum Omega^{+2e} - Tr A, each root z^T dM z;  hh: E_c = -sum Omega^{-2e} - Tr C
    // with d Omega^{-2e} = -z^T dM z (Eq. correlation_energy), so both sum z^T dM z
    const bool hh = c->last_channel == PPRPA_CHANNEL_HH;
    std::vector<double> f(c->last_nroots, 1.0);
    return grad_weighted(c, c->last_mult, c->d_lastZ, c->last_nroots, f.data(), hh ? 1 : 0, dL, deps, where);
}

int pprpa_grad_vector(pprpa_ctx* c, int mult, const double* z, double* dL, double* deps, int where) {
    if (mult == PPRPA_AB)
        return set_error(PPRPA_ERR_UNSUPPORTED, "gradients of the alpha-beta subspace are not built");
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if (!z) return set_error(PPRPA_ERR_ARG, "grad_vector: null z");
    PairTable* t;
    PP_TRY(ensure_pairs(c, mult, &t));
    const double* dz = z;
    if (where == PPRPA_HOST) {
        double* b;
        PP_TRY(ws_get(c, "gradv_z", sizeof(double) * t->N, (void**)&b));
        PP_CUDA(cudaMemcpyAsync(b, z, sizeof(double) * t->N, cudaMemcpyHostToDevice, c->stream));
        dz = b;
    }
    const double one = 1.0;
    return grad_weighted(c, mult, dz, 1, &one, -1, dL, deps, where);
}

int pprpa_sigma_batch(int nmol, pprpa_ctx* const* ctxs, const int* mults, const int* ks,
                      const double* const* z, double* const* sigma, int precision, int flags) {
    if (nmol <= 0 || !ctxs || !mults || !ks || !z || !sigma)
        return set_error(PPRPA_ERR_ARG, "sigma_batch: bad arguments");
    if (precision != PPRPA_PREC_BF16 && precision != PPRPA_PREC_BF16 + 16)
        return set_error(PPRPA_ERR_ARG, "sigma_batch: precision must be BF16 or BF16x3");
    PP_TRY(check_ctx(ctxs[0]));
    for (int m = 0; m < nmol; ++m) {
        if (!ctxs[m] || ctxs[m]->device != ctxs[0]->device)
            return set_error(PPRPA_ERR_ARG, "sigma_batch: all contexts must share one device");
        PP_TRY(need_L(ctxs[m]));
        if ((mults[m] != 1 && mults[m] != 3) || ks[m] <= 0 || !z[m] || !sigma[m])
            return set_error(PPRPA_ERR_ARG, "sigma_batch: bad molecule arguments");
    }
    cudaStream_t st = ctxs[0]->stream;
    const int nterms = precision == PPRPA_PREC_BF16 ? 1 : 3;
    PP_TRY(sigma_tc_batch(nmol, ctxs, mults, ks, z, sigma, nterms, st, ctxs[0], (flags & 1) != 0));
    PP_TRY(check_status(ctxs[0]));
    return PPRPA_OK;
}

int pprpa_autotune(pprpa_ctx* c, int mult, int k, int precision, int* tiles) {
    PP_TRY(check_ctx(c));
    PP_TRY(need_L(c));
    if ((mult != 1 && mult != 3) || k <= 0) return set_error(PPRPA_ERR_ARG, "autotune: bad arguments");
    if (precision != PPRPA_PREC_BF16 && precision != PPRPA_PREC_BF16 + 16)
        return set_error(PPRPA_ERR_ARG, "autotune: precision must be BF16 or BF16x3");
    return autotune_tiles(c, mult, k, precision == PPRPA_PREC_BF16 ? 1 : 3, tiles);
}

int pprpa_profile(pprpa_ctx* c, int enable, double* out) {
    PP_TRY(check_ctx(c));
    if (out) {
        PP_CUDA(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < 12; ++i) out[i] = 0.0;
        for (auto& r : c->prof) {
            float ms = 0.f;
            PP_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
            out[3 * r.kind + 0] += 1.0;
            out[3 * r.kind + 1] += ms;
            out[3 * r.kind + 2] += r.flops;
        }
    }
    if (enable >= 0) {
        for (auto& r : c->prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        c->prof.clear();
        c->profile = enable != 0;
    }
    return PPRPA_OK;
}

}  // extern "C"
