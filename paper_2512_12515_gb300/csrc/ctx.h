// Internal state of a ppRPA context (host runtime of the C ABI).
#pragma once
#include <cmath>
#include <cuda.h>

#include <map>
#include <string>
#include <vector>

#include "kernels.h"
#include "tc.h"

namespace pprpa {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct ProfRec {
    cudaEvent_t a = nullptr, b = nullptr;
    int kind = 0;        // 0 s1 bf16, 1 s2 bf16, 2 s1 split, 3 s2 split
    double flops = 0.0;  // algorithmic sigma flops of the launch
};

struct PairTable {
    int nvv = 0, noo = 0, N = 0;
    std::vector<int> pp, pq;
    int* d_pp = nullptr;
    int* d_pq = nullptr;
    bool ready = false;
};

}  // namespace pprpa

struct pprpa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 152;

    int nmo = 0, nocc = 0;  // orbitals, orbitals with occupation n > 0 (hole candidates)
    int nfull = 0;          // orbitals with n = 1; those with n < 1 are particle candidates
    std::vector<double> occ, eps;
    int no = -1, nv = -1;  // active space: hole slots, particle slots
    bool have_L = false;
    int naux = 0;
    double* d_eps = nullptr;  // slot energies (n)
    double* d_slot_w = nullptr;  // slot weights (n): sqrt(n_p) on holes, sqrt(1 - n_p) on particles
    int* d_slot_orb = nullptr;   // MO index of every slot (n)
    // MO index of slot s: the highest `no` orbitals with n > 0, then the lowest `nv` with n < 1
    // (a fractionally occupied orbital can be both)
    int orb(int s) const { return s < no ? nocc - no + s : nfull + (s - no); }
    double slot_w(int s) const {
        const double f = occ[orb(s)];
        return s < no ? std::sqrt(f) : std::sqrt(1.0 - f);
    }
    bool weighted() const {  // some active slot has a weight other than 1
        for (int s = 0; s < no + nv; ++s)
            if (slot_w(s) != 1.0) return true;
        return false;
    }
    double* d_L = nullptr;    // [naux][n][n]

    pprpa::PairTable pairs[3];  // [0] singlet, [1] triplet, [2] alpha-beta (unrestricted)
    // beta set of the spin-unrestricted alpha-beta subspace (the context's own set is alpha)
    double* d_Lb = nullptr;    // [naux][nb][nb]
    double* d_epsb = nullptr;  // [nb]
    int nob = 0, nvb = 0;
    bool have_Lb = false;
    int nb() const { return nob + nvb; }

    // BF16 copies of L for the tensor-core sigma
    pprpa::PadMap pm;
    __nv_bfloat16* d_Lhi = nullptr;
    __nv_bfloat16* d_Llo = nullptr;
    bool bf16_ready = false;
    // E4M3 copy of L (stage 1 of the FP8 form) and its per-P scales
    void* d_L8 = nullptr;
    float* d_L8scale = nullptr;
    int ncol8 = 0, c_off8 = 0;
    bool fp8_ready = false;

    int* d_status = nullptr;
    std::map<std::string, pprpa::DevBuf> ws;  // grow-only named workspaces
    std::map<std::string, int> tuned_bn;      // autotuned N tile per problem key

    // per-launch profiling of the tensor-core GEMMs
    bool profile = false;
    std::vector<pprpa::ProfRec> prof;

    // batched-sigma plans (tensor maps, work items, CUDA graph) owned by this context: BF16
    // and BF16x3 forms
    void* batch_plan = nullptr;
    void* batch_plan3 = nullptr;

    // last solve (for gradients)
    int last_mult = 0;
    int last_channel = 0;  // PPRPA_CHANNEL_* of the last solve (sign of z^T W z)
    int last_nroots = 0;
    int last_N = 0;
    bool last_all_roots = false;  // the last solve returned every addition root (FULL)
    double* d_lastZ = nullptr;

    int n() const { return no + nv; }

    // bumped whenever device memory of the context is freed or moved (workspaces, integrals,
    // pair tables, energies): batched-sigma plans captured with its pointers compare it
    // before replaying
    unsigned long long mem_epoch = 0;

    // host waits on this context's stream: spin (cudaStreamSynchronize, lowest latency) or,
    // when many host threads each drive a context (pprpa_solve_batch), block on an event
    // created with cudaEventBlockingSync so that waiting threads do not occupy host cores
    bool blocking_sync = false;
    cudaEvent_t sync_ev = nullptr;

    // pinned host staging for the small per-iteration readbacks of a Davidson solve: a copy
    // into pageable memory waits for the stream by itself, a copy into this one does not, so
    // several readbacks share one wait
    // (slot 0: the Davidson readbacks; slot 1: the uploads of a batched-sigma plan)
    void* hstage[2] = {nullptr, nullptr};
    size_t hstage_bytes[2] = {0, 0};
};

namespace pprpa {

int ws_get(pprpa_ctx* c, const std::string& name, size_t bytes, void** out);
int ensure_pairs(pprpa_ctx* c, int mult, PairTable** out);
int ensure_bf16(pprpa_ctx* c);
int sigma_f64(pprpa_ctx* c, int mult, int k, const double* d_z, double* d_sigma);
// alpha-beta subspace of spin-unrestricted ppRPA (mult = PPRPA_AB): FP64 only
int ensure_pairs_ab(pprpa_ctx* c, PairTable** out);
int diag_ab(pprpa_ctx* c, PairTable* t, double* D);
int build_ab(pprpa_ctx* c, PairTable* t, double* M);
int sigma_ab_f64(pprpa_ctx* c, int k, const double* d_z, double* d_sigma);
int sigma_tc(pprpa_ctx* c, int mult, int k, const double* d_z, double* d_sigma, int nterms,
             bool f8 = false);
int ensure_fp8(pprpa_ctx* c);
int sigma_tc_batch(int nmol, pprpa_ctx* const* ctxs, const int* mults, const int* ks,
                   const double* const* z, double* const* sigma, int nterms, cudaStream_t st,
                   pprpa_ctx* owner, bool use_graph);
void destroy_batch_plan(void* plan);
int autotune_tiles(pprpa_ctx* c, int mult, int k, int nterms, int* bn_out);
int check_status(pprpa_ctx* c);
// Waits for the context's stream (see pprpa_ctx::blocking_sync).
int ctx_sync(pprpa_ctx* c);
// Pinned host staging of at least `bytes` (pprpa_ctx::hstage, slot 0 or 1), grown on demand.
int host_stage(pprpa_ctx* c, size_t bytes, void** out, int slot = 0);

// Tensor-core sigma provider of a Davidson solve run among others (pprpa_solve_batch): the
// solve hands its BF16 (nterms 1) or BF16x3 (nterms 3) products of k device vectors to it
// instead of launching them itself.
struct SigmaHook {
    virtual ~SigmaHook() {}
    virtual int sigma(pprpa_ctx* c, int mult, int k, const double* z, double* out, int nterms) = 0;
};
// pprpa_solve after its argument checks; hook may be null.
int solve_checked(pprpa_ctx* c, const pprpa_options* o, double* omega, double* X, double* Y,
                  double* ec, pprpa_info* info, SigmaHook* hook);

}  // namespace pprpa
