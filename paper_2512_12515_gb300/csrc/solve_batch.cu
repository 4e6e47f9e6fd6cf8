// pprpa_solve_batch: Davidson solves of many molecules at once, their tensor-core sigma
// products gathered into the batched persistent launch.
//
// Each molecule's Davidson iteration (Sec. "Implementation Details": the lowest roots of
// Eq. eigen_equation by the Davidson algorithm) runs on its own host thread and its own CUDA
// stream, so the per-molecule FP64 steps (projections, the one-CTA Rayleigh-Ritz
// eigensolve, residuals, corrections, orthonormalisation) of different molecules overlap on
// the GPU.  Whenever a solve needs a BF16 or BF16x3 sigma it hands its vectors to a
// rendezvous; when every molecule still iterating has posted, the last one runs a single
// batched sigma over all of them (sigma_tc_batch: one persistent tensor-core launch per stage
// for the small molecules, replayed from a CUDA graph while the batch keeps its shape, and
// clustered launches for the large ones) on the batch's stream, and releases them.  A solve
// that finishes leaves the rendezvous, so the others never wait for it.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

namespace pprpa {
namespace {

struct Request {
    bool on = false;
    int mult = 1, k = 0, nterms = 1;
    double* z = nullptr;  // staging copies (device, per molecule, stable between rounds)
    double* s = nullptr;
    int rc = PPRPA_OK;
};

class BatchSigma : public SigmaHook {
  public:
    BatchSigma(int nmol, pprpa_ctx* const* ctxs, pprpa_ctx* owner, int kcap)
        : ctxs_(ctxs, ctxs + nmol), owner_(owner), req_(nmol), active_(nmol), kcap_(kcap) {}

    // A block larger than kcap vectors (the guess, a collapse) goes over several rounds, so
    // that every molecule's intermediate T of a round holds at most kcap vectors.
    int sigma(pprpa_ctx* c, int mult, int k, const double* z, double* out, int nterms) override {
        PairTable* pt;
        PP_TRY(ensure_pairs(c, mult, &pt));
        for (int j0 = 0; j0 < k; j0 += kcap_) {
            const int kj = std::min(kcap_, k - j0);
            PP_TRY(round_trip(c, mult, kj, z + (size_t)j0 * pt->N, out + (size_t)j0 * pt->N, nterms, pt->N));
        }
        return PPRPA_OK;
    }

    int round_trip(pprpa_ctx* c, int mult, int k, const double* z, double* out, int nterms, int N) {
        const int m = index_of(c);
        if (m < 0) return set_error(PPRPA_ERR_ARG, "solve_batch: unknown context");
        const size_t bytes = sizeof(double) * (size_t)k * N;
        // staging buffers of kcap vectors: their addresses, and the batch's graph, stay fixed
        // between rounds
        double *zs, *ss;
        PP_TRY(ws_get(c, "bsolve_z", sizeof(double) * (size_t)kcap_ * N, (void**)&zs));
        PP_TRY(ws_get(c, "bsolve_s", sizeof(double) * (size_t)kcap_ * N, (void**)&ss));
        PP_CUDA(cudaMemcpyAsync(zs, z, bytes, cudaMemcpyDeviceToDevice, c->stream));
        PP_TRY(ctx_sync(c));
        int rc;
        {
            std::unique_lock<std::mutex> lk(mu_);
            Request& r = req_[m];
            r.on = true;
            r.mult = mult;
            r.k = k;
            r.nterms = nterms;
            r.z = zs;
            r.s = ss;
            r.rc = PPRPA_OK;
            ++posted_;
            const unsigned long long my = round_;
            if (posted_ == active_) run_locked();
            else cv_.wait(lk, [&] { return round_ != my; });
            rc = req_[m].rc;
        }
        if (rc != PPRPA_OK) return rc;
        PP_CUDA(cudaMemcpyAsync(out, ss, bytes, cudaMemcpyDeviceToDevice, c->stream));
        return PPRPA_OK;
    }

    // A solve is over: the others stop waiting for it.
    void leave() {
        std::unique_lock<std::mutex> lk(mu_);
        --active_;
        if (active_ > 0 && posted_ == active_) run_locked();
    }

    int rounds() const { return (int)round_; }
    double sigma_seconds() const { return sigma_s_; }
    double issue_seconds() const { return issue_s_; }
    double tensor_flops() const { return flops_; }

  private:
    int index_of(pprpa_ctx* c) const {
        for (size_t m = 0; m < ctxs_.size(); ++m)
            if (ctxs_[m] == c) return (int)m;
        return -1;
    }

    // Every molecule still iterating has posted: one batched sigma per arithmetic form.
    void run_locked() {
        for (int nterms : {1, 3}) {
            std::vector<pprpa_ctx*> cs;
            std::vector<int> mults, ks;
            std::vector<const double*> zs;
            std::vector<double*> ss;
            std::vector<int> who;
            for (size_t m = 0; m < req_.size(); ++m) {
                const Request& r = req_[m];
                if (!r.on || r.nterms != nterms) continue;
                cs.push_back(ctxs_[m]);
                mults.push_back(r.mult);
                ks.push_back(r.k);
                zs.push_back(r.z);
                ss.push_back(r.s);
                who.push_back((int)m);
            }
            if (cs.empty()) continue;
            const auto t0 = std::chrono::steady_clock::now();
            int rc = sigma_tc_batch((int)cs.size(), cs.data(), mults.data(), ks.data(), zs.data(), ss.data(),
                                    nterms, owner_->stream, owner_, use_graph_);
            issue_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            for (size_t q = 0; q < cs.size(); ++q)
                flops_ += (double)ks[q] * nterms * 3.0 * cs[q]->naux * cs[q]->n() *
                          ((double)cs[q]->nv * cs[q]->nv + (double)cs[q]->no * cs[q]->no);
            if (rc == PPRPA_OK) rc = ctx_sync(owner_);
            if (rc == PPRPA_OK) rc = check_status(owner_);
            sigma_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            for (int m : who) req_[m].rc = rc;
        }
        for (Request& r : req_) r.on = false;
        posted_ = 0;
        ++round_;
        cv_.notify_all();
    }

    std::vector<pprpa_ctx*> ctxs_;
    pprpa_ctx* owner_;
    // the batch changes shape almost every round (molecules converge and leave, blocks
    // shrink), so each round's graph runs once; PPRPA_SOLVE_BATCH_GRAPH=0 launches directly
    // (measured the same)
    bool use_graph_ = getenv("PPRPA_SOLVE_BATCH_GRAPH") ? atoi(getenv("PPRPA_SOLVE_BATCH_GRAPH")) != 0 : true;
    // time in the batched sigma rounds, of it the part before the final wait (host work and
    // the molecules that run on their own launches), and the tensor-core flop issued
    // (printed with PPRPA_BATCH_LOG=1)
    double sigma_s_ = 0.0, issue_s_ = 0.0, flops_ = 0.0;
    std::vector<Request> req_;
    int active_;
    int kcap_;
    int posted_ = 0;
    unsigned long long round_ = 0;
    std::mutex mu_;
    std::condition_variable cv_;
};

}  // namespace
}  // namespace pprpa

using namespace pprpa;

extern "C" int pprpa_solve_batch(int nmol, pprpa_ctx* const* ctxs, const pprpa_options* opts,
                                 double* const* omega, double* const* X, double* const* Y,
                                 pprpa_info* infos, int* rcs) {
    if (nmol <= 0 || !ctxs || !opts || !omega || !rcs) return set_error(PPRPA_ERR_ARG, "solve_batch: bad arguments");
    for (int m = 0; m < nmol; ++m) {
        if (!ctxs[m]) return set_error(PPRPA_ERR_ARG, "solve_batch: null context");
        if (ctxs[m]->device != ctxs[0]->device)
            return set_error(PPRPA_ERR_ARG, "solve_batch: all contexts must share one device");
        for (int q = 0; q < m; ++q)
            if (ctxs[q] == ctxs[m]) return set_error(PPRPA_ERR_ARG, "solve_batch: a context appears twice");
        if (opts[m].method != PPRPA_METHOD_DAVIDSON)
            return set_error(PPRPA_ERR_ARG, "solve_batch: every molecule must use the Davidson method");
        if (!omega[m]) return set_error(PPRPA_ERR_ARG, "solve_batch: null omega");
    }
    PP_CUDA(cudaSetDevice(ctxs[0]->device));
    // the batch's own context: its stream runs the batched sigma, and it owns the batch plans
    pprpa_ctx* owner = nullptr;
    PP_TRY(pprpa_create(&owner, ctxs[0]->device, nullptr));
    owner->blocking_sync = true;
    std::vector<std::thread> threads;
    std::vector<std::string> errs(nmol);
    {
        // vectors per molecule and round (PPRPA_BATCH_KCAP, default 8): bounds the sum over
        // molecules of the first-stage intermediates
        const char* kv = getenv("PPRPA_BATCH_KCAP");
        const int kcap = std::max(1, kv ? atoi(kv) : 8);
        BatchSigma hub(nmol, ctxs, owner, kcap);
        threads.reserve(nmol);
        for (int m = 0; m < nmol; ++m) {
            threads.emplace_back([&, m] {
                cudaSetDevice(ctxs[m]->device);
                const bool keep = ctxs[m]->blocking_sync;
                ctxs[m]->blocking_sync = true;  // many threads wait at once: block, do not spin
                rcs[m] = solve_checked(ctxs[m], &opts[m], omega[m], X ? X[m] : nullptr, Y ? Y[m] : nullptr,
                                       nullptr, infos ? &infos[m] : nullptr, &hub);
                if (rcs[m] != PPRPA_OK) errs[m] = pprpa_last_error();
                ctxs[m]->blocking_sync = keep;
                hub.leave();
            });
        }
        for (auto& t : threads) t.join();
        if (getenv("PPRPA_BATCH_LOG") && atoi(getenv("PPRPA_BATCH_LOG")))
            fprintf(stderr, "[pprpa] solve_batch: %d rounds, %.3f s in the batched sigma (%.3f s issuing), %.3g tensor flop\n",
                    hub.rounds(), hub.sigma_seconds(), hub.issue_seconds(), hub.tensor_flops());
    }
    pprpa_destroy(owner);
    for (int m = 0; m < nmol; ++m)
        if (rcs[m] != PPRPA_OK)
            return set_error(rcs[m], "solve_batch: molecule " + std::to_string(m) + ": " + errs[m]);
    return PPRPA_OK;
}
