// pprpa_sigma_noalloc: the FP64 sigma (sigma = M z through sum_P L^P Zt L^P) for callers
// that must not allocate device memory.
//
// Some host programs cannot call cudaMalloc at the point where they need sigma: code that
// runs inside another framework's memory pool with a fixed budget (where a raw allocation
// would bypass its accounting or fail), latency-critical loops where the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable, or plugins whose host forbids
// allocating from inside its callbacks.  This entry point takes every input and output
// from the caller and keeps its intermediates (pair tables, packed pair matrices, the
// per-P products and the output blocks) in one file-scope device array of fixed size.
//
// The array is part of the library image: every GPU that loads the library holds it until
// the process exits.  All calls share it and it keeps the previous call's contents, so the
// parts that must start at zero are cleared on every call, and two calls whose work
// overlaps on the GPU (different streams, or different host threads on one device) race
// on it: order them on one stream or serialise them.
#include <mutex>

#include "kernels.h"

namespace pprpa {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  Host code only has a
// host-side stand-in for the symbol, so the address is looked up once per device, with
// that device current, and cached.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(PPRPA_ERR_ARG, "sigma_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(PPRPA_ERR_CUDA, std::string("sigma_noalloc: cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PPRPA_OK;
}

// Pair tables (virtual pairs, then occupied pairs; row-major upper triangle) written by one
// thread per row of each block.
__global__ void noalloc_pairs_kernel(int no, int nv, int mult, int nvv, int* pp, int* pq) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int tri = mult == 1 ? 0 : 1;  // triplet rows start one past the diagonal
    if (r < nv) {
        const int off = r * nv - r * (r - 1) / 2 - tri * r;
        int t = off;
        for (int b = r + tri; b < nv; ++b, ++t) { pp[t] = no + r; pq[t] = no + b; }
    } else if (r < nv + no) {
        const int i = r - nv;
        const int off = nvv + i * no - i * (i - 1) / 2 - tri * i;
        int t = off;
        for (int j = i + tri; j < no; ++j, ++t) { pp[t] = i; pq[t] = j; }
    }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace pprpa

using namespace pprpa;

extern "C" int pprpa_sigma_noalloc(int mult, int nocc_act, int nvir_act, int naux, const double* L,
                                   const double* eps, int k, const double* z, double* sigma,
                                   void* cuda_stream) {
    if (mult != 1 && mult != 3) return set_error(PPRPA_ERR_ARG, "sigma_noalloc: mult must be 1 or 3");
    if (nocc_act < 0 || nvir_act < 0 || nocc_act + nvir_act == 0 || naux <= 0 || k < 0)
        return set_error(PPRPA_ERR_ARG, "sigma_noalloc: bad sizes");
    if (k == 0) return PPRPA_OK;
    if (!L || !eps || !z || !sigma) return set_error(PPRPA_ERR_ARG, "sigma_noalloc: null pointer");
    const int no = nocc_act, nv = nvir_act, n = no + nv;
    const int tri = mult == 1 ? 0 : 1;
    const int64_t nvv = (int64_t)nv * (nv + 1) / 2 - (int64_t)tri * nv;
    const int64_t noo = (int64_t)no * (no + 1) / 2 - (int64_t)tri * no;
    const int64_t N = nvv + noo;
    const int64_t n2 = (int64_t)n * n;
    // scratch: pair tables, Zt [k][n][n], O [k][n][n], then T [pc][k][n][n] with pc >= 1
    const size_t b_pairs = align256(sizeof(int) * (size_t)N);
    const size_t b_mat = align256(sizeof(double) * (size_t)(k * n2));
    const size_t fixed = 2 * b_pairs + 2 * b_mat;
    if (fixed + b_mat > kNoAllocScratchBytes)
        return set_error(PPRPA_ERR_ARG,
                         "sigma_noalloc: problem too large for the 64 MiB scratch (needs 3*k*n^2*8 + "
                         "8*N bytes; use pprpa_sigma)");
    int dev = 0;
    PP_CUDA(cudaGetDevice(&dev));
    unsigned char* base;
    PP_TRY(scratch_address(dev, (void**)&base));
    int* pp = (int*)base;
    int* pq = (int*)(base + b_pairs);
    double* Zt = (double*)(base + 2 * b_pairs);
    double* O = (double*)(base + 2 * b_pairs + b_mat);
    double* T = (double*)(base + fixed);
    // auxiliary slices per pass: as many products as the scratch holds (the batched GEMM
    // launches split themselves where pc * k products exceed one grid)
    const int pc = (int)std::min<int64_t>(naux, (int64_t)((kNoAllocScratchBytes - fixed) / b_mat));
    cudaStream_t st = (cudaStream_t)cuda_stream;

    noalloc_pairs_kernel<<<(unsigned)ceil_div(n, 128), 128, 0, st>>>(no, nv, mult, (int)nvv, pp, pq);
    PP_CHECK_LAUNCH();
    PP_CUDA(cudaMemsetAsync(Zt, 0, sizeof(double) * (size_t)(k * n2), st));
    PP_TRY(launch_unpack_f64(z, k, (int)N, pp, pq, n, mult, Zt, st));
    for (int P0 = 0; P0 < naux; P0 += pc) {
        const int np = std::min(pc, naux - P0);
        const double* L0 = L + (int64_t)P0 * n2;
        for (int blk = 0; blk < 2; ++blk) {  // T[P][j] = L^P Zt_j on the virtual / occupied columns
            const int off = blk == 0 ? no : 0, sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            Dgemm g;
            g.M = n; g.N = sz; g.K = sz;
            g.A = L0 + off; g.lda = n; g.sA1 = n2;
            g.B = Zt + (int64_t)off * n + off; g.ldb = n; g.sB2 = n2;
            g.C = T + off; g.ldc = n; g.sC1 = n2 * k; g.sC2 = n2;
            g.nb1 = np; g.nb2 = k;
            PP_TRY(dgemm(g, st));
        }
        for (int blk = 0; blk < 2; ++blk) {  // O_j[blk] (+)= sum_P T[P][j][blk rows] L^P[:, blk]
            const int off = blk == 0 ? no : 0, sz = blk == 0 ? nv : no;
            if (sz == 0) continue;
            Dgemm g;
            g.M = sz; g.N = sz; g.K = n;
            g.A = T + (int64_t)off * n; g.lda = n; g.sA1 = n2; g.sAr = n2 * k;
            g.B = L0 + off; g.ldb = n; g.sBr = n2;
            g.C = O + (int64_t)off * n + off; g.ldc = n; g.sC1 = n2;
            g.nb1 = k; g.nr = np;
            g.beta = P0 == 0 ? 0.0 : 1.0;
            PP_TRY(dgemm(g, st));
        }
    }
    PP_TRY(launch_pack_f64(O, z, k, (int)N, (int)nvv, pp, pq, n, eps, mult, sigma, st));
    return PPRPA_OK;
}
