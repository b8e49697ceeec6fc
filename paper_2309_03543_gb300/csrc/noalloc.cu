// Allocation-free solve: FP64 Jacobi-PCG on a matrix the caller already holds
// in the library's padded ELL form, for callers that cannot allocate device
// memory.  Some callers run where cudaMalloc is not available to them: inside
// a host that owns every device allocation through its own pool (and forbids
// other allocations), in code that must not trigger the implicit device
// synchronisation of cudaMalloc/cudaFree, or under a memory budget that has
// already been handed out.  This entry point only launches kernels; its
// working vectors live in one file-scope device array of fixed size.
//
// It runs the same kernels as cps_solve (pcg_kernels.cuh, compiled here in a
// namespace of their own) on the symmetrically scaled matrix, so its results
// agree with cps_solve's up to rounding.
#include "cps_internal.cuh"

#include <cmath>
#include <mutex>

namespace cps_noalloc {
using namespace ::cps;
#include "pcg_kernels.cuh"
}  // namespace cps_noalloc

namespace {

using cps::CgState;
using cps::kBlock;
using cps::kMaxGrid;

// Largest system this entry point accepts (rows), and the device scratch
// that size needs: scaled off-diagonals [3n], scale s [n], iterate, residual,
// direction and A p [4 x n], reduction partials and the iteration state.
constexpr int64_t kNoAllocMaxRows = 65536;
constexpr int kNoAllocGrid = (int)((kNoAllocMaxRows + kBlock - 1) / kBlock);   // 256 blocks
constexpr int kChunkIters = 32;
constexpr int kCheckEvery = 8;

struct Scratch {
    double a[3 * kNoAllocMaxRows];
    double s[kNoAllocMaxRows];
    double y[kNoAllocMaxRows];
    double r[kNoAllocMaxRows];
    double p[kNoAllocMaxRows];
    double q[kNoAllocMaxRows];
    double partials[cps::kNumPartials * kMaxGrid];
    CgState st;
    int err;
};

// About 4.3 MB per device that loads the library, held until the process
// exits.  Shared by every call: overlapping calls on the GPU race.
static __device__ __align__(256) unsigned char g_scratch[sizeof(Scratch)];

// Device address of g_scratch per device (host code cannot use the symbol
// itself as a pointer).
constexpr int kMaxDevices = 64;
static Scratch* g_addr[kMaxDevices] = {nullptr};
static std::mutex g_addr_mu;

int scratch_for_current_device(Scratch** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CPS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) return CPS_ERR_CUDA;
        g_addr[dev] = static_cast<Scratch*>(ptr);
    }
    *out = g_addr[dev];
    return CPS_OK;
}

__global__ void kn_sqrt_diag(const double* __restrict__ diag, int64_t n, double* __restrict__ s,
                             int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[e];
        if (!(d > 0.0) || !isfinite(d)) {
            atomicCAS(err, 0, CPS_ERR_NOT_SPD);
            s[e] = 1.0;
        } else {
            s[e] = sqrt(d);
        }
    }
}

__global__ void kn_scale(const int32_t* __restrict__ col, const double* __restrict__ val,
                         const double* __restrict__ s, int64_t n, double* __restrict__ a,
                         int* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < 3 * n;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k % n;
        const int32_t c = col[k];
        if (c < 0 || c >= n) {
            atomicCAS(err, 0, CPS_ERR_ARG);
            a[k] = 0.0;
            continue;
        }
        a[k] = val[k] / (s[e] * s[c]);
    }
}

int read_state(const Scratch* sc, cudaStream_t stream, CgState* h) {
    if (cudaMemcpyAsync(h, &sc->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return CPS_ERR_CUDA;
    return cudaStreamSynchronize(stream) == cudaSuccess ? CPS_OK : CPS_ERR_CUDA;
}

}  // namespace

extern "C" int cps_solve_ell_noalloc(int64_t n, const double* diag, const int32_t* col,
                                     const double* val, const double* b, double* x, double rtol,
                                     int64_t max_iter, cps_stats* stats, void* stream_ptr) {
    // Every return goes through finish(): stats, when given, always carries
    // the returned status (rel_res NaN where no residual was computed).
    int64_t total = 0, launches = 0;
    auto finish = [&](int status, double rel) -> int {
        if (stats) *stats = cps_stats{total, rel, status, 1, launches};
        return status;
    };
    const double kNoResidual = std::nan("");
    if (n < 0 || n > kNoAllocMaxRows) return finish(CPS_ERR_ARG, kNoResidual);
    if (n > 0 && (!diag || !col || !val || !b || !x)) return finish(CPS_ERR_ARG, kNoResidual);
    if (!(rtol >= 0.0) || max_iter < 0) return finish(CPS_ERR_ARG, kNoResidual);
    if (n == 0) return finish(CPS_OK, 0.0);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
    // An error left pending by the caller's earlier work is not this call's:
    // report it without clearing it, so that the caller still sees it.
    if (cudaPeekAtLastError() != cudaSuccess) return finish(CPS_ERR_CUDA, kNoResidual);
    Scratch* sc = nullptr;
    int rc = scratch_for_current_device(&sc);
    if (rc) return finish(rc, kNoResidual);
    namespace K = cps_noalloc::cps;
    const int g = kNoAllocGrid;
    // The state (including the reductions' arrival counters) and the error
    // flag must start at zero; the previous call's contents are stale.
    if (cudaMemsetAsync(&sc->st, 0, sizeof(CgState), stream) != cudaSuccess ||
        cudaMemsetAsync(&sc->err, 0, sizeof(int), stream) != cudaSuccess)
        return finish(CPS_ERR_CUDA, kNoResidual);
    kn_sqrt_diag<<<g, kBlock, 0, stream>>>(diag, n, sc->s, &sc->err);
    kn_scale<<<g, kBlock, 0, stream>>>(col, val, sc->s, n, sc->a, &sc->err);
    launches += 2;
    int herr = 0;
    if (cudaMemcpyAsync(&herr, &sc->err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return finish(CPS_ERR_CUDA, kNoResidual);
    if (herr) return finish(herr, kNoResidual);
    CgState h{};
    int status = CPS_OK;
    for (int restart = 0; restart < 8; ++restart) {
        const long long budget = (long long)(max_iter - total);
        K::k_init64<<<g, kBlock, 0, stream>>>(b, x, sc->s, sc->a, col, n, sc->y, sc->r, sc->p, rtol,
                                              budget, 1, sc->partials, &sc->st);
        ++launches;
        rc = read_state(sc, stream, &h);
        if (rc) return finish(rc, kNoResidual);
        while (!h.done && budget > 0) {
            for (int k = 0; k < kChunkIters; ++k) {
                K::k_spmv_dot<double, 2><<<g, kBlock, 0, stream>>>(sc->a, col, sc->p, sc->q, n,
                                                                 sc->partials, &sc->st);
                if (k % kCheckEvery == kCheckEvery - 1)
                    K::k_cg_b<double, true, true, 2><<<g, kBlock, 0, stream>>>(
                        sc->r, sc->q, sc->s, n, sc->partials, &sc->st);
                else
                    K::k_cg_b<double, false, true, 2><<<g, kBlock, 0, stream>>>(
                        sc->r, sc->q, sc->s, n, sc->partials, &sc->st);
                K::k_cg_c<double, 2><<<g, kBlock, 0, stream>>>(sc->y, sc->p, sc->r, n, &sc->st);
                launches += 3;
            }
            if (cudaGetLastError() != cudaSuccess) return finish(CPS_ERR_CUDA, kNoResidual);
            rc = read_state(sc, stream, &h);
            if (rc) return finish(rc, kNoResidual);
        }
        total += h.iter;
        status = h.status;
        K::k_final64<<<g, kBlock, 0, stream>>>(b, sc->y, sc->s, sc->a, col, n, x, sc->partials,
                                               &sc->st);
        ++launches;
        rc = read_state(sc, stream, &h);
        if (rc) return finish(rc, kNoResidual);
        if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
    }
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    if (status == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) status = CPS_ERR_NOT_CONVERGED;
    return finish(status, rel);
}
