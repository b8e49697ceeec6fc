// Batched solves: many independent corrector systems advanced together, one
// launch per phase for all of them (the ensemble use case: one assembled
// matrix per member, Sec. 3.1 assembly-once applies to each).
//
// Work is cut into tiles of kTileRows consecutive rows of one system.  A fixed
// grid walks a list of the tiles of systems still running; the list is
// rebuilt on the device at the start of every chunk of iterations from the
// systems' stop flags (the per-system convergence mask), so finished systems
// cost nothing.  Each system keeps its own scalar state (alpha, beta, rho,
// stop flag) and its own partial sums: a tile writes its partial, the block
// that completes a system's last tile adds them in tile order (deterministic)
// and updates that system's scalars.  The iteration is the FP64 Jacobi loop
// of pcg_kernels.cuh (three kernels); a chunk of iterations is one CUDA graph.
#include "cps_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

namespace cps {
namespace {

constexpr int kTileRows = 2048;   // 8 rows per thread per tile
constexpr int kBatchChunk = 32;
constexpr int kBatchCheck = 8;

struct BatchDesc {
    const double* a;
    const int32_t* col;
    const double* s;
    const double* b;
    double* x;
    double* y;
    double* r;
    double* p;
    double* q;
    double* partials;
    CgState* st;
    int64_t n;
    int32_t ntiles;
    int32_t pad;
};

struct TileRef {
    int32_t sys;
    int32_t tile;
};


// Sum of a per-tile partial over the block; returns true in the block that
// completed the system's last tile, with the system's totals in v[].
template <int NV>
__device__ __forceinline__ bool tile_sum(double (&v)[NV], const BatchDesc& d, int tile,
                                         unsigned int* arrive, bool* last) {
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) d.partials[k * kMaxGrid * 4 + tile] = v[k];
        __threadfence();
        const unsigned int t = atomicAdd(arrive, 1u);
        *last = (t == (unsigned)d.ntiles - 1u);
    }
    __syncthreads();
    if (!*last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < d.ntiles; i += blockDim.x)
            acc += __ldcg(&d.partials[k * kMaxGrid * 4 + i]);
        v[k] = acc;
    }
    block_sum<NV>(v);
    if (threadIdx.x == 0) *arrive = 0u;
    return true;
}

#define CPS_TILE_LOOP(tiles, ntile_ptr)                                                  \
    const int ntl_ = *(ntile_ptr);                                                       \
    for (int ti_ = blockIdx.x; ti_ < ntl_; ti_ += gridDim.x)

// The stop flag of a tile's system, read once and shared by the block so that
// the whole block takes the same branch.
__device__ __forceinline__ int block_done(const CgState* st) {
    __shared__ int v;
    __syncthreads();
    if (threadIdx.x == 0) v = *(volatile const int*)&st->done;
    __syncthreads();
    return v;
}

__global__ void kb_compact(const BatchDesc* __restrict__ d, int nsys, TileRef* tiles,
                           int* ntiles) {
    // one block: prefix over systems still running
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
        const int i = s0 + threadIdx.x;
        const int cnt = (i < nsys && d[i].st->done == 0) ? d[i].ntiles : 0;
        // inclusive scan of cnt across the block
        __shared__ int sc[1024];
        sc[threadIdx.x] = cnt;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
            __syncthreads();
            sc[threadIdx.x] += v;
            __syncthreads();
        }
        const int start = base + sc[threadIdx.x] - cnt;
        for (int t = 0; t < cnt; ++t) tiles[start + t] = TileRef{i, t};
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base += sc[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ntiles = base;
}

// Every tile of every system (for the run start and end).
__global__ void kb_all_tiles(const BatchDesc* __restrict__ d, int nsys, TileRef* tiles,
                             int* ntiles) {
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int s0 = 0; s0 < nsys; s0 += blockDim.x) {
        const int i = s0 + threadIdx.x;
        const int cnt = i < nsys ? d[i].ntiles : 0;
        __shared__ int sc[1024];
        sc[threadIdx.x] = cnt;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
            __syncthreads();
            sc[threadIdx.x] += v;
            __syncthreads();
        }
        const int start = base + sc[threadIdx.x] - cnt;
        for (int t = 0; t < cnt; ++t) tiles[start + t] = TileRef{i, t};
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base += sc[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ntiles = base;
}

// y = S x, r = S^-1 b - Ahat y, p = r; per system rho, ||b||^2, ||S r||^2.
__global__ void __launch_bounds__(kBlock) kb_init(const BatchDesc* __restrict__ dd,
                                                  const TileRef* __restrict__ tiles,
                                                  const int* ntile, double rtol,
                                                  long long budget) {
    __shared__ bool last;
    CPS_TILE_LOOP(tiles, ntile) {
        const TileRef tr = tiles[ti_];
        const BatchDesc d = dd[tr.sys];
        const int64_t n = d.n;
        double rr = 0.0, bb = 0.0, nn = 0.0;
        const int64_t r0 = (int64_t)tr.tile * kTileRows;
#pragma unroll 4
        for (int64_t e = r0 + threadIdx.x; e < r0 + kTileRows && e < n; e += blockDim.x) {
            const double se = d.s[e];
            const double ye = se * d.x[e];
            double ay = ye;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int32_t c = d.col[j * n + e];
                ay = fma(d.a[j * n + e], d.s[c] * d.x[c], ay);
            }
            const double be = d.b[e];
            const double re = be / se - ay;
            d.y[e] = ye;
            d.r[e] = re;
            d.p[e] = re;
            rr = fma(re, re, rr);
            bb = fma(be, be, bb);
            const double t = se * re;
            nn = fma(t, t, nn);
        }
        double v[3] = {rr, bb, nn};
        if (tile_sum<3>(v, d, tr.tile, &d.st->arrive[2], &last) && threadIdx.x == 0) {
            CgState* st = d.st;
            st->rho = v[0];
            st->bnorm2 = v[1];
            st->thresh2 = rtol * rtol * v[1];
            st->rnorm2 = v[2];
            st->alpha = 0.0;
            st->beta = 0.0;
            st->gamma = 0.0;
            st->iter = 0;
            st->max_iter = budget;
            st->status = CPS_OK;
            st->done = (v[1] == 0.0 || v[2] <= st->thresh2 || budget <= 0) ? 2 : 0;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) kb_spmv(const BatchDesc* __restrict__ dd,
                                                  const TileRef* __restrict__ tiles,
                                                  const int* ntile) {
    __shared__ bool last;
    CPS_TILE_LOOP(tiles, ntile) {
        const TileRef tr = tiles[ti_];
        const BatchDesc d = dd[tr.sys];
        const int dn = block_done(d.st);
        if (dn) {
            if (dn == 1 && tr.tile == 0 && threadIdx.x == 0) d.st->done = 2;
            continue;
        }
        const int64_t n = d.n;
        double acc = 0.0;
        const int64_t r0 = (int64_t)tr.tile * kTileRows;
#pragma unroll 4
        for (int64_t e = r0 + threadIdx.x; e < r0 + kTileRows && e < n; e += blockDim.x) {
            const double pe = d.p[e];
            double v = pe;
#pragma unroll
            for (int j = 0; j < 3; ++j) v = fma(d.a[j * n + e], d.p[d.col[j * n + e]], v);
            d.q[e] = v;
            acc = fma(pe, v, acc);
        }
        double t[1] = {acc};
        if (tile_sum<1>(t, d, tr.tile, &d.st->arrive[0], &last) && threadIdx.x == 0) {
            CgState* st = d.st;
            st->gamma = t[0];
            if (!(t[0] > 0.0) || !isfinite(t[0])) {
                st->status = CPS_ERR_NOT_SPD;
                st->done = 2;
            } else {
                st->alpha = st->rho / t[0];
            }
        }
        __syncthreads();
    }
}

template <bool NORM>
__global__ void __launch_bounds__(kBlock) kb_update(const BatchDesc* __restrict__ dd,
                                                    const TileRef* __restrict__ tiles,
                                                    const int* ntile) {
    __shared__ bool last;
    CPS_TILE_LOOP(tiles, ntile) {
        const TileRef tr = tiles[ti_];
        const BatchDesc d = dd[tr.sys];
        if (block_done(d.st)) continue;
        const int64_t n = d.n;
        const double al = d.st->alpha;
        double rr = 0.0, nn = 0.0;
        const int64_t r0 = (int64_t)tr.tile * kTileRows;
#pragma unroll 4
        for (int64_t e = r0 + threadIdx.x; e < r0 + kTileRows && e < n; e += blockDim.x) {
            const double re = fma(-al, d.q[e], d.r[e]);
            d.r[e] = re;
            rr = fma(re, re, rr);
            if (NORM) {
                const double t = d.s[e] * re;
                nn = fma(t, t, nn);
            }
        }
        double t[2] = {rr, nn};
        if (tile_sum<2>(t, d, tr.tile, &d.st->arrive[1], &last) && threadIdx.x == 0) {
            CgState* st = d.st;
            const long long it = st->iter + 1;
            st->iter = it;
            int done = 0;
            if (NORM) {
                st->rnorm2 = t[1];
                if (t[1] <= st->thresh2) done = 1;
            }
            if (it >= st->max_iter) done = 1;
            if (!(t[0] > 0.0)) done = 1;
            st->beta = t[0] / st->rho;
            st->rho = t[0];
            if (done) st->done = 1;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) kb_direction(const BatchDesc* __restrict__ dd,
                                                       const TileRef* __restrict__ tiles,
                                                       const int* ntile) {
    CPS_TILE_LOOP(tiles, ntile) {
        const TileRef tr = tiles[ti_];
        const BatchDesc d = dd[tr.sys];
        if (block_done(d.st) == 2) continue;
        const int64_t n = d.n;
        const double al = d.st->alpha, be = d.st->beta;
        const int64_t r0 = (int64_t)tr.tile * kTileRows;
#pragma unroll 4
        for (int64_t e = r0 + threadIdx.x; e < r0 + kTileRows && e < n; e += blockDim.x) {
            const double pe = d.p[e];
            d.y[e] = fma(al, pe, d.y[e]);
            d.p[e] = fma(be, pe, d.r[e]);
        }
    }
}

// x = S^-1 y and the true residual per system.
__global__ void __launch_bounds__(kBlock) kb_final(const BatchDesc* __restrict__ dd,
                                                   const TileRef* __restrict__ tiles,
                                                   const int* ntile) {
    __shared__ bool last;
    CPS_TILE_LOOP(tiles, ntile) {
        const TileRef tr = tiles[ti_];
        const BatchDesc d = dd[tr.sys];
        const int64_t n = d.n;
        const bool zero = d.st->bnorm2 == 0.0;
        double nn = 0.0;
        const int64_t r0 = (int64_t)tr.tile * kTileRows;
#pragma unroll 4
        for (int64_t e = r0 + threadIdx.x; e < r0 + kTileRows && e < n; e += blockDim.x) {
            if (zero) {
                d.x[e] = 0.0;
                continue;
            }
            const double se = d.s[e], ye = d.y[e];
            double ay = ye;
#pragma unroll
            for (int j = 0; j < 3; ++j) ay = fma(d.a[j * n + e], d.y[d.col[j * n + e]], ay);
            const double res = d.b[e] - se * ay;
            d.x[e] = ye / se;
            nn = fma(res, res, nn);
        }
        double t[1] = {nn};
        if (tile_sum<1>(t, d, tr.tile, &d.st->arrive[3], &last) && threadIdx.x == 0)
            d.st->rnorm2 = t[0];
        __syncthreads();
    }
}

// Systems still running after a chunk (0 when all have stopped).
__global__ void kb_count_running(const BatchDesc* __restrict__ d, int nsys, int* out) {
    int c = 0;
    for (int i = threadIdx.x; i < nsys; i += blockDim.x) c += d[i].st->done == 0 ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ int sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        *out = t;
    }
}

}  // namespace

// Mixed-precision ensemble.  Each system's binary32 solve takes its own
// residual-replacement decisions on the host between its graph chunks, so
// the systems cannot share one launch per phase as the FP64 batch does.
// Instead kMixedWorkers host threads take systems from a shared counter and
// run each system's whole solve on the thread's own stream: the graph chunks
// of different systems overlap on the GPU (most systems of an ensemble are
// small, and a small system's solve is bound by launch latency, not by
// bandwidth).  The caller's stream is ordered before and after all of it.
constexpr int kMixedWorkers = 8;

static int solve_batch_mixed(const cps_sys* systems, int nsys, const double* const* b,
                             double* const* x, double rtol, int64_t max_iter, int precision,
                             cps_stats* stats, cudaStream_t stream) {
    cps_ctx ctx = systems[0]->ctx;
    const int nw = std::min(nsys, kMixedWorkers);
    std::vector<cudaStream_t> streams(nw, nullptr);
    std::vector<cudaEvent_t> done(nw, nullptr);
    cudaEvent_t ready = nullptr;
    int rc = CPS_OK;
    auto cleanup = [&]() {
        for (auto& st : streams)
            if (st) cudaStreamDestroy(st);
        for (auto& ev : done)
            if (ev) cudaEventDestroy(ev);
        if (ready) cudaEventDestroy(ready);
    };
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) rc = CPS_ERR_CUDA;
    for (int w = 0; w < nw && rc == CPS_OK; ++w)
        if (cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) != cudaSuccess)
            rc = CPS_ERR_CUDA;
    if (rc == CPS_OK && cudaEventRecord(ready, stream) != cudaSuccess) rc = CPS_ERR_CUDA;
    if (rc != CPS_OK) {
        cudaGetLastError();
        cleanup();
        cps::set_error(ctx, "solve_batch: could not create worker streams");
        return rc;
    }
    std::vector<int> rcs(nsys, CPS_OK);
    std::atomic<int> next{0};
    auto work = [&](int w) {
        cudaSetDevice(ctx->device);
        cudaStreamWaitEvent(streams[w], ready, 0);
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nsys) break;
            rcs[i] = solve_impl(systems[i], b[i], x[i], rtol, max_iter, precision,
                                stats ? &stats[i] : nullptr, streams[w]);
        }
        cudaEventRecord(done[w], streams[w]);
    };
    std::vector<std::thread> threads;
    threads.reserve(nw);
    for (int w = 0; w < nw; ++w) threads.emplace_back(work, w);
    for (auto& th : threads) th.join();
    for (int w = 0; w < nw; ++w) cudaStreamWaitEvent(stream, done[w], 0);
    cleanup();
    for (int i = 0; i < nsys; ++i)
        if (rcs[i] != CPS_OK) return rcs[i];
    return CPS_OK;
}

int solve_batch_impl(const cps_sys* systems, int nsys, const double* const* b,
                     double* const* x, double rtol, int64_t max_iter, int precision,
                     cps_stats* stats, cudaStream_t stream) {
    cps_ctx ctx = systems[0]->ctx;
    for (int i = 0; i < nsys; ++i) {
        if (!b[i] || !x[i]) {
            cps::set_error(ctx, "solve_batch: null vector");
            return CPS_ERR_ARG;
        }
    }
    if (!(rtol >= 0.0) || max_iter < 0) {
        cps::set_error(ctx, "solve_batch: bad argument");
        return CPS_ERR_ARG;
    }
    if (precision != CPS_FP64) return solve_batch_mixed(systems, nsys, b, x, rtol, max_iter,
                                                        precision, stats, stream);
    std::vector<BatchDesc> hd(nsys);
    int64_t total_tiles = 0;
    for (int i = 0; i < nsys; ++i) {
        cps_sys s = systems[i];
        BatchDesc& d = hd[i];
        d.a = s->a;
        d.col = s->col;
        d.s = s->s;
        d.b = b[i];
        d.x = x[i];
        d.y = s->wy;
        d.r = s->wr;
        d.p = s->wp0;
        d.q = s->wq;
        d.partials = s->partials;
        d.st = s->st;
        d.n = s->nt;
        d.ntiles = (int32_t)((s->nt + kTileRows - 1) / kTileRows);
        d.pad = 0;
        if (d.ntiles > 4 * kMaxGrid) {
            cps::set_error(ctx, "solve_batch: a system is too large for the batched path");
            return CPS_ERR_ARG;
        }
        total_tiles += d.ntiles;
    }
    BatchDesc* dd = nullptr;
    TileRef* tiles = nullptr;
    int* counts = nullptr;       // [0] tiles in the list, [1] systems running
    int* hcount = nullptr;
    CPS_CUDA_TRY(ctx, cudaMallocAsync((void**)&dd, sizeof(BatchDesc) * nsys, stream));
    CPS_CUDA_TRY(ctx, cudaMallocAsync((void**)&tiles, sizeof(TileRef) * total_tiles, stream));
    CPS_CUDA_TRY(ctx, cudaMallocAsync((void**)&counts, sizeof(int) * 2, stream));
    CPS_CUDA_TRY(ctx, cudaMallocHost((void**)&hcount, sizeof(int)));
    CPS_CUDA_TRY(ctx, cudaMemcpyAsync(dd, hd.data(), sizeof(BatchDesc) * nsys,
                                      cudaMemcpyHostToDevice, stream));
    const int grid = grid_for(ctx, total_tiles * kTileRows, 8);
    const int cblock = nsys < 1024 ? ((nsys + 31) / 32) * 32 : 1024;
    int rc = CPS_OK;
    int64_t launches = 0;
    std::vector<int64_t> iters(nsys, 0);
    std::vector<int> status(nsys, CPS_OK);
    cudaStream_t cap = nullptr;
    cudaGraphExec_t ge = nullptr;
    do {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
            rc = CPS_ERR_CUDA;
            break;
        }
        cudaGraph_t g = nullptr;
        cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        kb_compact<<<1, cblock, 0, cap>>>(dd, nsys, tiles, counts);
        for (int k = 0; k < kBatchChunk; ++k) {
            kb_spmv<<<grid, kBlock, 0, cap>>>(dd, tiles, counts);
            if (k % kBatchCheck == kBatchCheck - 1)
                kb_update<true><<<grid, kBlock, 0, cap>>>(dd, tiles, counts);
            else
                kb_update<false><<<grid, kBlock, 0, cap>>>(dd, tiles, counts);
            kb_direction<<<grid, kBlock, 0, cap>>>(dd, tiles, counts);
        }
        kb_count_running<<<1, cblock, 0, cap>>>(dd, nsys, counts + 1);
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        if (ce != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            rc = CPS_ERR_CUDA;
            break;
        }
        cudaGraphDestroy(g);
        const int64_t per_chunk = 2 + 3 * kBatchChunk;
        // Restart rounds: systems whose true residual misses rtol start again
        // from their x (those that met it stop at once in kb_init).
        for (int round = 0; round < 8 && rc == CPS_OK; ++round) {
            int64_t spent = 0;
            for (int i = 0; i < nsys; ++i) spent = iters[i] > spent ? iters[i] : spent;
            kb_all_tiles<<<1, cblock, 0, stream>>>(dd, nsys, tiles, counts);
            kb_init<<<grid, kBlock, 0, stream>>>(dd, tiles, counts, rtol,
                                                 (long long)(max_iter - spent));
            launches += 2;
            for (;;) {
                if (cudaGraphLaunch(ge, stream) != cudaSuccess) {
                    rc = CPS_ERR_CUDA;
                    break;
                }
                launches += per_chunk;
                cudaMemcpyAsync(hcount, counts + 1, sizeof(int), cudaMemcpyDeviceToHost, stream);
                if (cudaStreamSynchronize(stream) != cudaSuccess) {
                    rc = CPS_ERR_CUDA;
                    break;
                }
                if (*hcount == 0) break;
            }
            if (rc) break;
            kb_all_tiles<<<1, cblock, 0, stream>>>(dd, nsys, tiles, counts);
            kb_final<<<grid, kBlock, 0, stream>>>(dd, tiles, counts);
            launches += 2;
            bool again = false;
            for (int i = 0; i < nsys; ++i) {
                CgState h;
                if (cudaMemcpyAsync(&h, systems[i]->st, sizeof(CgState), cudaMemcpyDeviceToHost,
                                    stream) != cudaSuccess ||
                    cudaStreamSynchronize(stream) != cudaSuccess) {
                    rc = CPS_ERR_CUDA;
                    break;
                }
                iters[i] += h.iter;
                const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
                int st = h.status;
                if (st == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) {
                    st = CPS_ERR_NOT_CONVERGED;
                    if (iters[i] < max_iter) again = true;
                }
                status[i] = st;
                if (stats) {
                    stats[i].iters = iters[i];
                    stats[i].rel_res = rel;
                    stats[i].status = st;
                    stats[i].refinements = round + 1;
                    stats[i].launches = launches;
                }
            }
            if (!again) break;
        }
    } while (false);
    if (ge) cudaGraphExecDestroy(ge);
    if (cap) cudaStreamDestroy(cap);
    cudaFreeAsync(dd, stream);
    cudaFreeAsync(tiles, stream);
    cudaFreeAsync(counts, stream);
    cudaStreamSynchronize(stream);
    cudaFreeHost(hcount);
    if (rc != CPS_OK) {
        cps::set_error(ctx, "solve_batch: CUDA failure");
        return rc;
    }
    int first = CPS_OK;
    for (int i = 0; i < nsys; ++i)
        if (status[i] != CPS_OK && first == CPS_OK) first = status[i];
    if (first == CPS_ERR_NOT_CONVERGED) cps::set_error(ctx, "solve_batch: max_iter reached");
    if (first == CPS_ERR_NOT_SPD) cps::set_error(ctx, "solve_batch: p.Ap <= 0");
    return first;
}

}  // namespace cps
