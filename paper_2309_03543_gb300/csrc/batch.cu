// Batched solves: many independent corrector systems advanced together (the
// ensemble use case: one assembled matrix per member, Sec. 3.1 assembly-once
// applies to each).  Two FP64 designs:
//
// One launch (the default).  A cooperative launch of two 512-thread blocks
// per SM solves the whole ensemble: static teams of blocks take the largest
// systems (rows split, sums combined through bounded waits on a per-team
// arrival counter), every other block takes whole systems from a device work
// queue, and a team's blocks join the queue when their system is done.  The
// iteration is the single-reduction (Chronopoulos-Gear) Jacobi CG: a block
// alone on its rows is bound by memory latency, so two passes and two
// synchronisations per iteration beat the textbook three and three.
//
// Graph chunks.  Work is cut into tiles of kTileRows consecutive rows of one
// system.  A fixed grid walks a list of the tiles of systems still running;
// the list is rebuilt on the device at the start of every chunk of
// iterations from the systems' stop flags (the per-system convergence mask),
// so finished systems cost nothing.  Each system keeps its own scalar state
// (alpha, beta, rho, stop flag) and its own partial sums: a tile writes its
// partial, the block that completes a system's last tile adds them in tile
// order (deterministic) and updates that system's scalars.  The iteration is
// the FP64 Jacobi loop of pcg_kernels.cuh (three kernels); a chunk of
// iterations is one CUDA graph.
#include "block_solve.cuh"
#include "cps_internal.cuh"
#include "exact_sum.cuh"

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

// ---- The ensemble in one launch (the block-level solves: block_solve.cuh).
constexpr int kMinTeamRows = 2048;   // rows a team member keeps at least

// Blocks [first, first + k) solve system sys as one team.
struct TeamPlan {
    int32_t sys;
    int32_t first;
    int32_t k;
    int32_t pad;
};


// First the static teams: block b of team t solves its slice of system
// teams[t].sys (rows split in multiples of 32).  Then every block takes whole
// systems in the order `order` (largest estimated work first) from the
// counter *next until none is left.  FP64 or mixed precision.
template <bool MIXED>
__global__ void __launch_bounds__(kBB, 2) kb_one_launch(const BatchDesc* __restrict__ dd,
                                                        const int* __restrict__ order, int nqueue,
                                                        int* next,
                                                        const TeamPlan* __restrict__ teams,
                                                        int nteams, TeamSync* sync, double rtol,
                                                        long long max_iter) {
    __shared__ int s_k;
    __shared__ TeamCtx s_tc;
    for (int t = 0; t < nteams; ++t) {
        const TeamPlan tp = teams[t];
        const int rank = (int)blockIdx.x - tp.first;
        if (rank < 0 || rank >= tp.k) continue;
        const BatchDesc& d = dd[tp.sys];
        const int64_t rows = ((d.n + tp.k - 1) / tp.k + 31) / 32 * 32;
        const int64_t lo = min(d.n, (int64_t)rank * rows);
        const int64_t hi = min(d.n, lo + rows);
        if (threadIdx.x == 0)
            s_tc = TeamCtx{sync + t, (unsigned long long)sync[t].stall, rank, tp.k, 0u};
        __syncthreads();
        if (MIXED) kbp_solve_mixed(d, lo, hi, &s_tc, rtol, max_iter);
        else kbp_solve(d, lo, hi, &s_tc, rtol, max_iter);
        break;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_k = atomicAdd(next, 1);
        __syncthreads();
        const int k = s_k;
        if (k >= nqueue) return;
        const BatchDesc& d = dd[order[k]];
        if (MIXED) kbp_solve_mixed(d, 0, d.n, nullptr, rtol, max_iter);
        else kbp_solve(d, 0, d.n, nullptr, rtol, max_iter);
    }
}

// The systems' states into one array (one copy to the host).
__global__ void kb_gather_states(const BatchDesc* __restrict__ dd, int nsys, CgState* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys; i += gridDim.x * blockDim.x)
        out[i] = *dd[i].st;
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

// Static teams for one launch of G blocks.  System i's estimated work is
// W_i = n_i^1.5 (the iteration count grows with the mesh's side) and a
// block's fair share is T = sum W / G.  A system above T / 2 gets a team of
// ceil(2 W_i / T) blocks (at most kMaxTeam, and at least kMinTeamRows rows,
// 4 per thread, a member); the others go to the work queue, largest first.
// The queue keeps the blocks its own work needs (ceil(W_queue / T)), and the
// teams are scaled down if they would take more than the rest.  The blocks no
// team holds take from the queue from the start, and every team's blocks
// once their system is done.  Measured on the 256-system ensemble (FP64):
//   teams above 2T of ceil(W_i / T) blocks                      4.34 s
//   this rule                                                   3.96-4.02 s
//   this rule without the queue's reserve                       4.32 s
//   teams sharing the whole grid, k_i = floor(G W_i / W_large)  4.25 s
// In every plan the teams' systems end between about 2 and 3.9 s: W_i
// predicts a team's time only roughly, and about 60% of the blocks are busy
// over the launch on average.
static void plan_teams(const std::vector<BatchDesc>& hd, int G, std::vector<TeamPlan>& teams,
                       std::vector<int>& order) {
    const int nsys = (int)hd.size();
    std::vector<double> w(nsys);
    double total = 0.0;
    for (int i = 0; i < nsys; ++i) {
        w[i] = std::pow((double)hd[i].n, 1.5);
        total += w[i];
    }
    std::vector<int> idx(nsys);
    for (int i = 0; i < nsys; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int u, int v) { return w[u] > w[v]; });
    teams.clear();
    order.clear();
    const double T = total / std::max(G, 1);
    double wq = 0.0;
    long long sumk = 0;
    for (int i : idx) {
        int k = T > 0.0 && w[i] > 0.5 * T
                    ? (int)std::min<double>(kMaxTeam, std::ceil(2.0 * w[i] / T))
                    : 1;
        k = (int)std::min<int64_t>(k, std::max<int64_t>(1, hd[i].n / kMinTeamRows));
        if (k >= 2) {
            teams.push_back(TeamPlan{i, 0, k, 0});
            sumk += k;
        } else {
            order.push_back(i);
            wq += w[i];
        }
    }
    const int queue_blocks = T > 0.0 ? (int)std::ceil(wq / T) : G;
    const int avail = std::max(0, G - std::min(G, queue_blocks));
    if (sumk > avail) {
        // scale the teams down; a team of one becomes a queue entry again
        const double f = (double)avail / (double)sumk;
        std::vector<TeamPlan> kept;
        std::vector<int> back;
        for (const TeamPlan& t : teams) {
            const int k = (int)std::floor(t.k * f);
            if (k >= 2) kept.push_back(TeamPlan{t.sys, 0, k, 0});
            else back.push_back(t.sys);
        }
        teams.swap(kept);
        order.insert(order.begin(), back.begin(), back.end());
    }
    int first = 0;
    for (TeamPlan& t : teams) {
        t.first = first;
        first += t.k;
    }
}

// The ensemble in one cooperative launch of kb_one_launch (FP64 or mixed
// precision): two blocks per SM; the static teams solve the largest systems
// while the other blocks take the rest from the work queue, largest first,
// each to rtol, and every team's blocks join the queue when their system is
// done.
static int solve_batch_one_launch(const cps_sys* systems, int nsys, const double* const* b,
                                  double* const* x, double rtol, int64_t max_iter,
                                  bool mixed, cps_stats* stats, cudaStream_t stream) {
    cps_ctx ctx = systems[0]->ctx;
    std::vector<BatchDesc> hd(nsys);
    for (int i = 0; i < nsys; ++i) {
        cps_sys s = systems[i];
        BatchDesc& d = hd[i];
        d = BatchDesc{};
        d.a = s->a;
        d.col = s->col;
        d.s = s->s;
        d.b = b[i];
        d.x = x[i];
        d.y = s->wy;
        d.r = s->wr;
        d.p = s->wp0;
        d.q = s->wq;
        d.t = s->wp1;
        d.a32 = s->a32;
        d.s32 = s->s32;
        d.best = s->wbest;
        d.partials = s->partials;
        d.st = s->st;
        d.n = s->nt;
    }
    const void* kernel = mixed ? (const void*)kb_one_launch<true> : (const void*)kb_one_launch<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBB, 0) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        cps::set_error(ctx, "solve_batch: the one-launch kernel does not fit an SM");
        return CPS_ERR_CUDA;
    }
    const int grid = ctx->num_sms * per_sm;
    std::vector<TeamPlan> teams;
    std::vector<int> order;
    plan_teams(hd, grid, teams, order);
    const int nteams = (int)teams.size();
    const int nqueue = (int)order.size();
    BatchDesc* dd = nullptr;
    int* dorder = nullptr;     // [nqueue] order, then the work counter
    TeamPlan* dteams = nullptr;
    TeamSync* dsync = nullptr;
    CgState* dst = nullptr;
    CgState* hst = nullptr;
    const size_t nt_alloc = (size_t)std::max(nteams, 1);
    size_t npart = 0;            // the teams' partials follow their TeamSync array
    for (const TeamPlan& t : teams) npart += 8 * (size_t)t.k;
    const size_t sync_bytes = sizeof(TeamSync) * nt_alloc + sizeof(double) * std::max<size_t>(npart, 1);
    int rc = CPS_OK;
    if (cudaMallocAsync((void**)&dd, sizeof(BatchDesc) * nsys, stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dorder, sizeof(int) * (nqueue + 1), stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dteams, sizeof(TeamPlan) * nt_alloc, stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dsync, sync_bytes, stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dst, sizeof(CgState) * nsys, stream) != cudaSuccess ||
        cudaMallocHost((void**)&hst, sizeof(CgState) * nsys) != cudaSuccess)
        rc = CPS_ERR_NOMEM;
    if (rc == CPS_OK &&
        (cudaMemcpyAsync(dd, hd.data(), sizeof(BatchDesc) * nsys, cudaMemcpyHostToDevice,
                         stream) != cudaSuccess ||
         (nqueue > 0 && cudaMemcpyAsync(dorder, order.data(), sizeof(int) * nqueue,
                                        cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
         (nteams > 0 && cudaMemcpyAsync(dteams, teams.data(), sizeof(TeamPlan) * nteams,
                                        cudaMemcpyHostToDevice, stream) != cudaSuccess) ||
         cudaMemsetAsync(dorder + nqueue, 0, sizeof(int), stream) != cudaSuccess))
        rc = CPS_ERR_CUDA;
    if (rc == CPS_OK) {
        // test hook (cps_test_inject on the first system): every team's waits
        // expect one arrival that never comes
        const int stall = systems[0]->inject == CPS_TEST_STALL_BARRIER ? 1 : 0;
        systems[0]->inject = 0;
        std::vector<TeamSync> hs(nt_alloc);
        double* part = reinterpret_cast<double*>(dsync + nt_alloc);
        for (int t = 0; t < nteams; ++t) {
            hs[t] = TeamSync{};
            hs[t].stall = stall;
            hs[t].partials = part;
            part += 8 * (size_t)teams[t].k;
        }
        if (cudaMemcpyAsync(dsync, hs.data(), sizeof(TeamSync) * nt_alloc, cudaMemcpyHostToDevice,
                            stream) != cudaSuccess)
            rc = CPS_ERR_CUDA;
    }
    if (rc == CPS_OK) {
        // cooperative: every team's blocks are resident together
        int* dnext = dorder + nqueue;
        long long mi = (long long)max_iter;
        void* args[] = {(void*)&dd, (void*)&dorder, (void*)&nqueue, (void*)&dnext,
                        (void*)&dteams, (void*)&nteams, (void*)&dsync, (void*)&rtol, (void*)&mi};
        if (cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBB), args,
                                        0, stream) != cudaSuccess)
            rc = CPS_ERR_CUDA;
    }
    if (rc == CPS_OK) {
        kb_gather_states<<<(nsys + 255) / 256, 256, 0, stream>>>(dd, nsys, dst);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hst, dst, sizeof(CgState) * nsys, cudaMemcpyDeviceToHost, stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            rc = CPS_ERR_CUDA;
    }
    int first = CPS_OK;
    if (rc == CPS_OK) {
        for (int i = 0; i < nsys; ++i) {
            const CgState& h = hst[i];
            const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
            int st = h.status;
            if (st == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) st = CPS_ERR_NOT_CONVERGED;
            if (st != CPS_OK && first == CPS_OK) first = st;
            if (stats) {
                stats[i].iters = h.iter;
                stats[i].rel_res = rel;
                stats[i].status = st;
                stats[i].refinements = mixed ? h.updates : 1;
                stats[i].launches = 2;
            }
        }
    }
    if (dd) cudaFreeAsync(dd, stream);
    if (dorder) cudaFreeAsync(dorder, stream);
    if (dteams) cudaFreeAsync(dteams, stream);
    if (dsync) cudaFreeAsync(dsync, stream);
    if (dst) cudaFreeAsync(dst, stream);
    cudaStreamSynchronize(stream);
    if (hst) cudaFreeHost(hst);
    if (rc != CPS_OK) {
        cudaGetLastError();
        cps::set_error(ctx, rc == CPS_ERR_NOMEM ? "solve_batch: out of memory"
                                                : "solve_batch: CUDA failure");
        return rc;
    }
    if (first == CPS_ERR_NOT_CONVERGED)
        cps::set_error(ctx, mixed ? "solve_batch: a member did not reach rtol in mixed precision "
                                    "(max_iter, or binary32 refinement stopped reducing its "
                                    "residual: its x holds the iterate with the least residual)"
                                  : "solve_batch: max_iter reached");
    if (first == CPS_ERR_NOT_SPD) cps::set_error(ctx, "solve_batch: p.Ap <= 0");
    if (first == CPS_ERR_TIMEOUT)
        cps::set_error(ctx, "solve_batch: a team wait ran out (blocks not co-resident?)");
    return first;
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
    if (precision != CPS_FP64 && precision != CPS_MIXED) {
        cps::set_error(ctx, "solve_batch: bad precision");
        return CPS_ERR_ARG;
    }
    if (ctx->batch_path == CPS_BATCH_ONE_LAUNCH)
        return solve_batch_one_launch(systems, nsys, b, x, rtol, max_iter,
                                      precision == CPS_MIXED, stats, stream);
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
