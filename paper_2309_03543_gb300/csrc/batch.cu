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
    double* t;                    // one-launch solve only: w = Ahat r
    const float* a32;             // one-launch mixed solve: binary32 matrix and S
    const float* s32;
    double* best;                 // one-launch mixed solve: the best FP64 iterate
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

// ---- The ensemble in one launch.  The systems are independent, so they need
// no common barrier: a block (or a team of blocks) solves a system to rtol by
// itself, and takes the next one the moment it converges.  FP64 Jacobi-PCG on
// the scaled matrix with restarts from the true residual as in the single
// solve.  Every sum is an exact integer sum (block_sum_exact, and the team
// sum over the members' block totals), so a team's members take identical
// decisions.
constexpr int kBB = 512;          // threads per block: two blocks per SM

// A system whose estimated work is several blocks' fair share is solved by a
// static team of blocks instead (one launch is cooperative, so a team's
// blocks are co-resident): each member owns a slice of the rows, and the
// team's sums combine the members' exact block totals through a per-team
// arrival counter and a double-buffered partials array.  Every wait is
// bounded (about one second of %globaltimer and a poll cap); a member whose
// wait runs out records it in the team's state, and the others stop at their
// next wait.
constexpr int kMaxTeam = 32;
constexpr int kMinTeamRows = 2048;
constexpr long long kTeamSpinCap = 1LL << 26;
constexpr unsigned long long kTeamWaitNs = 1000000000ull;

struct TeamSync {
    unsigned long long count;   // arrivals since the launch
    int timeout;
    int pad[13];
    double partials[2][4][kMaxTeam];
};

// Blocks [first, first + k) solve system sys as one team.
struct TeamPlan {
    int32_t sys;
    int32_t first;
    int32_t k;
    int32_t pad;
};

__device__ __forceinline__ void team_red_add(unsigned long long* p) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long team_ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long team_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread: bounded wait until the team's count reaches target.  False if
// it ran out, or if a member has already recorded a timeout.
__device__ bool team_wait(TeamSync* ts, unsigned long long target) {
    if (team_ld_acquire(&ts->count) < target) {
        const unsigned long long t0 = team_ns();
        for (long long spins = 1;; ++spins) {
            if (team_ld_acquire(&ts->count) >= target) break;
            if (spins > kTeamSpinCap || ((spins & 255) == 0 && team_ns() - t0 > kTeamWaitNs)) {
                atomicExch(&ts->timeout, 1);
                return false;
            }
        }
    }
    return *(volatile int*)&ts->timeout == 0;
}

// A member's view of its team, in shared memory; only thread 0 reads or
// writes it.
struct TeamCtx {
    TeamSync* ts;
    unsigned long long target;   // arrivals that complete the latest sync
    int rank;
    int k;
    unsigned int epoch;          // syncs passed (the parity picks the partials)
};

// Thread 0: arrive at the team's next sync (its partials, if any, already
// stored in slot tc.epoch & 1) and wait for it; returns that slot, or -1 if a
// wait ran out.
__device__ __noinline__ int team_arrive_wait(TeamCtx& tc) {
    const int par = tc.epoch & 1;
    tc.target += (unsigned long long)tc.k;
    ++tc.epoch;
    team_red_add(&tc.ts->count);
    return team_wait(tc.ts, tc.target) ? par : -1;
}

// Team-wide exact sum of v[0..NV) (NV <= 4): the block's exact total, then
// the k members' totals aligned to their largest exponent and summed in
// integers by warp 0 (the same set in every member: bit-identical results,
// so all members take the same decisions).  Also a team barrier.
template <int NV>
__device__ __forceinline__ bool team_sum(double (&v)[NV], TeamCtx& tc) {
    static_assert(NV >= 1 && NV <= 4, "team sum width");
    __shared__ double s_tot[NV];
    __shared__ int s_par;
    block_sum_exact<NV, kBB>(v);
    if (threadIdx.x == 0) {
        const int par = tc.epoch & 1;
#pragma unroll
        for (int q = 0; q < NV; ++q) tc.ts->partials[par][q][tc.rank] = v[q];
        s_par = team_arrive_wait(tc);
    }
    __syncthreads();
    const int par = s_par;
    if (par < 0) return false;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int k = tc.k;
        const TeamSync* ts = tc.ts;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double w = lane < k ? __ldcg(&ts->partials[par][q][lane]) : 0.0;
            const int E = __reduce_max_sync(0xffffffffu, align_exp(w));
            const long long T = warp_sum_fixed<52>(align_fixed(w, E, 1));
            if (lane == 0) s_tot[q] = fixed_to_double(T, E, 1);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = s_tot[q];
    return true;
}

// Team barrier: the block's writes before it are visible to every member
// after it.
__device__ __forceinline__ bool team_barrier(TeamCtx& tc) {
    __shared__ int s_par;
    __syncthreads();
    if (threadIdx.x == 0) s_par = team_arrive_wait(tc);
    __syncthreads();
    return s_par >= 0;
}

// Rows [lo, hi) of one system by the block's threads, U rows per trip (one
// block apart), all loads of a trip before any use.  Before a trip's loads,
// PF(f) is issued for the rows f of the next trip (an L1 prefetch holds no
// register: a block's loads in flight are otherwise capped by the 64
// registers a thread has at two blocks per SM, and a block alone on its
// rows is bound by memory latency).
#define CPS_BLK_LOOP(lo, hi, U, PF, LOAD, BODY)                                        \
    {                                                                                  \
        const int64_t hi_ = (hi);                                                      \
        int64_t i0_ = (lo) + threadIdx.x;                                              \
        for (; i0_ + (U - 1) * (int64_t)kBB < hi_; i0_ += U * (int64_t)kBB) {          \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t f = i0_ + (U + u) * (int64_t)kBB;                        \
                if (f < hi_) PF;                                                       \
            }                                                                          \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = i0_ + u * (int64_t)kBB;                              \
                LOAD;                                                                  \
            }                                                                          \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = i0_ + u * (int64_t)kBB;                              \
                BODY;                                                                  \
            }                                                                          \
        }                                                                              \
        for (; i0_ < hi_; i0_ += kBB) {                                                \
            const int u = 0;                                                           \
            const int64_t e = i0_;                                                     \
            LOAD;                                                                      \
            BODY;                                                                      \
        }                                                                              \
    }

__device__ __forceinline__ void pf_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Scalars of one block's solve, in shared memory: thread 0 takes every
// decision, the other threads read alpha, beta and the flag after a barrier.
struct SolveScalars {
    double gamma, alpha, beta, bnorm2, rnorm2, thresh2;
    double ig;                    // 1 / gamma
    double c;                     // 1 / (gamma alpha)
    long long total, it, budget;
    int flag;                     // 0 run, 1 stop, 2 breakdown, 3 b = 0
    int status;
};

// w = Ahat r on rows [lo, hi) with gamma = r.r, delta = w.r and, if check,
// ||S r||^2 into v[0..3).
#define CPS_BLK_SPMV_W(lo, hi, check, v)                                               \
    {                                                                                  \
        double re[2], a0[2], a1[2], a2[2];                                             \
        int32_t c0[2], c1[2], c2[2];                                                   \
        CPS_BLK_LOOP(lo, hi, 2,                                                        \
            (pf_l1(r + f), pf_l1(A + f), pf_l1(A + n + f), pf_l1(A + 2 * n + f),       \
             pf_l1(C + f), pf_l1(C + n + f), pf_l1(C + 2 * n + f)),                    \
            (re[u] = r[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],       \
             c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),                    \
            {                                                                          \
                double wv = fma(a0[u], r[c0[u]], re[u]);                               \
                wv = fma(a1[u], r[c1[u]], wv);                                         \
                wv = fma(a2[u], r[c2[u]], wv);                                         \
                w[e] = wv;                                                             \
                v[0] = fma(re[u], re[u], v[0]);                                        \
                v[1] = fma(wv, re[u], v[1]);                                           \
                if (check) {                                                           \
                    const double tt = S[e] * re[u];                                    \
                    v[2] = fma(tt, tt, v[2]);                                          \
                }                                                                      \
            })                                                                         \
    }

// One system, rows [lo, hi) solved by this block: the whole system (tc null)
// or this member's slice of a team's system (tc in shared memory).  FP64
// Jacobi CG on the scaled matrix with the single-reduction (Chronopoulos-Gear)
// recurrences: s = Ahat p and w = Ahat r carried so that one SpMV gives both
// inner products of an iteration,
//   p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s   | barrier
//   w = Ahat r; gamma = r.r, delta = w.r (every 8th: ||S r||^2)   | one sum
//   beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
// A block alone is bound by memory latency, not bandwidth: two passes and two
// synchronisations an iteration instead of the textbook three and three.
// Restarts from the true residual (at most 8 rounds).  The result and the
// status go to the system's CgState (iter, rnorm2, bnorm2, status; done = 2),
// written by the block that holds row 0.
__device__ __forceinline__ void kbp_solve(const BatchDesc& d, int64_t lo, int64_t hi,
                                          TeamCtx* tc, double rtol, long long max_iter) {
    __shared__ SolveScalars sc;
    const int64_t n = d.n;
    const double* __restrict__ A = d.a;
    const int32_t* __restrict__ C = d.col;
    const double* __restrict__ S = d.s;
    double* __restrict__ y = d.y;
    double* __restrict__ r = d.r;
    double* __restrict__ p = d.p;
    double* __restrict__ sv = d.q;
    double* __restrict__ w = d.t;
    bool ok = true;               // false once a team wait ran out
    auto sum1 = [&](double (&v)[1]) {
        if (tc) ok = team_sum<1>(v, *tc) && ok;
        else block_sum_exact<1, kBB>(v);
    };
    auto sum3 = [&](double (&v)[3]) {
        if (tc) ok = team_sum<3>(v, *tc) && ok;
        else block_sum_exact<3, kBB>(v);
    };
    auto barrier = [&]() {
        if (tc) ok = team_barrier(*tc) && ok;
        else __syncthreads();
    };
    if (threadIdx.x == 0) {
        sc.total = 0;
        sc.it = 0;
        sc.status = CPS_OK;
        sc.bnorm2 = sc.rnorm2 = sc.thresh2 = 0.0;
    }
    for (int round = 0; round < 8; ++round) {
        // y = S x, r = S^-1 b - Ahat y, p = s = 0
        double v3[3] = {0.0, 0.0, 0.0};
        for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) {
            const double se = S[e];
            const double ye = se * d.x[e];
            double ay = ye;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int32_t c = C[j * n + e];
                ay = fma(A[j * n + e], S[c] * d.x[c], ay);
            }
            const double be = d.b[e];
            const double re = be / se - ay;
            y[e] = ye;
            r[e] = re;
            p[e] = 0.0;
            sv[e] = 0.0;
            v3[0] = fma(re, re, v3[0]);
            v3[1] = fma(be, be, v3[1]);
            const double t = se * re;
            v3[2] = fma(t, t, v3[2]);
        }
        sum3(v3);                 // also the barrier before x is overwritten
        if (!ok) break;
        if (threadIdx.x == 0) {
            sc.bnorm2 = v3[1];
            sc.thresh2 = rtol * rtol * v3[1];
            sc.rnorm2 = v3[2];
            sc.budget = max_iter - sc.total;
            sc.it = 0;
            sc.flag = v3[1] == 0.0 ? 3
                      : (v3[2] > sc.thresh2 && sc.budget > 0 && v3[0] > 0.0) ? 0 : 1;
        }
        __syncthreads();
        if (sc.flag == 3) {           // b = 0: x = 0
            for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) d.x[e] = 0.0;
            if (threadIdx.x == 0) sc.rnorm2 = 0.0;
            break;
        }
        if (sc.flag == 0) {
            // w = Ahat r: alpha = gamma / delta, beta = 0
            double g3[3] = {0.0, 0.0, 0.0};
            CPS_BLK_SPMV_W(lo, hi, false, g3)
            sum3(g3);
            if (!ok) break;
            if (threadIdx.x == 0) {
                const double g = g3[0], dl = g3[1];
                if (!(dl > 0.0) || !isfinite(dl)) {
                    sc.flag = 2;
                    sc.status = CPS_ERR_NOT_SPD;
                } else {
                    sc.gamma = g;
                    sc.alpha = g / dl;
                    sc.beta = 0.0;
                    sc.ig = 1.0 / g;
                    sc.c = dl * sc.ig * sc.ig;
                }
            }
            __syncthreads();
        }
        while (sc.flag == 0) {
            {
                const double alpha = sc.alpha, beta = sc.beta;
                double pe[2], se[2], we[2], re[2], ye[2];
                CPS_BLK_LOOP(lo, hi, 2,
                    (pf_l1(p + f), pf_l1(sv + f), pf_l1(w + f), pf_l1(r + f), pf_l1(y + f)),
                    (pe[u] = p[e], se[u] = sv[e], we[u] = w[e], re[u] = r[e], ye[u] = y[e]),
                    {
                        const double pn = fma(beta, pe[u], re[u]);
                        const double sn = fma(beta, se[u], we[u]);
                        p[e] = pn;
                        sv[e] = sn;
                        y[e] = fma(alpha, pn, ye[u]);
                        r[e] = fma(-alpha, sn, re[u]);
                    })
            }
            barrier();
            if (!ok) break;
            const bool check = ((sc.it + 1) % 8) == 0;
            double g3[3] = {0.0, 0.0, 0.0};
            CPS_BLK_SPMV_W(lo, hi, check, g3)
            sum3(g3);
            if (!ok) break;
            if (threadIdx.x == 0) {
                const long long it = ++sc.it;
                const double g = g3[0], dl = g3[1];
                bool halt = !(g > 0.0) || it >= sc.budget;
                if (check) {
                    sc.rnorm2 = g3[2];
                    if (g3[2] <= sc.thresh2) halt = true;
                }
                int f = halt ? 1 : 0;
                if (!halt) {
                    const double den = fma(-(g * g), sc.c, dl);
                    if (!(den > 0.0) || !isfinite(den)) {
                        // on a round's first iteration p.Ap <= 0: not SPD;
                        // later the recurrence lost its digits at the FP64
                        // floor: stop, and let the true residual decide
                        f = it > 1 ? 1 : 2;
                        if (f == 2) sc.status = CPS_ERR_NOT_SPD;
                    } else {
                        const double ig = 1.0 / g;
                        sc.alpha = g / den;
                        sc.beta = g * sc.ig;
                        sc.ig = ig;
                        sc.c = den * ig * ig;
                    }
                }
                sc.gamma = g;
                sc.flag = f;
            }
            __syncthreads();
        }
        if (!ok) break;
        // x = S^-1 y and the true residual ||b - A x||^2 (y read at
        // neighbours: every exit above follows a team-wide sum)
        double nn[1] = {0.0};
        for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) {
            const double se = S[e];
            const double ye = y[e];
            double ay = ye;
#pragma unroll
            for (int j = 0; j < 3; ++j) ay = fma(A[j * n + e], y[C[j * n + e]], ay);
            const double res = d.b[e] - se * ay;
            d.x[e] = ye / se;
            nn[0] = fma(res, res, nn[0]);
        }
        sum1(nn);
        if (!ok) break;
        if (threadIdx.x == 0) {
            sc.total += sc.it;
            sc.it = 0;
            sc.rnorm2 = nn[0];
            sc.flag = (sc.status != CPS_OK || nn[0] <= sc.thresh2 || sc.total >= max_iter) ? 1 : 0;
        }
        __syncthreads();
        if (sc.flag) break;
    }
    __syncthreads();
    if (threadIdx.x == 0 && lo == 0) {
        CgState* st = d.st;
        st->iter = sc.total + sc.it;
        st->rnorm2 = sc.rnorm2;
        st->bnorm2 = sc.bnorm2;
        st->thresh2 = sc.thresh2;
        st->status = ok ? sc.status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
    __syncthreads();
}

// ---- Mixed precision in the one launch.  The single solve's reliable-update
// refinement with every decision taken on the device: binary32 matrix,
// vectors and SpMV in the inner iteration (the textbook recurrences, as in the
// single solve: the single-reduction ones carry s = Ahat p by recurrence,
// which drifts in binary32; FP64 inner products and scalars), an FP64 true
// residual after every run, the best FP64 iterate kept, and the same stop,
// divergence and restart rules.  Two passes an iteration: the direction
// update is fused into the SpMV (q = Ahat (r + beta p_old) gathered from r
// and the old direction at the neighbours; p double-buffered), then the
// residual and correction update.
constexpr double kMxDelta = 0.5;      // residual drop between replacements
constexpr int kMxMaxUpdates = 2000;
constexpr double kMxDiverge = 1e4;

// Thread 0's refinement state of one mixed solve.
struct MixedScalars {
    double rho, rho_prev, alpha, beta;    // inner scalars (rho = r.r, rho_prev its last value)
    double bnorm2, rnorm2, thresh2, outer2, rho_rep;
    double best, prev, last;
    long long total, it;                  // inner iterations: whole solve, this run
    int updates, stall, restarts;
    int first;                            // next run starts from p = 0
    int par;                              // which buffer holds the current direction
    int flag;                             // per phase: 0 go on, 1 stop
    int action;                           // after a residual: 0 run, 1 end, 2 end + restore
    int copy;                             // keep x as the best iterate
    int status;
};

// One system by this block (tc null) or this member's rows of a team's
// system: Jacobi PCG on the scaled matrix, binary32 inner iteration with FP64
// residual replacement.  x receives the final (or best) FP64 iterate; the
// result goes to the system's CgState (iter, rnorm2, bnorm2, status,
// updates; done = 2) from the block that holds row 0.
__device__ __forceinline__ void kbp_solve_mixed(const BatchDesc& d, int64_t lo, int64_t hi,
                                                TeamCtx* tc, double rtol, long long max_iter) {
    __shared__ MixedScalars sm;
    const int64_t n = d.n;
    const double* __restrict__ A = d.a;       // FP64 scaled matrix (residuals)
    const int32_t* __restrict__ C = d.col;
    const double* __restrict__ S = d.s;
    const float* __restrict__ A32 = d.a32;
    const float* __restrict__ S32 = d.s32;
    double* __restrict__ x = d.x;
    float* __restrict__ r = reinterpret_cast<float*>(d.r);
    float* __restrict__ pb0 = reinterpret_cast<float*>(d.p);
    float* __restrict__ pb1 = reinterpret_cast<float*>(d.t);
    float* __restrict__ q = reinterpret_cast<float*>(d.q);
    float* __restrict__ dy = reinterpret_cast<float*>(d.y);
    bool ok = true;
    auto sum1 = [&](double (&v)[1]) {
        if (tc) ok = team_sum<1>(v, *tc) && ok;
        else block_sum_exact<1, kBB>(v);
    };
    auto sum2 = [&](double (&v)[2]) {
        if (tc) ok = team_sum<2>(v, *tc) && ok;
        else block_sum_exact<2, kBB>(v);
    };
    auto sum3 = [&](double (&v)[3]) {
        if (tc) ok = team_sum<3>(v, *tc) && ok;
        else block_sum_exact<3, kBB>(v);
    };
    auto barrier = [&]() {
        if (tc) ok = team_barrier(*tc) && ok;
        else __syncthreads();
    };
    if (threadIdx.x == 0) {
        sm.total = 0;
        sm.it = 0;
        sm.updates = sm.stall = sm.restarts = 0;
        sm.first = 1;
        sm.best = sm.prev = sm.last = INFINITY;
        sm.bnorm2 = sm.rnorm2 = sm.thresh2 = 0.0;
        sm.rho = sm.rho_prev = 0.0;
        sm.par = 0;
        sm.status = CPS_OK;
    }
    __syncthreads();
    for (;;) {
        // FP64 true residual of x: r = S^-1 b - Ahat (S x), rounded to
        // binary32; the correction d = 0
        {
            double v3[3] = {0.0, 0.0, 0.0};   // r32.r32, b.b, ||S r||^2
            for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) {
                const double se = S[e];
                double ay = se * x[e];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int32_t c = C[j * n + e];
                    ay = fma(A[j * n + e], S[c] * x[c], ay);
                }
                const double be = d.b[e];
                const double re = be / se - ay;
                const float rf = (float)re;
                r[e] = rf;
                dy[e] = 0.0f;
                v3[0] = fma((double)rf, (double)rf, v3[0]);
                v3[1] = fma(be, be, v3[1]);
                const double t = se * re;
                v3[2] = fma(t, t, v3[2]);
            }
            sum3(v3);
            if (!ok) break;
            if (threadIdx.x == 0) {
                const double rr = v3[0], bb = v3[1], nn = v3[2];
                sm.bnorm2 = bb;
                sm.outer2 = rtol * rtol * bb;
                sm.rnorm2 = nn;
                sm.copy = 0;
                int act = 0;
                if (bb == 0.0 || nn <= sm.outer2) {
                    act = 1;                              // converged (b = 0: x = 0 below)
                } else {
                    if (nn < sm.best) {
                        sm.best = nn;
                        sm.copy = 1;
                    } else if (!(nn <= kMxDiverge * sm.best)) {
                        sm.status = CPS_ERR_NOT_CONVERGED;  // refinement diverging
                        act = 2;
                    }
                    if (act == 0 && (sm.total >= max_iter || sm.updates >= kMxMaxUpdates)) {
                        sm.status = CPS_ERR_NOT_CONVERGED;
                        act = nn > sm.best ? 2 : 1;
                    }
                    if (act == 0) {
                        // a replaced residual that stops falling (no 10% gain
                        // over 8 replacements) restarts the directions, at
                        // most 4 times; one that rose since the last
                        // replacement restarts them without counting
                        if (nn < 0.81 * sm.prev) {
                            sm.prev = nn;
                            sm.stall = 0;
                        } else {
                            ++sm.stall;
                        }
                        const bool rose = nn > sm.last;
                        sm.last = nn;
                        if (sm.stall >= 8 && !sm.first) {
                            if (++sm.restarts > 4) {
                                sm.status = CPS_ERR_NOT_CONVERGED;
                                act = nn > sm.best ? 2 : 1;
                            } else {
                                sm.first = 1;
                                sm.stall = 0;
                            }
                        } else if (rose && !sm.first) {
                            sm.first = 1;
                        }
                    }
                    if (act == 0) {
                        const double inner2 = kMxDelta * kMxDelta * nn;
                        sm.thresh2 = inner2 > 0.25 * sm.outer2 ? inner2 : 0.25 * sm.outer2;
                        sm.rho_rep = rr;
                        // continue the directions: p = r_true + beta p_k with
                        // beta = rho_true / rho_k (0 on a fresh start)
                        sm.beta = sm.first || !(sm.rho_prev > 0.0) ? 0.0 : rr / sm.rho_prev;
                        sm.rho = rr;
                        sm.it = 0;
                        ++sm.updates;
                        if (!(rr > 0.0)) act = 1;
                    }
                }
                sm.action = act;
            }
            __syncthreads();
        }
        const int act = sm.action;
        if (act != 0) {
            if (sm.bnorm2 == 0.0) {
                for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) x[e] = 0.0;
                if (threadIdx.x == 0) sm.rnorm2 = 0.0;
            } else if (act == 2) {
                for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) x[e] = d.best[e];
                if (threadIdx.x == 0) sm.rnorm2 = sm.best;
            }
            break;
        }
        if (sm.copy)
            for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) d.best[e] = x[e];
        if (sm.first) {       // a fresh start: clear the direction
            float* pz = sm.par ? pb1 : pb0;
            for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) pz[e] = 0.0f;
        }
        if (threadIdx.x == 0) sm.flag = 0;
        barrier();            // r and the direction final everywhere
        if (!ok) break;
        if (threadIdx.x == 0) sm.first = 0;
        while (sm.flag == 0) {
            const int par = sm.par;
            const float* __restrict__ po = par ? pb1 : pb0;
            float* __restrict__ pn = par ? pb0 : pb1;
            // p = r + beta p_old; q = Ahat p (gathered); gamma = p.q
            double g[1] = {0.0};
            {
                const float beta = (float)sm.beta;
                float ro[2], pol[2], a0[2], a1[2], a2[2];
                int32_t c0[2], c1[2], c2[2];
                CPS_BLK_LOOP(lo, hi, 2,
                    (pf_l1(r + f), pf_l1(po + f), pf_l1(A32 + f), pf_l1(A32 + n + f),
                     pf_l1(A32 + 2 * n + f), pf_l1(C + f), pf_l1(C + n + f), pf_l1(C + 2 * n + f)),
                    (ro[u] = r[e], pol[u] = po[e], a0[u] = A32[e], a1[u] = A32[n + e],
                     a2[u] = A32[2 * n + e], c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                    {
                        const float pe = fmaf(beta, pol[u], ro[u]);
                        float v = fmaf(a0[u], fmaf(beta, po[c0[u]], r[c0[u]]), pe);
                        v = fmaf(a1[u], fmaf(beta, po[c1[u]], r[c1[u]]), v);
                        v = fmaf(a2[u], fmaf(beta, po[c2[u]], r[c2[u]]), v);
                        pn[e] = pe;
                        q[e] = v;
                        g[0] = fma((double)pe, (double)v, g[0]);
                    })
            }
            sum1(g);
            if (!ok) break;
            if (threadIdx.x == 0) {
                const double gamma = g[0];
                if (!(gamma > 0.0) || !isfinite(gamma)) {
                    sm.status = CPS_ERR_NOT_SPD;
                    sm.flag = 2;
                } else {
                    sm.alpha = sm.rho / gamma;
                }
                sm.par = par ^ 1;
            }
            __syncthreads();
            if (sm.flag == 2) break;
            // r -= alpha q, d += alpha p; rho' = r.r (every 8th: ||S r||^2)
            const bool check = ((sm.it + 1) % 8) == 0;
            double rr[2] = {0.0, 0.0};
            {
                const float alpha = (float)sm.alpha;
                float qe[2], re[2], pe[2], ye[2];
                CPS_BLK_LOOP(lo, hi, 2,
                    (pf_l1(q + f), pf_l1(r + f), pf_l1(pn + f), pf_l1(dy + f)),
                    (qe[u] = q[e], re[u] = r[e], pe[u] = pn[e], ye[u] = dy[e]),
                    {
                        const float rv = fmaf(-alpha, qe[u], re[u]);
                        r[e] = rv;
                        dy[e] = fmaf(alpha, pe[u], ye[u]);
                        rr[0] = fma((double)rv, (double)rv, rr[0]);
                        if (check) {
                            const double tt = (double)S32[e] * (double)rv;
                            rr[1] = fma(tt, tt, rr[1]);
                        }
                    })
            }
            sum2(rr);
            if (!ok) break;
            if (threadIdx.x == 0) {
                const long long it = ++sm.it;
                const double rho_new = rr[0];
                // stop the run: the recursive residual fell below the
                // replacement threshold, the budget is spent, or r.r reached
                // the binary32 rounding floor (1e-13 of the replaced one)
                bool halt = !(rho_new > 0.0) || sm.total + it >= max_iter ||
                            rho_new <= 1e-13 * sm.rho_rep;
                if (check && rr[1] <= sm.thresh2) halt = true;
                sm.beta = rho_new / sm.rho;
                sm.rho_prev = sm.rho;
                sm.rho = rho_new;
                sm.flag = halt ? 1 : 0;
            }
            __syncthreads();
        }
        if (!ok || sm.flag == 2) break;
        // x += S^-1 d in FP64 (own rows), then every member's x is final
        // before the next residual reads it at neighbours
        for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) x[e] += (double)dy[e] / S[e];
        if (threadIdx.x == 0) {
            sm.total += sm.it;
            sm.it = 0;
        }
        barrier();
        if (!ok) break;
    }
    __syncthreads();
    if (threadIdx.x == 0 && lo == 0) {
        CgState* st = d.st;
        st->iter = sm.total + sm.it;
        st->rnorm2 = sm.rnorm2;
        st->bnorm2 = sm.bnorm2;
        st->thresh2 = sm.outer2;
        st->updates = sm.updates;
        st->status = ok ? sm.status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
    __syncthreads();
}

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
        if (threadIdx.x == 0) s_tc = TeamCtx{sync + t, 0ull, rank, tp.k, 0u};
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

// Static teams for one launch of G blocks: system i's estimated work is
// W_i = n_i^1.5 (the iteration count grows with the mesh's side), the fair
// share of a block is T = sum W / G, and a system with W_i > 2 T gets a team
// of ceil(W_i / T) blocks (at most kMaxTeam), so that it ends near the fair
// makespan instead of dominating it; a member keeps at least kMinTeamRows
// rows (4 per thread).  The teams' blocks are scaled down if
// they would leave the queue of the other systems fewer blocks than its own
// work needs.  `order` receives the other systems, largest work first.
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
    std::vector<int> ks;
    double wq = 0.0;
    long long sumk = 0;
    for (int i : idx) {
        int k = T > 0.0 && w[i] > 2.0 * T
                    ? (int)std::min<double>(kMaxTeam, std::ceil(w[i] / T))
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
    int rc = CPS_OK;
    if (cudaMallocAsync((void**)&dd, sizeof(BatchDesc) * nsys, stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dorder, sizeof(int) * (nqueue + 1), stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dteams, sizeof(TeamPlan) * nt_alloc, stream) != cudaSuccess ||
        cudaMallocAsync((void**)&dsync, sizeof(TeamSync) * nt_alloc, stream) != cudaSuccess ||
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
         cudaMemsetAsync(dsync, 0, sizeof(TeamSync) * nt_alloc, stream) != cudaSuccess ||
         cudaMemsetAsync(dorder + nqueue, 0, sizeof(int), stream) != cudaSuccess))
        rc = CPS_ERR_CUDA;
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
