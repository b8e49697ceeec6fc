// Persistent grid-synchronised FP64 solves: the whole Jacobi-PCG run (or the
// reduced-system run) is one cooperative launch whose blocks step through the
// iterations together, separated by software synchronisation instead of
// kernel boundaries (a kernel boundary with a grid reduction costs several
// microseconds on GB300, more than the memory time of a small system).
//
// Block b owns the contiguous rows [b R, (b+1) R) of every vector (R a
// multiple of 32), in every phase.
//
// Dot products: every block stores its partial sums into its own slot of one
// of two partial buffers (alternating, so that a block already in the next
// reduction never overwrites a slot another block is still reading), then
// adds 1 to a 64-bit arrival counter with release semantics; reduction k is
// complete when the counter reaches G (k + 1).  After an acquire load has
// seen that value, warp 0 of every block adds all G slots itself, in slot
// order with the same shuffle tree: every block obtains bit-identical totals
// (the same alpha, beta and stop decisions everywhere).
//
// The direction update -> SpMV dependency is local: the SpMV of block b reads
// p only at the rows its matrix rows reference, which on meshes numbered with
// locality (lattices, banded orderings) lie in a few neighbouring blocks.
// Each block computes that block range once; after its direction update a
// block publishes its iteration number in its own flag (release), and before
// the next SpMV it waits only for the flags of the blocks in its range
// (acquire).  If any block's range spans more than kMaxDeps blocks, every
// block uses a grid-wide barrier there instead.
//
// Co-residency of all blocks is guaranteed by the cooperative launch.  Every
// wait is bounded (about one second of %globaltimer, and a poll cap): a
// block whose wait runs out records CPS_ERR_TIMEOUT and leaves; the blocks
// waiting on it then run out too, so the kernel always ends.
#include "cps_internal.cuh"
#include "exact_sum.cuh"

#include <cmath>
#include <cstddef>

namespace cps {
namespace {

constexpr int kPBlock = 1024;
constexpr long long kSpinCap = 1LL << 26;           // polls; each one an L2 round trip
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr int kFlagStride = 16;                      // one 128-byte line per block flag
constexpr int kMaxDeps = 8;
constexpr int kPartialSlots = 4;                     // quantities per reduction buffer

struct GridSync {
    unsigned long long count;   // arrivals since the launch
    int timeout;
    int pad[29];
    unsigned long long flag[kMaxGrid * kFlagStride];   // per-block iteration flags
};

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Hint: fetch the line holding p into this SM's L1 (no register result).
__device__ __forceinline__ void prefetch_l1(const void* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait until *p >= target (one thread).  False if it ran out, or if
// another block has already recorded a timeout.
__device__ bool wait_geq(const unsigned long long* p, unsigned long long target, GridSync* gs) {
    if (ld_acquire(p) < target) {
        const unsigned long long t0 = global_ns();
        for (long long spins = 1;; ++spins) {
            if (ld_acquire(p) >= target) break;
            if (spins > kSpinCap || ((spins & 255) == 0 && global_ns() - t0 > kWaitNs)) {
                atomicExch(&gs->timeout, 1);
                return false;
            }
        }
    }
    return *(volatile int*)&gs->timeout == 0;
}

// Barriers passed by this block: reductions (k picks the partial buffer) and
// the arrival count that completes the latest barrier (every barrier adds its
// arrivals per block x the grid; the test hook starts it one arrival high, so
// that every barrier waits for an arrival that never comes).
struct Epoch {
    unsigned int k = 0;
    unsigned long long target = 0;
};

__device__ __forceinline__ void named_barrier(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Grid-wide sum of v[0..NV) (NV <= 4), every stage in exact integer sums:
// the block aligns its 1024 values per quantity to their largest exponent
// and sums them (two warp-reduction rounds through shared memory); warp k
// stores the block total of quantity k and, after the grid's arrivals, stages
// the G block totals in buf[k] (G <= kPBlock) and sums them the same way.
// Lane 0 of warp 0 then derives the block's scalars from the totals,
// post(tot, sc, flag) (once per block: a FP64 divide per thread would cost
// more than a vector sweep), and every thread receives sc[0..NS) and the
// flag.  Returns false if a wait ran out somewhere.
template <int NV, int NS, typename Post>
__device__ __forceinline__ bool grid_allreduce(double (*buf)[kPBlock], double (&v)[NV],
                                               double (&out)[NS], int& flag, double* partials,
                                               GridSync* gs, Epoch& ep, Post post) {
    static_assert(NV >= 1 && NV <= kPartialSlots, "partial slots per buffer");
    __shared__ int s_e[kPartialSlots][32];
    __shared__ long long s_w[kPartialSlots][32];
    __shared__ int s_eb[kPartialSlots];
    __shared__ double tot[kPartialSlots];
    __shared__ double sc[NS];
    __shared__ int s_flag;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int em = __reduce_max_sync(0xffffffffu, align_exp(v[k]));
        if (lane == 0) s_e[k][warp] = em;
    }
    __syncthreads();            // also orders every thread's phase writes before the arrival
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int E = __reduce_max_sync(0xffffffffu, s_e[k][lane]);
        const long long w = warp_sum_fixed<52>(align_fixed(v[k], E, 1));
        if (lane == 0) {
            s_w[k][warp] = w;
            if (warp == 0) s_eb[k] = E;
        }
    }
    __syncthreads();
    const unsigned int G = gridDim.x;
    double* pb = partials + (size_t)(ep.k & 1) * (kPartialSlots * kMaxGrid);
    ++ep.k;
    ep.target += G;
    if (warp < NV) {
        const long long T = warp_sum_fixed<57>(s_w[warp][lane]);
        if (lane == 0) pb[warp * kMaxGrid + blockIdx.x] = fixed_to_double(T, s_eb[warp], 1);
        // the arrival (one per block) follows the NV partial stores; the
        // barrier among the NV warps orders them before warp 0's release
        if (NV > 1) named_barrier(1, NV * 32);
        if (warp == 0 && lane == 0) {
            red_release_add(&gs->count, 1ull);
            s_ok = wait_geq(&gs->count, ep.target, gs) ? 1 : 0;
        }
        if (NV > 1) named_barrier(1, NV * 32);
        else __syncwarp();
        int em = 1;
        for (unsigned int i = lane; i < G; i += 32) {
            const double t = __ldcg(&pb[warp * kMaxGrid + i]);
            buf[warp][i] = t;
            em = max(em, align_exp(t));
        }
        const int E = __reduce_max_sync(0xffffffffu, em);
        __syncwarp();
        long long acc = 0;       // at most G/32 <= 32 values of 2^50 a lane
        for (unsigned int i = lane; i < G; i += 32) acc += align_fixed(buf[warp][i], E, 3);
        const long long T2 = warp_sum_fixed<57>(acc);
        if (lane == 0) tot[warp] = fixed_to_double(T2, E, 3);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] = tot[k];
        post(t, sc, s_flag);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NS; ++k) out[k] = sc[k];
    flag = s_flag;
    return s_ok != 0;
}

// Plain grid barrier.
__device__ bool grid_barrier(GridSync* gs, Epoch& ep) {
    __shared__ int s_ok;
    __syncthreads();
    ep.target += gridDim.x;
    if (threadIdx.x == 0) {
        red_release_add(&gs->count, 1ull);
        s_ok = wait_geq(&gs->count, ep.target, gs) ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// This block has finished phase `slot` (0: direction update, 1: the reduced
// system's red phase) `it` times.
__device__ __forceinline__ void halo_post(GridSync* gs, unsigned long long it, int slot = 0) {
    __syncthreads();
    if (threadIdx.x == 0) st_release(&gs->flag[blockIdx.x * kFlagStride + slot], it);
}

// Wait until the blocks [dlo, dhi] (other than this one) have posted `it`
// in `slot`.
__device__ bool halo_wait(GridSync* gs, int dlo, int dhi, unsigned long long it, int slot = 0) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        for (int d = dlo; d <= dhi && ok; ++d)
            if (d != (int)blockIdx.x && !wait_geq(&gs->flag[d * kFlagStride + slot], it, gs))
                ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Range [*lo, *hi] of blocks owning the columns that rows [r0, r1) read
// (the self column of an empty slot excluded), where block k owns rows
// base + [k R, (k+1) R) of the columns' range; this block if there is none.
__device__ void column_blocks(const int32_t* __restrict__ C, int64_t n, int64_t r0, int64_t r1,
                              int64_t base, int64_t R, int* lo, int* hi) {
    __shared__ int s_lo, s_hi;
    if (threadIdx.x == 0) {
        s_lo = INT32_MAX;
        s_hi = -1;
    }
    __syncthreads();
    int cmin = INT32_MAX, cmax = -1;
    for (int64_t e = r0 + threadIdx.x; e < r1; e += kPBlock)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int c = C[j * n + e];
            if (c == (int)e) continue;
            const int k = (int)(((int64_t)c - base) / R);
            cmin = k < cmin ? k : cmin;
            cmax = k > cmax ? k : cmax;
        }
    if (cmax >= 0) {
        atomicMin(&s_lo, cmin);
        atomicMax(&s_hi, cmax);
    }
    __syncthreads();
    *lo = s_hi >= 0 ? s_lo : (int)blockIdx.x;
    *hi = s_hi >= 0 ? s_hi : (int)blockIdx.x;
    __syncthreads();
}

struct PersistArgs {
    const double* a;
    const int32_t* col;
    const double* s;
    double* y;
    double* r;
    double* p;
    double* q;
    double* t;          // reduced system: red scratch
    int64_t n;
    int64_t nR;         // reduced system: first black row
    double* partials;
    GridSync* gs;
    CgState* st;
    int stall;          // test hook: 1 makes every barrier wait for one arrival too many
    double dmin;        // single-reduction loops: smallest diagonal entry (stop-test gate)
    double* z;          // IC(0): preconditioned residual
    const double* dinv; // IC(0): inverse pivots
    const double* dpiv; // IC(0), Eisenstat form: the pivots themselves
};

// Rows per block for m rows over the grid: a multiple of 32.
__device__ __forceinline__ int64_t rows_per_block(int64_t m) {
    const int64_t r = (m + gridDim.x - 1) / gridDim.x;
    return (r + 31) & ~(int64_t)31;
}

// Unrolled loop over rows [lo, hi) by the block's threads: U rows per trip
// (one block apart, so every access stays coalesced) with all their loads
// issued before any use.
#define CPS_B_LOOP(lo, hi, U, LOAD, BODY)                                              \
    {                                                                                  \
        const int64_t hi_ = (hi);                                                      \
        int64_t i0_ = (lo) + threadIdx.x;                                              \
        for (; i0_ + (U - 1) * (int64_t)kPBlock < hi_; i0_ += U * (int64_t)kPBlock) {  \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = i0_ + u * (int64_t)kPBlock;                          \
                LOAD;                                                                  \
            }                                                                          \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = i0_ + u * (int64_t)kPBlock;                          \
                BODY;                                                                  \
            }                                                                          \
        }                                                                              \
        for (; i0_ < hi_; i0_ += kPBlock) {                                            \
            const int u = 0;                                                           \
            const int64_t e = i0_;                                                     \
            LOAD;                                                                      \
            BODY;                                                                      \
        }                                                                              \
    }

constexpr int kU = 4;    // rows per trip in the SpMV phases (7 loads per row)
constexpr int kUV = 4;   // rows per trip in the vector phases (2 or 3 loads per row)

// FP64 Jacobi CG on the scaled matrix from the state k_init64 left:
//   [wait for the halo] q = Ahat p, gamma | alpha; r -= alpha q; rho',
//   ||S r||^2 | beta, stop; y += alpha p; p = r + beta p; post
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_cg(PersistArgs P) {
    __shared__ double rbuf[2][kPBlock];
    // the run's scalars (the same in every block) in shared memory, so that
    // the streaming phases keep their registers: rho, ||S r||^2
    __shared__ double sc[2];
    CgState* st = P.st;
    if (st->done) return;                      // uniform: set before the launch
    const int64_t n = P.n;
    const double* __restrict__ A = P.a;
    const int32_t* __restrict__ C = P.col;
    double* __restrict__ p = P.p;
    double* __restrict__ q = P.q;
    double* __restrict__ r = P.r;
    double* __restrict__ y = P.y;
    GridSync* gs = P.gs;
    const int64_t R = rows_per_block(n);
    const int64_t lo = blockIdx.x * R < n ? blockIdx.x * R : n;
    const int64_t hi = lo + R < n ? lo + R : n;
    Epoch ep;
    ep.target = P.stall ? 1ull : 0ull;
    // the blocks whose rows this block's SpMV reads
    int dlo = blockIdx.x, dhi = blockIdx.x;
    {
        __shared__ int s_lo, s_hi;
        if (threadIdx.x == 0) {
            s_lo = (int)lo;
            s_hi = (int)(hi > lo ? hi - 1 : lo);
        }
        __syncthreads();
        int cmin = INT32_MAX, cmax = -1;
        for (int64_t e = lo + threadIdx.x; e < hi; e += kPBlock)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int c = C[j * n + e];
                cmin = c < cmin ? c : cmin;
                cmax = c > cmax ? c : cmax;
            }
        if (cmax >= 0) {
            atomicMin(&s_lo, cmin);
            atomicMax(&s_hi, cmax);
        }
        __syncthreads();
        dlo = (int)(s_lo / R);
        dhi = (int)(s_hi / R);
    }
    bool ok = true;
    bool halo;
    {
        double wide[1] = {(dhi - dlo + 1 > kMaxDeps) ? 1.0 : 0.0};
        double none[1];
        int any = 0;
        ok = grid_allreduce<1, 1>(rbuf, wide, none, any, P.partials, gs, ep,
                                  [](const double (&t)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = t[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    // the run's scalars (the same values in every thread of every block)
    if (threadIdx.x == 0) {
        sc[0] = st->rho;
        sc[1] = st->rnorm2;
    }
    long long it = 0;
    int status = CPS_OK;
    while (ok) {
        if (halo && it > 0) {
            ok = halo_wait(gs, dlo, dhi, (unsigned long long)it);
            if (!ok) break;
        }
        double g[1] = {0.0};
        {
            double pe[kU], a0[kU], a1[kU], a2[kU];
            int32_t c0[kU], c1[kU], c2[kU];
            CPS_B_LOOP(lo, hi, kU,
                (pe[u] = p[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double v = fma(a0[u], p[c0[u]], pe[u]);
                    v = fma(a1[u], p[c1[u]], v);
                    v = fma(a2[u], p[c2[u]], v);
                    q[e] = v;
                    g[0] = fma(pe[u], v, g[0]);
                })
        }
        double sa[1];
        int bad = 0;
        ok = grid_allreduce<1, 1>(rbuf, g, sa, bad, P.partials, gs, ep,
                                  [&](const double (&t)[1], double* o, int& f) {
                                      f = (t[0] > 0.0 && isfinite(t[0])) ? 0 : 1;
                                      o[0] = f ? 0.0 : sc[0] / t[0];
                                  });
        if (!ok) break;
        if (bad) {
            status = CPS_ERR_NOT_SPD;
            break;
        }
        const double alpha = sa[0];
        const bool check = ((it + 1) % 8) == 0;
        double rr[2] = {0.0, 0.0};
        {
            double qe[kUV], re0[kUV];
            CPS_B_LOOP(lo, hi, kUV, (qe[u] = q[e], re0[u] = r[e]), {
                const double re = fma(-alpha, qe[u], re0[u]);
                r[e] = re;
                rr[0] = fma(re, re, rr[0]);
                if (check) {
                    const double tt = P.s[e] * re;
                    rr[1] = fma(tt, tt, rr[1]);
                }
            })
        }
        double sb[1];
        int stop = 0;
        const long long it1 = it + 1;
        ok = grid_allreduce<2, 1>(rbuf, rr, sb, stop, P.partials, gs, ep,
                                  [&](const double (&t)[2], double* o, int& f) {
                                      bool halt = !(t[0] > 0.0) || it1 >= st->max_iter;
                                      if (check) {
                                          sc[1] = t[1];  // ||S r||^2
                                          if (t[1] <= st->thresh2) halt = true;
                                      }
                                      o[0] = t[0] / sc[0];   // beta
                                      sc[0] = t[0];          // rho'
                                      f = halt ? 1 : 0;
                                  });
        if (!ok) break;
        ++it;
        const double beta = sb[0];
        {
            double pe[kUV], ye[kUV], re[kUV];
            CPS_B_LOOP(lo, hi, kUV, (pe[u] = p[e], ye[u] = y[e], re[u] = stop ? 0.0 : r[e]), {
                y[e] = fma(alpha, pe[u], ye[u]);
                if (!stop) p[e] = fma(beta, pe[u], re[u]);
            })
        }
        if (stop) break;
        if (halo) {
            halo_post(gs, (unsigned long long)it);
        } else {
            ok = grid_barrier(gs, ep);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = it;
        st->rho = sc[0];
        st->rnorm2 = sc[1];
        st->status = ok ? status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

constexpr int kUG = 2;    // rows per trip in the single-reduction update (5 loads per row)
constexpr int kUGS = 2;   // rows per trip in its SpMV phase
constexpr double kNormGate = 64.0;   // margin of the stop-test gate (see k_persistent_gear)

// FP64 Jacobi CG with the single-reduction (Chronopoulos-Gear) recurrences,
// from the state k_init64 + k_gear_start left (w = Ahat r, p = s = 0,
// alpha = rho / delta, beta = 0), s = Ahat p and w = Ahat r carried by
// recurrence so that both inner products of an iteration come from one SpMV:
//   p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s       | post
//   [wait for the halo] w = Ahat r; gamma = r.r, delta = w.r (every 8th:
//   ||S r||^2) | one grid reduction: stop test, beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old)
// One neighbour wait and one grid reduction per iteration (the textbook
// persistent loop has two reductions), at 9 FP64 FMAs per row.  The
// reduction after the SpMV also orders the next update's writes of r after
// every block's reads of it.  s lives in P.q, w in P.t.
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_gear(PersistArgs P) {
    __shared__ double rbuf[3][kPBlock];
    // The run's scalars, the same values in every block: kept in shared
    // memory (thread 0 updates them inside the reduction) so that the
    // streaming phases keep their registers.
    // rho, alpha, beta, ||S r||^2, 1/rho, 1/(rho alpha), stop threshold
    __shared__ double sc[7];
    __shared__ long long s_max_iter;
    __shared__ int s_stop;        // 1 stop, 2 breakdown
    CgState* st = P.st;
    if (st->done) return;                      // uniform: set before the launch
    const int64_t n = P.n;
    const double* __restrict__ A = P.a;
    const int32_t* __restrict__ C = P.col;
    double* __restrict__ y = P.y;
    double* __restrict__ r = P.r;
    double* __restrict__ p = P.p;
    double* __restrict__ s = P.q;
    double* __restrict__ w = P.t;
    GridSync* gs = P.gs;
    const int64_t R = rows_per_block(n);
    const int64_t lo = blockIdx.x * R < n ? blockIdx.x * R : n;
    const int64_t hi = lo + R < n ? lo + R : n;
    Epoch ep;
    ep.target = P.stall ? 1ull : 0ull;
    int dlo, dhi;
    column_blocks(C, n, lo, hi, 0, R, &dlo, &dhi);
    if (threadIdx.x == 0) {
        sc[0] = st->rho;
        sc[1] = st->alpha;
        sc[2] = st->beta;
        sc[3] = st->rnorm2;
        sc[4] = 1.0 / st->rho;
        sc[5] = 1.0 / (st->rho * st->alpha);
        sc[6] = st->thresh2;
        s_max_iter = st->max_iter;
        s_stop = 0;
    }
    bool ok;
    bool halo;
    {
        double wide[1] = {(dhi - dlo + 1 > kMaxDeps) ? 1.0 : 0.0};
        double none[1];
        int any = 0;
        ok = grid_allreduce<1, 1>(rbuf, wide, none, any, P.partials, gs, ep,
                                  [](const double (&t)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = t[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    long long it = 0;
    while (ok) {
        {
            const double alpha = sc[1], beta = sc[2];
            double pe[kUG], se[kUG], we[kUG], re[kUG], ye[kUG];
            CPS_B_LOOP(lo, hi, kUG,
                (pe[u] = p[e], se[u] = s[e], we[u] = w[e], re[u] = r[e], ye[u] = y[e]),
                {
                    const double pn = fma(beta, pe[u], re[u]);
                    const double sn = fma(beta, se[u], we[u]);
                    p[e] = pn;
                    s[e] = sn;
                    y[e] = fma(alpha, pn, ye[u]);
                    r[e] = fma(-alpha, sn, re[u]);
                })
        }
        if (halo) {
            halo_post(gs, (unsigned long long)(it + 1));
            // the SpMV's first trip reads this block's rows only up to the
            // gathers: fetch them into L1 while waiting on the neighbours
#pragma unroll
            for (int u = 0; u < kUGS; ++u) {
                const int64_t e = lo + threadIdx.x + u * (int64_t)kPBlock;
                if (e < hi) {
                    prefetch_l1(r + e);
                    prefetch_l1(A + e);
                    prefetch_l1(A + n + e);
                    prefetch_l1(A + 2 * n + e);
                    prefetch_l1(C + e);
                    prefetch_l1(C + n + e);
                    prefetch_l1(C + 2 * n + e);
                }
            }
            ok = halo_wait(gs, dlo, dhi, (unsigned long long)(it + 1));
        } else {
            ok = grid_barrier(gs, ep);
        }
        if (!ok) break;
        // Stop test on ||S r||^2 every 8th iteration, and only once it can
        // hold: ||S r||^2 >= min(diag) r.r, so while min(diag) gamma stays
        // above kNormGate times the threshold the test cannot pass (gamma of
        // the last iteration stands in for this one's, with that margin) and
        // the sum is skipped (two FP64 operations a row).
        const bool check = ((it + 1) % 8) == 0 && P.dmin * sc[0] <= kNormGate * sc[6];
        double sums[3] = {0.0, 0.0, 0.0};
        {
            double re[kUGS], a0[kUGS], a1[kUGS], a2[kUGS];
            int32_t c0[kUGS], c1[kUGS], c2[kUGS];
            CPS_B_LOOP(lo, hi, kUGS,
                (re[u] = r[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double v = fma(a0[u], r[c0[u]], re[u]);
                    v = fma(a1[u], r[c1[u]], v);
                    v = fma(a2[u], r[c2[u]], v);
                    w[e] = v;
                    sums[0] = fma(re[u], re[u], sums[0]);
                    sums[1] = fma(v, re[u], sums[1]);
                    if (check) {
                        const double tt = P.s[e] * re[u];
                        sums[2] = fma(tt, tt, sums[2]);
                    }
                })
        }
        // the next update's first trip reads only this block's own rows,
        // final now: fetch them into L1 during the reduction
#pragma unroll
        for (int u = 0; u < kUG; ++u) {
            const int64_t e = lo + threadIdx.x + u * (int64_t)kPBlock;
            if (e < hi) {
                prefetch_l1(p + e);
                prefetch_l1(s + e);
                prefetch_l1(w + e);
                prefetch_l1(r + e);
                prefetch_l1(y + e);
            }
        }
        // thread 0, from the totals: the stop test, beta = gamma/gamma_old
        // and alpha = gamma/den with den = delta - beta gamma/alpha_old =
        // delta - gamma^2/(gamma_old alpha_old).  1/gamma_old and
        // 1/(gamma_old alpha_old) are carried, so one divide stays on the
        // critical path; 1/gamma issues beside it.
        const long long it1 = it + 1;
        auto post = [&](const double* t, bool chk, int& f) {
            const double g = t[0], d = t[1];
            bool halt = !(g > 0.0) || it1 >= s_max_iter;       // exact solution, budget
            if (chk) {
                sc[3] = t[2];
                if (t[2] <= sc[6]) halt = true;
            }
            f = halt ? 1 : 0;
            if (!halt) {
                const double den = fma(-(g * g), sc[5], d);
                if (!(den > 0.0) || !isfinite(den)) {
                    // on a run's first iteration p.Ap <= 0: not SPD; later, the
                    // recurrence's difference lost its digits at the FP64
                    // floor: stop, and let the true residual decide
                    f = it > 0 ? 1 : 2;
                } else {
                    const double ig = 1.0 / g;
                    sc[1] = g / den;
                    sc[2] = g * sc[4];
                    sc[4] = ig;
                    sc[5] = den * ig * ig;
                }
            }
            sc[0] = g;
        };
        double none[1];
        int flag = 0;
        if (check) {
            double v3[3] = {sums[0], sums[1], sums[2]};
            ok = grid_allreduce<3, 1>(rbuf, v3, none, flag, P.partials, gs, ep,
                                      [&](const double (&t)[3], double* o, int& f) {
                                          o[0] = 0.0;
                                          post(t, true, f);
                                      });
        } else {
            double v2[2] = {sums[0], sums[1]};
            ok = grid_allreduce<2, 1>(rbuf, v2, none, flag, P.partials, gs, ep,
                                      [&](const double (&t)[2], double* o, int& f) {
                                          o[0] = 0.0;
                                          post(t, false, f);
                                      });
        }
        if (!ok) break;
        it = it1;
        if (flag) {
            if (threadIdx.x == 0) s_stop = flag;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = it;
        st->rho = sc[0];
        st->alpha = sc[1];
        st->beta = sc[2];
        st->rnorm2 = sc[3];
        st->status = ok ? (s_stop == 2 ? CPS_ERR_NOT_SPD : CPS_OK) : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

// FP64 IC(0)-PCG in a two-colour order by Eisenstat's form of the
// preconditioned iteration (S. C. Eisenstat, SIAM J. Sci. Stat. Comput. 2,
// 1981), in one persistent launch with the single-reduction recurrences.
// With Ahat = [[I, E], [E^T, I]] (red rows [0, nR) first), the strictly lower
// part Lt = [[0, 0], [E^T, 0]] and Dt = diag(I, D_B), the IC(0) factor is
// M = (Dt + Lt) Dt^-1 (Dt + Lt^T).  PCG on Ahat with M gives the same
// iterates as PCG on T = (Dt + Lt)^-1 Ahat (Dt + Lt^T)^-1 (symmetric) with
// the diagonal preconditioner Dt, under xh = (Dt + Lt^T) y and
// rh = (Dt + Lt)^-1 r; and from Ahat = (Dt + Lt) + (Dt + Lt^T) - (2 Dt - I),
//   T = diag(I, D_B^-1 (I - E^T E) D_B^-1):
// the red block is the identity, the black one needs E then E^T once.  One
// pass over the matrix per iteration instead of two sweeps and an SpMV.  With
// z = Dt rh (z_R = rh_R, z_B = D_B rh_B) and w = T z:
//   w_R = z_R, and w_B = D_B^-1 (rh_B - E^T v) with v_R = E rh_B,
// so in the recurrences s = T p stays equal to p on the red rows.  Per
// iteration, from the state k_init64 left (y, r):
//   all    p = z + beta p; s = w + beta s (black; red s = p);
//          xh += alpha p; rh -= alpha s                                   | post 0
//   red    [wait: black owners' rh_B] v_R = E rh_B; gamma_R = delta_R = rh_R.rh_R | post 1
//   black  [wait: red owners' v] w_B = D_B^-1 (rh_B - E^T v), z_B = D_B rh_B;
//          gamma_B = rh_B.z_B, delta_B = (rh_B - E^T v).rh_B
//   one grid reduction: stop test, beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old)
// Pass 0 transforms instead of updating (xh_R = y_R + E y_B, rh_B =
// D_B^-1 (r_B - E^T r_R), p = s = 0; xh_B = D_B y_B after the red rows have
// read y_B); after the stop, y = (Dt + Lt^T)^-1 xh: y_B = D_B^-1 xh_B, then
// y_R = xh_R - E y_B.  The stop test (every 8th pass) sums ||S r||^2 of the
// true-form residual r = (Dt + Lt) rh: r_R = rh_R, r_B = z_B + E^T rh_R.
// xh lives in P.y, rh in P.r, s_B in P.q, w_B in P.t, v_R and z_B in P.z.
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_ic0(PersistArgs P) {
    __shared__ double rbuf[3][kPBlock];
    // gamma, alpha, beta, ||S r||^2, 1/gamma, 1/(gamma alpha), stop threshold
    __shared__ double sc[7];
    __shared__ long long s_max_iter;
    __shared__ int s_stop;        // 1 stop, 2 breakdown
    __shared__ int s_dep[4];      // [lo, hi] owners for black rows, then for red rows
    CgState* st = P.st;
    if (st->done) return;                      // uniform: set before the launch
    const int n = (int)P.n, nR = (int)P.nR, nB = n - nR;
    const double* __restrict__ A = P.a;
    const int32_t* __restrict__ C = P.col;
    const double* __restrict__ dinv = P.dinv;
    const double* __restrict__ dpiv = P.dpiv;
    double* __restrict__ y = P.y;
    double* __restrict__ r = P.r;
    double* __restrict__ p = P.p;
    double* __restrict__ s = P.q;
    double* __restrict__ w = P.t;
    double* __restrict__ z = P.z;
    GridSync* gs = P.gs;
    const int Rr = (int)rows_per_block(nR), Rb = (int)rows_per_block(nB);
    const int rlo = (int)blockIdx.x * Rr < nR ? (int)blockIdx.x * Rr : nR;
    const int rhi = rlo + Rr < nR ? rlo + Rr : nR;
    const int blo = nR + ((int)blockIdx.x * Rb < nB ? (int)blockIdx.x * Rb : nB);
    const int bhi = blo + Rb < n ? blo + Rb : n;
    Epoch ep;
    ep.target = P.stall ? 1ull : 0ull;
    {
        int lo_, hi_;
        column_blocks(C, n, blo, bhi, 0, Rr, &lo_, &hi_);
        if (threadIdx.x == 0) {
            s_dep[0] = lo_;
            s_dep[1] = hi_;
        }
        column_blocks(C, n, rlo, rhi, nR, Rb, &lo_, &hi_);
        if (threadIdx.x == 0) {
            s_dep[2] = lo_;
            s_dep[3] = hi_;
        }
        __syncthreads();          // every thread reads s_dep below
    }
    if (threadIdx.x == 0) {
        sc[0] = 0.0;
        sc[1] = 0.0;
        sc[2] = 0.0;
        sc[3] = st->rnorm2;
        sc[4] = 0.0;
        sc[5] = 0.0;
        sc[6] = st->thresh2;
        s_max_iter = st->max_iter;
        s_stop = 0;
    }
    bool ok;
    bool halo;
    {
        const bool wide = s_dep[1] - s_dep[0] + 1 > kMaxDeps || s_dep[3] - s_dep[2] + 1 > kMaxDeps;
        double wv[1] = {wide ? 1.0 : 0.0};
        double none[1];
        int any = 0;
        ok = grid_allreduce<1, 1>(rbuf, wv, none, any, P.partials, gs, ep,
                                  [](const double (&t)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = t[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    auto post = [&](int slot, int ps) {
        if (halo) halo_post(gs, (unsigned long long)(ps + 1), slot);
    };
    // wait for phase `slot` of this pass at the owners of the black rows'
    // columns (which = 0) or of the red rows' columns (which = 1)
    auto wait = [&](int slot, int ps, int which) -> bool {
        if (!halo) return grid_barrier(gs, ep);
        return halo_wait(gs, s_dep[2 * which], s_dep[2 * which + 1],
                         (unsigned long long)(ps + 1), slot);
    };
    int pass = 0;              // passes 1, 2, ... each begin with an update: iterations = pass
    for (; ok; ++pass) {
        const bool upd = pass > 0;
        const bool check = upd && (pass % 8) == 0;
        const double alpha = sc[1], beta = sc[2];
        double sums[3] = {0.0, 0.0, 0.0};
        if (upd) {
            // red: z = w = rh (old), so s = p: p = rh + beta p, xh += alpha p,
            // rh -= alpha p
            {
                double re[2], pe[2], ye[2];
                CPS_B_LOOP(rlo, rhi, 2, (re[u] = r[e], pe[u] = p[e], ye[u] = y[e]), {
                    const double pn = fma(beta, pe[u], re[u]);
                    p[e] = pn;
                    y[e] = fma(alpha, pn, ye[u]);
                    r[e] = fma(-alpha, pn, re[u]);
                })
            }
            // black: p = z + beta p, s = w + beta s, xh += alpha p,
            // rh -= alpha s
            double pe[2], se[2], we[2], ze[2], re[2], ye[2];
            CPS_B_LOOP(blo, bhi, 2,
                (pe[u] = p[e], se[u] = s[e], we[u] = w[e], ze[u] = z[e], re[u] = r[e],
                 ye[u] = y[e]),
                {
                    const double pn = fma(beta, pe[u], ze[u]);
                    const double sn = fma(beta, se[u], we[u]);
                    p[e] = pn;
                    s[e] = sn;
                    y[e] = fma(alpha, pn, ye[u]);
                    r[e] = fma(-alpha, sn, re[u]);
                })
        } else {
            // xh_R = y_R + E y_B (y_B still the untransformed iterate)
            for (int e = rlo + (int)threadIdx.x; e < rhi; e += kPBlock) {
                double v = fma(A[e], y[C[e]], y[e]);
                v = fma(A[n + e], y[C[n + e]], v);
                v = fma(A[2 * n + e], y[C[2 * n + e]], v);
                y[e] = v;
                p[e] = 0.0;
            }
            // rh_B = D_B^-1 (r_B - E^T r_R) (r_R is never written here)
            for (int e = blo + (int)threadIdx.x; e < bhi; e += kPBlock) {
                double v = fma(-A[e], r[C[e]], r[e]);
                v = fma(-A[n + e], r[C[n + e]], v);
                v = fma(-A[2 * n + e], r[C[2 * n + e]], v);
                r[e] = v * dinv[e];
                p[e] = 0.0;
                s[e] = 0.0;
            }
        }
        post(0, pass);
        // the red phase's first trip reads this block's rows up to the
        // gathers: fetch them into L1 while waiting on the neighbours
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = rlo + (int)threadIdx.x + u * kPBlock;
            if (e < rhi) {
                prefetch_l1(r + e);
                prefetch_l1(A + e);
                prefetch_l1(A + n + e);
                prefetch_l1(A + 2 * n + e);
                prefetch_l1(C + e);
                prefetch_l1(C + n + e);
                prefetch_l1(C + 2 * n + e);
            }
        }
        if (!(ok = wait(0, pass, 1))) break;
        // red: v_R = E rh_B; gamma_R = delta_R = rh_R.rh_R
        {
            double re[2], a0[2], a1[2], a2[2];
            int c0[2], c1[2], c2[2];
            CPS_B_LOOP(rlo, rhi, 2,
                (re[u] = r[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double v = a0[u] * r[c0[u]];
                    v = fma(a1[u], r[c1[u]], v);
                    v = fma(a2[u], r[c2[u]], v);
                    z[e] = v;
                    sums[0] = fma(re[u], re[u], sums[0]);
                    if (check) {
                        const double tt = P.s[e] * re[u];
                        sums[2] = fma(tt, tt, sums[2]);
                    }
                })
        }
        sums[1] = sums[0];
        post(1, pass);
        // likewise the black phase's first trip
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = blo + (int)threadIdx.x + u * kPBlock;
            if (e < bhi) {
                prefetch_l1(r + e);
                prefetch_l1(A + e);
                prefetch_l1(A + n + e);
                prefetch_l1(A + 2 * n + e);
                prefetch_l1(C + e);
                prefetch_l1(C + n + e);
                prefetch_l1(C + 2 * n + e);
                prefetch_l1(dpiv + e);
                prefetch_l1(dinv + e);
            }
        }
        if (!(ok = wait(1, pass, 0))) break;
        // black: w_B = D_B^-1 (rh_B - E^T v), z_B = D_B rh_B; gamma_B, delta_B
        {
            double re[2], a0[2], a1[2], a2[2];
            int c0[2], c1[2], c2[2];
            CPS_B_LOOP(blo, bhi, 2,
                (re[u] = r[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double t = fma(-a0[u], z[c0[u]], re[u]);
                    t = fma(-a1[u], z[c1[u]], t);
                    t = fma(-a2[u], z[c2[u]], t);
                    const double d = dpiv[e];
                    const double ze = d * re[u];
                    w[e] = t * dinv[e];
                    z[e] = ze;
                    if (!upd) y[e] = d * y[e];        // xh_B = D_B y_B
                    sums[0] = fma(re[u], ze, sums[0]);
                    sums[1] = fma(t, re[u], sums[1]);
                    if (check) {
                        double rb = fma(a0[u], r[c0[u]], ze);
                        rb = fma(a1[u], r[c1[u]], rb);
                        rb = fma(a2[u], r[c2[u]], rb);
                        const double tt = P.s[e] * rb;
                        sums[2] = fma(tt, tt, sums[2]);
                    }
                })
        }
        // the next update's first trips read only this block's own rows,
        // final now: fetch them into L1 during the reduction
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int er = rlo + (int)threadIdx.x + u * kPBlock;
            if (er < rhi) {
                prefetch_l1(r + er);
                prefetch_l1(p + er);
                prefetch_l1(y + er);
            }
        }
        auto step = [&](const double* t, bool chk, int& f) {
            const double g = t[0], d = t[1];
            bool halt = !(g > 0.0) || (upd && pass >= s_max_iter);   // exact, budget
            if (chk) {
                sc[3] = t[2];
                if (t[2] <= sc[6]) halt = true;
            }
            f = halt ? 1 : 0;
            if (!halt) {
                const double den = fma(-(g * g), sc[5], d);
                if (!(den > 0.0) || !isfinite(den)) {
                    // pass 0: z.Tz <= 0, not SPD; later the recurrence's
                    // difference lost its digits at the FP64 floor: stop,
                    // and let the true residual decide
                    f = upd ? 1 : 2;
                } else {
                    const double ig = 1.0 / g;
                    sc[1] = g / den;
                    sc[2] = g * sc[4];
                    sc[4] = ig;
                    sc[5] = den * ig * ig;
                }
            }
            sc[0] = g;
        };
        double none[1];
        int flag = 0;
        if (check) {
            double v3[3] = {sums[0], sums[1], sums[2]};
            ok = grid_allreduce<3, 1>(rbuf, v3, none, flag, P.partials, gs, ep,
                                      [&](const double (&t)[3], double* o, int& f) {
                                          o[0] = 0.0;
                                          step(t, true, f);
                                      });
        } else {
            double v2[2] = {sums[0], sums[1]};
            ok = grid_allreduce<2, 1>(rbuf, v2, none, flag, P.partials, gs, ep,
                                      [&](const double (&t)[2], double* o, int& f) {
                                          o[0] = 0.0;
                                          step(t, false, f);
                                      });
        }
        if (!ok) break;
        if (flag) {
            if (threadIdx.x == 0) s_stop = flag;
            break;
        }
    }
    if (ok) {
        // y = (Dt + Lt^T)^-1 xh: y_B = D_B^-1 xh_B, then y_R = xh_R - E y_B
        for (int e = blo + (int)threadIdx.x; e < bhi; e += kPBlock) y[e] *= dinv[e];
        post(2, 0);
        ok = wait(2, 0, 1);
        if (ok) {
            for (int e = rlo + (int)threadIdx.x; e < rhi; e += kPBlock) {
                double v = fma(-A[e], y[C[e]], y[e]);
                v = fma(-A[n + e], y[C[n + e]], v);
                v = fma(-A[2 * n + e], y[C[2 * n + e]], v);
                y[e] = v;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = pass;
        st->rho = sc[0];
        st->alpha = sc[1];
        st->beta = sc[2];
        st->rnorm2 = sc[3];
        st->status = ok ? (s_stop == 2 ? CPS_ERR_NOT_SPD : CPS_OK) : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

// Reduced system (two colours, colour order): CG on S = I - E^T E over the
// black rows [nR, n) from the state k_black_init left.  Block b owns red rows
// [b Rr, (b+1) Rr) and black rows nR + [b Rb, (b+1) Rb).
//   t_R = E p_B | q_B = p_B - E^T t_R, gamma | r -= alpha q, rho' | y, p |
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_reduced(PersistArgs P) {
    __shared__ double rbuf[2][kPBlock];
    // the run's scalars (the same in every block) in shared memory, so that
    // the streaming phases keep their registers: rho, ||S r||^2
    __shared__ double sc[2];
    CgState* st = P.st;
    if (st->done) return;
    const int64_t n = P.n, nR = P.nR, nB = n - nR;
    const double* __restrict__ A = P.a;
    const int32_t* __restrict__ C = P.col;
    double* __restrict__ p = P.p;
    double* __restrict__ q = P.q;
    double* __restrict__ r = P.r;
    double* __restrict__ y = P.y;
    double* __restrict__ t = P.t;
    GridSync* gs = P.gs;
    // row ranges fit 32 bits (the columns are int32): fewer registers
    const int Rr = (int)rows_per_block(nR), Rb = (int)rows_per_block(nB);
    const int rlo = (int)blockIdx.x * Rr < nR ? (int)blockIdx.x * Rr : (int)nR;
    const int rhi = rlo + Rr < nR ? rlo + Rr : (int)nR;
    const int blo = (int)nR + ((int)blockIdx.x * Rb < nB ? (int)blockIdx.x * Rb : (int)nB);
    const int bhi = blo + Rb < n ? blo + Rb : (int)n;
    if (threadIdx.x == 0) {
        sc[0] = st->rho;
        sc[1] = st->rnorm2;
    }
    long long it = 0;
    int status = CPS_OK;
    bool ok = true;
    Epoch ep;
    ep.target = P.stall ? 1ull : 0ull;
    // The red phase reads p at black rows, the black phase t at red rows:
    // on banded numberings both lie in a few neighbouring blocks, and the
    // two grid barriers become waits on those blocks' flags (slot 0: p
    // updated, slot 1: t computed), as in k_persistent_cg.
    int dplo, dphi, dtlo, dthi;
    column_blocks(C, n, rlo, rhi, nR, Rb, &dplo, &dphi);
    column_blocks(C, n, blo, bhi, 0, Rr, &dtlo, &dthi);
    bool halo;
    {
        const bool wide = dphi - dplo + 1 > kMaxDeps || dthi - dtlo + 1 > kMaxDeps;
        double w[1] = {wide ? 1.0 : 0.0};
        double none[1];
        int any = 0;
        ok = grid_allreduce<1, 1>(rbuf, w, none, any, P.partials, gs, ep,
                                  [](const double (&tt)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = tt[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    while (ok) {
        if (halo && it > 0) {
            ok = halo_wait(gs, dplo, dphi, (unsigned long long)it, 0);
            if (!ok) break;
        }
        {
            double a0[kU], a1[kU], a2[kU];
            int32_t c0[kU], c1[kU], c2[kU];
            CPS_B_LOOP(rlo, rhi, kU,
                (a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e], c0[u] = C[e],
                 c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double acc = 0.0;
                    if (c0[u] != (int32_t)e) acc = fma(a0[u], p[c0[u]], acc);
                    if (c1[u] != (int32_t)e) acc = fma(a1[u], p[c1[u]], acc);
                    if (c2[u] != (int32_t)e) acc = fma(a2[u], p[c2[u]], acc);
                    t[e] = acc;
                })
        }
        if (halo) {
            halo_post(gs, (unsigned long long)(it + 1), 1);
            ok = halo_wait(gs, dtlo, dthi, (unsigned long long)(it + 1), 1);
        } else {
            ok = grid_barrier(gs, ep);
        }
        if (!ok) break;
        double g[1] = {0.0};
        {
            double pe[kU], a0[kU], a1[kU], a2[kU];
            int32_t c0[kU], c1[kU], c2[kU];
            CPS_B_LOOP(blo, bhi, kU,
                (pe[u] = p[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double v = pe[u];
                    if (c0[u] != (int32_t)e) v = fma(-a0[u], t[c0[u]], v);
                    if (c1[u] != (int32_t)e) v = fma(-a1[u], t[c1[u]], v);
                    if (c2[u] != (int32_t)e) v = fma(-a2[u], t[c2[u]], v);
                    q[e] = v;
                    g[0] = fma(pe[u], v, g[0]);
                })
        }
        double sa[1];
        int bad = 0;
        ok = grid_allreduce<1, 1>(rbuf, g, sa, bad, P.partials, gs, ep,
                                  [&](const double (&t)[1], double* o, int& f) {
                                      f = (t[0] > 0.0 && isfinite(t[0])) ? 0 : 1;
                                      o[0] = f ? 0.0 : sc[0] / t[0];
                                  });
        if (!ok) break;
        if (bad) {
            status = CPS_ERR_NOT_SPD;
            break;
        }
        const double alpha = sa[0];
        const bool check = ((it + 1) % 8) == 0;
        double rr[2] = {0.0, 0.0};
        {
            double qe[kUV], re0[kUV];
            CPS_B_LOOP(blo, bhi, kUV, (qe[u] = q[e], re0[u] = r[e]), {
                const double re = fma(-alpha, qe[u], re0[u]);
                r[e] = re;
                rr[0] = fma(re, re, rr[0]);
                if (check) {
                    const double tt = P.s[e] * re;
                    rr[1] = fma(tt, tt, rr[1]);
                }
            })
        }
        double sb[1];
        int stop = 0;
        const long long it1 = it + 1;
        ok = grid_allreduce<2, 1>(rbuf, rr, sb, stop, P.partials, gs, ep,
                                  [&](const double (&t)[2], double* o, int& f) {
                                      bool halt = !(t[0] > 0.0) || it1 >= st->max_iter;
                                      if (check) {
                                          sc[1] = t[1];  // ||S r||^2
                                          if (t[1] <= st->thresh2) halt = true;
                                      }
                                      o[0] = t[0] / sc[0];   // beta
                                      sc[0] = t[0];          // rho'
                                      f = halt ? 1 : 0;
                                  });
        if (!ok) break;
        ++it;
        const double beta = sb[0];
        {
            double pe[kUV], ye[kUV], re[kUV];
            CPS_B_LOOP(blo, bhi, kUV, (pe[u] = p[e], ye[u] = y[e], re[u] = stop ? 0.0 : r[e]), {
                y[e] = fma(alpha, pe[u], ye[u]);
                if (!stop) p[e] = fma(beta, pe[u], re[u]);
            })
        }
        if (stop) break;
        if (halo) {
            halo_post(gs, (unsigned long long)it, 0);
        } else {
            ok = grid_barrier(gs, ep);
            if (!ok) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = it;
        st->rho = sc[0];
        st->rnorm2 = sc[1];
        st->status = ok ? status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

// The reduced (black-cell Schur complement) CG with the single-reduction
// (Chronopoulos-Gear) recurrences, from the state k_black_init left (y_B,
// r_B, ||b||^2, ||S r||^2): s_B = Schur p_B and w_B = Schur r_B are carried,
// so that both inner products of an iteration come from one Schur product:
//   [wait for the halo] t_R = E r_B | post, [wait] w_B = r_B - E^T t_R,
//   gamma = r.r, delta = w.r (every 8th: ||S r||^2) | one grid reduction:
//   stop test; first pass alpha = gamma/delta, beta = 0; later beta =
//   gamma/gamma_old, alpha = gamma/(delta - beta gamma/alpha_old) |
//   p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s | post
// Two neighbour waits and one grid reduction per iteration (the textbook
// reduced loop, k_persistent_reduced, has two reductions), at 9 FP64 FMAs a
// black row plus 3 a red row.  s lives in q, w in z; p and s start at zero.
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_reduced1(PersistArgs P) {
    __shared__ double rbuf[3][kPBlock];
    // gamma, alpha, beta, ||S r||^2, 1/gamma, 1/(gamma alpha), stop threshold
    __shared__ double sc[7];
    __shared__ long long s_max_iter;
    __shared__ int s_stop;
    CgState* st = P.st;
    if (st->done) return;                      // uniform: set before the launch
    const int64_t n = P.n, nR = P.nR, nB = n - nR;
    const double* __restrict__ A = P.a;
    const int32_t* __restrict__ C = P.col;
    double* __restrict__ p = P.p;
    double* __restrict__ sv = P.q;
    double* __restrict__ w = P.z;
    double* __restrict__ r = P.r;
    double* __restrict__ y = P.y;
    double* __restrict__ t = P.t;
    GridSync* gs = P.gs;
    const int Rr = (int)rows_per_block(nR), Rb = (int)rows_per_block(nB);
    const int rlo = (int)blockIdx.x * Rr < nR ? (int)blockIdx.x * Rr : (int)nR;
    const int rhi = rlo + Rr < nR ? rlo + Rr : (int)nR;
    const int blo = (int)nR + ((int)blockIdx.x * Rb < nB ? (int)blockIdx.x * Rb : (int)nB);
    const int bhi = blo + Rb < n ? blo + Rb : (int)n;
    if (threadIdx.x == 0) {
        sc[0] = st->rho;
        sc[1] = 0.0;
        sc[2] = 0.0;
        sc[3] = st->rnorm2;
        sc[4] = 0.0;
        sc[5] = 0.0;
        sc[6] = st->thresh2;
        s_max_iter = st->max_iter;
        s_stop = 0;
    }
    bool ok = true;
    Epoch ep;
    ep.target = P.stall ? 1ull : 0ull;
    // the red phase reads r at black rows, the black phase t at red rows
    // (slot 0: r updated, slot 1: t computed), as in k_persistent_reduced
    int dplo, dphi, dtlo, dthi;
    column_blocks(C, n, rlo, rhi, nR, Rb, &dplo, &dphi);
    column_blocks(C, n, blo, bhi, 0, Rr, &dtlo, &dthi);
    bool halo;
    {
        const bool wide = dphi - dplo + 1 > kMaxDeps || dthi - dtlo + 1 > kMaxDeps;
        double wv[1] = {wide ? 1.0 : 0.0};
        double none[1];
        int any = 0;
        ok = grid_allreduce<1, 1>(rbuf, wv, none, any, P.partials, gs, ep,
                                  [](const double (&tt)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = tt[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    // the recurrences start from p = s = 0 (own rows only)
    for (int64_t e = blo + threadIdx.x; e < bhi; e += kPBlock) {
        p[e] = 0.0;
        sv[e] = 0.0;
    }
    long long it = 0;
    while (ok) {
        if (halo && it > 0) {
            ok = halo_wait(gs, dplo, dphi, (unsigned long long)it, 0);
            if (!ok) break;
        }
        {
            double a0[kU], a1[kU], a2[kU];
            int32_t c0[kU], c1[kU], c2[kU];
            CPS_B_LOOP(rlo, rhi, kU,
                (a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e], c0[u] = C[e],
                 c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double acc = 0.0;
                    if (c0[u] != (int32_t)e) acc = fma(a0[u], r[c0[u]], acc);
                    if (c1[u] != (int32_t)e) acc = fma(a1[u], r[c1[u]], acc);
                    if (c2[u] != (int32_t)e) acc = fma(a2[u], r[c2[u]], acc);
                    t[e] = acc;
                })
        }
        if (halo) {
            halo_post(gs, (unsigned long long)(it + 1), 1);
            ok = halo_wait(gs, dtlo, dthi, (unsigned long long)(it + 1), 1);
        } else {
            ok = grid_barrier(gs, ep);
        }
        if (!ok) break;
        const bool check = ((it + 1) % 8) == 0;
        double sums[3] = {0.0, 0.0, 0.0};
        {
            double re[kUGS], a0[kUGS], a1[kUGS], a2[kUGS];
            int32_t c0[kUGS], c1[kUGS], c2[kUGS];
            CPS_B_LOOP(blo, bhi, kUGS,
                (re[u] = r[e], a0[u] = A[e], a1[u] = A[n + e], a2[u] = A[2 * n + e],
                 c0[u] = C[e], c1[u] = C[n + e], c2[u] = C[2 * n + e]),
                {
                    double v = re[u];
                    if (c0[u] != (int32_t)e) v = fma(-a0[u], t[c0[u]], v);
                    if (c1[u] != (int32_t)e) v = fma(-a1[u], t[c1[u]], v);
                    if (c2[u] != (int32_t)e) v = fma(-a2[u], t[c2[u]], v);
                    w[e] = v;
                    sums[0] = fma(re[u], re[u], sums[0]);
                    sums[1] = fma(v, re[u], sums[1]);
                    if (check) {
                        const double tt = P.s[e] * re[u];
                        sums[2] = fma(tt, tt, sums[2]);
                    }
                })
        }
        // thread 0, from the totals: the stop test and the step scalars (1/gamma
        // and 1/(gamma alpha) carried, one divide on the critical path)
        const long long it0 = it;
        auto post = [&](const double* tt, bool chk, int& f) {
            const double g = tt[0], d = tt[1];
            bool halt = !(g > 0.0) || it0 >= s_max_iter;       // exact solution, budget
            if (chk) {
                sc[3] = tt[2];
                if (tt[2] <= sc[6]) halt = true;
            }
            f = halt ? 1 : 0;
            if (!halt) {
                const double den = it0 == 0 ? d : fma(-(g * g), sc[5], d);
                if (!(den > 0.0) || !isfinite(den)) {
                    // on the run's first pass p.Sp <= 0: not SPD; later, the
                    // recurrence's difference lost its digits at the FP64
                    // floor: stop, and let the true residual decide
                    f = it0 > 0 ? 1 : 2;
                } else {
                    const double ig = 1.0 / g;
                    sc[1] = g / den;
                    sc[2] = it0 == 0 ? 0.0 : g * sc[4];
                    sc[4] = ig;
                    sc[5] = den * ig * ig;
                }
            }
            sc[0] = g;
        };
        double none[1];
        int flag = 0;
        if (check) {
            double v3[3] = {sums[0], sums[1], sums[2]};
            ok = grid_allreduce<3, 1>(rbuf, v3, none, flag, P.partials, gs, ep,
                                      [&](const double (&tt)[3], double* o, int& f) {
                                          o[0] = 0.0;
                                          post(tt, true, f);
                                      });
        } else {
            double v2[2] = {sums[0], sums[1]};
            ok = grid_allreduce<2, 1>(rbuf, v2, none, flag, P.partials, gs, ep,
                                      [&](const double (&tt)[2], double* o, int& f) {
                                          o[0] = 0.0;
                                          post(tt, false, f);
                                      });
        }
        if (!ok) break;
        if (flag) {
            if (threadIdx.x == 0) s_stop = flag;
            break;
        }
        {
            const double alpha = sc[1], beta = sc[2];
            double pe[kUG], se[kUG], we[kUG], re[kUG], ye[kUG];
            CPS_B_LOOP(blo, bhi, kUG,
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
        ++it;
        if (halo) {
            halo_post(gs, (unsigned long long)it, 0);
        } else {
            ok = grid_barrier(gs, ep);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->iter = it;
        st->rho = sc[0];
        st->rnorm2 = sc[3];
        st->status = ok ? (s_stop == 2 ? CPS_ERR_NOT_SPD : CPS_OK) : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

}  // namespace

// The persistent kernel of a solve kind: 0 textbook Jacobi, 1 the reduced
// system, 2 single-reduction Jacobi, 3 single-reduction IC(0) in a
// two-colour order, 4 the reduced system with the single-reduction
// recurrences.
static void (*persistent_kernel(int kind))(PersistArgs) {
    switch (kind) {
        case 1: return k_persistent_reduced;
        case 2: return k_persistent_gear;
        case 3: return k_persistent_ic0;
        case 4: return k_persistent_reduced1;
        default: return k_persistent_cg;
    }
}

// Largest grid of a persistent launch on this device (blocks that stay
// resident together), 0 if the kernel does not fit.
int persistent_max_grid(cps_sys s, int reduced) {
    auto kern = persistent_kernel(reduced);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int G = s->ctx->num_sms * (per_sm < 4 ? per_sm : 4);
    return G > kPBlock ? kPBlock : G;
}

// Launches the persistent solve (reduced = 0: Jacobi on all rows; 1: the
// reduced system; 2: single-reduction Jacobi on all rows, after k_init64 and
// k_gear_start, with s = A p in q and w = A r in t; 3: single-reduction IC(0)
// in the two-colour order after k_init64, s in q, w in t, z and the inverse
// pivots in z, dinv; 4: the reduced system with the single-reduction
// recurrences after k_black_init, s in q, w in z, the red scratch in t)
// after the caller's init kernel; state in s->st.  With
// win_bytes > 0 the launch carries a persisting L2 access-policy window over
// [win_base, win_base + win_bytes) (the caller holds the set-aside).  grid:
// blocks of the launch, at most what stays resident (0: that maximum).
int persistent_solve(cps_sys s, int reduced, const double* a, const int32_t* col,
                     const double* sc, double* y, double* r, double* p, double* q, double* t,
                     int64_t n, int64_t nR, const void* win_base, size_t win_bytes, int grid,
                     cudaStream_t stream, double* z, const double* dinv, const double* dpiv) {
    if (!s->gsync) {
        cudaError_t e = cudaMalloc((void**)&s->gsync, sizeof(GridSync));
        if (e != cudaSuccess) {
            cudaGetLastError();
            cps::set_error(s->ctx, "persistent: cudaMalloc failed");
            return CPS_ERR_NOMEM;
        }
    }
    auto kern = persistent_kernel(reduced);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        cps::set_error(s->ctx, "persistent: kernel does not fit an SM");
        return CPS_ERR_ARG;
    }
    int G = s->ctx->num_sms * (per_sm < 4 ? per_sm : 4);
    if (G > kPBlock) G = kPBlock;          // the reductions stage one value per block in a row
    if (grid > 0 && grid < G) G = grid;
    // counter, timeout and the G flags in use start at zero
    CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(s->gsync, 0,
                                         offsetof(GridSync, flag) +
                                             sizeof(unsigned long long) * kFlagStride * G,
                                         stream));
    const int stall = s->inject == CPS_TEST_STALL_BARRIER ? 1 : 0;
    s->inject = 0;
    PersistArgs P{a, col, sc, y, r, p, q, t, n, nR, s->partials,
                  reinterpret_cast<GridSync*>(s->gsync), s->st, stall, s->diag_min, z, dinv,
                  dpiv};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G, 1, 1);
    cfg.blockDim = dim3(kPBlock, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributeAccessPolicyWindow;
    at[1].val.accessPolicyWindow.base_ptr = const_cast<void*>(win_base);
    at[1].val.accessPolicyWindow.num_bytes = win_bytes;
    at[1].val.accessPolicyWindow.hitRatio = 1.0f;
    at[1].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[1].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = at;
    cfg.numAttrs = win_bytes > 0 ? 2 : 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, P);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cps::set_error(s->ctx, std::string("persistent launch: ") + cudaGetErrorString(e));
        return CPS_ERR_CUDA;
    }
    return CPS_OK;
}

}  // namespace cps
