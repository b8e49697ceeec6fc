// Device code of the block-level solves shared by the one-launch ensemble
// (batch.cu) and the one-launch CP1 step (cp1step.cu): teams of blocks with
// bounded-wait synchronisation, and FP64 / mixed-precision Jacobi PCG of one
// system (or one member's rows of it) by one block.
#pragma once

#include "cps_internal.cuh"
#include "exact_sum.cuh"

#include <cstdint>

namespace cps {
namespace {

// One system as the block-level solves see it (the graph-chunk batch path
// uses the tile fields).
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
constexpr int kMaxTeam = kBB;     // members (a team sum gives each thread one)
constexpr long long kTeamSpinCap = 1LL << 26;
constexpr unsigned long long kTeamWaitNs = 1000000000ull;

// One team's synchronisation state (count and timeout zero before the
// launch; partials a buffer of 2 x 4 x k doubles).
struct TeamSync {
    unsigned long long count;   // arrivals since the launch
    int timeout;
    int stall;                  // test hook: every wait expects one more arrival
    double* partials;           // [2][4][k]: per sync parity, quantity, member
    int pad[10];
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
// the k members' totals (one per thread, k <= kMaxTeam) summed exactly by the
// block -- the same set in every member, so bit-identical results and the
// same decisions in all of them.  Also a team barrier.
template <int NV>
__device__ __forceinline__ bool team_sum(double (&v)[NV], TeamCtx& tc) {
    static_assert(NV >= 1 && NV <= 4, "team sum width");
    __shared__ int s_par;
    block_sum_exact<NV, kBB>(v);
    if (threadIdx.x == 0) {
        double* P = tc.ts->partials + (size_t)(tc.epoch & 1) * 4 * tc.k;
#pragma unroll
        for (int q = 0; q < NV; ++q) P[q * tc.k + tc.rank] = v[q];
        s_par = team_arrive_wait(tc);
    }
    __syncthreads();
    const int par = s_par;
    if (par < 0) return false;
    const int k = tc.k;
    const double* P = tc.ts->partials + (size_t)par * 4 * k;
    const int m = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = m < k ? __ldcg(P + q * k + m) : 0.0;
    block_sum_exact<NV, kBB>(v);
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
// written by the block that holds row 0.  Returns false if a team wait ran
// out (the status is then CPS_ERR_TIMEOUT).
__device__ __forceinline__ bool kbp_solve(const BatchDesc& d, int64_t lo, int64_t hi,
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
    return ok;
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
// updates; done = 2) from the block that holds row 0.  Returns false if a
// team wait ran out.
__device__ __forceinline__ bool kbp_solve_mixed(const BatchDesc& d, int64_t lo, int64_t hi,
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
    return ok;
}

}  // namespace
}  // namespace cps
