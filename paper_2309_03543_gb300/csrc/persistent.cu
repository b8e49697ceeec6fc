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

#include <cmath>
#include <cstddef>

namespace cps {
namespace {

constexpr int kPBlock = 1024;
constexpr long long kSpinCap = 1LL << 26;           // polls; each one an L2 round trip
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr int kFlagStride = 16;                      // one 128-byte line per block flag
constexpr int kMaxDeps = 8;

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

// Barriers passed by this block (reductions and grid barriers).
struct Epoch {
    unsigned long long k = 0;
    unsigned long long extra = 0;   // test hook: arrivals a barrier waits for beyond the grid
};

// Grid-wide sum of v[0..NV) (NV <= 2).  Lane 0 of warp 0 then derives the
// block's scalars from the totals, post(tot, sc, flag) (once per block: a
// FP64 divide per thread would cost GB300 more than a vector sweep), and
// every thread receives sc[0..NS) and the flag.  Returns false if a wait ran
// out somewhere.
template <int NV, int NS, typename Post>
__device__ bool grid_allreduce(double (&v)[NV], double (&out)[NS], int& flag, double* partials,
                               GridSync* gs, Epoch& ep, Post post) {
    static_assert(NV >= 1 && NV <= 2, "two partial slots per buffer");
    __shared__ double buf[NV][kPBlock];
    __shared__ double sc[NS];
    __shared__ int s_flag;
    __shared__ int s_ok;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
    __syncthreads();            // also orders every thread's phase writes before the arrival
    const unsigned int G = gridDim.x;
    double* pb = partials + (size_t)(ep.k & 1) * (2 * kMaxGrid);
    ++ep.k;
    if (threadIdx.x < 32) {
        double t[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = buf[k][lane];
#pragma unroll
            for (int j = lane + 32; j < kPBlock; j += 32) a += buf[k][j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            t[k] = a;
        }
        int ok = 1;
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) pb[k * kMaxGrid + blockIdx.x] = t[k];
            red_release_add(&gs->count, 1ull);
            ok = wait_geq(&gs->count, ep.k * (unsigned long long)G + ep.extra, gs) ? 1 : 0;
        }
        __syncwarp();
        ok = __shfl_sync(0xffffffffu, ok, 0);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double a = 0.0;
            for (unsigned int i = lane; i < G; i += 32) a += __ldcg(&pb[k * kMaxGrid + i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            t[k] = a;
        }
        if (lane == 0) {
            s_ok = ok;
            post(t, sc, s_flag);
        }
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
    ++ep.k;
    if (threadIdx.x == 0) {
        red_release_add(&gs->count, 1ull);
        s_ok = wait_geq(&gs->count, ep.k * (unsigned long long)gridDim.x + ep.extra, gs) ? 1 : 0;
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
    ep.extra = P.stall ? 1ull : 0ull;
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
        ok = grid_allreduce<1, 1>(wide, none, any, P.partials, gs, ep,
                                  [](const double (&t)[1], double* o, int& f) {
                                      o[0] = 0.0;
                                      f = t[0] > 0.0 ? 1 : 0;
                                  });
        halo = any == 0;
    }
    // the run's scalars (the same values in every thread of every block)
    double rho = st->rho;
    const double thresh2 = st->thresh2;
    const long long max_iter = st->max_iter;
    long long it = 0;
    int status = CPS_OK;
    double rnorm2 = st->rnorm2;
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
        ok = grid_allreduce<1, 1>(g, sa, bad, P.partials, gs, ep,
                                  [&](const double (&t)[1], double* o, int& f) {
                                      f = (t[0] > 0.0 && isfinite(t[0])) ? 0 : 1;
                                      o[0] = f ? 0.0 : rho / t[0];
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
        double sb[3];
        int stop = 0;
        ok = grid_allreduce<2, 3>(rr, sb, stop, P.partials, gs, ep,
                                  [&](const double (&t)[2], double* o, int& f) {
                                      bool halt = !(t[0] > 0.0) || it + 1 >= max_iter;
                                      if (check && t[1] <= thresh2) halt = true;
                                      o[0] = t[0] / rho;     // beta
                                      o[1] = t[0];           // rho'
                                      o[2] = t[1];           // ||S r||^2
                                      f = halt ? 1 : 0;
                                  });
        if (!ok) break;
        ++it;
        if (check) rnorm2 = sb[2];
        const double beta = sb[0];
        rho = sb[1];
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
        st->rho = rho;
        st->rnorm2 = rnorm2;
        st->status = ok ? status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

// Reduced system (two colours, colour order): CG on S = I - E^T E over the
// black rows [nR, n) from the state k_black_init left.  Block b owns red rows
// [b Rr, (b+1) Rr) and black rows nR + [b Rb, (b+1) Rb).
//   t_R = E p_B | q_B = p_B - E^T t_R, gamma | r -= alpha q, rho' | y, p |
__global__ void __launch_bounds__(kPBlock, 1) k_persistent_reduced(PersistArgs P) {
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
    const int64_t Rr = rows_per_block(nR), Rb = rows_per_block(nB);
    const int64_t rlo = blockIdx.x * Rr < nR ? blockIdx.x * Rr : nR;
    const int64_t rhi = rlo + Rr < nR ? rlo + Rr : nR;
    const int64_t blo = nR + (blockIdx.x * Rb < nB ? blockIdx.x * Rb : nB);
    const int64_t bhi = blo + Rb < n ? blo + Rb : n;
    double rho = st->rho;
    const double thresh2 = st->thresh2;
    const long long max_iter = st->max_iter;
    long long it = 0;
    int status = CPS_OK;
    double rnorm2 = st->rnorm2;
    bool ok = true;
    Epoch ep;
    ep.extra = P.stall ? 1ull : 0ull;
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
        ok = grid_allreduce<1, 1>(w, none, any, P.partials, gs, ep,
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
        ok = grid_allreduce<1, 1>(g, sa, bad, P.partials, gs, ep,
                                  [&](const double (&t)[1], double* o, int& f) {
                                      f = (t[0] > 0.0 && isfinite(t[0])) ? 0 : 1;
                                      o[0] = f ? 0.0 : rho / t[0];
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
        double sb[3];
        int stop = 0;
        ok = grid_allreduce<2, 3>(rr, sb, stop, P.partials, gs, ep,
                                  [&](const double (&t)[2], double* o, int& f) {
                                      bool halt = !(t[0] > 0.0) || it + 1 >= max_iter;
                                      if (check && t[1] <= thresh2) halt = true;
                                      o[0] = t[0] / rho;     // beta
                                      o[1] = t[0];           // rho'
                                      o[2] = t[1];           // ||S r||^2
                                      f = halt ? 1 : 0;
                                  });
        if (!ok) break;
        ++it;
        if (check) rnorm2 = sb[2];
        const double beta = sb[0];
        rho = sb[1];
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
        st->rho = rho;
        st->rnorm2 = rnorm2;
        st->status = ok ? status : CPS_ERR_TIMEOUT;
        st->done = 2;
    }
}

}  // namespace

// Largest grid of a persistent launch on this device (blocks that stay
// resident together), 0 if the kernel does not fit.
int persistent_max_grid(cps_sys s, int reduced) {
    auto kern = reduced ? k_persistent_reduced : k_persistent_cg;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int G = s->ctx->num_sms * (per_sm < 4 ? per_sm : 4);
    return G > kMaxGrid ? kMaxGrid : G;
}

// Launches the persistent solve (reduced = 0: Jacobi on all rows; 1: the
// reduced system) after the caller's init kernel; state in s->st.  With
// win_bytes > 0 the launch carries a persisting L2 access-policy window over
// [win_base, win_base + win_bytes) (the caller holds the set-aside).  grid:
// blocks of the launch, at most what stays resident (0: that maximum).
int persistent_solve(cps_sys s, int reduced, const double* a, const int32_t* col,
                     const double* sc, double* y, double* r, double* p, double* q, double* t,
                     int64_t n, int64_t nR, const void* win_base, size_t win_bytes, int grid,
                     cudaStream_t stream) {
    if (!s->gsync) {
        cudaError_t e = cudaMalloc((void**)&s->gsync, sizeof(GridSync));
        if (e != cudaSuccess) {
            cudaGetLastError();
            cps::set_error(s->ctx, "persistent: cudaMalloc failed");
            return CPS_ERR_NOMEM;
        }
    }
    auto kern = reduced ? k_persistent_reduced : k_persistent_cg;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPBlock, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        cps::set_error(s->ctx, "persistent: kernel does not fit an SM");
        return CPS_ERR_ARG;
    }
    int G = s->ctx->num_sms * (per_sm < 4 ? per_sm : 4);
    if (G > kMaxGrid) G = kMaxGrid;
    if (grid > 0 && grid < G) G = grid;
    // counter, timeout and the G flags in use start at zero
    CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(s->gsync, 0,
                                         offsetof(GridSync, flag) +
                                             sizeof(unsigned long long) * kFlagStride * G,
                                         stream));
    const int stall = s->inject == CPS_TEST_STALL_BARRIER ? 1 : 0;
    s->inject = 0;
    PersistArgs P{a, col, sc, y, r, p, q, t, n, nR, s->partials,
                  reinterpret_cast<GridSync*>(s->gsync), s->st, stall};
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
