// Persistent solve of a small system inside one thread-block cluster.
//
// For meshes of up to a few tens of thousands of cells every kernel launch of
// the streaming loop costs more than its work, so the whole Jacobi-PCG run is
// one launch of a single cluster of C CTAs (C = 16 where the GPU allows it).
// CTA k owns rows [k R, (k+1) R): its slice of the scaled matrix and of the
// vectors y, r, p, q, s stay in its shared memory for the whole run.  The
// SpMV reads a neighbour's p from the owning CTA's shared memory through the
// cluster's distributed shared memory.  A dot product is summed per CTA and
// the CTA's partial is stored into a slot of every CTA's shared memory (C
// remote stores, one per lane); after the cluster barrier each CTA adds the C
// slots in rank order from its own shared memory (the same order everywhere,
// so all CTAs hold bit-identical alpha, beta and stop decisions).  The cluster barrier is the hardware one: all CTAs of a
// cluster are resident together, and no CTA waits on a software flag.
//
// Iteration (3 cluster barriers):
//   q = Ahat p, gamma = p.q | alpha = rho/gamma; r -= alpha q; y += alpha p;
//   rho' = r.r (and ||S r||^2) | beta = rho'/rho; stop test; p = r + beta p |
//
// Single-reduction variant (Chronopoulos-Gear recurrences; 2 cluster barriers):
// the CTA also keeps s = Ahat p and w = Ahat r, so that both inner products of
// an iteration come out of the one SpMV:
//   p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s |
//   w = Ahat r, gamma = r.r, delta = w.r (and ||S r||^2) |
//   beta = gamma/gamma_old, alpha = gamma/(delta - beta gamma/alpha_old).
// Same iterates as the textbook recurrence in exact arithmetic; one barrier
// fewer per iteration for the latency-bound small systems this path serves.
//
// Two more variants, pinned only (described at their kernels): the pipelined
// (Ghysels-Vanroose) recurrences with one split cluster barrier per
// iteration, and s-step CG (s = 2, 3) with s + 1 barriers per s iterations.
#include "cps_internal.cuh"
#include "exact_sum.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <cmath>

namespace cg = cooperative_groups;

namespace cps {
namespace {

constexpr int kClusterThreads = 1024;
constexpr int kCheck = 8;

struct ClusterArgs {
    const double* a;        // scaled off-diagonals [3][n]
    const int32_t* col;     // [3][n]
    const double* s;        // [n]
    const double* b;        // [n]
    const double* x;        // [n] initial guess
    double* y_out;          // [n] final scaled iterate
    CgState* st;
    int64_t n;
    int rows;               // R, rows per CTA
    double rtol;
    long long max_iter;
};

// Shared-memory layout of one CTA (R rows): a [3][R], p, r, y, q, s [R]
// doubles, col [3][R] int32, then (16-byte aligned) a reduction buffer of 3
// doubles per thread.
constexpr size_t kRowBytes = 3 * sizeof(double) + 3 * sizeof(int32_t) + 5 * sizeof(double);
constexpr size_t kRedBufBytes = 3 * kClusterThreads * sizeof(double);
__host__ __device__ inline size_t cluster_red_offset(int R) {
    return ((size_t)R * kRowBytes + 15) / 16 * 16;
}
__host__ __device__ inline size_t cluster_smem_bytes(int R) {
    return cluster_red_offset(R) + kRedBufBytes;
}

// Block sum of v[0..NV) through buf (NV x kClusterThreads doubles): warp k
// adds the values of quantity k (few FP64 adds: GB300 issues FP64 at 1/64
// of the FP32 rate); every thread then holds the totals.  Needs at least NV
// warps.
template <int NV>
__device__ __forceinline__ void block_sum_buf(double (&v)[NV], double* buf, double* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k * kClusterThreads + threadIdx.x] = v[k];
    __syncthreads();
    if (warp < NV) {
        double a = buf[warp * kClusterThreads + lane];
        for (int j = lane + 32; j < (int)blockDim.x; j += 32) a += buf[warp * kClusterThreads + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) tot[warp] = a;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = tot[k];
}

__global__ void __launch_bounds__(kClusterThreads, 1) k_cluster_cg(ClusterArgs A) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int R = A.rows;
    const int64_t n = A.n;
    const int64_t r0 = (int64_t)rank * R;
    const int nloc = (int)((r0 + R <= n) ? R : (n > r0 ? n - r0 : 0));

    extern __shared__ __align__(16) unsigned char smem[];
    double* a_s = reinterpret_cast<double*>(smem);          // [3][R]
    double* p_s = a_s + 3 * R;
    double* r_s = p_s + R;
    double* y_s = r_s + R;
    double* q_s = y_s + R;
    double* s_s = q_s + R;
    int32_t* c_s = reinterpret_cast<int32_t*>(s_s + R);      // [3][R] packed (rank << 16) | local
    double* rbuf = reinterpret_cast<double*>(smem + cluster_red_offset(R));
    __shared__ double red[3][16];   // red[k][c]: partial k of CTA c
    __shared__ double tot[3];
    __shared__ double sc[2];        // scalars derived once per CTA by thread 0
    __shared__ int s_stop;

    const int tid = threadIdx.x;
    for (int i = tid; i < nloc; i += blockDim.x) {
        const int64_t e = r0 + i;
        for (int j = 0; j < 3; ++j) {
            a_s[j * R + i] = A.a[j * n + e];
            const int32_t c = A.col[j * n + e];
            const int cr = c / R;
            c_s[j * R + i] = (cr << 16) | (c - cr * R);
        }
        const double se = A.s[e];
        s_s[i] = se;
        y_s[i] = se * A.x[e];
    }
    cluster.sync();

    auto gather = [&](double* base, int32_t packed) -> double {
        const int cr = packed >> 16, li = packed & 0xFFFF;
        if (cr == rank) return base[li];
        return cluster.map_shared_rank(base, cr)[li];
    };
    // This CTA's partial k (held by every thread after block_sum) goes to slot
    // [k][rank] of every CTA; lane c of warp 0 stores to CTA c.
    auto push = [&](int k, double v) {
        if (tid < C) cluster.map_shared_rank(&red[k][0], tid)[rank] = v;
    };
    // sum of slot k over the cluster, in rank order (thread 0 only: a FP64
    // add per thread per slot would cost more than the iteration's work)
    auto cluster_sum = [&](int k) -> double {
        double t = 0.0;
        for (int c = 0; c < C; ++c) t += red[k][c];
        return t;
    };

    // r = S^-1 b - Ahat y, p = r
    double v3[3] = {0.0, 0.0, 0.0};
    for (int i = tid; i < nloc; i += blockDim.x) {
        double ay = y_s[i];
        for (int j = 0; j < 3; ++j) ay = fma(a_s[j * R + i], gather(y_s, c_s[j * R + i]), ay);
        const double be = A.b[r0 + i];
        const double re = be / s_s[i] - ay;
        r_s[i] = re;
        p_s[i] = re;
        v3[0] = fma(re, re, v3[0]);
        v3[1] = fma(be, be, v3[1]);
        const double t = s_s[i] * re;
        v3[2] = fma(t, t, v3[2]);
    }
    block_sum_buf<3>(v3, rbuf, tot);
    push(0, v3[0]);
    push(1, v3[1]);
    push(2, v3[2]);
    cluster.sync();
    // run scalars: kept by thread 0 of every CTA (identical everywhere)
    double rho = 0.0, bnorm2 = 0.0, rnorm2 = 0.0, thresh2 = 0.0;
    if (tid == 0) {
        rho = cluster_sum(0);
        bnorm2 = cluster_sum(1);
        rnorm2 = cluster_sum(2);
        thresh2 = A.rtol * A.rtol * bnorm2;
        s_stop = (bnorm2 == 0.0 || rnorm2 <= thresh2 || A.max_iter <= 0) ? 1 : 0;
    }
    __syncthreads();
    int status = CPS_OK;
    long long it = 0;
    bool stop = s_stop != 0;
    while (!stop) {
        cluster.sync();     // p complete everywhere; partials of the last step read
        double g1[1] = {0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            const double pe = p_s[i];
            double v = pe;
            for (int j = 0; j < 3; ++j) v = fma(a_s[j * R + i], gather(p_s, c_s[j * R + i]), v);
            q_s[i] = v;
            g1[0] = fma(pe, v, g1[0]);
        }
        block_sum_buf<1>(g1, rbuf, tot);
        push(0, g1[0]);
        cluster.sync();
        if (tid == 0) {
            const double gamma = cluster_sum(0);
            const bool bad = !(gamma > 0.0) || !isfinite(gamma);
            sc[0] = bad ? 0.0 : rho / gamma;
            s_stop = bad ? 1 : 0;
        }
        __syncthreads();
        if (s_stop) {
            status = CPS_ERR_NOT_SPD;
            break;
        }
        const double alpha = sc[0];
        const bool check = ((it + 1) % kCheck) == 0;
        double g2[2] = {0.0, 0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            y_s[i] = fma(alpha, p_s[i], y_s[i]);
            const double re = fma(-alpha, q_s[i], r_s[i]);
            r_s[i] = re;
            g2[0] = fma(re, re, g2[0]);
            if (check) {
                const double t = s_s[i] * re;
                g2[1] = fma(t, t, g2[1]);
            }
        }
        block_sum_buf<2>(g2, rbuf, tot);
        push(1, g2[0]);
        push(2, g2[1]);
        cluster.sync();
        ++it;
        if (tid == 0) {
            const double rho_new = cluster_sum(1);
            bool halt = !(rho_new > 0.0) || it >= A.max_iter;
            if (check) {
                rnorm2 = cluster_sum(2);
                if (rnorm2 <= thresh2) halt = true;
            }
            sc[1] = rho_new / rho;
            rho = rho_new;
            s_stop = halt ? 1 : 0;
        }
        __syncthreads();
        stop = s_stop != 0;
        const double beta = sc[1];
        if (!stop)
            for (int i = tid; i < nloc; i += blockDim.x) p_s[i] = fma(beta, p_s[i], r_s[i]);
    }
    for (int i = tid; i < nloc; i += blockDim.x) A.y_out[r0 + i] = y_s[i];
    if (rank == 0 && tid == 0) {
        CgState* st = A.st;
        st->rho = rho;
        st->bnorm2 = bnorm2;
        st->thresh2 = thresh2;
        st->rnorm2 = rnorm2;
        st->iter = it;
        st->max_iter = A.max_iter;
        st->status = status;
        st->done = 2;
        st->alpha = 0.0;
        st->beta = 0.0;
    }
    cluster.sync();         // no CTA leaves while others may still read its memory
}

// Single-reduction layout: a [3][R], p, r, y, w, q (= Ahat p), s [R] doubles,
// col [3][R] int32, then the reduction buffer.
constexpr size_t kRowBytes1 = 3 * sizeof(double) + 3 * sizeof(int32_t) + 6 * sizeof(double);
__host__ __device__ inline size_t cluster1_red_offset(int R) {
    return ((size_t)R * kRowBytes1 + 15) / 16 * 16;
}
__host__ __device__ inline size_t cluster1_smem_bytes(int R) {
    return cluster1_red_offset(R) + kRedBufBytes;
}

__global__ void __launch_bounds__(kClusterThreads, 1) k_cluster_cg1(ClusterArgs A) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int R = A.rows;
    const int64_t n = A.n;
    const int64_t r0 = (int64_t)rank * R;
    const int nloc = (int)((r0 + R <= n) ? R : (n > r0 ? n - r0 : 0));

    extern __shared__ __align__(16) unsigned char smem[];
    double* a_s = reinterpret_cast<double*>(smem);          // [3][R]
    double* p_s = a_s + 3 * R;
    double* r_s = p_s + R;
    double* y_s = r_s + R;
    double* w_s = y_s + R;
    double* q_s = w_s + R;
    double* s_s = q_s + R;
    int32_t* c_s = reinterpret_cast<int32_t*>(s_s + R);      // [3][R] packed (rank << 16) | local
    double* rbuf = reinterpret_cast<double*>(smem + cluster1_red_offset(R));
    __shared__ double red[4][16];   // red[k][c]: partial k of CTA c
    __shared__ double tot[4];
    __shared__ double sc[2];        // alpha, beta, derived once per CTA by thread 0
    __shared__ int s_stop;

    const int tid = threadIdx.x;
    for (int i = tid; i < nloc; i += blockDim.x) {
        const int64_t e = r0 + i;
        for (int j = 0; j < 3; ++j) {
            a_s[j * R + i] = A.a[j * n + e];
            const int32_t c = A.col[j * n + e];
            const int cr = c / R;
            c_s[j * R + i] = (cr << 16) | (c - cr * R);
        }
        const double se = A.s[e];
        s_s[i] = se;
        y_s[i] = se * A.x[e];
        p_s[i] = 0.0;
        q_s[i] = 0.0;
    }
    cluster.sync();
    auto gather = [&](double* base, int32_t packed) -> double {
        const int cr = packed >> 16, li = packed & 0xFFFF;
        if (cr == rank) return base[li];
        return cluster.map_shared_rank(base, cr)[li];
    };
    auto push = [&](int k, double v) {
        if (tid < C) cluster.map_shared_rank(&red[k][0], tid)[rank] = v;
    };
    auto cluster_sum = [&](int k) -> double {
        double t = 0.0;
        for (int c = 0; c < C; ++c) t += red[k][c];
        return t;
    };

    // r = S^-1 b - Ahat y; ||b||^2, ||S r||^2
    {
        double v1[1] = {0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            double ay = y_s[i];
            for (int j = 0; j < 3; ++j) ay = fma(a_s[j * R + i], gather(y_s, c_s[j * R + i]), ay);
            const double be = A.b[r0 + i];
            r_s[i] = be / s_s[i] - ay;
            v1[0] = fma(be, be, v1[0]);
        }
        block_sum_buf<1>(v1, rbuf, tot);
        push(3, v1[0]);
    }
    cluster.sync();         // r complete everywhere
    // w = Ahat r, gamma = r.r, delta = w.r, ||S r||^2
    auto spmv_dots = [&](bool norm) {
        double v3[3] = {0.0, 0.0, 0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            const double re = r_s[i];
            double v = re;
            for (int j = 0; j < 3; ++j) v = fma(a_s[j * R + i], gather(r_s, c_s[j * R + i]), v);
            w_s[i] = v;
            v3[0] = fma(re, re, v3[0]);
            v3[1] = fma(v, re, v3[1]);
            if (norm) {
                const double t = s_s[i] * re;
                v3[2] = fma(t, t, v3[2]);
            }
        }
        block_sum_buf<3>(v3, rbuf, tot);
        push(0, v3[0]);
        push(1, v3[1]);
        push(2, v3[2]);
    };
    spmv_dots(true);
    cluster.sync();
    double gamma = 0.0, alpha = 0.0, bnorm2 = 0.0, rnorm2 = 0.0, thresh2 = 0.0;
    int status = CPS_OK;
    if (tid == 0) {
        gamma = cluster_sum(0);
        const double delta = cluster_sum(1);
        rnorm2 = cluster_sum(2);
        bnorm2 = cluster_sum(3);
        thresh2 = A.rtol * A.rtol * bnorm2;
        int stop = (bnorm2 == 0.0 || rnorm2 <= thresh2 || A.max_iter <= 0) ? 1 : 0;
        if (!stop && (!(delta > 0.0) || !isfinite(delta))) stop = 2;
        alpha = stop ? 0.0 : gamma / delta;
        sc[0] = alpha;
        sc[1] = 0.0;
        s_stop = stop;
    }
    __syncthreads();
    long long it = 0;
    int stop = s_stop;
    if (stop == 2) status = CPS_ERR_NOT_SPD;
    while (!stop) {
        const double al = sc[0], be = sc[1];
        for (int i = tid; i < nloc; i += blockDim.x) {
            const double pe = fma(be, p_s[i], r_s[i]);
            const double qe = fma(be, q_s[i], w_s[i]);
            p_s[i] = pe;
            q_s[i] = qe;
            y_s[i] = fma(al, pe, y_s[i]);
            r_s[i] = fma(-al, qe, r_s[i]);
        }
        cluster.sync();     // new r everywhere; last step's partials read
        ++it;
        const bool check = (it % kCheck) == 0;
        spmv_dots(check);
        cluster.sync();
        if (tid == 0) {
            const double g = cluster_sum(0);
            const double delta = cluster_sum(1);
            int halt = (!(g > 0.0) || it >= A.max_iter) ? 1 : 0;
            if (check) {
                rnorm2 = cluster_sum(2);
                if (rnorm2 <= thresh2) halt = 1;
            }
            const double beta = g / gamma;
            const double den = delta - beta * g / alpha;
            if (!halt && (!(den > 0.0) || !isfinite(den))) halt = 2;
            alpha = halt ? alpha : g / den;
            gamma = g;
            sc[0] = alpha;
            sc[1] = beta;
            s_stop = halt;
        }
        __syncthreads();
        stop = s_stop;
        if (stop == 2) status = CPS_ERR_NOT_SPD;
    }
    for (int i = tid; i < nloc; i += blockDim.x) A.y_out[r0 + i] = y_s[i];
    if (rank == 0 && tid == 0) {
        CgState* st = A.st;
        st->rho = gamma;
        st->bnorm2 = bnorm2;
        st->thresh2 = thresh2;
        st->rnorm2 = rnorm2;
        st->iter = it;
        st->max_iter = A.max_iter;
        st->status = status;
        st->done = 2;
        st->alpha = 0.0;
        st->beta = 0.0;
    }
    cluster.sync();         // no CTA leaves while others may still read its memory
}

// Pipelined variant (Ghysels-Vanroose recurrences; one split cluster barrier
// per iteration): besides s = Ahat p and w = Ahat r the CTA keeps
// z = Ahat s, so that the SpMV of an iteration, q = Ahat w, needs only the
// current w and can run while the iteration's reduction is in flight:
//   gamma = r.r, delta = w.r: block sum, partials pushed | cluster arrive
//   q = Ahat w over this CTA's own columns | cluster wait | q += remote columns
//   beta = gamma/gamma_old, alpha = gamma/(delta - beta gamma/alpha_old)
//   z = q + beta z; s = w + beta s; p = r + beta p; y += alpha p;
//   r -= alpha s; w -= alpha z
// w and the partials are double-buffered by iteration parity, so that the one
// barrier also orders each CTA's writes after every other CTA's reads of the
// iteration before.  Same iterates as the textbook recurrence in exact
// arithmetic; 11 FP64 FMAs a row against 9, and the recurrences drift sooner
// near the FP64 floor (the host's true residual then decides on a restart).
constexpr size_t kRowBytes2 = 3 * sizeof(double) + 3 * sizeof(int32_t) + 9 * sizeof(double);
__host__ __device__ inline size_t cluster2_red_offset(int R) {
    return ((size_t)R * kRowBytes2 + 15) / 16 * 16;
}
__host__ __device__ inline size_t cluster2_smem_bytes(int R) {
    return cluster2_red_offset(R) + kRedBufBytes;
}

__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kClusterThreads, 1) k_cluster_cgp(ClusterArgs A) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int R = A.rows;
    const int64_t n = A.n;
    const int64_t r0 = (int64_t)rank * R;
    const int nloc = (int)((r0 + R <= n) ? R : (n > r0 ? n - r0 : 0));

    extern __shared__ __align__(16) unsigned char smem[];
    double* a_s = reinterpret_cast<double*>(smem);          // [3][R]
    double* p_s = a_s + 3 * R;
    double* r_s = p_s + R;
    double* y_s = r_s + R;
    double* sv_s = y_s + R;         // s = Ahat p
    double* z_s = sv_s + R;         // z = Ahat s
    double* q_s = z_s + R;          // q = Ahat w
    double* w_s[2] = {q_s + R, q_s + 2 * R};
    double* s_s = q_s + 3 * R;      // the scaling S
    int32_t* c_s = reinterpret_cast<int32_t*>(s_s + R);      // [3][R] packed (rank << 16) | local
    double* rbuf = reinterpret_cast<double*>(smem + cluster2_red_offset(R));
    __shared__ double red[2][4][16];   // red[parity][k][c]: partial k of CTA c
    __shared__ double tot[4];
    __shared__ double sc[2];           // alpha, beta, derived once per CTA by thread 0
    __shared__ int s_stop;

    const int tid = threadIdx.x;
    for (int i = tid; i < nloc; i += blockDim.x) {
        const int64_t e = r0 + i;
        for (int j = 0; j < 3; ++j) {
            a_s[j * R + i] = A.a[j * n + e];
            const int32_t c = A.col[j * n + e];
            const int cr = c / R;
            c_s[j * R + i] = (cr << 16) | (c - cr * R);
        }
        const double se = A.s[e];
        s_s[i] = se;
        y_s[i] = se * A.x[e];
        p_s[i] = 0.0;
        sv_s[i] = 0.0;
        z_s[i] = 0.0;
    }
    cluster.sync();
    auto gather = [&](double* base, int32_t packed) -> double {
        const int cr = packed >> 16, li = packed & 0xFFFF;
        if (cr == rank) return base[li];
        return cluster.map_shared_rank(base, cr)[li];
    };
    auto push = [&](int par, int k, double v) {
        if (tid < C) cluster.map_shared_rank(&red[par][k][0], tid)[rank] = v;
    };
    auto cluster_sum = [&](int par, int k) -> double {
        double t = 0.0;
        for (int c = 0; c < C; ++c) t += red[par][k][c];
        return t;
    };

    // r = S^-1 b - Ahat y; ||b||^2
    {
        double v1[1] = {0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            double ay = y_s[i];
            for (int j = 0; j < 3; ++j) ay = fma(a_s[j * R + i], gather(y_s, c_s[j * R + i]), ay);
            const double be = A.b[r0 + i];
            r_s[i] = be / s_s[i] - ay;
            v1[0] = fma(be, be, v1[0]);
        }
        block_sum_buf<1>(v1, rbuf, tot);
        push(0, 3, v1[0]);
    }
    cluster.sync();         // r complete everywhere
    // w = Ahat r; gamma = r.r, delta = w.r, ||S r||^2
    {
        double v3[3] = {0.0, 0.0, 0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            const double re = r_s[i];
            double v = re;
            for (int j = 0; j < 3; ++j) v = fma(a_s[j * R + i], gather(r_s, c_s[j * R + i]), v);
            w_s[0][i] = v;
            v3[0] = fma(re, re, v3[0]);
            v3[1] = fma(v, re, v3[1]);
            const double t = s_s[i] * re;
            v3[2] = fma(t, t, v3[2]);
        }
        block_sum_buf<3>(v3, rbuf, tot);
        push(0, 0, v3[0]);
        push(0, 1, v3[1]);
        push(0, 2, v3[2]);
    }
    cluster.sync();         // w complete everywhere; the partials are in place
    double gamma = 0.0, alpha = 0.0, bnorm2 = 0.0, rnorm2 = 0.0, thresh2 = 0.0;
    int status = CPS_OK;
    if (tid == 0) {
        gamma = cluster_sum(0, 0);
        const double delta = cluster_sum(0, 1);
        rnorm2 = cluster_sum(0, 2);
        bnorm2 = cluster_sum(0, 3);
        thresh2 = A.rtol * A.rtol * bnorm2;
        int stop = (bnorm2 == 0.0 || rnorm2 <= thresh2 || A.max_iter <= 0) ? 1 : 0;
        if (!stop && (!(delta > 0.0) || !isfinite(delta))) stop = 2;
        alpha = stop ? 0.0 : gamma / delta;
        sc[0] = alpha;
        sc[1] = 0.0;
        s_stop = stop;
    }
    // q = Ahat w
    for (int i = tid; i < nloc; i += blockDim.x) {
        double v = w_s[0][i];
        for (int j = 0; j < 3; ++j) v = fma(a_s[j * R + i], gather(w_s[0], c_s[j * R + i]), v);
        q_s[i] = v;
    }
    __syncthreads();
    long long it = 0;
    int par = 0;            // w_s[par] holds the current w
    int stop = s_stop;
    if (stop == 2) status = CPS_ERR_NOT_SPD;
    while (!stop) {
        const double al = sc[0], be = sc[1];
        {
            const double* __restrict__ wc = w_s[par];
            double* __restrict__ wn = w_s[par ^ 1];
            for (int i = tid; i < nloc; i += blockDim.x) {
                const double ze = fma(be, z_s[i], q_s[i]);
                const double se = fma(be, sv_s[i], wc[i]);
                const double pe = fma(be, p_s[i], r_s[i]);
                z_s[i] = ze;
                sv_s[i] = se;
                p_s[i] = pe;
                y_s[i] = fma(al, pe, y_s[i]);
                r_s[i] = fma(-al, se, r_s[i]);
                wn[i] = fma(-al, ze, wc[i]);
            }
        }
        ++it;
        par ^= 1;
        const int rp = (int)(it & 1);
        const bool check = (it % kCheck) == 0;
        {
            double v3[3] = {0.0, 0.0, 0.0};
            const double* __restrict__ wc = w_s[par];
            for (int i = tid; i < nloc; i += blockDim.x) {
                const double re = r_s[i];
                v3[0] = fma(re, re, v3[0]);
                v3[1] = fma(wc[i], re, v3[1]);
                if (check) {
                    const double t = s_s[i] * re;
                    v3[2] = fma(t, t, v3[2]);
                }
            }
            block_sum_buf<3>(v3, rbuf, tot);   // also orders this CTA's w writes
            push(rp, 0, v3[0]);
            push(rp, 1, v3[1]);
            push(rp, 2, v3[2]);
        }
        cluster_arrive_release();
        // q = Ahat w: this CTA's own columns while the reduction completes
        for (int i = tid; i < nloc; i += blockDim.x) {
            double v = w_s[par][i];
            for (int j = 0; j < 3; ++j) {
                const int32_t pk = c_s[j * R + i];
                if ((pk >> 16) == rank) v = fma(a_s[j * R + i], w_s[par][pk & 0xFFFF], v);
            }
            q_s[i] = v;
        }
        cluster_wait_acquire();
        for (int i = tid; i < nloc; i += blockDim.x) {
            double v = q_s[i];
            bool any = false;
            for (int j = 0; j < 3; ++j) {
                const int32_t pk = c_s[j * R + i];
                const int cr = pk >> 16;
                if (cr != rank) {
                    v = fma(a_s[j * R + i], cluster.map_shared_rank(w_s[par], cr)[pk & 0xFFFF], v);
                    any = true;
                }
            }
            if (any) q_s[i] = v;
        }
        if (tid == 0) {
            const double g = cluster_sum(rp, 0);
            const double delta = cluster_sum(rp, 1);
            int halt = (!(g > 0.0) || it >= A.max_iter) ? 1 : 0;
            if (check) {
                rnorm2 = cluster_sum(rp, 2);
                if (rnorm2 <= thresh2) halt = 1;
            }
            const double beta = g / gamma;
            const double den = delta - beta * g / alpha;
            // a difference that lost its digits at the FP64 floor: stop and
            // let the true residual decide (restart or not converged)
            if (!halt && (!(den > 0.0) || !isfinite(den))) halt = 1;
            alpha = halt ? alpha : g / den;
            gamma = g;
            sc[0] = alpha;
            sc[1] = beta;
            s_stop = halt;
        }
        __syncthreads();
        stop = s_stop;
    }
    for (int i = tid; i < nloc; i += blockDim.x) A.y_out[r0 + i] = y_s[i];
    if (rank == 0 && tid == 0) {
        CgState* st = A.st;
        st->rho = gamma;
        st->bnorm2 = bnorm2;
        st->thresh2 = thresh2;
        st->rnorm2 = rnorm2;
        st->iter = it;
        st->max_iter = A.max_iter;
        st->status = status;
        st->done = 2;
        st->alpha = 0.0;
        st->beta = 0.0;
    }
    cluster.sync();         // no CTA leaves while others may still read its memory
}


// s-step variant (s inner iterations per outer step; the s-step CG of
// Chronopoulos and Gear, in the communication-avoiding form that carries the
// coefficients of the iterates in a Krylov basis).  Per outer step:
//   basis  V = [P_0 .. P_s, R_0 .. R_{s-1}], P_k = T_k(N) p, R_k = T_k(N) r,
//          with N = Ahat - I (the scaled off-diagonals) and T_k the Chebyshev
//          polynomials (T_0 = 1, T_1 = z, T_{k+1} = 2 z T_k - T_{k-1}): the
//          spectrum of N lies in [-1, 1] (Ahat is SPD with unit diagonal and
//          2I - Ahat is diagonally dominant), so every basis vector stays of
//          the size of p and r; s sweeps, one cluster barrier before each;
//   Gram   G = V^T V (and ||S r||^2 for the stop test) from the last sweep,
//          one exact block sum and one cluster barrier;
//   inner  s CG steps on the coefficient vectors (length m = 2s + 1) with
//          Ahat V = V B on the columns that have an image in the basis:
//          B e_{P_0} = e_{P_0} + e_{P_1}, B e_{P_k} = (e_{P_{k-1}} + e_{P_{k+1}})/2
//          + e_{P_k}, and the same in the R block; warp 0 of every CTA, one
//          lane per coefficient, identical in every CTA;
//   update p = V p', r = V r', y += V y' (row-local).
// s + 1 cluster barriers per s iterations (the single-reduction solve: 2s).
// The iterates are those of CG in exact arithmetic; the stop test runs once
// per outer step, on ||S r|| of the residual at its start.
constexpr int kSStepThreads = 512;   // <= 128 registers a thread for the Gram sums

template <int SS>
struct SStep {
    static constexpr int M = 2 * SS + 1;        // basis vectors
    static constexpr int NG = M * (M + 1) / 2;  // Gram entries, upper triangle
    static constexpr int QSR = NG;              // ||S R_0||^2
    static constexpr int QB = NG + 1;           // ||b||^2 (set-up)
    static constexpr int NQ = NG + 2;
    static_assert(NQ <= 32, "one lane per reduced quantity in the scalar stage");
};

// Index of Gram entry (i, j), i <= j, in the upper triangle stored row by row.
__host__ __device__ constexpr int gram_index(int i, int j, int M) {
    return i * M - i * (i - 1) / 2 + (j - i);
}

template <int M>
__host__ __device__ constexpr size_t sstep_row_bytes() {
    return (size_t)(3 + 2 + M) * sizeof(double) + 3 * sizeof(int32_t);
}

// Exact, order-independent sum over the CTA's warps of v[0..NV) (integer
// sums of the values aligned to each quantity's largest exponent in the CTA,
// exact_sum.cuh); totals into tot[0..NV) in shared memory.  FP64 adds would
// cost 16 SM clocks a warp instruction on GB300's FP64 pipe.
template <int NV>
__device__ __forceinline__ void cta_sum_exact(const double (&v)[NV], double* tot) {
    __shared__ int s_e[NV][32];
    __shared__ long long s_w[NV][32];
    __shared__ int s_eb[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int em = __reduce_max_sync(0xffffffffu, align_exp(v[k]));
        if (lane == 0) s_e[k][warp] = em;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int E = __reduce_max_sync(0xffffffffu, lane < W ? s_e[k][lane] : 1);
        const long long w = warp_sum_fixed<52>(align_fixed(v[k], E, 1));
        if (lane == 0) {
            s_w[k][warp] = w;
            if (warp == 0) s_eb[k] = E;
        }
    }
    __syncthreads();
    for (int k = warp; k < NV; k += W) {
        const long long T = warp_sum_fixed<57>(lane < W ? s_w[k][lane] : 0LL);
        if (lane == 0) tot[k] = fixed_to_double(T, s_eb[k], 1);
    }
    __syncthreads();
}

// Sum of v over lanes 0..7, returned to every lane of the warp.
__device__ __forceinline__ double sum8(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

template <int SS>
__global__ void __launch_bounds__(kSStepThreads, 1) k_cluster_cgs(ClusterArgs A) {
    using Q = SStep<SS>;
    constexpr int M = Q::M;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int R = A.rows;
    const int64_t n = A.n;
    const int64_t r0 = (int64_t)rank * R;
    const int nloc = (int)((r0 + R <= n) ? R : (n > r0 ? n - r0 : 0));

    // a [3][R], S, y, then the basis V [M][R] (P_0..P_s, R_0..R_{s-1}),
    // then col [3][R] int32 packed (rank << 16) | local
    extern __shared__ __align__(16) unsigned char smem[];
    double* a_s = reinterpret_cast<double*>(smem);
    double* s_s = a_s + 3 * R;
    double* y_s = s_s + R;
    double* V = y_s + R;
    int32_t* c_s = reinterpret_cast<int32_t*>(V + M * R);
    double* P0 = V;
    double* R0 = V + (SS + 1) * R;
    __shared__ double red[Q::NQ][16];   // red[k][c]: quantity k of CTA c
    __shared__ double tot[Q::NQ];
    __shared__ double coef[3][M];       // new p, new r, y increment (basis coordinates)
    __shared__ int s_stop, s_nin;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nloc; i += blockDim.x) {
        const int64_t e = r0 + i;
        for (int j = 0; j < 3; ++j) {
            a_s[j * R + i] = A.a[j * n + e];
            const int32_t c = A.col[j * n + e];
            const int cr = c / R;
            c_s[j * R + i] = (cr << 16) | (c - cr * R);
        }
        const double se = A.s[e];
        s_s[i] = se;
        y_s[i] = se * A.x[e];
    }
    cluster.sync();
    auto gather = [&](const double* base, int32_t packed) -> double {
        const int cr = packed >> 16, li = packed & 0xFFFF;
        if (cr == rank) return base[li];
        return cluster.map_shared_rank(const_cast<double*>(base), cr)[li];
    };
    // this CTA's totals tot[0..nq) go to slots [q0 + k][rank] of every CTA
    auto push = [&](int q0, int nq) {
        for (int t = tid; t < nq * C; t += blockDim.x) {
            const int k = t / C, c = t - k * C;
            cluster.map_shared_rank(&red[q0 + k][0], c)[rank] = tot[k];
        }
    };

    // r = S^-1 b - Ahat y, p = r; ||b||^2
    {
        double v1[1] = {0.0};
        for (int i = tid; i < nloc; i += blockDim.x) {
            double ay = y_s[i];
            for (int j = 0; j < 3; ++j) ay = fma(a_s[j * R + i], gather(y_s, c_s[j * R + i]), ay);
            const double be = A.b[r0 + i];
            const double re = be / s_s[i] - ay;
            P0[i] = re;
            R0[i] = re;
            v1[0] = fma(be, be, v1[0]);
        }
        cta_sum_exact<1>(v1, tot);
        push(Q::QB, 1);
    }

    // B of the coefficient space, row of this lane: (B x)_i = bcm x_{i-1} +
    // bc0 x_i + bcp x_{i+1}, within the lane's block (P or R); column k of a
    // block has an image in the basis for k <= K (P: s - 1, R: s - 2)
    double bcm = 0.0, bc0 = 0.0, bcp = 0.0;
    if (lane < M) {
        const bool inP = lane <= SS;
        const int k = inP ? lane : lane - (SS + 1);
        const int K = inP ? SS - 1 : SS - 2;
        if (k >= 1 && k - 1 <= K) bcm = (k == 1) ? 1.0 : 0.5;
        if (k <= K) bc0 = 1.0;
        if (k + 1 <= K) bcp = 0.5;
    }
    // run scalars, held by warp 0 of every CTA (identical everywhere)
    double gam = 0.0, bnorm2 = 0.0, rnorm2 = 0.0, thresh2 = 0.0;
    long long it = 0;
    int status = CPS_OK;
    bool first = true;
    for (;;) {
        cluster.sync();     // P_0, R_0 complete everywhere; the last step's slots read
#pragma unroll
        for (int k = 1; k <= SS; ++k) {
            if (k > 1) cluster.sync();      // P_{k-1}, R_{k-1} complete everywhere
            const double* Pp = V + (k - 1) * R;
            const double* Rp = R0 + (k - 1) * R;
            double* Pk = V + k * R;
            double* Rk = R0 + k * R;
            double g[Q::NG + 1];
            if (k == SS) {
#pragma unroll
                for (int q = 0; q <= Q::NG; ++q) g[q] = 0.0;
            }
            for (int i = tid; i < nloc; i += blockDim.x) {
                double np = 0.0, nr = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double aj = a_s[j * R + i];
                    const int32_t pk = c_s[j * R + i];
                    np = fma(aj, gather(Pp, pk), np);
                    if (k <= SS - 1) nr = fma(aj, gather(Rp, pk), nr);
                }
                const double pv = (k == 1) ? np : fma(2.0, np, -V[(k - 2) * R + i]);
                Pk[i] = pv;
                if (k <= SS - 1) Rk[i] = (k == 1) ? nr : fma(2.0, nr, -R0[(k - 2) * R + i]);
                if (k == SS) {
                    double vv[M];
#pragma unroll
                    for (int c = 0; c < M; ++c) vv[c] = (c == SS) ? pv : V[c * R + i];
#pragma unroll
                    for (int a = 0; a < M; ++a)
#pragma unroll
                        for (int b2 = a; b2 < M; ++b2)
                            g[gram_index(a, b2, M)] = fma(vv[a], vv[b2], g[gram_index(a, b2, M)]);
                    const double t = s_s[i] * vv[SS + 1];
                    g[Q::NG] = fma(t, t, g[Q::NG]);
                }
            }
            if (k == SS) {
                cta_sum_exact<Q::NG + 1>(g, tot);
                push(0, Q::NG + 1);
            }
        }
        cluster.sync();     // every CTA's Gram partials in place
        if (warp == 0) {
            double tq = 0.0;
            if (lane < Q::NQ)
                for (int c = 0; c < C; ++c) tq += red[lane][c];   // rank order everywhere
            if (lane < Q::NQ) tot[lane] = tq;
            __syncwarp();
            if (first) {
                bnorm2 = tot[Q::QB];
                thresh2 = A.rtol * A.rtol * bnorm2;
            }
            rnorm2 = tot[Q::QSR];
            int halt = (bnorm2 == 0.0 || rnorm2 <= thresh2 || it >= A.max_iter) ? 1 : 0;
            double gr[M];
#pragma unroll
            for (int j = 0; j < M; ++j)
                gr[j] = lane < M ? tot[gram_index(min(lane, j), max(lane, j), M)] : 0.0;
            double pc = lane == 0 ? 1.0 : 0.0;          // p' = e_{P_0}
            double rc = lane == SS + 1 ? 1.0 : 0.0;     // r' = e_{R_0}
            double yc = 0.0;
            double grc = lane < M ? gr[SS + 1] : 0.0;   // G r'
            gam = tot[gram_index(SS + 1, SS + 1, M)];   // r.r
            if (!halt && !(gam > 0.0 && isfinite(gam))) halt = 1;
            int nin = 0;
            const long long room = A.max_iter - it;
            for (int j = 0; j < SS && !halt && j < room; ++j) {
                const double pm = __shfl_up_sync(0xffffffffu, pc, 1);
                const double pp = __shfl_down_sync(0xffffffffu, pc, 1);
                const double qc = fma(bcp, pp, fma(bcm, pm, bc0 * pc));   // B p'
                double u = 0.0;                                             // G B p'
#pragma unroll
                for (int c = 0; c < M; ++c) u = fma(gr[c], __shfl_sync(0xffffffffu, qc, c), u);
                const double d = sum8(pc * u);                              // p.Ahat p
                if (!(d > 0.0) || !isfinite(d)) {
                    // on the first step of the run the matrix is not SPD;
                    // later, a difference that lost its digits at the FP64
                    // floor: stop and let the true residual decide
                    halt = (it == 0 && j == 0) ? 2 : 1;
                    break;
                }
                const double al = gam / d;
                yc = fma(al, pc, yc);
                rc = fma(-al, qc, rc);
                grc = fma(-al, u, grc);
                ++nin;
                const double gn = sum8(rc * grc);                           // r.r
                if (!(gn > 0.0) || !isfinite(gn)) {
                    halt = 1;
                    break;
                }
                const double be = gn / gam;
                gam = gn;
                pc = fma(be, pc, rc);
            }
            it += nin;
            if (!halt && it >= A.max_iter) halt = 1;
            if (lane < M) {
                coef[0][lane] = pc;
                coef[1][lane] = rc;
                coef[2][lane] = yc;
            }
            if (lane == 0) {
                s_stop = halt;
                s_nin = nin;
            }
        }
        __syncthreads();
        first = false;
        if (s_stop == 2) status = CPS_ERR_NOT_SPD;
        if (s_nin > 0)
            for (int i = tid; i < nloc; i += blockDim.x) {
                double pn = 0.0, rn = 0.0, dy = 0.0;
#pragma unroll
                for (int c = 0; c < M; ++c) {
                    const double vc = V[c * R + i];
                    pn = fma(coef[0][c], vc, pn);
                    rn = fma(coef[1][c], vc, rn);
                    dy = fma(coef[2][c], vc, dy);
                }
                P0[i] = pn;
                R0[i] = rn;
                y_s[i] += dy;
            }
        if (s_stop) break;
    }
    for (int i = tid; i < nloc; i += blockDim.x) A.y_out[r0 + i] = y_s[i];
    if (rank == 0 && tid == 0) {
        CgState* st = A.st;
        st->rho = gam;
        st->bnorm2 = bnorm2;
        st->thresh2 = thresh2;
        st->rnorm2 = rnorm2;
        st->iter = it;
        st->max_iter = A.max_iter;
        st->status = status;
        st->done = 2;
        st->alpha = 0.0;
        st->beta = 0.0;
    }
    cluster.sync();         // no CTA leaves while others may still read its memory
}

}  // namespace

// The cluster kernel of a variant: 0 textbook, 1 single reduction, 2 pipelined,
// 3 s-step with s = 2, 4 s-step with s = 3.
static void (*cluster_kernel(int variant))(ClusterArgs) {
    switch (variant) {
        case 1: return k_cluster_cg1;
        case 2: return k_cluster_cgp;
        case 3: return k_cluster_cgs<2>;
        case 4: return k_cluster_cgs<3>;
        default: return k_cluster_cg;
    }
}

static size_t cluster_row_bytes(int variant) {
    switch (variant) {
        case 1: return kRowBytes1;
        case 2: return kRowBytes2;
        case 3: return sstep_row_bytes<SStep<2>::M>();
        case 4: return sstep_row_bytes<SStep<3>::M>();
        default: return kRowBytes;
    }
}

static size_t cluster_smem_for(int variant, int R) {
    switch (variant) {
        case 1: return cluster1_smem_bytes(R);
        case 2: return cluster2_smem_bytes(R);
        case 3:
        case 4: return ((size_t)R * cluster_row_bytes(variant) + 15) / 16 * 16;
        default: return cluster_smem_bytes(R);
    }
}

// Dynamic shared memory a CTA of the cluster kernel may use on this device:
// the opt-in limit minus the kernel's static shared memory.
static size_t cluster_dyn_smem_limit(int dev, int variant) {
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, cluster_kernel(variant)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (size_t)smem_optin > fa.sharedSizeBytes ? (size_t)smem_optin - fa.sharedSizeBytes : 0;
}

// Largest system the cluster path (variant 0 textbook, 1 single reduction,
// 2 pipelined, 3 and 4 s-step with s = 2 and 3) takes on this GPU (0: not
// available).
int64_t cluster_max_rows(cps_ctx ctx, int variant) {
    const size_t lim = cluster_dyn_smem_limit(ctx->device, variant);
    const size_t fixed = kRedBufBytes + 16;
    if (lim <= fixed) return 0;
    const int64_t R = (int64_t)((lim - fixed) / cluster_row_bytes(variant));
    return std::min<int64_t>(R, 0xFFFF) * 16;
}

// Runs a whole FP64 Jacobi solve (from x) in one cluster launch; leaves the
// scaled iterate in y and the final scalars in s->st (done = 2).
int cluster_solve(cps_sys s, const double* b, const double* x, double* y, double rtol,
                  long long max_iter, cudaStream_t stream, int variant) {
    static std::atomic<bool> configured[5][64];   // zero-initialised (static storage)
    variant = (variant >= 1 && variant <= 4) ? variant : 0;
    void (*kern)(ClusterArgs) = cluster_kernel(variant);
    const int64_t n = s->nt;
    int csize = 16;
    cudaError_t e = cudaSuccess;
    const int dev = s->ctx->device;
    const size_t lim = cluster_dyn_smem_limit(dev, variant);
    if (!configured[variant][dev & 63].load()) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cps::set_error(s->ctx, std::string("cluster path: ") + cudaGetErrorString(e));
            return CPS_ERR_ARG;
        }
        configured[variant][dev & 63].store(true);
    }
    ClusterArgs A;
    A.a = s->a;
    A.col = s->col;
    A.s = s->s;
    A.b = b;
    A.x = x;
    A.y_out = y;
    A.st = s->st;
    A.n = n;
    A.rtol = rtol;
    A.max_iter = max_iter;
    for (; csize >= 2; csize /= 2) {
        const int R = (int)((n + csize - 1) / csize);
        const size_t smem = cluster_smem_for(variant, R);
        if (R > 0xFFFF || smem > lim) continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(csize, 1, 1);
        // one row per thread where the rows allow (fewer threads: cheaper
        // block reductions); at least 4 warps for the 3-quantity sums
        const int tmax = variant >= 3 ? kSStepThreads : kClusterThreads;
        const int threads = R >= tmax ? tmax : (R < 128 ? 128 : (R + 31) / 32 * 32);
        cfg.blockDim = dim3(threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess ||
            nclusters < 1) {
            cudaGetLastError();
            continue;
        }
        A.rows = R;
        e = cudaLaunchKernelEx(&cfg, kern, A);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cps::set_error(s->ctx, std::string("cluster launch: ") + cudaGetErrorString(e));
            return CPS_ERR_CUDA;
        }
        s->cluster_size = csize;
        return CPS_OK;
    }
    cps::set_error(s->ctx, "cluster path: no cluster shape fits this system");
    return CPS_ERR_ARG;
}

}  // namespace cps
