// Kernels of the conjugate-gradient solve.
//
// All vectors of a run live in the symmetrically scaled space (yhat = S x,
// rhat = S^-1 r, S = diag(sqrt(a_ee))); matrix rows are padded ELL with three
// off-diagonal slots, slot-major (entry j*n + e), and a unit diagonal.  Every
// reduction is deterministic (fixed grid, fixed summation order).
//
// FP64 iteration (GB300 issues FP64 at 1/64 of the FP32 rate, so nothing is
// recomputed): three streaming kernels,
//   k_spmv_dot: q = Ahat p, gamma = p.q;           last block: alpha = rho/gamma
//   k_cg_b:     r -= alpha q; Jacobi: rho' = r.r;  last block: beta, stop test
//   k_cg_c:     y += alpha p; p = z + beta p
// (with IC(0) the preconditioner sweeps run between k_cg_b and k_cg_c).
// FP64 Jacobi, single-reduction alternative (Chronopoulos-Gear): two kernels,
//   k_gear_update: p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s
//   k_gear_spmv:   w = Ahat r, gamma = r.r, delta = w.r; last block: alpha, beta
// (the autotuner picks between the two loops per system).
// Binary32 iteration of the mixed solve: two fused kernels,
//   k_cg_a: y += alpha_{k-1} p_{k-1} (x update one iteration late);
//           p_k = z_k + beta_{k-1} p_{k-1} for the own row and, recomputed
//           bit-identically, the three neighbours' rows; q = Ahat p_k,
//           gamma = p_k . q
//   k_cg_b: as above,
// with the search direction alternating between two buffers by the parity of
// the device iteration counter, so the same captured graph serves any
// starting iteration.
#pragma once

#include "cps_internal.cuh"

namespace cps {

#define CPS_GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Unrolled grid-stride loop: each thread takes U rows per trip, spaced one
// grid apart (every access stays coalesced), so that the loads of U rows are
// in flight together.  body(e, u) is called for the U rows of a trip after
// load(e, u) has been called for all of them; the tail runs one row a trip.
#define CPS_UNROLLED_LOOP(n, U, LOAD, BODY)                                            \
    {                                                                                  \
        const int64_t stride_ = (int64_t)gridDim.x * blockDim.x;                       \
        int64_t e0_ = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;                  \
        for (; e0_ + (U - 1) * stride_ < (n); e0_ += U * stride_) {                    \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = e0_ + u * stride_;                                   \
                LOAD;                                                                  \
            }                                                                          \
            _Pragma("unroll") for (int u = 0; u < U; ++u) {                            \
                const int64_t e = e0_ + u * stride_;                                   \
                BODY;                                                                  \
            }                                                                          \
        }                                                                              \
        for (; e0_ < (n); e0_ += stride_) {                                            \
            const int u = 0;                                                           \
            const int64_t e = e0_;                                                     \
            LOAD;                                                                      \
            BODY;                                                                      \
        }                                                                              \
    }

// Stop protocol of a run: st->done = 0 running; 1 stop after the current
// iteration's last kernel (set by k_cg_b); 2 stopped (set by the next
// k_spmv_dot when it finds 1, by a breakdown, or at the start of a run).

// ---- FP64 iteration: three kernels, 8 FP64 FMAs per row (GB300's FP64 rate
// is ~1/64 of FP32, so recomputing p at the neighbours would make the loop
// FP64-bound); 116 algorithmic bytes per row.
//   k_spmv_dot: q = Ahat p, gamma = p.q; last block: alpha = rho / gamma
//   k_cg_b:     r -= alpha q; Jacobi: rho' = r.r, beta = rho'/rho; stop test
//   k_cg_c:     y += alpha p; p = z + beta p

template <typename V, int U, int BS = kBlock>
__global__ void __launch_bounds__(BS) k_spmv_dot(const V* __restrict__ a,
                                                     const int32_t* __restrict__ col,
                                                     const V* __restrict__ p, V* __restrict__ q,
                                                     int64_t n, double* partials, CgState* st) {
    {
        const int d = st->done;
        if (d) {
            if (d == 1 && blockIdx.x == 0 && threadIdx.x == 0) st->done = 2;
            return;
        }
    }
    double acc = 0.0;
    V pe[U], a0[U], a1[U], a2[U];
    int32_t c0[U], c1[U], c2[U];
    CPS_UNROLLED_LOOP(n, U,
        (pe[u] = p[e], a0[u] = a[e], a1[u] = a[n + e], a2[u] = a[2 * n + e],
         c0[u] = col[e], c1[u] = col[n + e], c2[u] = col[2 * n + e]),
        {
            V v = fma(a0[u], p[c0[u]], pe[u]);
            v = fma(a1[u], p[c1[u]], v);
            v = fma(a2[u], p[c2[u]], v);
            q[e] = v;
            acc = fma((double)pe[u], (double)v, acc);
        })
    double t[1] = {acc};
    if (grid_sum<1, BS>(t, partials, &st->arrive[0]) && threadIdx.x == 0) {
        const double gamma = t[0];
        st->gamma = gamma;
        if (!(gamma > 0.0) || !isfinite(gamma)) {
            st->status = CPS_ERR_NOT_SPD;
            st->done = 2;
        } else {
            st->alpha = st->rho / gamma;
        }
    }
}

template <typename V, int U, int BS = kBlock>
__global__ void __launch_bounds__(BS) k_cg_c(V* __restrict__ y, V* __restrict__ p,
                                                 const V* __restrict__ z, int64_t n,
                                                 const CgState* st) {
    if (st->done == 2) return;
    const V al = (V)st->alpha;
    const V be = (V)st->beta;
    V pe[U], ye[U], ze[U];
    CPS_UNROLLED_LOOP(n, U, (pe[u] = p[e], ye[u] = y[e], ze[u] = z[e]),
        {
            y[e] = fma(al, pe[u], ye[u]);
            p[e] = fma(be, pe[u], ze[u]);
        })
}

// ---- binary32 iteration: two fused kernels (FP32 arithmetic is cheap, so p
// is recomputed at the neighbours instead of stored and re-read).
//   k_cg_a: y += alpha_{k-1} p_{k-1}   (x update one iteration late)
//           p_k = z_k + beta_{k-1} p_{k-1}   (own row and the neighbours')
//           q = Ahat p_k, gamma = p_k . q;  last block: alpha_k
//   k_cg_b: as above.
// p alternates between two buffers chosen by the parity of the iteration
// counter, so one captured graph serves any starting iteration.
template <typename V, int U>
__global__ void __launch_bounds__(kBlock) k_cg_a(const V* __restrict__ a,
                                                 const int32_t* __restrict__ col,
                                                 const V* __restrict__ z, V* __restrict__ p0,
                                                 V* __restrict__ p1, V* __restrict__ y,
                                                 V* __restrict__ q, int64_t n, double* partials,
                                                 CgState* st) {
    if (st->done) return;
    const bool odd = (st->iter & 1) != 0;
    const V* __restrict__ po = odd ? p1 : p0;
    V* __restrict__ pn = odd ? p0 : p1;
    const V al = (V)st->alpha;
    const V be = (V)st->beta;
    double acc = 0.0;
    V pold[U], ze[U], ye[U], a0[U], a1[U], a2[U];
    int32_t c0[U], c1[U], c2[U];
    CPS_UNROLLED_LOOP(n, U,
        (pold[u] = po[e], ze[u] = z[e], ye[u] = y[e], a0[u] = a[e], a1[u] = a[n + e],
         a2[u] = a[2 * n + e], c0[u] = col[e], c1[u] = col[n + e], c2[u] = col[2 * n + e]),
        {
            y[e] = fma(al, pold[u], ye[u]);
            const V pe = fma(be, pold[u], ze[u]);
            V v = fma(a0[u], fma(be, po[c0[u]], z[c0[u]]), pe);
            v = fma(a1[u], fma(be, po[c1[u]], z[c1[u]]), v);
            v = fma(a2[u], fma(be, po[c2[u]], z[c2[u]]), v);
            pn[e] = pe;
            q[e] = v;
            acc = fma((double)pe, (double)v, acc);
        })
    double t[1] = {acc};
    if (grid_sum<1>(t, partials, &st->arrive[0]) && threadIdx.x == 0) {
        const double gamma = t[0];
        st->gamma = gamma;
        if (!(gamma > 0.0) || !isfinite(gamma)) {
            st->status = CPS_ERR_NOT_SPD;
            st->done = 2;
        } else {
            st->alpha = st->rho / gamma;
        }
    }
}

template <typename V, bool NORM, bool JACOBI, int U, int BS = kBlock>
__global__ void __launch_bounds__(BS) k_cg_b(V* __restrict__ r, const V* __restrict__ q,
                                                 const V* __restrict__ s, int64_t n,
                                                 double* partials, CgState* st) {
    if (st->done) return;
    const V al = (V)st->alpha;
    double rr = 0.0, nn = 0.0;
    V re[U], qe[U], se[U];
    CPS_UNROLLED_LOOP(n, U, (re[u] = r[e], qe[u] = q[e], se[u] = NORM ? s[e] : (V)0),
        {
            const V rv = fma(-al, qe[u], re[u]);
            r[e] = rv;
            if (JACOBI) rr = fma((double)rv, (double)rv, rr);
            if (NORM) {
                const double t = (double)se[u] * (double)rv;
                nn = fma(t, t, nn);
            }
        })
    double t[2] = {rr, nn};
    if (grid_sum<2, BS>(t, partials, &st->arrive[1]) && threadIdx.x == 0) {
        const long long it = st->iter + 1;
        st->iter = it;
        int done = 0;
        if (NORM) {
            st->rnorm2 = t[1];
            if (t[1] <= st->thresh2) done = 1;
        }
        if (it >= st->max_iter) done = 1;
        if (JACOBI) {
            const double rho_new = t[0];
            if (!(rho_new > 0.0)) done = 1;      // exact solution reached
            // binary32: a recursive residual 1e-13 below the replaced one is
            // at the format's rounding floor (a system of a few cells gets
            // there in a few iterations); replace it before rounding noise
            // builds up in the update
            if (sizeof(V) == 4 && rho_new <= 1e-13 * st->rho_rep) done = 1;
            st->beta = rho_new / st->rho;
            st->rho = rho_new;
        }
        if (done) st->done = 1;
    }
}

// ---- FP64 single-reduction iteration (Jacobi; Chronopoulos-Gear recurrences):
// two streaming kernels and one grid reduction per iteration,
//   k_gear_update: p = r + beta p; s = w + beta s; y += alpha p; r -= alpha s
//   k_gear_spmv:   w = Ahat r; gamma = r.r, delta = w.r (and ||S r||^2);
//                  last block: stop test, beta = gamma/gamma_old,
//                  alpha = gamma/(delta - beta gamma/alpha_old)
// with s = Ahat p carried by recurrence.  The same iterates as the textbook
// loop in exact arithmetic; 125 algorithmic bytes and 9 FP64 FMAs per row
// (117 and 8), for one kernel boundary and one grid reduction fewer.  The stop
// is decided where the iteration ends (after the SpMV of the new residual), so
// k_gear_spmv sets done = 2 directly.  s lives in q, w in p1.

// After k_init64: w = Ahat r, delta = w.r, p = s = 0; alpha = rho/delta, beta = 0.
__global__ void __launch_bounds__(kBlock) k_gear_start(const double* __restrict__ a,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ r,
                                                       double* __restrict__ w,
                                                       double* __restrict__ p,
                                                       double* __restrict__ q, int64_t n,
                                                       double* partials, CgState* st) {
    if (st->done) return;
    double dd = 0.0;
    CPS_GRID_STRIDE(e, n) {
        const double re = r[e];
        double v = re;
#pragma unroll
        for (int j = 0; j < 3; ++j) v = fma(a[j * n + e], r[col[j * n + e]], v);
        w[e] = v;
        p[e] = 0.0;
        q[e] = 0.0;
        dd = fma(v, re, dd);
    }
    double t[1] = {dd};
    if (grid_sum<1>(t, partials, &st->arrive[1]) && threadIdx.x == 0) {
        const double delta = t[0];
        st->gamma = delta;
        st->beta = 0.0;
        if (!(delta > 0.0) || !isfinite(delta)) {
            st->status = CPS_ERR_NOT_SPD;
            st->done = 2;
        } else {
            st->alpha = st->rho / delta;
        }
    }
}

template <int U, int BS = kBlock>
__global__ void __launch_bounds__(BS) k_gear_update(double* __restrict__ y,
                                                    double* __restrict__ r,
                                                    double* __restrict__ p,
                                                    double* __restrict__ s,
                                                    const double* __restrict__ w, int64_t n,
                                                    const CgState* st) {
    if (st->done) return;
    const double al = st->alpha;
    const double be = st->beta;
    double pe[U], se[U], we[U], re[U], ye[U];
    CPS_UNROLLED_LOOP(n, U, (pe[u] = p[e], se[u] = s[e], we[u] = w[e], re[u] = r[e], ye[u] = y[e]),
        {
            const double pn = fma(be, pe[u], re[u]);
            const double sn = fma(be, se[u], we[u]);
            p[e] = pn;
            s[e] = sn;
            y[e] = fma(al, pn, ye[u]);
            r[e] = fma(-al, sn, re[u]);
        })
}

template <bool NORM, int U, int BS = kBlock>
__global__ void __launch_bounds__(BS) k_gear_spmv(const double* __restrict__ a,
                                                  const int32_t* __restrict__ col,
                                                  const double* __restrict__ r,
                                                  double* __restrict__ w,
                                                  const double* __restrict__ sc, int64_t n,
                                                  double* partials, CgState* st) {
    if (st->done) return;
    double gg = 0.0, dd = 0.0, nn = 0.0;
    double re[U], a0[U], a1[U], a2[U], se[U];
    int32_t c0[U], c1[U], c2[U];
    CPS_UNROLLED_LOOP(n, U,
        (re[u] = r[e], a0[u] = a[e], a1[u] = a[n + e], a2[u] = a[2 * n + e],
         c0[u] = col[e], c1[u] = col[n + e], c2[u] = col[2 * n + e], se[u] = NORM ? sc[e] : 0.0),
        {
            double v = fma(a0[u], r[c0[u]], re[u]);
            v = fma(a1[u], r[c1[u]], v);
            v = fma(a2[u], r[c2[u]], v);
            w[e] = v;
            gg = fma(re[u], re[u], gg);
            dd = fma(v, re[u], dd);
            if (NORM) {
                const double t = se[u] * re[u];
                nn = fma(t, t, nn);
            }
        })
    double t[3] = {gg, dd, nn};
    if (grid_sum<3, BS>(t, partials, &st->arrive[0]) && threadIdx.x == 0) {
        const long long it = st->iter + 1;
        st->iter = it;
        int done = 0;
        if (NORM) {
            st->rnorm2 = t[2];
            if (t[2] <= st->thresh2) done = 1;
        }
        if (it >= st->max_iter) done = 1;
        const double g = t[0], d = t[1];
        if (!(g > 0.0)) done = 1;                // exact solution reached
        if (!done) {
            const double be = g / st->rho;
            const double den = d - be * g / st->alpha;
            if (!(den > 0.0) || !isfinite(den)) {
                // on a run's first iteration p.Ap <= 0: not SPD; later, the
                // recurrence's difference lost its digits at the FP64 floor:
                // stop, and let the true residual decide
                if (it <= 1) st->status = CPS_ERR_NOT_SPD;
                done = 1;
            } else {
                st->beta = be;
                st->alpha = g / den;
            }
        }
        st->rho = g;
        st->gamma = d;
        if (done) st->done = 2;
    }
}

// Autotuning: keep the iteration kernels running whatever the data does.
__global__ void k_tune_prime(CgState* st) {
    st->done = 0;
    st->status = CPS_OK;
    st->rho = 1.0;
    st->alpha = 1e-3;
    st->beta = 0.5;
    st->max_iter = 1LL << 62;
    st->thresh2 = -1.0;
}

// p = z (start of an IC(0) run, after the first preconditioner application).
template <typename V>
__global__ void __launch_bounds__(kBlock) k_copy(V* __restrict__ dst, const V* __restrict__ src,
                                                 int64_t n) {
    CPS_GRID_STRIDE(e, n) { dst[e] = src[e]; }
}

// Pending x update of the binary32 iteration after its last k_cg_b:
// y += alpha p_last (the next run start resets alpha).
template <typename V>
__global__ void __launch_bounds__(kBlock) k_flush_y(V* __restrict__ y, const V* __restrict__ p0,
                                                    const V* __restrict__ p1, int64_t n,
                                                    CgState* st) {
    // iteration k wrote p_k to p1 (k even) or p0 (k odd); iter = k + 1 now
    const V* __restrict__ pl = (st->iter & 1) ? p1 : p0;
    if (st->status != CPS_OK) return;
    const V al = (V)st->alpha;
    if (al == (V)0) return;
    CPS_GRID_STRIDE(e, n) { y[e] = fma(al, pl[e], y[e]); }
}

// Start of a FP64 run from x: y = S x, r = S^-1 b - Ahat y, p_{-1} = 0.
// Jacobi: rho = r.r.  IC(0): rho = +inf so that the first preconditioner
// application yields beta = 0.
__global__ void __launch_bounds__(kBlock) k_init64(const double* __restrict__ b,
                                                   const double* __restrict__ x,
                                                   const double* __restrict__ s,
                                                   const double* __restrict__ a,
                                                   const int32_t* __restrict__ col, int64_t n,
                                                   double* __restrict__ y, double* __restrict__ r,
                                                   double* __restrict__ p0, double rtol,
                                                   long long budget, int jacobi, double* partials,
                                                   CgState* st) {
    double rr = 0.0, bb = 0.0, nn = 0.0;
    CPS_GRID_STRIDE(e, n) {
        const double se = s[e];
        const double ye = se * x[e];
        double ay = ye;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            ay = fma(a[j * n + e], s[c] * x[c], ay);
        }
        const double be = b[e];
        const double re = be / se - ay;
        y[e] = ye;
        r[e] = re;
        p0[e] = jacobi ? re : 0.0;
        rr = fma(re, re, rr);
        bb = fma(be, be, bb);
        const double t = se * re;
        nn = fma(t, t, nn);
    }
    double t[3] = {rr, bb, nn};
    if (grid_sum<3>(t, partials, &st->arrive[2]) && threadIdx.x == 0) {
        st->rho = jacobi ? t[0] : INFINITY;
        st->bnorm2 = t[1];
        st->thresh2 = rtol * rtol * t[1];
        st->rnorm2 = t[2];
        st->alpha = 0.0;
        st->beta = 0.0;
        st->gamma = 0.0;
        st->iter = 0;
        st->max_iter = budget;
        st->status = CPS_OK;
        st->done = (t[1] == 0.0 || t[2] <= st->thresh2 || budget <= 0) ? 2 : 0;
    }
}

// End of a FP64 run: x = S^-1 y and the true residual ||b - A x||^2.
__global__ void __launch_bounds__(kBlock) k_final64(const double* __restrict__ b,
                                                    const double* __restrict__ y,
                                                    const double* __restrict__ s,
                                                    const double* __restrict__ a,
                                                    const int32_t* __restrict__ col, int64_t n,
                                                    double* __restrict__ x, double* partials,
                                                    CgState* st) {
    const bool zero = st->bnorm2 == 0.0;
    double nn = 0.0;
    CPS_GRID_STRIDE(e, n) {
        if (zero) {
            x[e] = 0.0;
            continue;
        }
        const double se = s[e];
        const double ye = y[e];
        double ay = ye;
#pragma unroll
        for (int j = 0; j < 3; ++j) ay = fma(a[j * n + e], y[col[j * n + e]], ay);
        const double res = b[e] - se * ay;
        x[e] = ye / se;
        nn = fma(res, res, nn);
    }
    double t[1] = {nn};
    if (grid_sum<1>(t, partials, &st->arrive[3]) && threadIdx.x == 0) st->rnorm2 = t[0];
}

// Mixed precision, residual replacement: r = b - A x in FP64 from the FP64
// iterate x; the binary32 run continues with r32 = S^-1 r and d32 = 0.
// first: start a new run (p_{-1} = 0, beta = 0, iteration 0).  Otherwise the
// search direction is kept and beta is rescaled to the replaced residual
// (beta = rho_true / rho_k).  Stop of the binary32 run:
// ||S r|| <= max(delta ||r_true||, rtol ||b|| / 2).
__global__ void __launch_bounds__(kBlock) k_res64(const double* __restrict__ b,
                                                  const double* __restrict__ x,
                                                  const double* __restrict__ s,
                                                  const double* __restrict__ a,
                                                  const int32_t* __restrict__ col, int64_t n,
                                                  float* __restrict__ r32, float* __restrict__ p32_0,
                                                  float* __restrict__ d32, double rtol,
                                                  double delta, long long budget, int first,
                                                  int jacobi, double* partials, CgState* st) {
    double rr = 0.0, bb = 0.0, nn = 0.0;
    CPS_GRID_STRIDE(e, n) {
        const double se = s[e];
        double ay = se * x[e];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            ay = fma(a[j * n + e], s[c] * x[c], ay);
        }
        const double be = b[e];
        const double re = be / se - ay;
        const float rf = (float)re;
        r32[e] = rf;
        d32[e] = 0.0f;
        if (first) p32_0[e] = 0.0f;
        rr = fma((double)rf, (double)rf, rr);
        bb = fma(be, be, bb);
        const double t = se * re;
        nn = fma(t, t, nn);
    }
    double t[3] = {rr, bb, nn};
    if (grid_sum<3>(t, partials, &st->arrive[2]) && threadIdx.x == 0) {
        const double outer2 = rtol * rtol * t[1];
        const double inner2 = delta * delta * t[2];
        st->bnorm2 = t[1];
        st->rnorm2 = t[2];
        st->thresh2 = inner2 > 0.25 * outer2 ? inner2 : 0.25 * outer2;
        st->alpha = 0.0;
        st->status = CPS_OK;
        if (first) {
            st->iter = 0;
            st->beta = 0.0;
            st->rho = jacobi ? t[0] : INFINITY;
        } else if (jacobi) {
            // beta_k = rho_{k+1}/rho_k with rho_{k+1} taken from the true residual
            const double rho_k = st->beta > 0.0 ? st->rho / st->beta : INFINITY;
            st->beta = t[0] / rho_k;
            st->rho = t[0];
        } else {
            // the preconditioner application that follows computes
            // beta = rho_true / st->rho: hand it rho_k
            st->rho = st->beta > 0.0 ? st->rho / st->beta : INFINITY;
        }
        st->max_iter = st->iter + budget;
        st->rho_rep = t[0];
        st->done = (t[1] == 0.0 || t[2] <= outer2 || budget <= 0 || !(t[0] > 0.0)) ? 2 : 0;
    }
}

// Mixed precision: x += S^-1 d in FP64.
__global__ void __launch_bounds__(kBlock) k_correct(double* __restrict__ x,
                                                    const float* __restrict__ d,
                                                    const double* __restrict__ s, int64_t n) {
    CPS_GRID_STRIDE(e, n) { x[e] += (double)d[e] / s[e]; }
}

// y = A x = S (Ahat (S x)) in FP64.
__global__ void __launch_bounds__(kBlock) k_matvec64(const double* __restrict__ x,
                                                     const double* __restrict__ s,
                                                     const double* __restrict__ a,
                                                     const int32_t* __restrict__ col, int64_t n,
                                                     double* __restrict__ y) {
    CPS_GRID_STRIDE(e, n) {
        const double se = s[e];
        double v = se * x[e];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            v = fma(a[j * n + e], s[c] * x[c], v);
        }
        y[e] = se * v;
    }
}

__global__ void k_unscale_offdiag(const double* __restrict__ a, const int32_t* __restrict__ col,
                                  const double* __restrict__ s, int64_t n, double* __restrict__ v) {
    CPS_GRID_STRIDE(k, 3 * n) {
        const int64_t e = k % n;
        v[k] = a[k] * (s[e] * s[col[k]]);
    }
}

// Gather/scatter between the mesh order and the solver's (colour) order.
__global__ void k_permute_in(const double* __restrict__ b, const double* __restrict__ x,
                             const int32_t* __restrict__ perm, int64_t n,
                             double* __restrict__ bp, double* __restrict__ xp) {
    CPS_GRID_STRIDE(i, n) {
        const int32_t o = perm[i];
        bp[i] = b[o];
        xp[i] = x[o];
    }
}

__global__ void k_permute_out(const double* __restrict__ xp, const int32_t* __restrict__ perm,
                              int64_t n, double* __restrict__ x) {
    CPS_GRID_STRIDE(i, n) { x[perm[i]] = xp[i]; }
}

// dL/dT per side slot for one solve (A lambda = g):
//   interior: -(lambda_e - lambda_ep)(x_e - x_ep); Dirichlet: -lambda_e x_e.
// Optional chain to the cell log-permeability: dtheta_e += dxi_e sum_j dT_j gfac_j.
__global__ void __launch_bounds__(kBlock) k_adjoint_scatter(
    const double* __restrict__ x, const double* __restrict__ lam, const int32_t* __restrict__ col,
    const int32_t* __restrict__ kind, const double* __restrict__ gfac,
    const double* __restrict__ dxi, int64_t n, double* __restrict__ dT,
    double* __restrict__ dtheta) {
    CPS_GRID_STRIDE(e, n) {
        const double xe = x[e], le = lam[e];
        double g = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t k = j * n + e;
            const int sk = kind[k];
            double v = 0.0;
            if (sk == 1) {
                const int32_t c = col[k];
                v = -(le - lam[c]) * (xe - x[c]);
            } else if (sk == 2) {
                v = -le * xe;
            }
            if (dT) dT[k] += v;
            if (dtheta) g = fma(v, gfac[k], g);
        }
        if (dtheta) dtheta[e] += g * dxi[e];
    }
}

// ------------------------------------------------------------------ IC(0)
// Apply z = (L D L^T)^-1 r in colour order, L unit lower triangular with the
// pattern of Ahat (IC(0) factor), per colour c of rows [cs, ce):
//   forward  (c >= 1): w_i = r_i - sum_{lower slots} l_ik w_k   (w of colour 0 is r)
//   backward (c <= C-2): z_i = w_i / d_i - sum_{upper slots} l_ki z_k
// The last colour has no upper slots: forward and backward fuse.  Each kernel
// adds r_i z_i of its final rows into its own partial segment; the colour-0
// kernel (always last) sums every segment and sets rho, beta.

// Partial-sum segment of colour c.
__device__ __forceinline__ double* ic0_segment(double* partials, int c) {
    return partials + (size_t)(kNumPartials + c) * kMaxGrid;
}

template <typename V>
__global__ void __launch_bounds__(kBlock) k_ic0_fwd(const V* __restrict__ l,
                                                    const int32_t* __restrict__ col,
                                                    const V* __restrict__ dinv,
                                                    const V* __restrict__ r, V* __restrict__ z,
                                                    int64_t n, int64_t cs, int64_t ce,
                                                    int64_t first_end, int last, int colour,
                                                    double* partials, const CgState* st) {
    if (st->done) return;
    double acc = 0.0;
    for (int64_t i = cs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ce;
         i += (int64_t)gridDim.x * blockDim.x) {
        V w = r[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t k = col[j * n + i];
            if (k < cs) {
                const V wk = k < first_end ? r[k] : z[k];
                w = fma(-l[j * n + i], wk, w);
            }
        }
        if (last) {
            const V zi = w * dinv[i];
            z[i] = zi;
            acc = fma((double)r[i], (double)zi, acc);
        } else {
            z[i] = w;
        }
    }
    if (last) {
        double t[1] = {acc};
        block_sum<1>(t);
        if (threadIdx.x == 0) ic0_segment(partials, colour)[blockIdx.x] = t[0];
    }
}

template <typename V>
__global__ void __launch_bounds__(kBlock) k_ic0_bwd(const V* __restrict__ l,
                                                    const int32_t* __restrict__ col,
                                                    const V* __restrict__ dinv,
                                                    const V* __restrict__ r, V* __restrict__ z,
                                                    int64_t n, int64_t cs, int64_t ce,
                                                    int ncolours, int colour, double* partials,
                                                    CgState* st) {
    if (st->done) return;
    double acc = 0.0;
    for (int64_t i = cs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ce;
         i += (int64_t)gridDim.x * blockDim.x) {
        const V ri = r[i];
        const V wi = colour == 0 ? ri : z[i];
        V zi = wi * dinv[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t k = col[j * n + i];
            if (k >= ce) zi = fma(-l[j * n + i], z[k], zi);
        }
        z[i] = zi;
        acc = fma((double)ri, (double)zi, acc);
    }
    double t[1] = {acc};
    block_sum<1>(t);
    if (colour != 0) {
        if (threadIdx.x == 0) ic0_segment(partials, colour)[blockIdx.x] = t[0];
        return;
    }
    __shared__ bool lastb;
    if (threadIdx.x == 0) {
        ic0_segment(partials, 0)[blockIdx.x] = t[0];
        __threadfence();
        const unsigned int v = atomicAdd(&st->arrive[2], 1u);
        lastb = (v == gridDim.x - 1u);
    }
    __syncthreads();
    if (!lastb) return;
    __threadfence();
    double tot = 0.0;
    for (int c = 0; c < ncolours; ++c) {
        const double* seg = ic0_segment(partials, c);
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) tot += __ldcg(&seg[i]);
    }
    double u[1] = {tot};
    block_sum<1>(u);
    if (threadIdx.x == 0) {
        st->arrive[2] = 0u;
        const double rho_new = u[0];
        if (!(rho_new > 0.0)) st->done = 1;      // exact solution reached
        st->beta = rho_new / st->rho;
        st->rho = rho_new;
    }
}

// ------------------------------------------------------- reduced system
// Two-coloured cell graph, colour order: red rows [0, nR), black rows
// [nR, n); red rows couple only to black ones and vice versa, and Ahat has a
// unit diagonal.  Eliminating the red unknowns, y_R = bhat_R - E y_B, leaves
// the Schur complement system on the black cells
//   S y_B = bhat_B - E^T bhat_R,   S = I - E^T E,
// whose residual is exactly the black part of the full residual (the red part
// is zero by construction).  S p is applied as t_R = E p_B, q_B = p_B - E^T t_R.

// y_R = S_R^-1 b_R - E y_B with y_B given (from_x = 0) or taken as S_B x_B.
__global__ void __launch_bounds__(kBlock) k_red_recover(const double* __restrict__ b,
                                                        const double* __restrict__ xy,
                                                        const double* __restrict__ s,
                                                        const double* __restrict__ a,
                                                        const int32_t* __restrict__ col,
                                                        int64_t n, int64_t nR, int from_x,
                                                        double* __restrict__ y) {
    CPS_GRID_STRIDE(i, nR) {
        double acc = b[i] / s[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + i];
            if (c == (int32_t)i) continue;             // unused slot
            const double v = from_x ? s[c] * xy[c] : xy[c];
            acc = fma(-a[j * n + i], v, acc);
        }
        y[i] = acc;
    }
}

// Black rows: y_B = S_B x_B, r_B = bhat_B - y_B - E^T y_R, p_B = r_B; per run
// rho = r.r, ||b||^2 over all rows, ||S r||^2.
__global__ void __launch_bounds__(kBlock) k_black_init(const double* __restrict__ b,
                                                       const double* __restrict__ x,
                                                       const double* __restrict__ s,
                                                       const double* __restrict__ a,
                                                       const int32_t* __restrict__ col,
                                                       int64_t n, int64_t nR,
                                                       double* __restrict__ y,
                                                       double* __restrict__ r,
                                                       double* __restrict__ p, double rtol,
                                                       long long budget, double* partials,
                                                       CgState* st) {
    double rr = 0.0, bb = 0.0, nn = 0.0;
    CPS_GRID_STRIDE(k, n) {
        const double bk = b[k];
        bb = fma(bk, bk, bb);
    }
    CPS_GRID_STRIDE(k, n - nR) {
        const int64_t i = nR + k;
        const double se = s[i];
        const double ye = se * x[i];
        double ay = ye;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + i];
            if (c == (int32_t)i) continue;
            ay = fma(a[j * n + i], y[c], ay);
        }
        const double re = b[i] / se - ay;
        y[i] = ye;
        r[i] = re;
        p[i] = re;
        rr = fma(re, re, rr);
        const double t = se * re;
        nn = fma(t, t, nn);
    }
    double t[3] = {rr, bb, nn};
    if (grid_sum<3>(t, partials, &st->arrive[2]) && threadIdx.x == 0) {
        st->rho = t[0];
        st->bnorm2 = t[1];
        st->thresh2 = rtol * rtol * t[1];
        st->rnorm2 = t[2];
        st->alpha = 0.0;
        st->beta = 0.0;
        st->gamma = 0.0;
        st->iter = 0;
        st->max_iter = budget;
        st->status = CPS_OK;
        st->done = (t[1] == 0.0 || t[2] <= st->thresh2 || budget <= 0) ? 2 : 0;
    }
}

// t_R = E p_B (red rows).  First kernel of a reduced iteration: it also
// turns "stop after this iteration" into "stopped".
__global__ void __launch_bounds__(kBlock) k_schur_red(const double* __restrict__ a,
                                                      const int32_t* __restrict__ col,
                                                      const double* __restrict__ p,
                                                      double* __restrict__ t, int64_t n,
                                                      int64_t nR, CgState* st) {
    {
        const int d = st->done;
        if (d) {
            if (d == 1 && blockIdx.x == 0 && threadIdx.x == 0) st->done = 2;
            return;
        }
    }
    CPS_GRID_STRIDE(i, nR) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + i];
            if (c == (int32_t)i) continue;
            acc = fma(a[j * n + i], p[c], acc);
        }
        t[i] = acc;
    }
}

// q_B = p_B - E^T t_R (black rows), gamma = p_B . q_B; last block: alpha.
__global__ void __launch_bounds__(kBlock) k_schur_black(const double* __restrict__ a,
                                                        const int32_t* __restrict__ col,
                                                        const double* __restrict__ p,
                                                        const double* __restrict__ t,
                                                        double* __restrict__ q, int64_t n,
                                                        int64_t nR, double* partials,
                                                        CgState* st) {
    if (st->done) return;
    double acc = 0.0;
    CPS_GRID_STRIDE(k, n - nR) {
        const int64_t i = nR + k;
        const double pe = p[i];
        double v = pe;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + i];
            if (c == (int32_t)i) continue;
            v = fma(-a[j * n + i], t[c], v);
        }
        q[i] = v;
        acc = fma(pe, v, acc);
    }
    double g[1] = {acc};
    if (grid_sum<1>(g, partials, &st->arrive[0]) && threadIdx.x == 0) {
        const double gamma = g[0];
        st->gamma = gamma;
        if (!(gamma > 0.0) || !isfinite(gamma)) {
            st->status = CPS_ERR_NOT_SPD;
            st->done = 2;
        } else {
            st->alpha = st->rho / gamma;
        }
    }
}

}  // namespace cps
