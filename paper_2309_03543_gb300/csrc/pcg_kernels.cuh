// Kernels of the conjugate-gradient solve.  All vectors of one run are in the
// symmetrically scaled space (yhat = S x, rhat = S^-1 r); matrix rows are
// padded ELL with 3 off-diagonal slots, slot-major (entry j*n + e), and a
// unit diagonal.  Every reduction is deterministic (fixed grid, fixed order).
#pragma once

#include "cps_internal.cuh"

namespace cps {

#define CPS_GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// q = Ahat p, gamma = p.q; last block: alpha = rho / gamma.
template <typename V>
__global__ void __launch_bounds__(kBlock) k_spmv_dot(const V* __restrict__ a,
                                                     const int32_t* __restrict__ col,
                                                     const V* __restrict__ p, V* __restrict__ q,
                                                     int64_t n, double* partials, CgState* st) {
    if (st->done) return;
    double acc = 0.0;
    CPS_GRID_STRIDE(e, n) {
        const V pe = p[e];
        V v = pe;
#pragma unroll
        for (int j = 0; j < 3; ++j) v = fma(a[j * n + e], p[col[j * n + e]], v);
        q[e] = v;
        acc = fma((double)pe, (double)v, acc);
    }
    double t[1] = {acc};
    if (grid_sum<1>(t, partials, &st->arrive[0]) && threadIdx.x == 0) {
        const double gamma = t[0];
        st->gamma = gamma;
        if (!(gamma > 0.0) || !isfinite(gamma)) {
            st->status = CPS_ERR_NOT_SPD;
            st->done = 1;
        } else {
            st->alpha = st->rho / gamma;
        }
    }
}

// y += alpha p, r -= alpha q, rho' = r.r; with NORM also ||S r||^2 and the
// stop test.  Last block: beta = rho'/rho, iteration count, stop flag.
template <typename V, bool NORM>
__global__ void __launch_bounds__(kBlock) k_update(V* __restrict__ y, V* __restrict__ r,
                                                   const V* __restrict__ p,
                                                   const V* __restrict__ q,
                                                   const V* __restrict__ s, int64_t n,
                                                   double* partials, CgState* st) {
    if (st->done) return;
    const V al = (V)st->alpha;
    double rr = 0.0, nn = 0.0;
    CPS_GRID_STRIDE(e, n) {
        const V pe = p[e], qe = q[e];
        y[e] = fma(al, pe, y[e]);
        const V re = fma(-al, qe, r[e]);
        r[e] = re;
        rr = fma((double)re, (double)re, rr);
        if (NORM) {
            const double t = (double)s[e] * (double)re;
            nn = fma(t, t, nn);
        }
    }
    double t[2] = {rr, nn};
    if (grid_sum<2>(t, partials, &st->arrive[1]) && threadIdx.x == 0) {
        const double rho_new = t[0];
        const long long it = st->iter + 1;
        st->iter = it;
        int done = 0;
        if (NORM) {
            st->rnorm2 = t[1];
            if (t[1] <= st->thresh2) done = 1;
        }
        if (!(rho_new > 0.0)) done = 1;          // exact solution reached
        if (it >= st->max_iter) done = 1;
        st->beta = rho_new / st->rho;
        st->rho = rho_new;
        if (done) st->done = 1;
    }
}

// p = r + beta p
template <typename V>
__global__ void __launch_bounds__(kBlock) k_pupdate(V* __restrict__ p, const V* __restrict__ r,
                                                    int64_t n, const CgState* st) {
    if (st->done) return;
    const V be = (V)st->beta;
    CPS_GRID_STRIDE(e, n) { p[e] = fma(be, p[e], r[e]); }
}

// Start of a FP64 run from the user's x: y = S x, r = S^-1 b - Ahat y, p = r.
__global__ void __launch_bounds__(kBlock) k_init64(const double* __restrict__ b,
                                                   const double* __restrict__ x,
                                                   const double* __restrict__ s,
                                                   const double* __restrict__ a,
                                                   const int32_t* __restrict__ col, int64_t n,
                                                   double* __restrict__ y, double* __restrict__ r,
                                                   double* __restrict__ p, double rtol,
                                                   long long budget, double* partials,
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
        if (p) p[e] = re;
        rr = fma(re, re, rr);
        bb = fma(be, be, bb);
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
        st->done = (t[1] == 0.0 || t[2] <= st->thresh2 || budget <= 0) ? 1 : 0;
    }
}

// End of a FP64 run: x = S^-1 y and the true residual ||b - A x||^2 in FP64.
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

// Mixed precision, outer step: r = b - A x in FP64 from the FP64 iterate x;
// the inner run starts from d = 0 with r32 = p32 = S^-1 r rounded to binary32.
// Inner stop: ||S r_inner|| <= max(eta ||r||, rtol ||b|| / 2).
__global__ void __launch_bounds__(kBlock) k_res64(const double* __restrict__ b,
                                                  const double* __restrict__ x,
                                                  const double* __restrict__ s,
                                                  const double* __restrict__ a,
                                                  const int32_t* __restrict__ col, int64_t n,
                                                  float* __restrict__ r32, float* __restrict__ p32,
                                                  float* __restrict__ d32, double rtol, double eta,
                                                  long long budget, double* partials, CgState* st) {
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
        p32[e] = rf;
        d32[e] = 0.0f;
        rr = fma((double)rf, (double)rf, rr);
        bb = fma(be, be, bb);
        const double t = se * re;
        nn = fma(t, t, nn);
    }
    double t[3] = {rr, bb, nn};
    if (grid_sum<3>(t, partials, &st->arrive[2]) && threadIdx.x == 0) {
        st->rho = t[0];
        st->bnorm2 = t[1];
        st->rnorm2 = t[2];
        const double outer2 = rtol * rtol * t[1];
        const double inner2 = eta * eta * t[2];
        st->thresh2 = inner2 > 0.25 * outer2 ? inner2 : 0.25 * outer2;
        st->alpha = 0.0;
        st->beta = 0.0;
        st->gamma = 0.0;
        st->iter = 0;
        st->max_iter = budget;
        st->status = CPS_OK;
        st->done = (t[1] == 0.0 || t[2] <= outer2 || budget <= 0 || !(t[0] > 0.0)) ? 1 : 0;
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

}  // namespace cps
