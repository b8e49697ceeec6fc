// The CP2 step around the two corrector solves (Sec. 3.2.3, App. A, App. C).
//
// Per time step, given the cell velocity u^{k+2/3} of the first corrector and
// the cell field eps grad(Psi^k):
//   1. Fbar_j = ((u_e.n_j) A_ep + (u_ep.n_j) A_e)/(A_e + A_ep) l_j, the
//      area-weighted mean outward flux of each side (Eq. flux_k_+_2/3; n_jp =
//      -n_j), and B1_e = sum_j Fbar_j;
//   2. A eta~ = B1 (Eq. Cs2_7_1), the TPFA system of the library;
//   3. tau_j(eta~), the tangential part of the flux of Xi_j grad(eta) from the
//      co-normal decomposition of d_{j,tau} along the normals of the
//      neighbouring sides (Eq. Cs2_6, Eq. eta_flux, App. C), and
//      B2_e = B1_e + sum_j tau_j;
//   4. A eta = B2 (Eq. Cs2_7_2), warm-started from eta~;
//   5. outward fluxes Q_j = Fbar_j - T_j (eta_e - eta_ep) + tau_j, which sum to
//      zero over each cell (Eq. Cs2_5), the RT0 cell velocity
//      sum_j Q_j (centroid - x_j)/(2 A_e) (Eq. RT0) and
//      eps grad(Psi^{k+1}) = eps grad(Psi^k) + Mbar_e (u^{k+1} - u^{k+2/3})
//      (Eq. grad_PSI).
// Every flux is the physical flux leaving the cell.  The tangential flux of a
// side averages two one-sided estimates of d_{j,tau}.grad(eta): from e, with
// d_{j,tau} = c_1 n_1 + c_2 n_2 over e's other two sides and n_k.grad(eta) ~
// (eta_across - eta_e)/d_k, and the same from ep.  An estimate that needs the
// derivative across a no-flux side does not exist (the other is used alone);
// across a Dirichlet side eta = 0 at the midpoint.
//
// Set-up folds the geometry, the side tensor and the co-normal components into
// per-slot weights (the area weight of the mean flux, l_j n_j zeroed on no-flux
// sides, four co-normal weights and cell indices), so the step itself is three
// branch-free streaming kernels (1, 3, 5) around the two solves, one thread per
// cell.  A boundary slot is recognised by its column (col = e); no-flux slots
// carry zero coefficients and need no test.
#include "cps_internal.cuh"

#include <string>

namespace cps {
namespace {

// Per cell: RT0 weights (centroid - x_j)/(2 A_e) and Mbar_e, the mean over
// the cell's nodes of M = (I + nu eps Kinv dt)/dt (the cell's own M for cell
// fields).
__device__ __forceinline__ bool vertices_ok(const int32_t* __restrict__ tri, int64_t e,
                                            int64_t nv) {
    const int32_t a = tri[3 * e], b = tri[3 * e + 1], c = tri[3 * e + 2];
    return a >= 0 && a < nv && b >= 0 && b < nv && c >= 0 && c < nv;
}

__global__ void k_cp2_cell(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                           int64_t nt, int64_t nv, const double* __restrict__ eps,
                           const double* __restrict__ kinv, bool per_vertex, bool logk,
                           double nu, double dt, double* __restrict__ rt0,
                           double* __restrict__ mbar, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!vertices_ok(tri, e, nv)) {
            set_error(err, CPS_ERR_ARG);
            continue;
        }
        const int64_t v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        const double x0 = xy[2 * v[0]], y0 = xy[2 * v[0] + 1];
        const double x1 = xy[2 * v[1]], y1 = xy[2 * v[1] + 1];
        const double x2 = xy[2 * v[2]], y2 = xy[2 * v[2] + 1];
        const double a2 = (x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0);
        const double gx = (x0 + x1 + x2) / 3.0, gy = (y0 + y1 + y2) / 3.0;
        const double px[3] = {x0, x1, x2}, py[3] = {y0, y1, y2};
        for (int j = 0; j < 3; ++j) {
            rt0[(2 * j) * nt + e] = (gx - px[j]) / a2;
            rt0[(2 * j + 1) * nt + e] = (gy - py[j]) / a2;
        }
        double mb[3];
        cell_mbar(eps, kinv, v, e, per_vertex, logk, nu, dt, mb);
        mbar[e] = mb[0];
        mbar[nt + e] = mb[1];
        mbar[2 * nt + e] = mb[2];
    }
}

struct SideArgs {
    const double* xy;
    const int32_t* tri;
    const int32_t* col;
    const int32_t* slot_kind;
    const double* ccx;
    const double* ccy;
    const double* area;
    const double* xi;
    int64_t nt, nv;
    bool per_vertex;
    double* nx;     // [3nt] scratch
    double* ny;
    double* len;
    double* dist;   // d_{e,ep} (interior), delta_j (Dirichlet)
    double* dtx;    // [3nt] d_{j,tau}
    double* dty;
    double* lnx;    // [3nt] outputs
    double* lny;
    double* T;
    double* wgt;
    int* err;
};

// Per side slot: length, outward normal, circumcentre distance, side tensor
// Xi_j (the matrix's average), T_j = l_j d_{j,n}/d and d_{j,tau}.
__global__ void k_cp2_side(SideArgs A) {
    const int64_t nt = A.nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (!vertices_ok(A.tri, e, A.nv)) {
            set_error(A.err, CPS_ERR_ARG);
            for (int j = 0; j < 3; ++j) {
                const int64_t slot = (int64_t)j * nt + e;
                A.nx[slot] = A.ny[slot] = A.len[slot] = A.dist[slot] = 0.0;
                A.dtx[slot] = A.dty[slot] = A.lnx[slot] = A.lny[slot] = A.T[slot] = 0.0;
                A.wgt[slot] = 1.0;
            }
            continue;
        }
        const int32_t v[3] = {A.tri[3 * e], A.tri[3 * e + 1], A.tri[3 * e + 2]};
        const double cex = A.ccx[e], cey = A.ccy[e];
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int64_t ia = v[(j + 1) % 3], ib = v[(j + 2) % 3];
            const double px = A.xy[2 * ia], py = A.xy[2 * ia + 1];
            const double qx = A.xy[2 * ib], qy = A.xy[2 * ib + 1];
            const double tx = qx - px, ty = qy - py;
            const double l = sqrt(tx * tx + ty * ty);
            const double nx = ty / l, ny = -tx / l;
            const int sk = A.slot_kind[slot];
            const int32_t ep = A.col[slot];
            double d = 0.0;
            if (sk == 1) d = (A.ccx[ep] - cex) * nx + (A.ccy[ep] - cey) * ny;
            else if (sk == 2) d = (0.5 * (px + qx) - cex) * nx + (0.5 * (py + qy) - cey) * ny;
            if (sk != 0 && !(d > 1e-12 * l)) set_error(A.err, CPS_ERR_NONDELAUNAY);
            double x0, x1, x2;
            if (A.per_vertex) {
                x0 = 0.5 * (A.xi[3 * ia] + A.xi[3 * ib]);
                x1 = 0.5 * (A.xi[3 * ia + 1] + A.xi[3 * ib + 1]);
                x2 = 0.5 * (A.xi[3 * ia + 2] + A.xi[3 * ib + 2]);
            } else if (sk == 1) {
                x0 = 0.5 * (A.xi[3 * e] + A.xi[3 * (int64_t)ep]);
                x1 = 0.5 * (A.xi[3 * e + 1] + A.xi[3 * (int64_t)ep + 1]);
                x2 = 0.5 * (A.xi[3 * e + 2] + A.xi[3 * (int64_t)ep + 2]);
            } else {
                x0 = A.xi[3 * e];
                x1 = A.xi[3 * e + 1];
                x2 = A.xi[3 * e + 2];
            }
            const double dx = x0 * nx + x1 * ny, dy = x1 * nx + x2 * ny;
            const double dn = dx * nx + dy * ny;
            A.nx[slot] = nx;
            A.ny[slot] = ny;
            A.len[slot] = l;
            A.dist[slot] = d;
            A.dtx[slot] = dx - dn * nx;
            A.dty[slot] = dy - dn * ny;
            A.lnx[slot] = sk != 0 ? l * nx : 0.0;
            A.lny[slot] = sk != 0 ? l * ny : 0.0;
            A.T[slot] = sk != 0 ? l * dn / d : 0.0;
            A.wgt[slot] = sk == 1 ? A.area[ep] / (A.area[e] + A.area[ep]) : 1.0;
        }
    }
}

// Co-normal components of (dtx, dty) in the basis of the outward normals of
// cell c's sides other than local side jc (Cramer's rule), divided by the
// circumcentre distances across those sides; false if either is a no-flux side.
__device__ __forceinline__ bool conormal(int64_t c, int jc, int64_t nt, double dtx, double dty,
                                         const int32_t* __restrict__ col,
                                         const int32_t* __restrict__ slot_kind,
                                         const double* __restrict__ nx,
                                         const double* __restrict__ ny,
                                         const double* __restrict__ dist, double* w,
                                         int32_t* idx) {
    const int64_t s1 = (int64_t)((jc + 1) % 3) * nt + c, s2 = (int64_t)((jc + 2) % 3) * nt + c;
    const int k1 = slot_kind[s1], k2 = slot_kind[s2];
    if (k1 == 0 || k2 == 0) return false;
    const double n1x = nx[s1], n1y = ny[s1], n2x = nx[s2], n2y = ny[s2];
    const double det = n1x * n2y - n1y * n2x;
    w[0] = (dtx * n2y - dty * n2x) / det / dist[s1];
    w[1] = (n1x * dty - n1y * dtx) / det / dist[s2];
    idx[0] = k1 == 1 ? col[s1] : -1;
    idx[1] = k2 == 1 ? col[s2] : -1;
    return true;
}

struct WeightArgs {
    const int32_t* col;
    const int32_t* slot_kind;
    const double* nx;
    const double* ny;
    const double* len;
    const double* dist;
    const double* dtx;
    const double* dty;
    int64_t nt;
    double* tw;      // [4][3nt]
    int32_t* tidx;   // [4][3nt]
    int* err;
};

// Per side slot: the four weights w_k and cells i_k of
//   tau_j = sum_{k<2} w_k (eta[i_k] - eta_e) + sum_{k>=2} w_k (eta[i_k] - eta_ep),
// l_j / (number of estimates) folded into w.  Unused terms get w = 0 and a
// valid index.
__global__ void k_cp2_weights(WeightArgs A) {
    const int64_t nt = A.nt, ns = 3 * nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int sk = A.slot_kind[slot];
            double w[4] = {0.0, 0.0, 0.0, 0.0};
            int32_t idx[4] = {(int32_t)e, (int32_t)e, (int32_t)e, (int32_t)e};
            if (sk != 0) {
                const double dtx = A.dtx[slot], dty = A.dty[slot];
                const bool own = conormal(e, j, nt, dtx, dty, A.col, A.slot_kind, A.nx, A.ny,
                                          A.dist, w, idx);
                if (!own) w[0] = w[1] = 0.0, idx[0] = idx[1] = (int32_t)e;
                bool other = false;
                if (sk == 1) {
                    const int32_t ep = A.col[slot];
                    int jp = -1;
                    for (int k = 0; k < 3; ++k)
                        if (jp < 0 && A.slot_kind[(int64_t)k * nt + ep] == 1 &&
                            A.col[(int64_t)k * nt + ep] == (int32_t)e)
                            jp = k;
                    if (jp < 0) {
                        set_error(A.err, CPS_ERR_NONMANIFOLD);
                    } else {
                        other = conormal(ep, jp, nt, dtx, dty, A.col, A.slot_kind, A.nx, A.ny,
                                         A.dist, w + 2, idx + 2);
                    }
                    if (!other) w[2] = w[3] = 0.0, idx[2] = idx[3] = ep;
                }
                const int count = (own ? 1 : 0) + (other ? 1 : 0);
                const double f = count > 0 ? A.len[slot] / count : 0.0;
                for (int k = 0; k < 4; ++k) w[k] *= f;
            }
            for (int k = 0; k < 4; ++k) {
                A.tw[k * ns + slot] = w[k];
                A.tidx[k * ns + slot] = idx[k];
            }
        }
    }
}

// Step 1: Fbar per slot and B1_e = sum_j Fbar_j, as
// l_j n_j . (w u_e + (1 - w) u_ep) with w = A_ep/(A_e + A_ep) (Eq. flux_k_+_2/3
// with n_jp = -n_j).  A Dirichlet slot has col = e and w = 1 (e's own flux); a
// no-flux slot has l_j n_j = 0.
__global__ void __launch_bounds__(kBlock)
k_cp2_mean_flux(const double* __restrict__ u, const int32_t* __restrict__ col,
                const double* __restrict__ wgt, const double* __restrict__ lnx,
                const double* __restrict__ lny, int64_t nt, double* __restrict__ fbar,
                double* __restrict__ rhs) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double ue = u[e], ve = u[nt + e];
        double sum = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int32_t c = col[slot];
            const double w = wgt[slot];
            const double ux = w * ue + (1.0 - w) * u[c];
            const double uy = w * ve + (1.0 - w) * u[nt + c];
            const double f = lnx[slot] * ux + lny[slot] * uy;
            fbar[slot] = f;
            sum += f;
        }
        rhs[e] = sum;
    }
}

// Step 3: tau per slot from eta~ and B2_e = B1_e + sum_j tau_j.
__global__ void __launch_bounds__(kBlock)
k_cp2_tangential(const double* __restrict__ eta, const int32_t* __restrict__ col,
                                 const double* __restrict__ tw, const int32_t* __restrict__ tidx,
                                 int64_t nt, double* __restrict__ tau, double* __restrict__ rhs) {
    const int64_t ns = 3 * nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double ee = eta[e];
        double sum = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const double ep = eta[col[slot]];
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t i = tidx[k * ns + slot];
                const double ek = i >= 0 ? eta[i] : 0.0;
                t += tw[k * ns + slot] * (ek - (k < 2 ? ee : ep));
            }
            tau[slot] = t;
            sum += t;
        }
        rhs[e] += sum;
    }
}

// Step 5: side fluxes, RT0 cell velocity, eps grad(Psi) update.  On a
// boundary slot (col = e) eta across is 0 (Dirichlet); a no-flux slot has
// Fbar = T = tau = 0 and so Q = 0.
__global__ void __launch_bounds__(kBlock, 4)
k_cp2_update(const double* __restrict__ eta, const int32_t* __restrict__ col,
             const double* __restrict__ fbar, const double* __restrict__ T,
             const double* __restrict__ tau, const double* __restrict__ rt0,
             const double* __restrict__ mbar, const double* __restrict__ u23,
             const double* __restrict__ g_k, int64_t nt, double* __restrict__ flux,
             double* __restrict__ u_next, double* __restrict__ g_next) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double ee = eta[e];
        double ux = 0.0, uy = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int32_t c = col[slot];
            const double ec = eta[c];
            const double eb = c != (int32_t)e ? ec : 0.0;
            const double q = fbar[slot] - T[slot] * (ee - eb) + tau[slot];
            if (flux) flux[slot] = q;
            ux += q * rt0[(2 * j) * nt + e];
            uy += q * rt0[(2 * j + 1) * nt + e];
        }
        u_next[e] = ux;
        u_next[nt + e] = uy;
        const double du = ux - u23[e], dv = uy - u23[nt + e];
        const double m00 = mbar[e], m01 = mbar[nt + e], m11 = mbar[2 * nt + e];
        g_next[e] = g_k[e] + m00 * du + m01 * dv;
        g_next[nt + e] = g_k[nt + e] + m01 * du + m11 * dv;
    }
}

int fail(cps_sys s, int code, const std::string& msg) {
    set_error(s->ctx, msg);
    return code;
}

}  // namespace

void free_cp2(cps_sys s) {
    if (!s || !s->cp2) return;
    for (cudaEvent_t ev : s->cp2->ev)
        if (ev) cudaEventDestroy(ev);
    if (s->cp2->buf) cudaFree(s->cp2->buf);
    delete s->cp2;
    s->cp2 = nullptr;
}

int cp2_setup_impl(cps_sys s, const double* xy, const int32_t* tri, const double* eps,
                   const double* kinv, cudaStream_t stream) {
    if (s->kind != CPS_KIND_CP2) return fail(s, CPS_ERR_ARG, "cp2_setup: system is not CP2");
    if (!xy || !tri || !eps || !kinv) return fail(s, CPS_ERR_ARG, "cp2_setup: null pointer");
    const int64_t nt = s->nt, nv = s->nv, ns = 3 * nt;
    const bool per_vertex = s->field_loc == CPS_PER_VERTEX;
    const int64_t nf = per_vertex ? nv : nt;
    free_cp2(s);
    Cp2Data* c = new Cp2Data();
    // doubles: wgt 3, lnx 3, lny 3, T 3, tw 12, rt0 6, mbar 3, fbar 3, tau 3, rhs 1,
    // eta_t 1 (x nt, each slice 256-byte aligned); then tidx 12 nt int32
    const int64_t st = (nt + 31) / 32 * 32;
    const int64_t nd = 41 * st;
    const size_t bytes = sizeof(double) * (size_t)nd + sizeof(int32_t) * (size_t)(12 * st);
    cudaError_t ce = cudaMalloc(&c->buf, bytes);
    if (ce != cudaSuccess) {
        delete c;
        return fail(s, CPS_ERR_NOMEM, std::string("cp2_setup: cudaMalloc: ") + cudaGetErrorString(ce));
    }
    double* d = static_cast<double*>(c->buf);
    auto take = [&](int64_t k) { double* p = d; d += k * st; return p; };
    c->wgt = take(3);
    c->lnx = take(3);
    c->lny = take(3);
    c->T = take(3);
    c->tw = take(12);
    c->rt0 = take(6);
    c->mbar = take(3);
    c->fbar = take(3);
    c->tau = take(3);
    c->rhs = take(1);
    c->eta_t = take(1);
    c->tidx = reinterpret_cast<int32_t*>(d);
    s->cp2 = c;
    for (cudaEvent_t& ev : c->ev) {
        ce = cudaEventCreate(&ev);
        if (ce != cudaSuccess) {
            free_cp2(s);
            return fail(s, CPS_ERR_CUDA, std::string("cp2_setup: cudaEventCreate: ") +
                                             cudaGetErrorString(ce));
        }
    }
    // A slice of k st doubles holds the k rows [k][nt] at stride nt (k nt <= k st).

    double *ccx = nullptr, *ccy = nullptr, *area = nullptr, *xi = nullptr, *scratch = nullptr;
    int* err = nullptr;
    int h_err = 0;
    auto A = [&](void** p, size_t b) { return cudaMallocAsync(p, b, stream); };
    ce = A((void**)&ccx, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&ccy, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&area, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&xi, sizeof(double) * 3 * nf);
    if (ce == cudaSuccess) ce = A((void**)&scratch, sizeof(double) * 6 * ns);
    if (ce == cudaSuccess) ce = A((void**)&err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(int), stream);
    if (ce == cudaSuccess) {
        const int g = s->grid;
        k_cell_geometry<<<g, kBlock, 0, stream>>>(xy, tri, nt, nv, area, ccx, ccy, err);
        k_xi<<<g, kBlock, 0, stream>>>(eps, kinv, nf, s->nu, s->dt, s->logk, xi, err);
        k_cp2_cell<<<g, kBlock, 0, stream>>>(xy, tri, nt, nv, eps, kinv, per_vertex, s->logk,
                                             s->nu, s->dt, c->rt0, c->mbar, err);
        SideArgs sa{xy, tri, s->col, s->slot_kind, ccx, ccy, area, xi, nt, nv, per_vertex,
                    scratch, scratch + ns, scratch + 2 * ns, scratch + 3 * ns,
                    scratch + 4 * ns, scratch + 5 * ns, c->lnx, c->lny, c->T, c->wgt, err};
        k_cp2_side<<<g, kBlock, 0, stream>>>(sa);
        WeightArgs wa{s->col, s->slot_kind, sa.nx, sa.ny, sa.len, sa.dist, sa.dtx, sa.dty, nt,
                      c->tw, c->tidx, err};
        k_cp2_weights<<<g, kBlock, 0, stream>>>(wa);
        ce = cudaGetLastError();
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    }
    void* tmp[] = {ccx, ccy, area, xi, scratch, err};
    for (void* p : tmp)
        if (p) cudaFreeAsync(p, stream);
    cudaError_t se = cudaStreamSynchronize(stream);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) {
        free_cp2(s);
        return fail(s, ce == cudaErrorMemoryAllocation ? CPS_ERR_NOMEM : CPS_ERR_CUDA,
                    std::string("cp2_setup: ") + cudaGetErrorString(ce));
    }
    if (h_err != 0) {
        free_cp2(s);
        return fail(s, h_err, "cp2_setup: mesh or fields do not match the system (or bad input)");
    }
    return CPS_OK;
}

int cp2_step_impl(cps_sys s, const double* u23, const double* g_k, double* eta_tilde,
                  double* eta, double* u_next, double* g_next, double* flux, double rtol,
                  int64_t max_iter, int precision, cps_stats* stats, cudaStream_t stream) {
    Cp2Data* c = s->cp2;
    if (!c) return fail(s, CPS_ERR_ARG, "cp2_step: call cps_cp2_setup first");
    if (!u23 || !g_k || !eta || !u_next || !g_next)
        return fail(s, CPS_ERR_ARG, "cp2_step: null pointer");
    const int64_t nt = s->nt;
    // one thread per cell: the step kernels are short, gather-heavy streams
    const int g = (int)((nt + kBlock - 1) / kBlock);
    double* et = eta_tilde ? eta_tilde : c->eta_t;
    cps_stats st[2];
    // Events around each step kernel on the caller's stream; their durations
    // are read after the final synchronisation (cps_cp2_kernel_times).
    cudaEventRecord(c->ev[0], stream);
    k_cp2_mean_flux<<<g, kBlock, 0, stream>>>(u23, s->col, c->wgt, c->lnx, c->lny, nt, c->fbar,
                                              c->rhs);
    cudaEventRecord(c->ev[1], stream);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemsetAsync(et, 0, sizeof(double) * nt, stream);
    if (ce != cudaSuccess) return fail(s, CPS_ERR_CUDA, std::string("cp2_step: ") + cudaGetErrorString(ce));
    int rc1 = solve_impl(s, c->rhs, et, rtol, max_iter, precision, &st[0], stream);
    if (rc1 != CPS_OK && rc1 != CPS_ERR_NOT_CONVERGED) return rc1;
    cudaEventRecord(c->ev[2], stream);
    k_cp2_tangential<<<g, kBlock, 0, stream>>>(et, s->col, c->tw, c->tidx, nt, c->tau, c->rhs);
    cudaEventRecord(c->ev[3], stream);
    ce = cudaGetLastError();
    if (ce == cudaSuccess && eta != et)     // one buffer for both: the warm start is in place
        ce = cudaMemcpyAsync(eta, et, sizeof(double) * nt, cudaMemcpyDeviceToDevice, stream);
    if (ce != cudaSuccess) return fail(s, CPS_ERR_CUDA, std::string("cp2_step: ") + cudaGetErrorString(ce));
    int rc2 = solve_impl(s, c->rhs, eta, rtol, max_iter, precision, &st[1], stream);
    if (rc2 != CPS_OK && rc2 != CPS_ERR_NOT_CONVERGED) return rc2;
    cudaEventRecord(c->ev[4], stream);
    k_cp2_update<<<g, kBlock, 0, stream>>>(eta, s->col, c->fbar, c->T, c->tau, c->rt0, c->mbar,
                                           u23, g_k, nt, flux, u_next, g_next);
    cudaEventRecord(c->ev[5], stream);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) return fail(s, CPS_ERR_CUDA, std::string("cp2_step: ") + cudaGetErrorString(ce));
    for (int k = 0; k < 3; ++k)
        if (cudaEventElapsedTime(&c->kernel_ms[k], c->ev[2 * k], c->ev[2 * k + 1]) != cudaSuccess)
            c->kernel_ms[k] = -1.f;
    if (stats) {
        stats[0] = st[0];
        stats[1] = st[1];
    }
    return rc1 != CPS_OK ? rc1 : rc2;
}

int cp2_kernel_times(cps_sys s, float* ms) {
    if (!s->cp2 || !ms) return fail(s, CPS_ERR_ARG, "cp2_kernel_times: no CP2 step data");
    for (int k = 0; k < 3; ++k) ms[k] = s->cp2->kernel_ms[k];
    return CPS_OK;
}

}  // namespace cps
