// Assembly of the corrector matrices on the device.
//
//   1. side topology: a hash table keyed by the two vertex ids of each side
//      pairs the two cells sharing it (Sec. 3.1: each side has at most one
//      neighbour across it);
//   2. geometry per cell: area and circumcentre; per side: length, outward
//      normal and signed circumcentre distance d_{e,ep} (Eq. cs1_discr);
//   3. Xi = eps dt (I + nu eps dt Kinv)^-1 at every node or cell (Eq. Cs2_4);
//   4. side coefficients T_j = l_j (n_j . Xi_j n_j) / d_{e,ep} for CP2
//      (Eq. CS2_sys_coeff) or nu l_j / d_{e,ep} plus the mass term
//      Mbar_kk A_e for CP1 (Eq. CS1_sys_coeff), packed into a padded ELL
//      layout, slot-major [3][nt];
//   5. symmetric diagonal scaling s = sqrt(diag A), Ahat = S^-1 A S^-1.
//
// Every coefficient of a side is computed from each of its two cells with
// the same operation sequence on exactly negated inputs, so A is bitwise
// symmetric.
#include "cps_internal.cuh"

#include <cmath>
#include <cstring>

namespace cps {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    // MurmurHash3 64-bit finaliser.
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

constexpr unsigned long long kEmpty = ~0ULL;

__global__ void k_side_insert(const int32_t* __restrict__ tri, int64_t nt, int64_t nv,
                              unsigned long long* keys, int32_t* id0, int32_t* id1,
                              unsigned long long mask, int* err) {
    const int64_t n3 = 3 * nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / 3;
        const int j = (int)(t - 3 * e);
        const int64_t va = tri[3 * e + (j + 1) % 3];
        const int64_t vb = tri[3 * e + (j + 2) % 3];
        if (va < 0 || va >= nv || vb < 0 || vb >= nv || va == vb) {
            set_error(err, CPS_ERR_ARG);
            continue;
        }
        const unsigned long long lo = (unsigned long long)(va < vb ? va : vb);
        const unsigned long long hi = (unsigned long long)(va < vb ? vb : va);
        const unsigned long long key = lo * (unsigned long long)nv + hi;
        unsigned long long h = mix64(key) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            unsigned long long old = atomicCAS(&keys[h], kEmpty, key);
            if (old == kEmpty || old == key) {
                if (atomicCAS(&id0[h], -1, (int32_t)t) != -1) {
                    if (atomicCAS(&id1[h], -1, (int32_t)t) != -1) set_error(err, CPS_ERR_NONMANIFOLD);
                }
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

__global__ void k_side_lookup(const int32_t* __restrict__ tri, int64_t nt, int64_t nv,
                              const unsigned long long* __restrict__ keys,
                              const int32_t* __restrict__ id0, const int32_t* __restrict__ id1,
                              unsigned long long mask, int32_t* __restrict__ nbr) {
    const int64_t n3 = 3 * nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n3;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = t / 3;
        const int j = (int)(t - 3 * e);
        const int64_t va = tri[3 * e + (j + 1) % 3];
        const int64_t vb = tri[3 * e + (j + 2) % 3];
        int32_t other = -1;
        if (va >= 0 && va < nv && vb >= 0 && vb < nv && va != vb) {
            const unsigned long long lo = (unsigned long long)(va < vb ? va : vb);
            const unsigned long long hi = (unsigned long long)(va < vb ? vb : va);
            const unsigned long long key = lo * (unsigned long long)nv + hi;
            unsigned long long h = mix64(key) & mask;
            for (unsigned long long probe = 0; probe <= mask; ++probe) {
                const unsigned long long k = keys[h];
                if (k == key) {
                    const int32_t a = id0[h], b = id1[h];
                    other = (a == (int32_t)t) ? b : a;
                    break;
                }
                if (k == kEmpty) break;
                h = (h + 1) & mask;
            }
        }
        nbr[(int64_t)j * nt + e] = other >= 0 ? other / 3 : -1;
    }
}

}  // namespace

__global__ void k_cell_geometry(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                                int64_t nt, int64_t nv, double* __restrict__ area,
                                double* __restrict__ ccx, double* __restrict__ ccy, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = tri[3 * e], i1 = tri[3 * e + 1], i2 = tri[3 * e + 2];
        if (i0 < 0 || i0 >= nv || i1 < 0 || i1 >= nv || i2 < 0 || i2 >= nv) {
            set_error(err, CPS_ERR_ARG);
            area[e] = 0.0;
            ccx[e] = 0.0;
            ccy[e] = 0.0;
            continue;
        }
        const double ax = xy[2 * i0], ay = xy[2 * i0 + 1];
        const double bx = xy[2 * i1] - ax, by = xy[2 * i1 + 1] - ay;
        const double cx = xy[2 * i2] - ax, cy = xy[2 * i2 + 1] - ay;
        const double cross = bx * cy - by * cx;
        if (!(cross > 0.0)) set_error(err, CPS_ERR_ORIENTATION);
        area[e] = 0.5 * cross;
        const double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
        const double inv = 0.5 / cross;
        ccx[e] = ax + (cy * b2 - by * c2) * inv;
        ccy[e] = ay + (bx * c2 - cx * b2) * inv;
    }
}

// Xi = eps dt (I + c Kinv)^-1, c = nu eps dt, explicit 2x2 inverse.
__global__ void k_xi(const double* __restrict__ eps, const double* __restrict__ kinv, int64_t nf,
                     double nu, double dt, bool logk, double* __restrict__ xi, int* err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double ep = eps[i];
        const double kxx = kinv_at(kinv, i, 0, logk), kxy = kinv_at(kinv, i, 1, logk),
                     kyy = kinv_at(kinv, i, 2, logk);
        const double c = nu * ep * dt;
        const double m00 = 1.0 + c * kxx, m01 = c * kxy, m11 = 1.0 + c * kyy;
        const double det = m00 * m11 - m01 * m01;
        if (!(ep > 0.0) || !(det > 0.0) || !(m00 > 0.0)) set_error(err, CPS_ERR_ARG);
        const double sc = ep * dt / det;
        xi[3 * i] = sc * m11;
        xi[3 * i + 1] = -sc * m01;
        xi[3 * i + 2] = sc * m00;
    }
}

namespace {

__global__ void k_mark_dirichlet(const int32_t* __restrict__ dirichlet, int64_t nb, int64_t nt,
                                 const int32_t* __restrict__ nbr, int32_t* __restrict__ kind,
                                 int* err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sid = dirichlet[k];
        if (sid < 0 || sid >= 3 * nt) {
            set_error(err, CPS_ERR_ARG);
            continue;
        }
        const int64_t e = sid / 3;
        const int j = (int)(sid - 3 * e);
        const int64_t slot = (int64_t)j * nt + e;
        if (nbr[slot] >= 0) {
            set_error(err, CPS_ERR_ARG);
            continue;
        }
        kind[slot] = 2;
    }
}

struct TransArgs {
    const double* xy;
    const int32_t* tri;
    const int32_t* nbr;
    const double* ccx;
    const double* ccy;
    const double* area;
    const double* xi;      // [nf][3]
    const double* eps;
    const double* kinv;
    int32_t* slot_kind;    // in: 2 marks Dirichlet; out: 0/1/2
    double* diag;
    double* off;           // [3][nt] unscaled off-diagonals
    int32_t* col;
    double* gfac;          // may be null
    unsigned long long* n_interior;
    int64_t nt;
    int kind;
    int field_loc;     // CPS_PER_VERTEX or CPS_PER_CELL (log-permeability maps to cells)
    bool logk;
    double nu, dt;
    int* err;
};

__global__ void k_transmissibility(TransArgs A) {
    const int64_t nt = A.nt;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v[3] = {A.tri[3 * e], A.tri[3 * e + 1], A.tri[3 * e + 2]};
        const double cex = A.ccx[e], cey = A.ccy[e];
        double diag = 0.0;
        if (A.kind != CPS_KIND_CP2) {
            // Mbar_kk A_e, Mbar the mean over the cell's nodes of (I + nu eps Kinv dt)/dt
            const int comp = A.kind == CPS_KIND_CP1_X ? 0 : 2;
            double mkk;
            if (A.field_loc == CPS_PER_VERTEX) {
                mkk = 0.0;
                for (int k = 0; k < 3; ++k)
                    mkk += (1.0 + A.nu * A.eps[v[k]] * A.kinv[3 * (int64_t)v[k] + comp] * A.dt) / A.dt;
                mkk /= 3.0;
            } else {
                mkk = (1.0 + A.nu * A.eps[e] * kinv_at(A.kinv, e, comp, A.logk) * A.dt) / A.dt;
            }
            diag = mkk * A.area[e];
        }
        unsigned int interior = 0;
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int64_t ia = v[(j + 1) % 3], ib = v[(j + 2) % 3];
            const double px = A.xy[2 * ia], py = A.xy[2 * ia + 1];
            const double qx = A.xy[2 * ib], qy = A.xy[2 * ib + 1];
            const double tx = qx - px, ty = qy - py;
            const double l = sqrt(tx * tx + ty * ty);
            const double nx = ty / l, ny = -tx / l;
            const int32_t ep = A.nbr[slot];
            const bool dir = A.slot_kind[slot] == 2;
            double T = 0.0, g = 0.0;
            int32_t c = (int32_t)e;
            int sk = 0;
            if (ep >= 0 || dir) {
                double d;
                if (ep >= 0) {
                    d = (A.ccx[ep] - cex) * nx + (A.ccy[ep] - cey) * ny;
                } else {
                    d = (0.5 * (px + qx) - cex) * nx + (0.5 * (py + qy) - cey) * ny;
                }
                if (!(d > 1e-12 * l)) set_error(A.err, CPS_ERR_NONDELAUNAY);
                double coef;
                if (A.kind == CPS_KIND_CP2) {
                    double x0, x1, x2;
                    if (A.field_loc == CPS_PER_VERTEX) {
                        x0 = 0.5 * (A.xi[3 * ia] + A.xi[3 * ib]);
                        x1 = 0.5 * (A.xi[3 * ia + 1] + A.xi[3 * ib + 1]);
                        x2 = 0.5 * (A.xi[3 * ia + 2] + A.xi[3 * ib + 2]);
                    } else if (ep >= 0) {
                        x0 = 0.5 * (A.xi[3 * e] + A.xi[3 * (int64_t)ep]);
                        x1 = 0.5 * (A.xi[3 * e + 1] + A.xi[3 * (int64_t)ep + 1]);
                        x2 = 0.5 * (A.xi[3 * e + 2] + A.xi[3 * (int64_t)ep + 2]);
                    } else {
                        x0 = A.xi[3 * e];
                        x1 = A.xi[3 * e + 1];
                        x2 = A.xi[3 * e + 2];
                    }
                    const double dn = x0 * (nx * nx) + 2.0 * x1 * (nx * ny) + x2 * (ny * ny);
                    coef = dn;
                } else {
                    coef = A.nu;
                }
                T = l * coef / d;
                g = ep >= 0 ? l / (2.0 * d) : l / d;
                if (ep >= 0) {
                    c = ep;
                    sk = 1;
                    ++interior;
                } else {
                    sk = 2;
                }
            }
            diag += T;
            A.off[slot] = (sk == 1) ? -T : 0.0;
            A.col[slot] = c;
            A.slot_kind[slot] = sk;
            if (A.gfac) A.gfac[slot] = g;
        }
        A.diag[e] = diag;
        if (interior) atomicAdd(A.n_interior, (unsigned long long)interior);
    }
}

// s = sqrt(diag); also the smallest diagonal (as an ordered 64-bit pattern).
__global__ void k_sqrt_diag(const double* __restrict__ diag, int64_t nt, double* __restrict__ s,
                            float* __restrict__ s32, unsigned long long* dmin, int* err) {
    unsigned long long local = ~0ULL;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double d = diag[e];
        if (!(d > 0.0) || !isfinite(d)) {
            set_error(err, CPS_ERR_SINGULAR);
            s[e] = 1.0;
            s32[e] = 1.0f;
            local = 0ULL;
            continue;
        }
        const double r = sqrt(d);
        s[e] = r;
        s32[e] = (float)r;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
        local = bits < local ? bits : local;
    }
    atomicMin(dmin, local);
}

__global__ void k_scale_offdiag(const double* __restrict__ off, const int32_t* __restrict__ col,
                                const double* __restrict__ s, int64_t nt, double* __restrict__ a,
                                float* __restrict__ a32) {
    const int64_t n3 = 3 * nt;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n3;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k % nt;
        const int32_t c = col[k];
        const double v = off[k] / (s[e] * s[c]);
        a[k] = v;
        a32[k] = (float)v;
    }
}

// dxi/dtheta per cell for an isotropic cell field Kinv = exp(-theta) I:
// Xi = eps dt / (1 + s), s = nu eps dt Kinv, dXi/dtheta = Xi s / (1 + s).
// Flags a non-isotropic field by clearing *iso.
__global__ void k_dxi_dtheta(const double* __restrict__ eps, const double* __restrict__ kinv,
                             int64_t nt, double nu, double dt, bool logk,
                             double* __restrict__ dxi, int* iso) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double k = kinv_at(kinv, e, 0, logk);
        if (!logk && (kinv[3 * e + 1] != 0.0 || kinv[3 * e + 2] != k)) atomicExch(iso, 0);
        const double sv = nu * eps[e] * dt * k;
        const double xi = eps[e] * dt / (1.0 + sv);
        dxi[e] = xi * sv / (1.0 + sv);
    }
}

}  // namespace

template <typename T>
static int dev_alloc(cps_ctx ctx, T** p, size_t n) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n > 0 ? n : 1));
    if (e != cudaSuccess) {
        cps::set_error(ctx, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        *p = nullptr;
        return CPS_ERR_NOMEM;
    }
    return CPS_OK;
}

void free_sys(cps_sys s) {
    if (!s) return;
    free_cp2(s);
    free_cp1(s);
    // s->col lives inside s->a's allocation (one range for the L2 window)
    void* bufs[] = {s->s,     s->diag,  s->a,     s->a32,     s->s32,      s->gfac,
                    s->dxi,   s->slot_kind, s->perm, s->iperm, s->pa,  s->pcol,     s->pl,
                    s->pdinv, s->pdiag, s->ps, s->pa32, s->pl32, s->pdinv32, s->ps32,   s->wvec,
                    s->partials, s->st, s->gsync};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (s->hst) cudaFreeHost(s->hst);
    for (auto& ev : s->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& row : s->graph)
        for (auto& g : row)
            if (g) cudaGraphExecDestroy(g);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

static int fail(cps_ctx ctx, int code, const std::string& msg) {
    cps::set_error(ctx, msg);
    return code;
}

int assemble_impl(cps_ctx ctx, const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const int32_t* dirichlet, int64_t nb, const double* eps, const double* kinv,
                  int field_loc, int kind, double nu, double dt, cps_sys* out,
                  cudaStream_t stream) {
    *out = nullptr;
    if (nt <= 0 || nv < 3 || !xy || !tri || !eps || !kinv || nb < 0 || (nb > 0 && !dirichlet))
        return fail(ctx, CPS_ERR_ARG, "assemble: null pointer or bad size");
    if (nt > (int64_t)INT32_MAX / 3 || nv > (int64_t)INT32_MAX)
        return fail(ctx, CPS_ERR_ARG, "assemble: mesh too large for 32-bit indices");
    if (field_loc != CPS_PER_VERTEX && field_loc != CPS_PER_CELL && field_loc != CPS_PER_CELL_LOGK)
        return fail(ctx, CPS_ERR_ARG, "assemble: bad field_loc");
    const bool logk = field_loc == CPS_PER_CELL_LOGK;
    if (logk) field_loc = CPS_PER_CELL;
    if (kind != CPS_KIND_CP2 && kind != CPS_KIND_CP1_X && kind != CPS_KIND_CP1_Y)
        return fail(ctx, CPS_ERR_ARG, "assemble: bad kind");
    if (!(nu > 0.0) || !(dt > 0.0)) return fail(ctx, CPS_ERR_ARG, "assemble: nu and dt must be > 0");
    if (kind == CPS_KIND_CP2 && nb == 0)
        return fail(ctx, CPS_ERR_SINGULAR, "assemble: CP2 needs at least one Dirichlet side");

    cps_sys s = new cps_sys_s();
    s->ctx = ctx;
    s->nt = nt;
    s->nv = nv;
    s->kind = kind;
    s->field_loc = field_loc;
    s->logk = logk;
    s->nu = nu;
    s->dt = dt;
    const int64_t nf = field_loc == CPS_PER_VERTEX ? nv : nt;
    int rc = CPS_OK;
#define TRY_ALLOC(p, n)                        \
    do {                                       \
        rc = dev_alloc(ctx, &(p), (size_t)(n)); \
        if (rc) goto fail_free;                \
    } while (0)
    TRY_ALLOC(s->s, nt);
    TRY_ALLOC(s->diag, nt);
    // Off-diagonal values and columns in one allocation: a [3 nt] doubles,
    // then col [3 nt] int32 (256-byte aligned), so that one L2 access-policy
    // window covers the whole matrix the iteration streams.
    {
        const size_t a_elems = ((size_t)3 * nt + 31) / 32 * 32;
        const size_t col_elems = ((size_t)3 * nt * sizeof(int32_t) + sizeof(double) - 1) / sizeof(double);
        TRY_ALLOC(s->a, a_elems + col_elems);
        s->col = reinterpret_cast<int32_t*>(s->a + a_elems);
        s->mat_bytes = (a_elems + col_elems) * sizeof(double);
    }
    TRY_ALLOC(s->a32, 3 * nt);
    TRY_ALLOC(s->s32, nt);
    TRY_ALLOC(s->slot_kind, 3 * nt);
    {
        const int64_t vs = (nt + 31) / 32 * 32;     // 256-byte aligned slices
        TRY_ALLOC(s->wvec, 9 * vs);
        s->vec_stride = vs;
        double* w = s->wvec;
        s->wr = w;
        s->wp0 = w + vs;
        s->wq = w + 2 * vs;
        s->wy = w + 3 * vs;
        s->wp1 = w + 4 * vs;
        s->wz = w + 5 * vs;
        s->wb = w + 6 * vs;
        s->wx = w + 7 * vs;
        s->wbest = w + 8 * vs;
    }
    TRY_ALLOC(s->partials, (kNumPartials + 16) * kMaxGrid);
    TRY_ALLOC(s->st, 2);
    if (field_loc == CPS_PER_CELL && kind == CPS_KIND_CP2) {
        TRY_ALLOC(s->gfac, 3 * nt);
        TRY_ALLOC(s->dxi, nt);
    }
#undef TRY_ALLOC
    {
        cudaError_t e = cudaMallocHost((void**)&s->hst, 2 * sizeof(CgState));
        if (e != cudaSuccess) { rc = fail(ctx, CPS_ERR_NOMEM, "cudaMallocHost failed"); goto fail_free; }
        if (cudaEventCreateWithFlags(&s->ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev[1], cudaEventDisableTiming) != cudaSuccess) {
            rc = fail(ctx, CPS_ERR_CUDA, "cudaEventCreate failed");
            goto fail_free;
        }
    }
    s->grid = grid_for(ctx, nt);
    {
        // Scratch of the assembly, stream ordered and released before return.
        unsigned long long cap = 1;
        while (cap < (unsigned long long)(3 * nt)) cap <<= 1;
        cap <<= 1;   // load factor <= 1/4 of the 3 nt side slots (<= 1/2 of sides)
        unsigned long long* keys = nullptr;
        int32_t *id0 = nullptr, *id1 = nullptr, *nbr = nullptr;
        double *area = nullptr, *ccx = nullptr, *ccy = nullptr, *xi = nullptr, *off = nullptr;
        int* err = nullptr;
        unsigned long long* counters = nullptr;  // [0] interior slot count, [1] dmin bits
        int* iso = nullptr;
        int h_err = 0;
        unsigned long long h_cnt[2] = {0, 0};
        int h_iso = 1;
        auto A = [&](void** p, size_t bytes) { return cudaMallocAsync(p, bytes, stream); };
        cudaError_t ce = cudaSuccess;
        ce = A((void**)&keys, sizeof(unsigned long long) * cap);
        if (ce == cudaSuccess) ce = A((void**)&id0, sizeof(int32_t) * cap);
        if (ce == cudaSuccess) ce = A((void**)&id1, sizeof(int32_t) * cap);
        if (ce == cudaSuccess) ce = A((void**)&nbr, sizeof(int32_t) * 3 * nt);
        if (ce == cudaSuccess) ce = A((void**)&area, sizeof(double) * nt);
        if (ce == cudaSuccess) ce = A((void**)&ccx, sizeof(double) * nt);
        if (ce == cudaSuccess) ce = A((void**)&ccy, sizeof(double) * nt);
        if (ce == cudaSuccess) ce = A((void**)&xi, sizeof(double) * 3 * nf);
        if (ce == cudaSuccess) ce = A((void**)&off, sizeof(double) * 3 * nt);
        if (ce == cudaSuccess) ce = A((void**)&err, sizeof(int) * 2);
        if (ce == cudaSuccess) ce = A((void**)&counters, sizeof(unsigned long long) * 2);
        if (ce == cudaSuccess) {
            iso = err + 1;
            const int g3 = grid_for(ctx, 3 * nt);
            const int g1 = grid_for(ctx, nt);
            const int gf = grid_for(ctx, nf);
            cudaMemsetAsync(keys, 0xFF, sizeof(unsigned long long) * cap, stream);
            cudaMemsetAsync(id0, 0xFF, sizeof(int32_t) * cap, stream);
            cudaMemsetAsync(id1, 0xFF, sizeof(int32_t) * cap, stream);
            cudaMemsetAsync(err, 0, sizeof(int), stream);
            cudaMemsetAsync(iso, 0x00, sizeof(int), stream);
            cudaMemsetAsync(counters, 0, sizeof(unsigned long long), stream);
            cudaMemsetAsync(counters + 1, 0xFF, sizeof(unsigned long long), stream);
            cudaMemsetAsync(s->slot_kind, 0, sizeof(int32_t) * 3 * nt, stream);
            const int one = 1;
            cudaMemcpyAsync(iso, &one, sizeof(int), cudaMemcpyHostToDevice, stream);
            k_side_insert<<<g3, kBlock, 0, stream>>>(tri, nt, nv, keys, id0, id1, cap - 1, err);
            k_side_lookup<<<g3, kBlock, 0, stream>>>(tri, nt, nv, keys, id0, id1, cap - 1, nbr);
            k_cell_geometry<<<g1, kBlock, 0, stream>>>(xy, tri, nt, nv, area, ccx, ccy, err);
            k_xi<<<gf, kBlock, 0, stream>>>(eps, kinv, nf, nu, dt, logk, xi, err);
            if (nb > 0)
                k_mark_dirichlet<<<grid_for(ctx, nb), kBlock, 0, stream>>>(dirichlet, nb, nt, nbr,
                                                                         s->slot_kind, err);
            TransArgs ta;
            ta.xy = xy; ta.tri = tri; ta.nbr = nbr; ta.ccx = ccx; ta.ccy = ccy; ta.area = area;
            ta.xi = xi; ta.eps = eps; ta.kinv = kinv; ta.slot_kind = s->slot_kind;
            ta.diag = s->diag; ta.off = off; ta.col = s->col; ta.gfac = s->gfac;
            ta.n_interior = counters; ta.nt = nt; ta.kind = kind; ta.field_loc = field_loc;
            ta.nu = nu; ta.dt = dt; ta.err = err; ta.logk = logk;
            k_transmissibility<<<g1, kBlock, 0, stream>>>(ta);
            k_sqrt_diag<<<g1, kBlock, 0, stream>>>(s->diag, nt, s->s, s->s32, counters + 1, err);
            k_scale_offdiag<<<g3, kBlock, 0, stream>>>(off, s->col, s->s, nt, s->a, s->a32);
            if (s->dxi) k_dxi_dtheta<<<g1, kBlock, 0, stream>>>(eps, kinv, nt, nu, dt, logk, s->dxi, iso);
            s->assembly_launches = 8 + (nb > 0 ? 1 : 0) + (s->dxi ? 1 : 0);
            ce = cudaGetLastError();
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_iso, iso, sizeof(int), cudaMemcpyDeviceToHost, stream);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(h_cnt, counters, sizeof(h_cnt), cudaMemcpyDeviceToHost, stream);
        }
        void* scratch[] = {keys, id0, id1, nbr, area, ccx, ccy, xi, off, err, counters};
        for (void* p : scratch)
            if (p) cudaFreeAsync(p, stream);
        cudaError_t se = cudaStreamSynchronize(stream);
        if (ce == cudaSuccess) ce = se;
        if (ce != cudaSuccess) {
            rc = fail(ctx, ce == cudaErrorMemoryAllocation ? CPS_ERR_NOMEM : CPS_ERR_CUDA,
                      std::string("assemble: ") + cudaGetErrorString(ce));
            goto fail_free;
        }
        if (h_err != 0) {
            const char* what = h_err == CPS_ERR_NONMANIFOLD   ? "a side is shared by more than two cells"
                               : h_err == CPS_ERR_NONDELAUNAY ? "mesh is not Delaunay (d_{e,ep} <= 0)"
                               : h_err == CPS_ERR_ORIENTATION ? "a triangle is not counter-clockwise"
                               : h_err == CPS_ERR_SINGULAR    ? "a row has no positive diagonal"
                                                              : "bad mesh, boundary or field input";
            rc = fail(ctx, h_err, std::string("assemble: ") + what);
            goto fail_free;
        }
        s->n_interior = (int64_t)(h_cnt[0] / 2);
        std::memcpy(&s->diag_min, &h_cnt[1], sizeof(double));
        s->is_mmatrix = s->diag_min > 0.0 ? 1 : 0;   // off-diagonals are -T <= 0 by construction
        s->iso_cell = (s->dxi != nullptr) && h_iso == 1;
    }
    *out = s;
    return CPS_OK;
fail_free:
    cudaStreamSynchronize(stream);
    free_sys(s);
    return rc;
}

}  // namespace cps
