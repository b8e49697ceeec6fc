/*
 * cps_oracle.c -- plain, slow FP64 reference of the corrector-step solves.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle the CUDA library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the library never does.  It shares no code, header or
 * table with the CUDA path.
 *
 * What it computes (arXiv 2309.03543, Aricò et al.):
 *   1. mesh topology and geometry of the Delaunay triangulation (Sec. 3.1):
 *      cell areas, circumcentres, side lengths l_j, outward normals n_j and
 *      signed circumcentre distances d_{e,ep} (Eq. cs1_discr);
 *   2. the side tensor Xi = eps * M^-1 = eps*dt*(I + nu*eps*Kinv*dt)^-1
 *      (Eq. Cs2_4, with M = M0/dt and M0 = I + m dt, m = nu eps Kinv, Sec. 3.1)
 *      averaged over the two nodes of a side (Sec. 3.2);
 *   3. the CP2 matrix A_ee = sum_j l_j d_{j,n} / d_{e,ep},
 *      A_e,ep = -l_j d_{j,n} / d_{e,ep}, d_{j,n} = n_j . Xi_j n_j
 *      (Eq. CS2_sys_coeff, Eq. Cs2_5) and the CP1 matrix
 *      A_ee = Mbar_kk A_e + nu sum_j l_j/d_{e,ep}, A_e,ep = -nu l_j/d_{e,ep}
 *      (Eq. CS1_sys_coeff), as CSR;
 *   4. textbook preconditioned conjugate gradients (Hestenes-Stiefel) with
 *      Jacobi or incomplete Cholesky IC(0) in a given ordering -- the paper
 *      solves both corrector problems by PCG with incomplete Cholesky
 *      (Sec. 3.2.2, Sec. 3.2.3);
 *   5. a dense Cholesky solve for tiny meshes.
 *
 * Readings where the paper is silent (each is listed with its reason in the
 * design notes of the repository):
 *   - the side tensor is the mean of the two nodal tensors Xi_a, Xi_b (nodal
 *     fields) or of the two cell tensors (cell fields; a boundary side takes
 *     its own cell's);
 *   - d_{e,ep} = (c_ep - c_e) . n_j with n_j the outward normal of side j of e;
 *   - a Dirichlet side holds eta = 0 at its midpoint and adds
 *     l_j d_{j,n} / delta_j to the diagonal, delta_j = (m_j - c_e) . n_j;
 *     a no-flux side adds nothing;
 *   - Mbar of a cell is the mean of the nodal M = (I + nu eps Kinv dt)/dt.
 * Status codes mirror the library's: 0 ok, <0 error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NONMANIFOLD -2
#define OR_ERR_NONDELAUNAY -3
#define OR_ERR_ORIENTATION -4
#define OR_ERR_NOT_SPD -5
#define OR_ERR_NOT_CONVERGED -6
#define OR_ERR_SINGULAR -7
#define OR_ERR_NOMEM -8

#define OR_CP2 0
#define OR_CP1_X 1
#define OR_CP1_Y 2

#define OR_PER_VERTEX 0
#define OR_PER_CELL 1

#define OR_PC_NONE 0
#define OR_PC_JACOBI 1
#define OR_PC_IC0 2

/* ------------------------------------------------------------------ */
/* 1. Topology: which cell lies across each local side (Sec. 3.1: each  */
/*    side j of e is shared with at most one neighbour ep, side jp).    */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t lo, hi;   /* vertex ids of the side, lo < hi */
    int64_t id;       /* e*3 + j */
} side_key;

static int cmp_side(const void* a, const void* b) {
    const side_key* x = (const side_key*)a;
    const side_key* y = (const side_key*)b;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    return x->id < y->id ? -1 : (x->id > y->id);
}

/* nbr[e*3+j] = neighbour cell across local side j (joining vertices
 * (j+1)%3 and (j+2)%3) or -1 on the boundary. */
int or_topology(int64_t nt, const int32_t* tri, int32_t* nbr) {
    if (nt < 0 || (nt > 0 && (!tri || !nbr))) return OR_ERR_ARG;
    side_key* s = (side_key*)malloc(sizeof(side_key) * (size_t)(3 * nt + 1));
    if (!s) return OR_ERR_NOMEM;
    for (int64_t e = 0; e < nt; ++e)
        for (int j = 0; j < 3; ++j) {
            int64_t a = tri[e * 3 + (j + 1) % 3], b = tri[e * 3 + (j + 2) % 3];
            side_key* k = &s[e * 3 + j];
            k->lo = a < b ? a : b;
            k->hi = a < b ? b : a;
            k->id = e * 3 + j;
        }
    qsort(s, (size_t)(3 * nt), sizeof(side_key), cmp_side);
    for (int64_t i = 0; i < 3 * nt; ++i) nbr[i] = -1;
    int rc = OR_OK;
    for (int64_t i = 0; i < 3 * nt;) {
        int64_t k = i + 1;
        while (k < 3 * nt && s[k].lo == s[i].lo && s[k].hi == s[i].hi) ++k;
        if (k - i == 2) {
            nbr[s[i].id] = (int32_t)(s[i + 1].id / 3);
            nbr[s[i + 1].id] = (int32_t)(s[i].id / 3);
        } else if (k - i > 2) {
            rc = OR_ERR_NONMANIFOLD;
        }
        i = k;
    }
    free(s);
    return rc;
}

/* ------------------------------------------------------------------ */
/* 2. Geometry (Sec. 3.1; Eq. cs1_discr for d_{e,ep}).                  */
/* ------------------------------------------------------------------ */

/* area[e]; cc[2e..] circumcentre; per local side (e*3+j): len, nrm (2),
 * dist = d_{e,ep} for an interior side, the circumcentre-to-side distance
 * delta_j for a boundary side. */
int or_geometry(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                const int32_t* nbr, double* area, double* cc, double* len,
                double* nrm, double* dist) {
    for (int64_t e = 0; e < nt; ++e) {
        for (int k = 0; k < 3; ++k)
            if (tri[e * 3 + k] < 0 || tri[e * 3 + k] >= nv) return OR_ERR_ARG;
        const double* a = &xy[2 * (int64_t)tri[e * 3 + 0]];
        const double* b = &xy[2 * (int64_t)tri[e * 3 + 1]];
        const double* c = &xy[2 * (int64_t)tri[e * 3 + 2]];
        double bx = b[0] - a[0], by = b[1] - a[1];
        double cx = c[0] - a[0], cy = c[1] - a[1];
        double cross = bx * cy - by * cx;
        if (!(cross > 0.0)) return OR_ERR_ORIENTATION;
        area[e] = 0.5 * cross;
        /* circumcentre: the point equidistant from a, b, c */
        double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
        cc[2 * e + 0] = a[0] + (cy * b2 - by * c2) / (2.0 * cross);
        cc[2 * e + 1] = a[1] + (bx * c2 - cx * b2) / (2.0 * cross);
    }
    for (int64_t e = 0; e < nt; ++e)
        for (int j = 0; j < 3; ++j) {
            const double* p = &xy[2 * (int64_t)tri[e * 3 + (j + 1) % 3]];
            const double* q = &xy[2 * (int64_t)tri[e * 3 + (j + 2) % 3]];
            double tx = q[0] - p[0], ty = q[1] - p[1];
            double l = sqrt(tx * tx + ty * ty);
            double nx = ty / l, ny = -tx / l; /* outward for a CCW triangle */
            len[e * 3 + j] = l;
            nrm[(e * 3 + j) * 2 + 0] = nx;
            nrm[(e * 3 + j) * 2 + 1] = ny;
            int32_t ep = nbr[e * 3 + j];
            double d;
            if (ep >= 0) {
                d = (cc[2 * ep] - cc[2 * e]) * nx + (cc[2 * ep + 1] - cc[2 * e + 1]) * ny;
            } else {
                double mx = 0.5 * (p[0] + q[0]), my = 0.5 * (p[1] + q[1]);
                d = (mx - cc[2 * e]) * nx + (my - cc[2 * e + 1]) * ny;
            }
            dist[e * 3 + j] = d;
        }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 3. Xi = eps * M^-1 = eps*dt*(I + nu*eps*dt*Kinv)^-1 (Eq. Cs2_4).     */
/* ------------------------------------------------------------------ */

static void xi_tensor(double eps, const double* kinv, double nu, double dt, double* xi) {
    double c = nu * eps * dt;
    double m00 = 1.0 + c * kinv[0], m01 = c * kinv[1], m11 = 1.0 + c * kinv[2];
    double det = m00 * m11 - m01 * m01;
    double s = eps * dt / det;
    xi[0] = s * m11;
    xi[1] = -s * m01;
    xi[2] = s * m00;
}

void or_xi(int64_t n, const double* eps, const double* kinv, double nu, double dt,
           double* xi) {
    for (int64_t i = 0; i < n; ++i) xi_tensor(eps[i], &kinv[3 * i], nu, dt, &xi[3 * i]);
}

/* ------------------------------------------------------------------ */
/* 4. Assembly into CSR (Eq. CS2_sys_coeff, Eq. CS1_sys_coeff).         */
/* ------------------------------------------------------------------ */

/* Per local side coefficient T (the off-diagonal is -T).  For a Dirichlet
 * side T is the diagonal contribution l d_n / delta.  sigma[e] is the CP1
 * mass term Mbar_kk A_e (0 for CP2). */
int or_side_coefficients(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                         const int32_t* nbr, const int32_t* dirichlet, int64_t nb,
                         const double* eps, const double* kinv, int field_loc,
                         int kind, double nu, double dt, double* T, double* sigma,
                         int32_t* is_dirichlet) {
    if (nt <= 0 || !xy || !tri || !nbr || !T || !sigma || !is_dirichlet) return OR_ERR_ARG;
    if (field_loc != OR_PER_VERTEX && field_loc != OR_PER_CELL) return OR_ERR_ARG;
    if (kind < OR_CP2 || kind > OR_CP1_Y) return OR_ERR_ARG;
    int64_t nf = field_loc == OR_PER_VERTEX ? nv : nt;
    double* area = (double*)malloc(sizeof(double) * nt);
    double* cc = (double*)malloc(sizeof(double) * 2 * nt);
    double* len = (double*)malloc(sizeof(double) * 3 * nt);
    double* nrm = (double*)malloc(sizeof(double) * 6 * nt);
    double* dist = (double*)malloc(sizeof(double) * 3 * nt);
    double* xi = (double*)malloc(sizeof(double) * 3 * nf);
    int rc = OR_OK;
    if (!area || !cc || !len || !nrm || !dist || !xi) { rc = OR_ERR_NOMEM; goto done; }
    rc = or_geometry(nv, xy, nt, tri, nbr, area, cc, len, nrm, dist);
    if (rc) goto done;
    or_xi(nf, eps, kinv, nu, dt, xi);
    for (int64_t i = 0; i < 3 * nt; ++i) is_dirichlet[i] = 0;
    for (int64_t k = 0; k < nb; ++k) {
        int64_t s = dirichlet[k];
        if (s < 0 || s >= 3 * nt || nbr[s] >= 0) { rc = OR_ERR_ARG; goto done; }
        is_dirichlet[s] = 1;
    }
    for (int64_t e = 0; e < nt; ++e) {
        for (int j = 0; j < 3; ++j) {
            int64_t s = e * 3 + j;
            int32_t ep = nbr[s];
            double d = dist[s];
            T[s] = 0.0;
            if (ep < 0 && !is_dirichlet[s]) continue; /* no-flux side */
            if (!(d > 1e-12 * len[s])) { rc = OR_ERR_NONDELAUNAY; goto done; }
            if (kind == OR_CP2) {
                double xs[3];
                if (field_loc == OR_PER_VERTEX) {
                    const double* xa = &xi[3 * (int64_t)tri[e * 3 + (j + 1) % 3]];
                    const double* xb = &xi[3 * (int64_t)tri[e * 3 + (j + 2) % 3]];
                    for (int c = 0; c < 3; ++c) xs[c] = 0.5 * (xa[c] + xb[c]);
                } else if (ep >= 0) {
                    for (int c = 0; c < 3; ++c) xs[c] = 0.5 * (xi[3 * e + c] + xi[3 * (int64_t)ep + c]);
                } else {
                    for (int c = 0; c < 3; ++c) xs[c] = xi[3 * e + c];
                }
                double nx = nrm[2 * s], ny = nrm[2 * s + 1];
                double dn = xs[0] * nx * nx + 2.0 * xs[1] * nx * ny + xs[2] * ny * ny;
                T[s] = len[s] * dn / d;
            } else {
                T[s] = nu * len[s] / d;
            }
        }
        sigma[e] = 0.0;
        if (kind != OR_CP2) {
            /* Mbar = mean over the cell's nodes of M = (I + nu eps Kinv dt)/dt */
            int comp = kind == OR_CP1_X ? 0 : 2;
            double mkk;
            if (field_loc == OR_PER_VERTEX) {
                mkk = 0.0;
                for (int k = 0; k < 3; ++k) {
                    int64_t v = tri[e * 3 + k];
                    mkk += (1.0 + nu * eps[v] * kinv[3 * v + comp] * dt) / dt;
                }
                mkk /= 3.0;
            } else {
                mkk = (1.0 + nu * eps[e] * kinv[3 * e + comp] * dt) / dt;
            }
            sigma[e] = mkk * area[e];
        }
    }
done:
    free(area); free(cc); free(len); free(nrm); free(dist); free(xi);
    return rc;
}

/* CSR with the diagonal first in each row, then the neighbours in local side
 * order.  rowptr[nt+1], col/val sized 4*nt.  Returns nnz through *nnz. */
int or_assemble_csr(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                    const int32_t* dirichlet, int64_t nb, const double* eps,
                    const double* kinv, int field_loc, int kind, double nu, double dt,
                    int64_t* rowptr, int32_t* col, double* val, int64_t* nnz) {
    int32_t* nbr = (int32_t*)malloc(sizeof(int32_t) * 3 * (nt > 0 ? nt : 1));
    double* T = (double*)malloc(sizeof(double) * 3 * (nt > 0 ? nt : 1));
    double* sigma = (double*)malloc(sizeof(double) * (nt > 0 ? nt : 1));
    int32_t* isd = (int32_t*)malloc(sizeof(int32_t) * 3 * (nt > 0 ? nt : 1));
    int rc = OR_OK;
    if (!nbr || !T || !sigma || !isd) { rc = OR_ERR_NOMEM; goto done; }
    rc = or_topology(nt, tri, nbr);
    if (rc) goto done;
    rc = or_side_coefficients(nv, xy, nt, tri, nbr, dirichlet, nb, eps, kinv, field_loc,
                              kind, nu, dt, T, sigma, isd);
    if (rc) goto done;
    if (kind == OR_CP2 && nb == 0) { rc = OR_ERR_SINGULAR; goto done; }
    int64_t k = 0;
    for (int64_t e = 0; e < nt; ++e) {
        rowptr[e] = k;
        double diag = sigma[e];
        for (int j = 0; j < 3; ++j) diag += T[e * 3 + j];
        col[k] = (int32_t)e;
        val[k] = diag;
        ++k;
        for (int j = 0; j < 3; ++j) {
            int32_t ep = nbr[e * 3 + j];
            if (ep < 0) continue;
            col[k] = ep;
            val[k] = -T[e * 3 + j];
            ++k;
        }
    }
    rowptr[nt] = k;
    *nnz = k;
done:
    free(nbr); free(T); free(sigma); free(isd);
    return rc;
}

/* ------------------------------------------------------------------ */
/* 5. Preconditioned conjugate gradients (Sec. 3.2.2: PCG with          */
/*    incomplete Cholesky).                                            */
/* ------------------------------------------------------------------ */

static void csr_matvec(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                       const double* x, double* y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* IC(0) factor of P A P^T on the sparsity pattern of its lower triangle.
 * perm[new] = old (NULL: natural order).  Output: lower factor L in CSR with
 * the diagonal as the LAST entry of each row, columns ascending. */
typedef struct {
    int64_t n;
    int64_t* rp;
    int32_t* ci;
    double* v;
    int32_t* perm;   /* new -> old */
} ic0_factor;

typedef struct {
    int64_t c;
    double v;
} col_val;

static int cmp_col_val(const void* a, const void* b) {
    const col_val* x = (const col_val*)a;
    const col_val* y = (const col_val*)b;
    return x->c < y->c ? -1 : (x->c > y->c);
}

static void ic0_free(ic0_factor* f) {
    free(f->rp); free(f->ci); free(f->v); free(f->perm);
    memset(f, 0, sizeof(*f));
}

static int ic0_build(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                     const int32_t* perm_in, ic0_factor* f) {
    memset(f, 0, sizeof(*f));
    f->n = n;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    int32_t* iperm = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    if (!perm || !iperm) { free(perm); free(iperm); return OR_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) perm[i] = perm_in ? perm_in[i] : (int32_t)i;
    for (int64_t i = 0; i < n; ++i) iperm[i] = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (perm[i] < 0 || perm[i] >= n || iperm[perm[i]] >= 0) {
            free(perm); free(iperm); return OR_ERR_ARG;
        }
        iperm[perm[i]] = (int32_t)i;
    }
    /* lower triangle of B = P A P^T, row by row, columns sorted */
    int64_t cap = rp[n];
    f->rp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    f->ci = (int32_t*)malloc(sizeof(int32_t) * (cap > 0 ? cap : 1));
    f->v = (double*)malloc(sizeof(double) * (cap > 0 ? cap : 1));
    col_val* tmp = (col_val*)malloc(sizeof(col_val) * 64);
    if (!f->rp || !f->ci || !f->v || !tmp) { free(tmp); free(iperm); f->perm = perm; ic0_free(f); return OR_ERR_NOMEM; }
    f->perm = perm;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t old = perm[i];
        int64_t m = 0;
        f->rp[i] = k;
        for (int64_t q = rp[old]; q < rp[old + 1]; ++q) {
            int64_t c = iperm[ci[q]];
            if (c <= i) {
                if (m == 64) { free(tmp); free(iperm); ic0_free(f); return OR_ERR_ARG; }
                tmp[m].c = c;
                tmp[m].v = v[q];
                ++m;
            }
        }
        qsort(tmp, (size_t)m, sizeof(col_val), cmp_col_val);
        for (int64_t q = 0; q < m; ++q) {
            f->ci[k] = (int32_t)tmp[q].c;
            f->v[k] = tmp[q].v;
            ++k;
        }
        if (m == 0 || tmp[m - 1].c != i) { free(tmp); free(iperm); ic0_free(f); return OR_ERR_ARG; }
    }
    f->rp[n] = k;
    free(tmp);
    free(iperm);
    /* Incomplete Cholesky with no fill: for each row i and each k < i in its
     * pattern, L_ik = (b_ik - sum_{m<k} L_im L_km) / L_kk over the common
     * pattern; L_ii = sqrt(b_ii - sum_{k<i} L_ik^2). */
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = f->rp[i]; p < f->rp[i + 1] - 1; ++p) {
            int64_t kk = f->ci[p];
            double s = f->v[p];
            /* common pattern of rows i and kk below column kk */
            int64_t a = f->rp[i], b = f->rp[kk];
            while (a < p && b < f->rp[kk + 1] - 1) {
                if (f->ci[a] == f->ci[b]) { s -= f->v[a] * f->v[b]; ++a; ++b; }
                else if (f->ci[a] < f->ci[b]) ++a;
                else ++b;
            }
            f->v[p] = s / f->v[f->rp[kk + 1] - 1];
        }
        int64_t dpos = f->rp[i + 1] - 1;
        double s = f->v[dpos];
        for (int64_t p = f->rp[i]; p < dpos; ++p) s -= f->v[p] * f->v[p];
        if (!(s > 0.0)) { ic0_free(f); return OR_ERR_NOT_SPD; }
        f->v[dpos] = sqrt(s);
    }
    return OR_OK;
}

/* z = (L L^T)^-1 r in the original ordering; w is scratch of size n. */
static void ic0_apply(const ic0_factor* f, const double* r, double* z, double* w) {
    int64_t n = f->n;
    for (int64_t i = 0; i < n; ++i) {              /* L y = P r */
        double s = r[f->perm[i]];
        int64_t dpos = f->rp[i + 1] - 1;
        for (int64_t p = f->rp[i]; p < dpos; ++p) s -= f->v[p] * w[f->ci[p]];
        w[i] = s / f->v[dpos];
    }
    for (int64_t i = n - 1; i >= 0; --i) {         /* L^T u = y (column sweep) */
        int64_t dpos = f->rp[i + 1] - 1;
        w[i] /= f->v[dpos];
        for (int64_t p = f->rp[i]; p < dpos; ++p) w[f->ci[p]] -= f->v[p] * w[i];
    }
    for (int64_t i = 0; i < n; ++i) z[f->perm[i]] = w[i];
}

/* stats[0] = iterations, stats[1] = true relative residual ||b-Ax||/||b||,
 * stats[2] = recursive relative residual at exit. */
int or_pcg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
           const double* b, double* x, double rtol, int64_t maxit, int precond,
           const int32_t* perm, double* stats) {
    if (n < 0 || !stats) return OR_ERR_ARG;
    stats[0] = 0; stats[1] = 0; stats[2] = 0;
    if (n == 0) return OR_OK;
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* w = (double*)malloc(sizeof(double) * n);
    double* dinv = (double*)malloc(sizeof(double) * n);
    ic0_factor f;
    memset(&f, 0, sizeof(f));
    int rc = OR_OK;
    if (!r || !z || !p || !q || !w || !dinv) { rc = OR_ERR_NOMEM; goto done; }
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (ci[k] == i) d += v[k];
        if (!(d > 0.0)) { rc = OR_ERR_NOT_SPD; goto done; }
        dinv[i] = 1.0 / d;
    }
    if (precond == OR_PC_IC0) {
        rc = ic0_build(n, rp, ci, v, perm, &f);
        if (rc) goto done;
    } else if (precond != OR_PC_NONE && precond != OR_PC_JACOBI) {
        rc = OR_ERR_ARG; goto done;
    }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        goto done;
    }
    csr_matvec(n, rp, ci, v, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
#define APPLY_M(src, dst) do { \
        if (precond == OR_PC_IC0) ic0_apply(&f, src, dst, w); \
        else if (precond == OR_PC_JACOBI) for (int64_t i_ = 0; i_ < n; ++i_) dst[i_] = dinv[i_] * src[i_]; \
        else for (int64_t i_ = 0; i_ < n; ++i_) dst[i_] = src[i_]; } while (0)
    APPLY_M(r, z);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i];
    double rho = dot(n, r, z);
    double relres = sqrt(dot(n, r, r)) / bnorm;
    int64_t it = 0;
    while (relres > rtol && it < maxit) {
        csr_matvec(n, rp, ci, v, p, q);
        double gamma = dot(n, p, q);
        if (!(gamma > 0.0)) { rc = OR_ERR_NOT_SPD; break; }
        double alpha = rho / gamma;
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        ++it;
        relres = sqrt(dot(n, r, r)) / bnorm;
        if (relres <= rtol) break;
        APPLY_M(r, z);
        double rho_new = dot(n, r, z);
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
#undef APPLY_M
    stats[0] = (double)it;
    stats[2] = relres;
    csr_matvec(n, rp, ci, v, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    stats[1] = sqrt(dot(n, r, r)) / bnorm;
    if (rc == OR_OK && relres > rtol) rc = OR_ERR_NOT_CONVERGED;
done:
    ic0_free(&f);
    free(r); free(z); free(p); free(q); free(w); free(dinv);
    return rc;
}

/* y = A x for a CSR matrix (exported for tests and the adjoint). */
void or_matvec(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
               const double* x, double* y) {
    csr_matvec(n, rp, ci, v, x, y);
}

/* ------------------------------------------------------------------ */
/* 6. Dense Cholesky (textbook, for tiny meshes).  A is row-major n*n,   */
/*    overwritten by its factor; b is overwritten by the solution.     */
/* ------------------------------------------------------------------ */
int or_dense_cholesky_solve(int64_t n, double* A, double* b) {
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return OR_ERR_NOT_SPD;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int64_t i = 0; i < n; ++i) {              /* L y = b */
        double s = b[i];
        for (int64_t k = 0; k < i; ++k) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {         /* L^T x = y */
        double s = b[i];
        for (int64_t k = i + 1; k < n; ++k) s -= A[k * n + i] * b[k];
        b[i] = s / A[i * n + i];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 7. Adjoint of one solve A(T) x = b with respect to the side          */
/*    coefficients.  A = sum_interior T (e_e - e_ep)(e_e - e_ep)^T      */
/*    + sum_Dirichlet T e_e e_e^T (+ diag sigma), so with A lambda = g:  */
/*    dL/dT_side = -(lambda_e - lambda_ep)(x_e - x_ep) (interior) and   */
/*    -lambda_e x_e (Dirichlet).  Each interior side appears from both  */
/*    of its cells with the same value.                                */
/* ------------------------------------------------------------------ */
void or_side_gradient(int64_t nt, const int32_t* nbr, const int32_t* is_dirichlet,
                      const double* lambda, const double* x, double* dT) {
    for (int64_t e = 0; e < nt; ++e)
        for (int j = 0; j < 3; ++j) {
            int64_t s = e * 3 + j;
            int32_t ep = nbr[s];
            if (ep >= 0) dT[s] = -(lambda[e] - lambda[ep]) * (x[e] - x[ep]);
            else if (is_dirichlet[s]) dT[s] = -lambda[e] * x[e];
            else dT[s] = 0.0;
        }
}

/* Chain dL/dT to the per-cell log-permeability theta of an isotropic cell
 * field Kinv = exp(-theta) I (CP2, cell fields).  With xi_c the scalar of
 * Xi_c = eps dt / (1 + s) I, s = nu eps dt exp(-theta):
 *   dxi/dtheta = xi s / (1 + s);
 *   interior side: T = (l/d) (xi_e + xi_ep)/2  ->  dT/dxi_e = l/(2d);
 *   Dirichlet side: T = l xi_e / delta          ->  dT/dxi_e = l/delta. */
int or_theta_gradient(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                      const int32_t* nbr, const int32_t* is_dirichlet, const double* eps,
                      const double* theta, double nu, double dt, const double* dT,
                      double* dtheta) {
    double* area = (double*)malloc(sizeof(double) * nt);
    double* cc = (double*)malloc(sizeof(double) * 2 * nt);
    double* len = (double*)malloc(sizeof(double) * 3 * nt);
    double* nrm = (double*)malloc(sizeof(double) * 6 * nt);
    double* dist = (double*)malloc(sizeof(double) * 3 * nt);
    int rc = OR_OK;
    if (!area || !cc || !len || !nrm || !dist) { rc = OR_ERR_NOMEM; goto done; }
    rc = or_geometry(nv, xy, nt, tri, nbr, area, cc, len, nrm, dist);
    if (rc) goto done;
    for (int64_t e = 0; e < nt; ++e) {
        double s = nu * eps[e] * dt * exp(-theta[e]);
        double xi = eps[e] * dt / (1.0 + s);
        double dxi = xi * s / (1.0 + s);
        double g = 0.0;
        for (int j = 0; j < 3; ++j) {
            int64_t k = e * 3 + j;
            if (nbr[k] >= 0) g += dT[k] * len[k] / (2.0 * dist[k]);
            else if (is_dirichlet[k]) g += dT[k] * len[k] / dist[k];
        }
        dtheta[e] = g * dxi;
    }
done:
    free(area); free(cc); free(len); free(nrm); free(dist);
    return rc;
}

/* ------------------------------------------------------------------ */
/* 8. The CP2 step around the two solves (Sec. 3.2.3, App. A, App. C).  */
/*                                                                      */
/* Sign convention: every flux below is the PHYSICAL flux leaving cell  */
/* e through its local side j (n_j outward from e).  The velocity at    */
/* the end of the step has outward side fluxes Q_j = Fbar_j + Phi_j,    */
/* Phi_j the flux of Xi_j grad eta (Eq. Cs2_3, Eq. Cs2_5), and the     */
/* mass balance sum_j Q_j = 0 gives the two systems of Eq. Cs2_7:       */
/*   A eta~ = sum_j Fbar_j,  A eta = sum_j Fbar_j + sum_j tau_j(eta~),  */
/* with (A eta)_e = sum_j T_j (eta_e - eta_ep) (TPFA part of -Phi) and  */
/* tau_j the tangential part of Phi_j evaluated with eta~.              */
/* Readings (the paper is ambiguous or inconsistent here):              */
/*  - the m-terms carry the sign of Eq. Cs2_6 / Eq. A3.2, the only one   */
/*    with which the side fluxes of e and ep cancel (as the text after  */
/*    Eq. eta_flux states); Eq. eta_flux and the second right-hand      */
/*    side print the opposite sign;                                     */
/*  - d_{tau,n_l} alpha_l is the component of d_{j,tau} along n_l in    */
/*    the co-normal decomposition d_{j,tau} = c_1 n_1 + c_2 n_2 of      */
/*    Eq. A3.1 (oblique components); with it the flux is exact for      */
/*    linear eta under a uniform tensor;                                */
/*  - the two one-sided estimates (from e and from ep) are averaged;    */
/*    an estimate that needs the normal derivative across a no-flux     */
/*    side does not exist and the other is used alone (none: tau = 0);  */
/*    across a Dirichlet side eta = 0 at its midpoint;                  */
/*  - the extra 1/2 of Eq. A3.3 is not applied (Eq. Cs2_6 is followed). */
/* ------------------------------------------------------------------ */

/* Eq. flux_k_+_2/3: Fbar_j = ((u_e.n_j) A_ep - (u_ep.n_jp) A_e)/(A_e + A_ep)
 * l_j, with n_jp the outward normal of ep on the shared side.  Reading for
 * the boundary: a no-flux side carries no flux; a Dirichlet side carries
 * e's own normal flux (u_e.n_j) l_j.  u is [2*nt]: x components, then y. */
int or_cp2_mean_flux(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                     const int32_t* nbr, const int32_t* is_dirichlet, const double* u,
                     double* fbar) {
    double* area = (double*)malloc(sizeof(double) * nt);
    double* cc = (double*)malloc(sizeof(double) * 2 * nt);
    double* len = (double*)malloc(sizeof(double) * 3 * nt);
    double* nrm = (double*)malloc(sizeof(double) * 6 * nt);
    double* dist = (double*)malloc(sizeof(double) * 3 * nt);
    int rc = OR_OK;
    if (!area || !cc || !len || !nrm || !dist) { rc = OR_ERR_NOMEM; goto done; }
    rc = or_geometry(nv, xy, nt, tri, nbr, area, cc, len, nrm, dist);
    if (rc) goto done;
    for (int64_t e = 0; e < nt; ++e)
        for (int j = 0; j < 3; ++j) {
            int64_t s = e * 3 + j;
            int32_t ep = nbr[s];
            double une = u[e] * nrm[2 * s] + u[nt + e] * nrm[2 * s + 1];
            if (ep >= 0) {
                int jp = 0;
                while (jp < 3 && nbr[(int64_t)ep * 3 + jp] != (int32_t)e) ++jp;
                if (jp == 3) { rc = OR_ERR_NONMANIFOLD; goto done; }
                int64_t sp = (int64_t)ep * 3 + jp;
                double unp = u[ep] * nrm[2 * sp] + u[nt + ep] * nrm[2 * sp + 1];
                fbar[s] = (une * area[ep] - unp * area[e]) / (area[e] + area[ep]) * len[s];
            } else if (is_dirichlet[s]) {
                fbar[s] = une * len[s];
            } else {
                fbar[s] = 0.0;
            }
        }
done:
    free(area); free(cc); free(len); free(nrm); free(dist);
    return rc;
}

/* Side tensor Xi_j (xx, xy, yy) of local side s of cell e, the same
 * average as the matrix uses (Sec. 3.2). */
static void side_tensor(const double* xi, const int32_t* tri, const int32_t* nbr,
                        int field_loc, int64_t e, int j, double* xs) {
    int64_t s = e * 3 + j;
    if (field_loc == OR_PER_VERTEX) {
        const double* xa = &xi[3 * (int64_t)tri[e * 3 + (j + 1) % 3]];
        const double* xb = &xi[3 * (int64_t)tri[e * 3 + (j + 2) % 3]];
        for (int c = 0; c < 3; ++c) xs[c] = 0.5 * (xa[c] + xb[c]);
    } else if (nbr[s] >= 0) {
        for (int c = 0; c < 3; ++c) xs[c] = 0.5 * (xi[3 * e + c] + xi[3 * (int64_t)nbr[s] + c]);
    } else {
        for (int c = 0; c < 3; ++c) xs[c] = xi[3 * e + c];
    }
}

/* One-sided estimate of d_tau . grad(eta) from cell c, using the normal
 * derivatives across c's two sides other than local side jc: d_tau =
 * c1 n1 + c2 n2 (Cramer's rule on the 2x2 system), n_k . grad(eta) ~
 * (eta_across - eta_c)/d (Eq. A3.2).  Returns 0 and leaves *est alone if a
 * needed side is a no-flux side. */
static int one_sided(int64_t c, int jc, const double* dtau, const int32_t* nbr,
                     const int32_t* is_dirichlet, const double* nrm, const double* dist,
                     const double* eta, double* est) {
    int64_t s1 = c * 3 + (jc + 1) % 3, s2 = c * 3 + (jc + 2) % 3;
    if ((nbr[s1] < 0 && !is_dirichlet[s1]) || (nbr[s2] < 0 && !is_dirichlet[s2])) return 0;
    double n1x = nrm[2 * s1], n1y = nrm[2 * s1 + 1];
    double n2x = nrm[2 * s2], n2y = nrm[2 * s2 + 1];
    double det = n1x * n2y - n1y * n2x;
    double c1 = (dtau[0] * n2y - dtau[1] * n2x) / det;
    double c2 = (n1x * dtau[1] - n1y * dtau[0]) / det;
    double e1 = nbr[s1] >= 0 ? eta[nbr[s1]] : 0.0;
    double e2 = nbr[s2] >= 0 ? eta[nbr[s2]] : 0.0;
    *est = c1 * (e1 - eta[c]) / dist[s1] + c2 * (e2 - eta[c]) / dist[s2];
    return 1;
}

/* tau_j: tangential part of the outward flux of Xi_j grad(eta) through
 * local side j of e (Eq. Cs2_6, Eq. eta_flux, App. C): d_j = Xi_j n_j,
 * d_{j,tau} = d_j - (d_j.n_j) n_j, tau_j = l_j * mean of the one-sided
 * estimates of d_{j,tau} . grad(eta) from e and from ep.  Zero on a
 * no-flux side.  kinv/eps as for or_side_coefficients (CP2 tensor). */
int or_cp2_tangential_flux(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                           const int32_t* nbr, const int32_t* is_dirichlet, const double* eps,
                           const double* kinv, int field_loc, double nu, double dt,
                           const double* eta, double* tau) {
    if (field_loc != OR_PER_VERTEX && field_loc != OR_PER_CELL) return OR_ERR_ARG;
    int64_t nf = field_loc == OR_PER_VERTEX ? nv : nt;
    double* area = (double*)malloc(sizeof(double) * nt);
    double* cc = (double*)malloc(sizeof(double) * 2 * nt);
    double* len = (double*)malloc(sizeof(double) * 3 * nt);
    double* nrm = (double*)malloc(sizeof(double) * 6 * nt);
    double* dist = (double*)malloc(sizeof(double) * 3 * nt);
    double* xi = (double*)malloc(sizeof(double) * 3 * nf);
    int rc = OR_OK;
    if (!area || !cc || !len || !nrm || !dist || !xi) { rc = OR_ERR_NOMEM; goto done; }
    rc = or_geometry(nv, xy, nt, tri, nbr, area, cc, len, nrm, dist);
    if (rc) goto done;
    or_xi(nf, eps, kinv, nu, dt, xi);
    for (int64_t e = 0; e < nt; ++e)
        for (int j = 0; j < 3; ++j) {
            int64_t s = e * 3 + j;
            int32_t ep = nbr[s];
            tau[s] = 0.0;
            if (ep < 0 && !is_dirichlet[s]) continue;
            double xs[3];
            side_tensor(xi, tri, nbr, field_loc, e, j, xs);
            double nx = nrm[2 * s], ny = nrm[2 * s + 1];
            double dx = xs[0] * nx + xs[1] * ny, dy = xs[1] * nx + xs[2] * ny;
            double dn = dx * nx + dy * ny;
            double dtau[2] = {dx - dn * nx, dy - dn * ny};
            double sum = 0.0, est;
            int count = 0;
            if (one_sided(e, j, dtau, nbr, is_dirichlet, nrm, dist, eta, &est)) {
                sum += est;
                ++count;
            }
            if (ep >= 0) {
                int jp = 0;
                while (jp < 3 && nbr[(int64_t)ep * 3 + jp] != (int32_t)e) ++jp;
                if (jp == 3) { rc = OR_ERR_NONMANIFOLD; goto done; }
                if (one_sided(ep, jp, dtau, nbr, is_dirichlet, nrm, dist, eta, &est)) {
                    sum += est;
                    ++count;
                }
            }
            if (count > 0) tau[s] = len[s] * sum / count;
        }
done:
    free(area); free(cc); free(len); free(nrm); free(dist); free(xi);
    return rc;
}

/* End of the step.  Outward side fluxes Q_j = Fbar_j + Phi_j with
 * Phi_j = -T_j (eta_e - eta_ep) + tau_j (Dirichlet side: eta_ep = 0;
 * no-flux side: Q_j = 0).  Cell velocity (Eq. RT0): the RT0 field
 * sum_j Q_j (x - x_j)/(2 A_e), x_j the node opposite side j, taken at the
 * centroid (its mean over the cell; the field is constant in e when
 * sum_j Q_j = 0).  Eq. grad_PSI: g_next = g_k + Mbar_e (u_next - u23), g the
 * cell field eps grad(Psi), Mbar_e the mean over the cell's nodes of
 * M = (I + nu eps Kinv dt)/dt (the cell's own M for cell fields).
 * Q [nt*3] (e*3+j); u23, g_k, u_next, g_next [2*nt] (x, then y). */
int or_cp2_update(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                  const int32_t* nbr, const int32_t* is_dirichlet, const double* eps,
                  const double* kinv, int field_loc, double nu, double dt, const double* fbar,
                  const double* T, const double* tau, const double* eta, const double* u23,
                  const double* g_k, double* Q, double* u_next, double* g_next) {
    if (field_loc != OR_PER_VERTEX && field_loc != OR_PER_CELL) return OR_ERR_ARG;
    for (int64_t e = 0; e < nt; ++e) {
        for (int k = 0; k < 3; ++k)
            if (tri[e * 3 + k] < 0 || tri[e * 3 + k] >= nv) return OR_ERR_ARG;
        const double* p[3];
        for (int k = 0; k < 3; ++k) p[k] = &xy[2 * (int64_t)tri[e * 3 + k]];
        double a2 = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) -
                    (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]); /* 2 A_e */
        double gx = (p[0][0] + p[1][0] + p[2][0]) / 3.0;
        double gy = (p[0][1] + p[1][1] + p[2][1]) / 3.0;
        double ux = 0.0, uy = 0.0;
        for (int j = 0; j < 3; ++j) {
            int64_t s = e * 3 + j;
            int32_t ep = nbr[s];
            double q;
            if (ep >= 0) q = fbar[s] - T[s] * (eta[e] - eta[ep]) + tau[s];
            else if (is_dirichlet[s]) q = fbar[s] - T[s] * eta[e] + tau[s];
            else q = 0.0;
            Q[s] = q;
            ux += q * (gx - p[j][0]) / a2;
            uy += q * (gy - p[j][1]) / a2;
        }
        u_next[e] = ux;
        u_next[nt + e] = uy;
        double m00, m01, m11;
        if (field_loc == OR_PER_VERTEX) {
            m00 = m01 = m11 = 0.0;
            for (int k = 0; k < 3; ++k) {
                int64_t v = tri[e * 3 + k];
                double c = nu * eps[v] * dt;
                m00 += (1.0 + c * kinv[3 * v + 0]) / dt;
                m01 += c * kinv[3 * v + 1] / dt;
                m11 += (1.0 + c * kinv[3 * v + 2]) / dt;
            }
            m00 /= 3.0;
            m01 /= 3.0;
            m11 /= 3.0;
        } else {
            double c = nu * eps[e] * dt;
            m00 = (1.0 + c * kinv[3 * e + 0]) / dt;
            m01 = c * kinv[3 * e + 1] / dt;
            m11 = (1.0 + c * kinv[3 * e + 2]) / dt;
        }
        double du = ux - u23[e], dv = uy - u23[nt + e];
        g_next[e] = g_k[e] + m00 * du + m01 * dv;
        g_next[nt + e] = g_k[nt + e] + m01 * du + m11 * dv;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* 9. CP1 mass coupling (Sec. 3.2.2, Eq. cs1_sys2, App. B).             */
/* ------------------------------------------------------------------ */

/* Per cell the mass terms of the two CP1 systems and their coupling:
 * out[3e+0] = Mbar_11 A_e, out[3e+1] = Mbar_12 A_e, out[3e+2] = Mbar_22 A_e,
 * Mbar_e the mean over the cell's nodes of M = (I + nu eps Kinv dt)/dt (the
 * cell's own M for cell fields). */
int or_cp1_mass(int64_t nv, const double* xy, int64_t nt, const int32_t* tri,
                const double* eps, const double* kinv, int field_loc, double nu, double dt,
                double* out) {
    if (field_loc != OR_PER_VERTEX && field_loc != OR_PER_CELL) return OR_ERR_ARG;
    for (int64_t e = 0; e < nt; ++e) {
        for (int k = 0; k < 3; ++k)
            if (tri[e * 3 + k] < 0 || tri[e * 3 + k] >= nv) return OR_ERR_ARG;
        const double* a = &xy[2 * (int64_t)tri[e * 3 + 0]];
        const double* b = &xy[2 * (int64_t)tri[e * 3 + 1]];
        const double* c = &xy[2 * (int64_t)tri[e * 3 + 2]];
        double area = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));
        double m00 = 0.0, m01 = 0.0, m11 = 0.0;
        if (field_loc == OR_PER_VERTEX) {
            for (int k = 0; k < 3; ++k) {
                int64_t v = tri[e * 3 + k];
                double cf = nu * eps[v] * dt;
                m00 += (1.0 + cf * kinv[3 * v + 0]) / dt;
                m01 += cf * kinv[3 * v + 1] / dt;
                m11 += (1.0 + cf * kinv[3 * v + 2]) / dt;
            }
            m00 /= 3.0;
            m01 /= 3.0;
            m11 /= 3.0;
        } else {
            double cf = nu * eps[e] * dt;
            m00 = (1.0 + cf * kinv[3 * e + 0]) / dt;
            m01 = cf * kinv[3 * e + 1] / dt;
            m11 = (1.0 + cf * kinv[3 * e + 2]) / dt;
        }
        out[3 * e + 0] = m00 * area;
        out[3 * e + 1] = m01 * area;
        out[3 * e + 2] = m11 * area;
    }
    return OR_OK;
}
