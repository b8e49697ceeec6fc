// The CP1 solves of one time step (Sec. 3.2.2, Eq. cs1_sys2, App. B).
//
// The x and y velocity increments solve two CP1 systems that share the viscous
// operator nu L and differ in their mass terms.  They are coupled through the
// off-diagonal mass Mbar_12 A_e:
//   (Mbar_11 A_e + nu L) du_x = -nu L du_breve_x - Mbar_12 A_e du_y,
//   (Mbar_22 A_e + nu L) du_y = -nu L du_breve_y - Mbar_12 A_e du_x
// (Eq. CS1_sys_coeff; the right-hand side with the sign of Eq. CS1_2 and the
// outward normal derivative).  App. B (Eq. A1) solves them by an outer
// iteration: a first sweep without the coupling, then sweeps in which each
// component takes the other's previous iterate, until
// min(err_x, err_y) <= toll with err_k = ||du_k^{i+1} - du_k^i|| / ||du_k^i||.
//
// By default the whole outer iteration runs in one cooperative launch
// (k_cp1_step) after -nu L du_breve: per sweep the right-hand sides, the x and
// the y solve (Jacobi PCG, FP64 or mixed, by the whole grid as one team of
// blocks, block_solve.cuh), the change test as an exact team sum, and the
// stop decision, all on the device; the host reads the statistics once.  The
// host-driven loop (the library's PCG per solve, with the change sums read
// back after every sweep) serves systems with another preconditioner and can
// be chosen with cps_set_cp1_path.
#include "block_solve.cuh"
#include "cps_internal.cuh"

#include <algorithm>
#include <cmath>
#include <string>

namespace cps {
namespace {

// Per side slot T = nu l_j / d_{e,ep} (interior), nu l_j / delta_j (Dirichlet),
// 0 (no-flux); per cell Mbar_11 A_e, Mbar_12 A_e, Mbar_22 A_e.
__global__ void k_cp1_coeffs(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                             const int32_t* __restrict__ col,
                             const int32_t* __restrict__ slot_kind,
                             const double* __restrict__ ccx, const double* __restrict__ ccy,
                             const double* __restrict__ area, const double* __restrict__ eps,
                             const double* __restrict__ kinv, int64_t nt, int64_t nv,
                             bool per_vertex, bool logk, double nu, double dt,
                             double* __restrict__ T, double* __restrict__ mass, int* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v[3] = {tri[3 * e], tri[3 * e + 1], tri[3 * e + 2]};
        if (v[0] < 0 || v[0] >= nv || v[1] < 0 || v[1] >= nv || v[2] < 0 || v[2] >= nv) {
            set_error(err, CPS_ERR_ARG);
            for (int j = 0; j < 3; ++j) T[(int64_t)j * nt + e] = 0.0;
            mass[e] = mass[nt + e] = mass[2 * nt + e] = 0.0;
            continue;
        }
        const double cex = ccx[e], cey = ccy[e];
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int64_t ia = v[(j + 1) % 3], ib = v[(j + 2) % 3];
            const double px = xy[2 * ia], py = xy[2 * ia + 1];
            const double qx = xy[2 * ib], qy = xy[2 * ib + 1];
            const double tx = qx - px, ty = qy - py;
            const double l = sqrt(tx * tx + ty * ty);
            const double nx = ty / l, ny = -tx / l;
            const int sk = slot_kind[slot];
            double t = 0.0;
            if (sk != 0) {
                const int32_t ep = col[slot];
                const double d = sk == 1
                                     ? (ccx[ep] - cex) * nx + (ccy[ep] - cey) * ny
                                     : (0.5 * (px + qx) - cex) * nx + (0.5 * (py + qy) - cey) * ny;
                if (!(d > 1e-12 * l)) set_error(err, CPS_ERR_NONDELAUNAY);
                t = nu * l / d;
            }
            T[slot] = t;
        }
        double mb[3];
        cell_mbar(eps, kinv, v, e, per_vertex, logk, nu, dt, mb);
        const double a = area[e];
        mass[e] = mb[0] * a;
        mass[nt + e] = mb[1] * a;
        mass[2 * nt + e] = mb[2] * a;
    }
}

// lap_k = -nu L du_breve_k for both components; a boundary slot (col = e) has a
// zero increment across it, a no-flux slot T = 0.
__global__ void __launch_bounds__(kBlock)
k_cp1_laplacian(const double* __restrict__ u, const int32_t* __restrict__ col,
                const double* __restrict__ T, int64_t nt, double* __restrict__ lap) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double ux = u[e], uy = u[nt + e];
        double sx = 0.0, sy = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t slot = (int64_t)j * nt + e;
            const int32_t c = col[slot];
            const bool across = c != (int32_t)e;
            const double t = T[slot];
            const double cx = across ? u[c] : 0.0, cy = across ? u[nt + c] : 0.0;
            sx += t * (ux - cx);
            sy += t * (uy - cy);
        }
        lap[e] = -sx;
        lap[nt + e] = -sy;
    }
}

// Right-hand sides of a sweep from the current iterate du (coupled or not),
// and prev = du.
__global__ void __launch_bounds__(kBlock)
k_cp1_rhs(const double* __restrict__ lap, const double* __restrict__ m12,
          const double* __restrict__ du, int64_t nt, bool coupled, double* __restrict__ rhs,
          double* __restrict__ prev) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double ux = du[e], uy = du[nt + e];
        const double c = coupled ? m12[e] : 0.0;
        rhs[e] = lap[e] - c * uy;
        rhs[nt + e] = lap[nt + e] - c * ux;
        prev[e] = ux;
        prev[nt + e] = uy;
    }
}

// Per block: sum (du - prev)^2 and prev^2 for x and y, in a fixed order.
__global__ void __launch_bounds__(kBlock)
k_cp1_change(const double* __restrict__ du, const double* __restrict__ prev, int64_t nt,
             double* __restrict__ partials) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nt;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double px = prev[e], py = prev[nt + e];
        const double dx = du[e] - px, dy = du[nt + e] - py;
        v[0] += dx * dx;
        v[1] += px * px;
        v[2] += dy * dy;
        v[3] += py * py;
    }
    block_sum<4>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) partials[4 * (int64_t)blockIdx.x + k] = v[k];
}

// One block: the totals of nblocks partials (fixed order) into out[4].
__global__ void __launch_bounds__(kBlock)
k_cp1_change_total(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 4; ++k) v[k] += partials[4 * (int64_t)b + k];
    block_sum<4>(v);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) out[k] = v[k];
}

// ---- The one-launch step.  Statistics written by block 0, thread 0.
struct Cp1DevStats {
    long long outer;
    long long solve_iters;
    double err;
    double rel_res_max;
    int worst;          // first CPS_ERR_NOT_CONVERGED of a solve, else CPS_OK
    int fatal;          // a solve status other than OK / NOT_CONVERGED
    int settled;
    int pad;
};

// Layout of Cp1Data::dev: the team state, its partials, the two system
// descriptors and the statistics.
constexpr size_t kCp1SyncOff = 0;
constexpr size_t kCp1PartOff = 256;
constexpr size_t kCp1DescOff = kCp1PartOff + 8 * sizeof(double) * kMaxTeam;
constexpr size_t kCp1StatOff = kCp1DescOff + (2 * sizeof(BatchDesc) + 255) / 256 * 256;
constexpr size_t kCp1DevBytes = kCp1StatOff + 256;
static_assert(sizeof(TeamSync) <= 256 && sizeof(Cp1DevStats) <= 256, "one-launch CP1 layout");

struct Cp1DevArgs {
    const double* lap;       // [2][nt] -nu L du_breve
    const double* m12;       // [nt] Mbar_12 A_e
    double* du;              // [2][nt]
    double* prev;            // [2][nt]
    double* rhs;             // [2][nt]
    const BatchDesc* sys;    // [2]: the x and y systems (b = rhs_k, x = du_k)
    TeamSync* ts;            // the grid as one team
    Cp1DevStats* out;
    double toll, rtol;
    long long max_outer, max_iter;
    int64_t nt;
};

template <bool MIXED>
__global__ void __launch_bounds__(kBB, 2) k_cp1_step(Cp1DevArgs P) {
    __shared__ TeamCtx s_tc;
    __shared__ int s_stop;
    const int G = gridDim.x;
    const int64_t nt = P.nt;
    const int64_t rows = ((nt + G - 1) / G + 31) / 32 * 32;
    const int64_t lo = min(nt, (int64_t)blockIdx.x * rows);
    const int64_t hi = min(nt, lo + rows);
    if (threadIdx.x == 0) {
        s_tc = TeamCtx{P.ts, (unsigned long long)P.ts->stall, (int)blockIdx.x, G, 0u};
        if (blockIdx.x == 0) *P.out = Cp1DevStats{0, 0, INFINITY, 0.0, CPS_OK, CPS_OK, 0, 0};
    }
    __syncthreads();
    const double* __restrict__ lap = P.lap;
    const double* __restrict__ m12 = P.m12;
    double* __restrict__ du = P.du;
    double* __restrict__ prev = P.prev;
    double* __restrict__ rhs = P.rhs;
    bool ok = true;
    for (long long sweep = 0;; ++sweep) {
        // right-hand sides (sweep 0 without the coupling) and prev = du
        const bool coupled = sweep > 0;
        for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) {
            const double ux = du[e], uy = du[nt + e];
            const double c = coupled ? m12[e] : 0.0;
            rhs[e] = lap[e] - c * uy;
            rhs[nt + e] = lap[nt + e] - c * ux;
            prev[e] = ux;
            prev[nt + e] = uy;
        }
        ok = team_barrier(s_tc) && ok;
        if (!ok) break;
        // the two solves, each by the whole grid, warm-started from du
        for (int k = 0; k < 2 && ok; ++k)
            ok = (MIXED ? kbp_solve_mixed(P.sys[k], lo, hi, &s_tc, P.rtol, P.max_iter)
                        : kbp_solve(P.sys[k], lo, hi, &s_tc, P.rtol, P.max_iter)) && ok;
        if (!ok) break;
        // every block: the change sums of its rows (du final everywhere after
        // the team sum that ends each solve), one exact team sum; the solves'
        // states, written by block 0 before that sum, are final after it
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        if (coupled) {
            for (int64_t e = lo + threadIdx.x; e < hi; e += kBB) {
                const double px = prev[e], py = prev[nt + e];
                const double dx = du[e] - px, dy = du[nt + e] - py;
                v[0] = fma(dx, dx, v[0]);
                v[1] = fma(px, px, v[1]);
                v[2] = fma(dy, dy, v[2]);
                v[3] = fma(py, py, v[3]);
            }
        }
        ok = team_sum<4>(v, s_tc) && ok;
        if (!ok) break;
        if (threadIdx.x == 0) {
            // the same decision in every block (the same totals and states)
            int worst = CPS_OK, fatal = CPS_OK;
            long long iters = 0;
            double relmax = 0.0;
            for (int k = 0; k < 2; ++k) {
                const CgState* st = P.sys[k].st;
                const double b2 = __ldcg(&st->bnorm2), r2 = __ldcg(&st->rnorm2);
                const double rel = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
                int sk = __ldcg(&st->status);
                if (sk == CPS_OK && b2 > 0.0 && !(rel <= P.rtol)) sk = CPS_ERR_NOT_CONVERGED;
                if (sk == CPS_ERR_NOT_CONVERGED && worst == CPS_OK) worst = sk;
                if (sk != CPS_OK && sk != CPS_ERR_NOT_CONVERGED && fatal == CPS_OK) fatal = sk;
                iters += __ldcg(&st->iter);
                relmax = fmax(relmax, rel);
            }
            auto rel_change = [](double d2, double p2) {
                return d2 == 0.0 ? 0.0 : (p2 > 0.0 ? sqrt(d2) / sqrt(p2) : INFINITY);
            };
            const double err = coupled ? fmin(rel_change(v[0], v[1]), rel_change(v[2], v[3]))
                                       : INFINITY;
            const bool settled = coupled ? err <= P.toll : P.max_outer == 0;
            s_stop = (fatal != CPS_OK || settled || sweep >= P.max_outer) ? 1 : 0;
            if (blockIdx.x == 0) {
                Cp1DevStats* o = P.out;
                o->solve_iters += iters;
                o->rel_res_max = fmax(o->rel_res_max, relmax);
                if (o->worst == CPS_OK) o->worst = worst;
                o->fatal = fatal;
                if (coupled) {
                    o->outer = sweep;
                    o->err = err;
                }
                o->settled = settled ? 1 : 0;
            }
        }
        __syncthreads();
        if (s_stop) break;
    }
    if (!ok && blockIdx.x == 0 && threadIdx.x == 0) P.out->fatal = CPS_ERR_TIMEOUT;
}

int fail(cps_sys s, int code, const std::string& msg) {
    set_error(s->ctx, msg);
    return code;
}

double rel_change(double d2, double p2) {
    if (d2 == 0.0) return 0.0;
    return p2 > 0.0 ? std::sqrt(d2) / std::sqrt(p2) : INFINITY;
}

}  // namespace

void free_cp1(cps_sys s) {
    if (!s || !s->cp1) return;
    if (s->cp1->buf) cudaFree(s->cp1->buf);
    if (s->cp1->dev) cudaFree(s->cp1->dev);
    if (s->cp1->hstats) cudaFreeHost(s->cp1->hstats);
    delete s->cp1;
    s->cp1 = nullptr;
}

int cp1_setup_impl(cps_sys sx, cps_sys sy, const double* xy, const int32_t* tri,
                   const double* eps, const double* kinv, cudaStream_t stream) {
    if (!sy || sx->kind != CPS_KIND_CP1_X || sy->kind != CPS_KIND_CP1_Y)
        return fail(sx, CPS_ERR_ARG, "cp1_setup: needs a CP1_X and a CP1_Y system");
    if (sx->ctx != sy->ctx || sx->nt != sy->nt || sx->nv != sy->nv ||
        sx->field_loc != sy->field_loc || sx->logk != sy->logk)
        return fail(sx, CPS_ERR_ARG, "cp1_setup: the two systems differ in mesh or fields");
    if (!xy || !tri || !eps || !kinv) return fail(sx, CPS_ERR_ARG, "cp1_setup: null pointer");
    const int64_t nt = sx->nt, nv = sx->nv;
    free_cp1(sx);
    Cp1Data* c = new Cp1Data();
    c->nt = nt;
    const int64_t st = (nt + 31) / 32 * 32;
    // T 3, mass 3, lap 2, rhs 2, prev 2 slices of st doubles; then partials
    const size_t nd = (size_t)12 * st + 4 * (size_t)(kMaxGrid + 1);
    cudaError_t ce = cudaMalloc(&c->buf, sizeof(double) * nd);
    if (ce != cudaSuccess) {
        delete c;
        return fail(sx, CPS_ERR_NOMEM, std::string("cp1_setup: cudaMalloc: ") + cudaGetErrorString(ce));
    }
    ce = cudaMalloc(&c->dev, kCp1DevBytes);
    if (ce == cudaSuccess) ce = cudaMallocHost(&c->hstats, sizeof(Cp1DevStats));
    if (ce != cudaSuccess) {
        cudaFree(c->buf);
        if (c->dev) cudaFree(c->dev);
        delete c;
        return fail(sx, CPS_ERR_NOMEM, std::string("cp1_setup: ") + cudaGetErrorString(ce));
    }
    double* d = static_cast<double*>(c->buf);
    c->T = d;
    c->mass = d + 3 * st;
    c->lap = d + 6 * st;
    c->rhs = d + 8 * st;
    c->prev = d + 10 * st;
    c->partials = d + 12 * st;
    sx->cp1 = c;

    double *ccx = nullptr, *ccy = nullptr, *area = nullptr;
    int* err = nullptr;
    int h_err = 0;
    auto A = [&](void** p, size_t b) { return cudaMallocAsync(p, b, stream); };
    ce = A((void**)&ccx, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&ccy, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&area, sizeof(double) * nt);
    if (ce == cudaSuccess) ce = A((void**)&err, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(err, 0, sizeof(int), stream);
    if (ce == cudaSuccess) {
        const int g = sx->grid;
        k_cell_geometry<<<g, kBlock, 0, stream>>>(xy, tri, nt, nv, area, ccx, ccy, err);
        k_cp1_coeffs<<<g, kBlock, 0, stream>>>(xy, tri, sx->col, sx->slot_kind, ccx, ccy, area,
                                               eps, kinv, nt, nv,
                                               sx->field_loc == CPS_PER_VERTEX, sx->logk, sx->nu,
                                               sx->dt, c->T, c->mass, err);
        ce = cudaGetLastError();
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    }
    void* tmp[] = {ccx, ccy, area, err};
    for (void* p : tmp)
        if (p) cudaFreeAsync(p, stream);
    cudaError_t se = cudaStreamSynchronize(stream);
    if (ce == cudaSuccess) ce = se;
    if (ce != cudaSuccess) {
        free_cp1(sx);
        return fail(sx, ce == cudaErrorMemoryAllocation ? CPS_ERR_NOMEM : CPS_ERR_CUDA,
                    std::string("cp1_setup: ") + cudaGetErrorString(ce));
    }
    if (h_err != 0) {
        free_cp1(sx);
        return fail(sx, h_err, "cp1_setup: mesh or fields do not match the systems (or bad input)");
    }
    return CPS_OK;
}

// The step in one cooperative launch of k_cp1_step (both systems Jacobi).
static int cp1_step_one_launch(cps_sys sx, cps_sys sy, double* du, double toll,
                               int64_t max_outer, double rtol, int64_t max_iter, bool mixed,
                               cps_cp1_stats* stats, cudaStream_t stream) {
    Cp1Data* c = sx->cp1;
    const int64_t nt = sx->nt;
    const void* kernel = mixed ? (const void*)k_cp1_step<true> : (const void*)k_cp1_step<false>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBB, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return fail(sx, CPS_ERR_CUDA, "cp1_step: the one-launch kernel does not fit an SM");
    }
    const int grid = std::min(sx->ctx->num_sms * per_sm, kMaxTeam);
    char* dev = static_cast<char*>(c->dev);
    TeamSync hs{};
    hs.partials = reinterpret_cast<double*>(dev + kCp1PartOff);
    hs.stall = sx->inject == CPS_TEST_STALL_BARRIER ? 1 : 0;   // test hook, one-shot
    sx->inject = 0;
    BatchDesc hd[2];
    cps_sys sys[2] = {sx, sy};
    for (int k = 0; k < 2; ++k) {
        cps_sys s = sys[k];
        BatchDesc& d = hd[k];
        d = BatchDesc{};
        d.a = s->a;
        d.col = s->col;
        d.s = s->s;
        d.b = c->rhs + k * nt;
        d.x = du + k * nt;
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
        d.n = nt;
    }
    Cp1DevArgs a{};
    a.lap = c->lap;
    a.m12 = c->mass + nt;
    a.du = du;
    a.prev = c->prev;
    a.rhs = c->rhs;
    a.sys = reinterpret_cast<const BatchDesc*>(dev + kCp1DescOff);
    a.ts = reinterpret_cast<TeamSync*>(dev + kCp1SyncOff);
    a.out = reinterpret_cast<Cp1DevStats*>(dev + kCp1StatOff);
    a.toll = toll;
    a.rtol = rtol;
    a.max_outer = (long long)max_outer;
    a.max_iter = (long long)max_iter;
    a.nt = nt;
    Cp1DevStats* h = static_cast<Cp1DevStats*>(c->hstats);
    cudaError_t ce = cudaMemcpyAsync(dev + kCp1SyncOff, &hs, sizeof(hs), cudaMemcpyHostToDevice,
                                     stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(dev + kCp1DescOff, hd, sizeof(hd), cudaMemcpyHostToDevice, stream);
    if (ce == cudaSuccess) {
        void* args[] = {(void*)&a};
        ce = cudaLaunchCooperativeKernel(kernel, dim3(grid), dim3(kBB), args, 0, stream);
    }
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(h, a.out, sizeof(Cp1DevStats), cudaMemcpyDeviceToHost, stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return fail(sx, CPS_ERR_CUDA, std::string("cp1_step: ") + cudaGetErrorString(ce));
    }
    if (stats) *stats = cps_cp1_stats{h->outer, h->solve_iters, h->err, h->rel_res_max};
    if (h->fatal == CPS_ERR_TIMEOUT)
        return fail(sx, CPS_ERR_TIMEOUT, "cp1_step: a device-side wait ran out");
    if (h->fatal == CPS_ERR_NOT_SPD) return fail(sx, CPS_ERR_NOT_SPD, "cp1_step: p.Ap <= 0");
    if (h->fatal != CPS_OK) return fail(sx, h->fatal, "cp1_step: a solve failed");
    if (h->worst != CPS_OK) return fail(sx, h->worst, "cp1_step: a solve did not reach rtol");
    if (!h->settled) return fail(sx, CPS_ERR_NOT_CONVERGED, "cp1_step: outer iteration above toll");
    return CPS_OK;
}

int cp1_step_impl(cps_sys sx, cps_sys sy, const double* du_breve, double* du, double toll,
                  int64_t max_outer, double rtol, int64_t max_iter, int precision,
                  cps_cp1_stats* stats, cudaStream_t stream) {
    Cp1Data* c = sx->cp1;
    if (!c) return fail(sx, CPS_ERR_ARG, "cp1_step: call cps_cp1_setup first");
    if (!sy || sy->kind != CPS_KIND_CP1_Y || sy->nt != sx->nt || sy->ctx != sx->ctx)
        return fail(sx, CPS_ERR_ARG, "cp1_step: sys_y is not the CP1_Y partner");
    if (!du_breve || !du || !(toll >= 0.0) || max_outer < 0)
        return fail(sx, CPS_ERR_ARG, "cp1_step: bad argument");
    if (precision != CPS_FP64 && precision != CPS_MIXED)
        return fail(sx, CPS_ERR_ARG, "cp1_step: bad precision");
    const int64_t nt = sx->nt;
    const int g1 = (int)((nt + kBlock - 1) / kBlock);
    const bool jacobi = sx->precond == CPS_PC_JACOBI && sy->precond == CPS_PC_JACOBI;
    if (c->path == 0 && jacobi && nt > 0) {
        k_cp1_laplacian<<<g1, kBlock, 0, stream>>>(du_breve, sx->col, c->T, nt, c->lap);
        const cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return fail(sx, CPS_ERR_CUDA, std::string("cp1_step: ") + cudaGetErrorString(le));
        return cp1_step_one_launch(sx, sy, du, toll, max_outer, rtol, max_iter,
                                   precision == CPS_MIXED, stats, stream);
    }
    const int gr = sx->grid;   // <= kMaxGrid blocks for the change sums
    cps_cp1_stats st{0, 0, INFINITY, 0.0};
    int worst = CPS_OK;
    auto solve_pair = [&]() -> int {
        cps_stats a{}, b{};
        int r1 = solve_impl(sx, c->rhs, du, rtol, max_iter, precision, &a, stream);
        if (r1 != CPS_OK && r1 != CPS_ERR_NOT_CONVERGED) return r1;
        int r2 = solve_impl(sy, c->rhs + nt, du + nt, rtol, max_iter, precision, &b, stream);
        if (r2 != CPS_OK && r2 != CPS_ERR_NOT_CONVERGED) return r2;
        st.solve_iters += a.iters + b.iters;
        st.rel_res_max = std::fmax(st.rel_res_max, std::fmax(a.rel_res, b.rel_res));
        if (worst == CPS_OK) worst = r1 != CPS_OK ? r1 : r2;
        return CPS_OK;
    };
    k_cp1_laplacian<<<g1, kBlock, 0, stream>>>(du_breve, sx->col, c->T, nt, c->lap);
    k_cp1_rhs<<<g1, kBlock, 0, stream>>>(c->lap, c->mass + nt, du, nt, false, c->rhs, c->prev);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) return fail(sx, CPS_ERR_CUDA, std::string("cp1_step: ") + cudaGetErrorString(ce));
    int rc = solve_pair();
    if (rc) return rc;
    double h[4];
    bool settled = max_outer == 0;   // the uncoupled sweep only
    while (st.outer < max_outer) {
        k_cp1_rhs<<<g1, kBlock, 0, stream>>>(c->lap, c->mass + nt, du, nt, true, c->rhs, c->prev);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return fail(sx, CPS_ERR_CUDA, std::string("cp1_step: ") + cudaGetErrorString(ce));
        rc = solve_pair();
        if (rc) return rc;
        ++st.outer;
        k_cp1_change<<<gr, kBlock, 0, stream>>>(du, c->prev, nt, c->partials);
        k_cp1_change_total<<<1, kBlock, 0, stream>>>(c->partials, gr, c->partials + 4 * kMaxGrid);
        ce = cudaGetLastError();
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(h, c->partials + 4 * kMaxGrid, sizeof(h), cudaMemcpyDeviceToHost,
                                 stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(stream);
        if (ce != cudaSuccess) return fail(sx, CPS_ERR_CUDA, std::string("cp1_step: ") + cudaGetErrorString(ce));
        st.err = std::fmin(rel_change(h[0], h[1]), rel_change(h[2], h[3]));
        if (st.err <= toll) {
            settled = true;
            break;
        }
    }
    if (stats) *stats = st;
    if (worst != CPS_OK) return worst;
    if (!settled) return fail(sx, CPS_ERR_NOT_CONVERGED, "cp1_step: outer iteration above toll");
    return CPS_OK;
}

}  // namespace cps
