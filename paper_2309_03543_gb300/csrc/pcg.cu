// Preconditioned conjugate gradients on the device (Sec. 3.2.2: the
// corrector systems are solved by PCG; the matrix is assembled and factored
// once and reused for every right-hand side).
//
// Jacobi-PCG on A is run as plain CG on the symmetrically scaled matrix
// Ahat = S^-1 A S^-1 (S = diag(sqrt(a_ee)), unit diagonal): with yhat = S x
// and bhat = S^-1 b its iterates are exactly those of Jacobi-PCG on A, but the
// diagonal and its inverse are never read inside the loop.  One iteration is
//   k_spmv_dot : q = Ahat p,  gamma = p.q  (last block: alpha = rho/gamma)
//   k_update   : y += alpha p, r -= alpha q, rho' = r.r (and ||S r||^2 every
//                few iterations for the stop test; last block: beta, stop)
//   k_pupdate  : p = r + beta p
// All scalars live in device memory; the host only polls a stop flag once per
// chunk of iterations, which are replayed from a CUDA graph.
//
// Mixed precision (CPS_MIXED): FP64 outer iterative refinement
//   r = b - A x (FP64), inner CG on Ahat d = S^-1 r with binary32 matrix,
//   vectors and SpMV, FP64 dot products and alpha/beta, x += S^-1 d (FP64).
#include "cps_internal.cuh"
#include "pcg_kernels.cuh"

#include <cmath>

namespace cps {

namespace {
// Iterations per graph chunk and the stop-test period inside a chunk.
constexpr int kChunk = 32;
constexpr int kCheckEvery = 8;
// Inner residual reduction per refinement step of the mixed solver.
constexpr double kInnerEta = 1e-2;
constexpr int kMaxRefinements = 100;
}  // namespace

static int ensure_capture_stream(cps_sys s) {
    if (!s->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s->ctx->last_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            return CPS_ERR_CUDA;
        }
    }
    return CPS_OK;
}

// Vector views of one CG run in working precision V.
template <typename V>
struct CgVecs {
    const V* a;
    const int32_t* col;
    const V* s;        // scale, for the unscaled residual norm
    V* y;
    V* r;
    V* p;
    V* q;
    int64_t n;
};

template <typename V>
static void enqueue_iteration(cps_sys s, const CgVecs<V>& v, bool norm, cudaStream_t st) {
    const int g = s->grid;
    k_spmv_dot<V><<<g, kBlock, 0, st>>>(v.a, v.col, v.p, v.q, v.n, s->partials, s->st);
    if (norm)
        k_update<V, true><<<g, kBlock, 0, st>>>(v.y, v.r, v.p, v.q, v.s, v.n, s->partials, s->st);
    else
        k_update<V, false><<<g, kBlock, 0, st>>>(v.y, v.r, v.p, v.q, v.s, v.n, s->partials, s->st);
    k_pupdate<V><<<g, kBlock, 0, st>>>(v.p, v.r, v.n, s->st);
}

template <typename V>
static int get_chunk_graph(cps_sys s, int prec, const CgVecs<V>& v, cudaGraphExec_t* out) {
    cudaGraphExec_t& ge = s->graph[prec][0];
    if (!ge) {
        int rc = ensure_capture_stream(s);
        if (rc) return rc;
        cudaGraph_t graph = nullptr;
        CPS_CUDA_TRY(s->ctx, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kChunk; ++k)
            enqueue_iteration<V>(s, v, (k % kCheckEvery) == kCheckEvery - 1, s->cap_stream);
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            s->ctx->last_error = std::string("graph capture: ") +
                                 cudaGetErrorString(le != cudaSuccess ? le : ce);
            return CPS_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            ge = nullptr;
            s->ctx->last_error = std::string("graph instantiate: ") + cudaGetErrorString(ie);
            return CPS_ERR_CUDA;
        }
    }
    *out = ge;
    return CPS_OK;
}

// Replays iteration chunks until the device sets st->done.  One chunk of
// look-ahead keeps the GPU busy while the host reads the previous flag; a
// chunk enqueued after the stop returns at once in every kernel.
template <typename V>
static int run_chunks(cps_sys s, int prec, const CgVecs<V>& v, cudaStream_t stream,
                      CgState* final_state, int64_t* launches) {
    cudaGraphExec_t ge = nullptr;
    int rc = get_chunk_graph<V>(s, prec, v, &ge);
    if (rc) return rc;
    for (long long k = 0;; ++k) {
        const int slot = (int)(k & 1);
        CPS_CUDA_TRY(s->ctx, cudaGraphLaunch(ge, stream));
        *launches += 3 * kChunk;
        CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(&s->hst[slot], s->st, sizeof(CgState),
                                             cudaMemcpyDeviceToHost, stream));
        CPS_CUDA_TRY(s->ctx, cudaEventRecord(s->ev[slot], stream));
        if (k >= 1) {
            const int prev = 1 - slot;
            CPS_CUDA_TRY(s->ctx, cudaEventSynchronize(s->ev[prev]));
            if (s->hst[prev].done) break;
        }
    }
    CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(&s->hst[0], s->st, sizeof(CgState),
                                         cudaMemcpyDeviceToHost, stream));
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    *final_state = s->hst[0];
    return CPS_OK;
}

static int read_state(cps_sys s, cudaStream_t stream, CgState* h) {
    CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(&s->hst[0], s->st, sizeof(CgState),
                                         cudaMemcpyDeviceToHost, stream));
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    *h = s->hst[0];
    return CPS_OK;
}

// ------------------------------------------------------------------ FP64

static int solve_fp64(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
                      cps_stats* stats, cudaStream_t stream) {
    const int64_t n = s->nt;
    const int g = s->grid;
    CgVecs<double> v{s->a, s->col, s->s, s->wy, s->wr, s->wp, s->wq, n};
    int64_t total = 0, launches = 0;
    CgState h{};
    int status = CPS_OK;
    // A restart recomputes r = b - A x when the recursively updated residual
    // has met rtol but the true residual has not (rounding drift).
    for (int restart = 0; restart < 8; ++restart) {
        const long long budget = (long long)(max_iter - total);
        k_init64<<<g, kBlock, 0, stream>>>(b, x, v.s, v.a, v.col, n, v.y, v.r, v.p, rtol, budget,
                                            s->partials, s->st);
        ++launches;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        int rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (!h.done && budget > 0) {
            rc = run_chunks<double>(s, CPS_FP64, v, stream, &h, &launches);
            if (rc) return rc;
        }
        total += h.iter;
        status = h.status;
        k_final64<<<g, kBlock, 0, stream>>>(b, v.y, v.s, v.a, v.col, n, x, s->partials, s->st);
        ++launches;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
    }
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    if (status == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) status = CPS_ERR_NOT_CONVERGED;
    if (stats) {
        stats->iters = total;
        stats->rel_res = rel;
        stats->status = status;
        stats->refinements = 1;
        stats->launches = launches;
    }
    if (status == CPS_ERR_NOT_SPD) s->ctx->last_error = "solve: p.Ap <= 0 (matrix not SPD or NaN input)";
    if (status == CPS_ERR_NOT_CONVERGED) s->ctx->last_error = "solve: max_iter reached";
    return status;
}

// ------------------------------------------------------------------ mixed

static int solve_mixed(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
                       cps_stats* stats, cudaStream_t stream) {
    const int64_t n = s->nt;
    const int g = s->grid;
    // binary32 vectors reuse the first half of the FP64 work buffers.
    float* d32 = reinterpret_cast<float*>(s->wy);
    float* r32 = reinterpret_cast<float*>(s->wr);
    float* p32 = reinterpret_cast<float*>(s->wp);
    float* q32 = reinterpret_cast<float*>(s->wq);
    CgVecs<float> v{s->a32, s->col, s->s32, d32, r32, p32, q32, n};
    int64_t total = 0, launches = 0;
    int refinements = 0;
    CgState h{};
    int status = CPS_OK;
    for (;;) {
        k_res64<<<g, kBlock, 0, stream>>>(b, x, s->s, s->a, s->col, n, r32, p32, d32, rtol,
                                          kInnerEta, (long long)(max_iter - total), s->partials,
                                          s->st);
        ++launches;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        int rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (h.bnorm2 == 0.0 || h.rnorm2 <= rtol * rtol * h.bnorm2) break;   // converged
        if (total >= max_iter || refinements >= kMaxRefinements) {
            status = CPS_ERR_NOT_CONVERGED;
            break;
        }
        ++refinements;
        if (!h.done) {
            rc = run_chunks<float>(s, CPS_MIXED, v, stream, &h, &launches);
            if (rc) return rc;
        }
        total += h.iter;
        if (h.status != CPS_OK) {
            status = h.status;
            break;
        }
        k_correct<<<g, kBlock, 0, stream>>>(x, d32, s->s, n);
        ++launches;
    }
    if (h.bnorm2 == 0.0) {
        CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, stream));
    }
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    if (stats) {
        stats->iters = total;
        stats->rel_res = rel;
        stats->status = status;
        stats->refinements = refinements;
        stats->launches = launches;
    }
    if (status == CPS_ERR_NOT_CONVERGED) s->ctx->last_error = "solve: refinement did not reach rtol";
    if (status == CPS_ERR_NOT_SPD) s->ctx->last_error = "solve: p.Ap <= 0 in the inner solve";
    return status;
}

int solve_impl(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
               int precision, cps_stats* stats, cudaStream_t stream) {
    if (!b || !x || !(rtol >= 0.0) || max_iter < 0) {
        s->ctx->last_error = "solve: bad argument";
        return CPS_ERR_ARG;
    }
    if (s->precond != CPS_PC_JACOBI) {
        s->ctx->last_error = "solve: preconditioner not available";
        return CPS_ERR_ARG;
    }
    if (precision == CPS_FP64) return solve_fp64(s, b, x, rtol, max_iter, stats, stream);
    if (precision == CPS_MIXED) return solve_mixed(s, b, x, rtol, max_iter, stats, stream);
    s->ctx->last_error = "solve: bad precision";
    return CPS_ERR_ARG;
}

int precond_impl(cps_sys s, int precond, cudaStream_t) {
    if (precond == CPS_PC_JACOBI) {
        s->precond = precond;
        return CPS_OK;
    }
    s->ctx->last_error = "set_precond: unknown preconditioner";
    return CPS_ERR_ARG;
}

int matvec_impl(cps_sys s, const double* x, double* y, cudaStream_t stream) {
    if (!x || !y) {
        s->ctx->last_error = "matvec: null pointer";
        return CPS_ERR_ARG;
    }
    k_matvec64<<<s->grid, kBlock, 0, stream>>>(x, s->s, s->a, s->col, s->nt, y);
    CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    return CPS_OK;
}

int export_impl(cps_sys s, double* diag, int32_t* col, double* val, cudaStream_t stream) {
    if (!diag || !col || !val) {
        s->ctx->last_error = "export: null pointer";
        return CPS_ERR_ARG;
    }
    CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(diag, s->diag, sizeof(double) * s->nt,
                                         cudaMemcpyDeviceToDevice, stream));
    CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(col, s->col, sizeof(int32_t) * 3 * s->nt,
                                         cudaMemcpyDeviceToDevice, stream));
    k_unscale_offdiag<<<grid_for(s->ctx, 3 * s->nt), kBlock, 0, stream>>>(s->a, s->col, s->s,
                                                                          s->nt, val);
    CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    return CPS_OK;
}

int adjoint_impl(cps_sys s, const double* x, const double* g, double* lambda, double* dT,
                 double* dtheta, double rtol, int64_t max_iter, cps_stats* stats,
                 cudaStream_t stream) {
    if (!x || !g || !lambda) {
        s->ctx->last_error = "adjoint: null pointer";
        return CPS_ERR_ARG;
    }
    if (dtheta && !s->iso_cell) {
        s->ctx->last_error = "adjoint: dtheta needs a CP2 system with an isotropic per-cell field";
        return CPS_ERR_ARG;
    }
    int rc = solve_fp64(s, g, lambda, rtol, max_iter, stats, stream);
    if (rc != CPS_OK) return rc;
    if (dT || dtheta) {
        k_adjoint_scatter<<<s->grid, kBlock, 0, stream>>>(x, lambda, s->col, s->slot_kind, s->gfac,
                                                           s->dxi, s->nt, dT, dtheta);
        if (stats) stats->launches += 1;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    }
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    return CPS_OK;
}

int solve_batch_impl(const cps_sys* systems, int nsys, const double* const* b,
                     double* const* x, double rtol, int64_t max_iter, int precision,
                     cps_stats* stats, cudaStream_t stream) {
    int first = CPS_OK;
    for (int i = 0; i < nsys; ++i) {
        int rc = solve_impl(systems[i], b[i], x[i], rtol, max_iter, precision,
                            stats ? &stats[i] : nullptr, stream);
        if (rc != CPS_OK && first == CPS_OK) first = rc;
    }
    return first;
}

}  // namespace cps
