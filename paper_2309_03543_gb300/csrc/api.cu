// C ABI entry points (declared in include/cps.h).  Argument checks, device
// selection and handle bookkeeping; the work is in assemble.cu and pcg.cu.
#include "cps_internal.cuh"

#include <new>

#include <nvtx3/nvToolsExt.h>

namespace {

int set_device(cps_ctx ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        cps::set_error(ctx, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        return CPS_ERR_CUDA;
    }
    return CPS_OK;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

// NVTX range over one library call (the calls show up by name in Nsight
// Systems and select launches in Nsight Compute; free without a tool).
namespace {
struct CallRange {
    explicit CallRange(const char* name) { nvtxRangePushA(name); }
    ~CallRange() { nvtxRangePop(); }
};
}  // namespace

extern "C" {

int cps_create(cps_ctx* out, int device) {
    if (!out) return CPS_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
        return CPS_ERR_ARG;
    cps_ctx c = new (std::nothrow) cps_ctx_s();
    if (!c) return CPS_ERR_NOMEM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor,
                               device) != cudaSuccess) {
        delete c;
        return CPS_ERR_CUDA;
    }
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    c->l2_bytes = (size_t)l2;
    int lp = 0;
    cudaDeviceGetAttribute(&lp, cudaDevAttrMaxPersistingL2CacheSize, device);
    c->l2_persist_max = (size_t)lp;
    *out = c;
    return CPS_OK;
}

int cps_destroy(cps_ctx ctx) {
    if (!ctx) return CPS_ERR_ARG;
    cudaSetDevice(ctx->device);
    for (cps_sys s : ctx->systems) cps::free_sys(s);
    ctx->systems.clear();
    delete ctx;
    return CPS_OK;
}

const char* cps_last_error(cps_ctx ctx) {
    if (!ctx) return "null context";
    return ctx->last_error.c_str();
}

int cps_assemble(cps_ctx ctx, const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                 const int32_t* dirichlet, int64_t nb, const double* eps, const double* kinv,
                 int field_loc, int kind, double nu, double dt, cps_sys* out, void* stream) {
    CallRange range_("cps_assemble");
    if (!ctx || !out) return CPS_ERR_ARG;
    *out = nullptr;
    int rc = set_device(ctx);
    if (rc) return rc;
    cps::set_error(ctx, "");
    rc = cps::assemble_impl(ctx, xy, nv, tri, nt, dirichlet, nb, eps, kinv, field_loc, kind, nu,
                            dt, out, as_stream(stream));
    if (rc == CPS_OK) {
        ctx->systems.insert(*out);
        std::lock_guard<std::mutex> lock(ctx->mu);
        auto it = ctx->tune_cache.find({(*out)->nt, (*out)->nv});
        if (it != ctx->tune_cache.end())
            for (int p = 0; p < 2; ++p) (*out)->tune[p] = it->second[p];
    }
    return rc;
}

int cps_set_precond(cps_sys sys, int precond, void* stream) {
    CallRange range_("cps_set_precond");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::precond_impl(sys, precond, as_stream(stream));
}

int cps_sys_free(cps_sys sys) {
    if (!sys) return CPS_ERR_ARG;
    cps_ctx ctx = sys->ctx;
    if (!ctx || ctx->systems.erase(sys) == 0) return CPS_ERR_ARG;   // unknown or freed
    set_device(ctx);
    cps::free_sys(sys);
    return CPS_OK;
}

int cps_sys_info(cps_sys sys, int64_t* nt, int64_t* n_interior_sides, double* diag_min,
                 int* is_mmatrix, int64_t* setup_launches) {
    if (!sys) return CPS_ERR_ARG;
    if (setup_launches) *setup_launches = sys->assembly_launches;
    if (nt) *nt = sys->nt;
    if (n_interior_sides) *n_interior_sides = sys->n_interior;
    if (diag_min) *diag_min = sys->diag_min;
    if (is_mmatrix) *is_mmatrix = sys->is_mmatrix;
    return CPS_OK;
}

int cps_export_matrix(cps_sys sys, double* diag, int32_t* col, double* val, void* stream) {
    CallRange range_("cps_export_matrix");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::export_impl(sys, diag, col, val, as_stream(stream));
}

int cps_solve(cps_sys sys, const double* b, double* x, double rtol, int64_t max_iter,
              int precision, cps_stats* stats, void* stream) {
    CallRange range_("cps_solve");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::solve_impl(sys, b, x, rtol, max_iter, precision, stats, as_stream(stream));
}

int cps_solve_batch(const cps_sys* systems, int nsys, const double* const* b, double* const* x,
                    double rtol, int64_t max_iter, int precision, cps_stats* stats,
                    void* stream) {
    CallRange range_("cps_solve_batch");
    if (nsys < 0 || (nsys > 0 && (!systems || !b || !x))) return CPS_ERR_ARG;
    if (nsys == 0) return CPS_OK;
    for (int i = 0; i < nsys; ++i)
        if (!systems[i] || systems[i]->ctx != systems[0]->ctx) return CPS_ERR_ARG;
    int rc = set_device(systems[0]->ctx);
    if (rc) return rc;
    return cps::solve_batch_impl(systems, nsys, b, x, rtol, max_iter, precision, stats,
                                 as_stream(stream));
}

int cps_cp2_setup(cps_sys sys, const double* xy, const int32_t* tri, const double* eps,
                  const double* kinv, void* stream) {
    CallRange range_("cps_cp2_setup");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::cp2_setup_impl(sys, xy, tri, eps, kinv, as_stream(stream));
}

int cps_cp2_step(cps_sys sys, const double* u23, const double* g_k, double* eta_tilde,
                 double* eta, double* u_next, double* g_next, double* flux, double rtol,
                 int64_t max_iter, int precision, cps_stats* stats, void* stream) {
    CallRange range_("cps_cp2_step");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::cp2_step_impl(sys, u23, g_k, eta_tilde, eta, u_next, g_next, flux, rtol,
                              max_iter, precision, stats, as_stream(stream));
}

int cps_cp1_setup(cps_sys sys_x, cps_sys sys_y, const double* xy, const int32_t* tri,
                  const double* eps, const double* kinv, void* stream) {
    CallRange range_("cps_cp1_setup");
    if (!sys_x) return CPS_ERR_ARG;
    int rc = set_device(sys_x->ctx);
    if (rc) return rc;
    return cps::cp1_setup_impl(sys_x, sys_y, xy, tri, eps, kinv, as_stream(stream));
}

int cps_cp1_step(cps_sys sys_x, cps_sys sys_y, const double* du_breve, double* du, double toll,
                 int64_t max_outer, double rtol, int64_t max_iter, int precision,
                 cps_cp1_stats* stats, void* stream) {
    CallRange range_("cps_cp1_step");
    if (!sys_x) return CPS_ERR_ARG;
    int rc = set_device(sys_x->ctx);
    if (rc) return rc;
    return cps::cp1_step_impl(sys_x, sys_y, du_breve, du, toll, max_outer, rtol, max_iter,
                              precision, stats, as_stream(stream));
}

int cps_set_cp1_path(cps_sys sys_x, int path) {
    if (!sys_x || !sys_x->cp1 || (path != CPS_CP1_ONE_LAUNCH && path != CPS_CP1_HOST))
        return CPS_ERR_ARG;
    sys_x->cp1->path = path;
    return CPS_OK;
}

int cps_cp2_kernel_times(cps_sys sys, float* ms) {
    if (!sys) return CPS_ERR_ARG;
    return cps::cp2_kernel_times(sys, ms);
}

int cps_adjoint(cps_sys sys, const double* x, const double* g, double* lambda, double* dT,
                double* dtheta, double rtol, int64_t max_iter, cps_stats* stats, void* stream) {
    CallRange range_("cps_adjoint");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::adjoint_impl(sys, x, g, lambda, dT, dtheta, rtol, max_iter, stats,
                             as_stream(stream));
}

int cps_set_batch_path(cps_ctx ctx, int path) {
    if (!ctx || (path != CPS_BATCH_ONE_LAUNCH && path != CPS_BATCH_GRAPH)) return CPS_ERR_ARG;
    ctx->batch_path = path;
    return CPS_OK;
}

int cps_set_solver_path(cps_sys sys, int path) {
    if (!sys) return CPS_ERR_ARG;
    cps::Tuning& t = sys->tune[CPS_FP64];
    if (path >= CPS_PATH_STREAM && path <= CPS_PATH_PERSISTENT_1RED_L2) {
        // IC(0) in a two-colour order: the persistent single-reduction loop
        // for the CPS_PATH_PERSISTENT_1RED pins, the streaming kernels for
        // the others
        t.ic0_done = true;
        t.ic0_path = (path == CPS_PATH_PERSISTENT_1RED || path == CPS_PATH_PERSISTENT_1RED_L2) ? 1 : 0;
        t.ic0_win = path != CPS_PATH_PERSISTENT_1RED_L2 ? 0
                    : cps::l2_window_fits_mode(sys, 4) ? 4
                    : cps::l2_window_fits_mode(sys, 3) ? 3 : 0;
    }
    if (path == CPS_PATH_AUTO) {
        t.ic0_done = false;
        t.ic0_path = 0;
        t.path_done = false;
        t.path = 0;
        t.red_done = false;
        t.red_path = 0;
    } else if (path == CPS_PATH_STREAM) {
        t.path_done = true;
        t.path = 0;
        t.l2win = 0;
        t.red_done = true;
        t.red_path = 0;
        t.red_win = 0;
    } else if (path == CPS_PATH_STREAM_1RED || path == CPS_PATH_STREAM_1RED_L2) {
        // with L2: all five vectors of the loop where the set-aside holds them, else r, p, q
        int win = 0;
        if (path == CPS_PATH_STREAM_1RED_L2) {
            win = cps::l2_window_fits_mode(sys, 3) ? 3 : 2;
            if (!cps::l2_vectors_fit(sys)) {
                cps::set_error(sys->ctx, "set_solver_path: the persisting L2 set-aside cannot hold r, p, q");
                return CPS_ERR_ARG;
            }
        }
        t.path_done = true;
        t.path = 3;
        t.l2win = win;
    } else if (path == CPS_PATH_PERSISTENT_1RED || path == CPS_PATH_PERSISTENT_1RED_L2) {
        if (path == CPS_PATH_PERSISTENT_1RED_L2 && !cps::l2_window_fits_mode(sys, 3)) {
            cps::set_error(sys->ctx, "set_solver_path: the persisting L2 set-aside cannot hold "
                                     "the five vectors of the single-reduction loop");
            return CPS_ERR_ARG;
        }
        t.path_done = true;
        t.path = 4;
        t.l2win = path == CPS_PATH_PERSISTENT_1RED_L2 ? 3 : 0;
        t.pgrid = 0;
        t.red_done = true;
        t.red_path = 2;
        t.red_win = path == CPS_PATH_PERSISTENT_1RED_L2 ? 3 : 0;
        t.red_pgrid = 0;
    } else if (path == CPS_PATH_PERSISTENT) {
        t.path_done = true;
        t.path = 2;
        t.l2win = 0;
        t.red_done = true;
        t.red_path = 1;
        t.red_win = 0;
        t.pgrid = 0;
        t.red_pgrid = 0;
    } else if (path == CPS_PATH_PERSISTENT_L2) {
        if (!cps::l2_vectors_fit(sys)) {
            cps::set_error(sys->ctx, "set_solver_path: the persisting L2 set-aside cannot hold r, p, q");
            return CPS_ERR_ARG;
        }
        t.path_done = true;
        t.path = 2;
        t.l2win = 2;
        t.red_done = true;
        t.red_path = 1;
        t.red_win = 2;
        t.pgrid = 0;
        t.red_pgrid = 0;
    } else if (path == CPS_PATH_STREAM_L2) {
        if (!cps::l2_vectors_fit(sys)) {
            cps::set_error(sys->ctx, "set_solver_path: the persisting L2 set-aside cannot hold r, p, q");
            return CPS_ERR_ARG;
        }
        t.path_done = true;
        t.path = 0;
        t.l2win = 2;
        t.red_done = true;
        t.red_path = 0;
        t.red_win = 2;
    } else if (path == CPS_PATH_CLUSTER || path == CPS_PATH_CLUSTER_1RED ||
               path == CPS_PATH_CLUSTER_PIPE || path == CPS_PATH_CLUSTER_SSTEP2 ||
               path == CPS_PATH_CLUSTER_SSTEP3) {
        const int var = path == CPS_PATH_CLUSTER_SSTEP3   ? 4
                        : path == CPS_PATH_CLUSTER_SSTEP2 ? 3
                        : path == CPS_PATH_CLUSTER_PIPE   ? 2
                        : path == CPS_PATH_CLUSTER_1RED   ? 1
                                                          : 0;
        if (sys->nt > cps::cluster_max_rows(sys->ctx, var)) {
            cps::set_error(sys->ctx, "set_solver_path: system too large for one cluster");
            return CPS_ERR_ARG;
        }
        t.path_done = true;
        t.path = 1;
        t.l2win = 0;
        t.cluster_variant = var;
    } else {
        return CPS_ERR_ARG;
    }
    return CPS_OK;
}

int cps_test_inject(cps_sys sys, int fault) {
    if (!sys || (fault != 0 && fault != CPS_TEST_STALL_BARRIER)) return CPS_ERR_ARG;
    sys->inject = fault;
    return CPS_OK;
}

int cps_set_kernel_shapes(cps_sys sys, int precision, const int32_t* unroll, const int32_t* grid,
                          const int32_t* block) {
    if (!sys || !unroll || !grid || !block || (precision != CPS_FP64 && precision != CPS_MIXED))
        return CPS_ERR_ARG;
    const int nk = precision == CPS_FP64 ? 3 : 2;
    for (int k = 0; k < nk; ++k) {
        const bool ok_u = unroll[k] == 1 || unroll[k] == 2 || unroll[k] == 4 ||
                          (unroll[k] == 8 && precision == CPS_FP64 && k > 0);
        const bool ok_g = grid[k] >= 1 && grid[k] <= cps::kMaxGrid;
        const bool ok_b = block[k] == cps::kBlock || (precision == CPS_FP64 && block[k] == 1024);
        if (!ok_u || !ok_g || !ok_b) {
            cps::set_error(sys->ctx, "set_kernel_shapes: unroll 1/2/4 (8 for the FP64 vector "
                                   "kernels), grid 1..4096, block 256 (or 1024 for FP64)");
            return CPS_ERR_ARG;
        }
    }
    cps::Tuning& t = sys->tune[precision];
    for (int k = 0; k < nk; ++k) {
        t.k[k].unroll = unroll[k];
        t.k[k].grid = grid[k];
        t.k[k].block = block[k];
    }
    t.done = true;
    t.kg_set = false;        // the single-reduction update follows the pinned residual update
    cps::drop_graphs(sys, precision);       // captured with the old shapes
    return CPS_OK;
}

int cps_get_tuning(cps_sys sys, int precision, int32_t* unroll, int32_t* grid, int32_t* block,
                   int32_t* flags, double* probe_us) {
    if (!sys || !unroll || !grid || (precision != CPS_FP64 && precision != CPS_MIXED))
        return CPS_ERR_ARG;
    const cps::Tuning& t = sys->tune[precision];
    for (int k = 0; k < 3; ++k) {
        unroll[k] = t.done ? t.k[k].unroll : 0;
        grid[k] = t.done ? t.k[k].grid : 0;
        if (block) block[k] = t.done ? t.k[k].block : 0;
    }
    if (flags) {
        flags[0] = (t.path_done && t.path == 1) ? 1 + t.cluster_variant : 0;
        flags[1] = t.path_done ? t.l2win : 0;
        flags[2] = t.path_done && (t.path == 2 || t.path == 4);
        flags[3] = t.red_done ? t.red_path : 0;
        flags[4] = t.red_done ? t.red_win : 0;
        flags[5] = t.path_done && t.path == 3;
        flags[6] = t.path_done && t.path == 4;
        flags[7] = (t.ic0_done && t.ic0_path == 1 && sys->ncolours == 2)
                       ? (t.ic0_win == 4 ? 3 : (t.ic0_win == 3 ? 2 : 1))
                       : 0;
    }
    if (probe_us) {
        for (int k = 0; k < 6; ++k) probe_us[k] = t.probe_us[k];
        for (int k = 0; k < 4; ++k) probe_us[6 + k] = t.red_probe_us[k];
        probe_us[16] = t.red_probe_us[4];
        probe_us[17] = t.red_probe_us[5];
        probe_us[10] = t.probe_us[6];
        probe_us[11] = t.probe_us[7];
        probe_us[12] = t.probe_us[8];
        probe_us[13] = t.probe_us[9];
        probe_us[14] = t.ic0_probe_us[0];
        probe_us[15] = t.ic0_probe_us[1];
    }
    return CPS_OK;
}

int cps_get_gear_shape(cps_sys sys, int32_t* unroll, int32_t* grid, int32_t* block) {
    if (!sys || !unroll || !grid || !block) return CPS_ERR_ARG;
    const cps::Tuning& t = sys->tune[CPS_FP64];
    const cps::KCfg c = t.kg_set ? t.kg : t.k[1];
    *unroll = t.done ? (c.block == 1024 && c.unroll > 2 ? 2 : c.unroll) : 0;
    *grid = t.done ? c.grid : 0;
    *block = t.done ? c.block : 0;
    return CPS_OK;
}

int cps_matvec(cps_sys sys, const double* x, double* y, void* stream) {
    CallRange range_("cps_matvec");
    if (!sys) return CPS_ERR_ARG;
    int rc = set_device(sys->ctx);
    if (rc) return rc;
    return cps::matvec_impl(sys, x, y, as_stream(stream));
}

}  // extern "C"
