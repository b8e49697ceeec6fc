// Internal definitions of the corrector-step solver library (not part of the
// C ABI).  Device data layout, handle structs, launch helpers and the
// deterministic grid reduction shared by the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <array>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <unordered_set>

#include "cps.h"

namespace cps {

constexpr int kBlock = 256;          // threads per block for streaming kernels
constexpr int kMaxGrid = 4096;       // bound on blocks (size of partial buffers)
constexpr int kNumPartials = 4;      // doubles reduced per kernel at most

// Scalar state of one conjugate-gradient run, kept on the device so that the
// iteration never waits for the host.  Written only by the last block of a
// reduction kernel; read by every block of later kernels.
struct CgState {
    double rho;        // r^T z of the current residual
    double alpha;      // step length of the current iteration
    double beta;       // p-update coefficient of the current iteration
    double bnorm2;     // ||b||^2 of the outer system (unscaled)
    double thresh2;    // stop threshold on the residual norm squared
    double rnorm2;     // last evaluated residual norm squared (unscaled)
    double gamma;      // p^T A p of the current iteration
    long long iter;    // iterations completed in this run
    long long max_iter;
    int done;          // 1: stop (converged, breakdown or max_iter)
    int status;        // CPS_OK or an error code set on the device
    unsigned int arrive[4];   // arrival counters of the grid reductions
    double rho_rep;    // mixed precision: r.r of the last residual replacement
    int updates;       // mixed one-launch batch: residual replacements of the solve
    int pad;
};

// Launch configuration of one iteration kernel: rows per thread per trip of
// the grid-stride loop, and grid size (blocks of kBlock threads).
struct KCfg {
    int unroll = 2;
    int grid = 0;
    int block = kBlock;      // threads per block (FP64 iteration kernels: 256 or 1024)
};

// Autotuned configurations of the iteration kernels of one precision:
// k[0] SpMV (FP64) or fused SpMV (binary32), k[1] residual update, k[2]
// direction update (FP64 only).
struct Tuning {
    KCfg k[3];
    bool done = false;
    int path = 0;            // FP64 Jacobi: 0 graph-replayed kernels, 1 one-cluster launch,
                             // 2 one persistent grid-synchronised launch, 3 graph-replayed
                             // single-reduction kernels, 4 one persistent launch of the
                             // single-reduction recurrences
    int red_path = 0;        // reduced system: 0 graph-replayed kernels, 1 persistent launch,
                             // 2 persistent launch of the single-reduction recurrences
    bool red_done = false;
    bool path_done = false;
    int l2win = 0;           // FP64 Jacobi stream path, persisting L2 window: 0 none,
                             // 1 the matrix, 2 the vectors r, p, q, 3 r, p, q, y, p1
    double probe_us[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // us/iteration: stream,
                                               // cluster, stream + matrix in L2, persistent,
                                               // stream + vectors in L2, persistent + vectors
                                               // in L2, single-reduction stream (+ vectors in
                                               // L2), single-reduction persistent (+ vectors
                                               // in L2)
    double red_probe_us[6] = {0, 0, 0, 0, 0, 0};   // reduced system: stream, persistent,
                                             // the same with r, p, q in persisting L2, then
                                             // persistent single-reduction without and with
                                             // its five vectors in persisting L2
    int red_win = 0;         // reduced system: persisting L2 window (0 none, 2 r, p, q,
                             // 3 r, p, q, y, p1)
    int pgrid = 0;           // blocks of the persistent launch (0: all that stay resident)
    int red_pgrid = 0;       // the same for the reduced system
    int cluster_variant = 0; // one-cluster launch: 0 textbook CG, 1 single reduction,
                             // 2 pipelined, 3 / 4 s-step (s = 2 / 3)
    KCfg kg;                 // single-reduction update kernel (if kg_set; else k[1])
    bool kg_set = false;
    // FP64 IC(0) in a two-colour order: 0 graph-replayed streaming kernels,
    // 1 one persistent launch of the single-reduction recurrences
    int ic0_path = 0;
    int ic0_win = 0;         // persisting L2 window of the persistent IC(0) loop (0 or 4)
    bool ic0_done = false;
    double ic0_probe_us[2] = {0, 0};   // us/iteration: streaming, persistent (best window)
};

// Device error flag written by the assembly kernels (first error wins).
__device__ __forceinline__ void set_error(int* err, int code) {
    atomicCAS(err, 0, code);
}

// Component comp (0 xx, 1 xy, 2 yy) of K^-1 at field point i: stored, or
// exp(-theta_i) I for a log-permeability field.
__device__ __forceinline__ double kinv_at(const double* __restrict__ kinv, int64_t i, int comp,
                                          bool logk) {
    if (logk) return comp == 1 ? 0.0 : exp(-kinv[i]);
    return kinv[3 * i + comp];
}

// Mbar_e (xx, xy, yy): the mean over the cell's nodes v[0..3) of
// M = (I + nu eps Kinv dt)/dt, or the cell's own M for cell fields (Sec. 3.1,
// Sec. 3.2 cell averages).
__device__ __forceinline__ void cell_mbar(const double* __restrict__ eps,
                                          const double* __restrict__ kinv, const int64_t* v,
                                          int64_t e, bool per_vertex, bool logk, double nu,
                                          double dt, double* m) {
    double m00 = 0.0, m01 = 0.0, m11 = 0.0;
    if (per_vertex) {
        for (int k = 0; k < 3; ++k) {
            const double c = nu * eps[v[k]] * dt;
            m00 += (1.0 + c * kinv_at(kinv, v[k], 0, false)) / dt;
            m01 += c * kinv_at(kinv, v[k], 1, false) / dt;
            m11 += (1.0 + c * kinv_at(kinv, v[k], 2, false)) / dt;
        }
        m00 /= 3.0;
        m01 /= 3.0;
        m11 /= 3.0;
    } else {
        const double c = nu * eps[e] * dt;
        m00 = (1.0 + c * kinv_at(kinv, e, 0, logk)) / dt;
        m01 = c * kinv_at(kinv, e, 1, logk) / dt;
        m11 = (1.0 + c * kinv_at(kinv, e, 2, logk)) / dt;
    }
    m[0] = m00;
    m[1] = m01;
    m[2] = m11;
}

// Per cell area and circumcentre (Sec. 3.1); CPS_ERR_ARG / _ORIENTATION in err.
__global__ void k_cell_geometry(const double* __restrict__ xy, const int32_t* __restrict__ tri,
                                int64_t nt, int64_t nv, double* __restrict__ area,
                                double* __restrict__ ccx, double* __restrict__ ccy, int* err);
// Xi = eps dt (I + nu eps dt Kinv)^-1 at nf field points (Eq. Cs2_4), [nf][3].
__global__ void k_xi(const double* __restrict__ eps, const double* __restrict__ kinv, int64_t nf,
                     double nu, double dt, bool logk, double* __restrict__ xi, int* err);

// Data of the CP1 step (Sec. 3.2.2, App. B), set up once per pair of CP1
// systems (kept on the x system).  Slot-major like the matrix.
struct Cp1Data {
    void* buf = nullptr;
    double* T = nullptr;      // [3nt] nu l_j / d (interior), nu l_j / delta (Dirichlet), 0
    double* mass = nullptr;   // [3][nt] Mbar_11 A_e, Mbar_12 A_e, Mbar_22 A_e
    double* lap = nullptr;    // [2][nt] -nu L du_breve (x, y)
    double* rhs = nullptr;    // [2][nt]
    double* prev = nullptr;   // [2][nt] previous iterate
    double* partials = nullptr;  // [kMaxGrid][4] + [4] error sums
    void* dev = nullptr;         // one-launch step: team state, system descriptors, statistics
    void* hstats = nullptr;      // pinned copy of the one-launch statistics
    int path = 0;                // 0 one launch (Jacobi systems), 1 host-driven sweeps
    int64_t nt = 0;
};

// Data of the CP2 step around the two solves (Sec. 3.2.3), set up once per
// system by cps_cp2_setup; every array is a slice of buf.  Slot-major [k][nt]
// like the matrix: slot j*nt + e is local side j of cell e.
struct Cp2Data {
    void* buf = nullptr;
    double* wgt = nullptr;    // [3nt] A_ep/(A_e + A_ep) (1 on a boundary side)
    double* lnx = nullptr;    // [3nt] l_j n_j, x (0 on a no-flux side)
    double* lny = nullptr;    // [3nt] l_j n_j, y (0 on a no-flux side)
    double* T = nullptr;      // [3nt] side coefficient (interior, Dirichlet), 0 no-flux
    double* tw = nullptr;     // [4][3nt] co-normal weights of the tangential flux
    double* rt0 = nullptr;    // [6][nt] (centroid - x_j)/(2 A_e), j = 0..2, x then y
    double* mbar = nullptr;   // [3][nt] Mbar_e (xx, xy, yy)
    double* fbar = nullptr;   // [3nt] mean side flux of the current step
    double* tau = nullptr;    // [3nt] tangential flux of the current step
    double* rhs = nullptr;    // [nt] right-hand side of the current solve
    double* eta_t = nullptr;  // [nt] first solution when the caller keeps none
    int32_t* tidx = nullptr;  // [4][3nt] cell whose eta enters each weight (-1: eta = 0)
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    float kernel_ms[3] = {0.f, 0.f, 0.f};   // last step: mean flux, tangential, update
};

// Block-wide sum of v[0..NV) over BS threads (BS = blockDim.x); on return
// every thread holds the totals.  GB300 issues FP64 adds at 1/64 of the FP32
// rate, so the adds are kept few: every thread stores its values to shared
// memory and warp k alone adds the BS values of quantity k (BS/32 serial adds
// per lane, then a 5-step shuffle tree), NV (BS/32 + 5) warp-wide FP64 adds
// per block instead of the (BS/32 + 1) 5 of a shuffle tree in every warp.  The
// order is fixed, so the result is deterministic.
template <int NV, int BS = kBlock>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    static_assert(BS % 32 == 0 && BS <= 1024 && NV <= BS / 32, "block shape");
    __shared__ double buf[NV][BS];
    __shared__ double tot[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) buf[k][threadIdx.x] = v[k];
    __syncthreads();
    if (warp < NV) {
        double t = buf[warp][lane];
#pragma unroll
        for (int j = lane + 32; j < BS; j += 32) t += buf[warp][j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) tot[warp] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = tot[k];
}

// Deterministic sum over the grid: every block writes its partial sums, the
// last block to arrive adds them up in a fixed order.  Returns true only in
// the last block, where v[] then holds the totals in every thread.
template <int NV, int BS = kBlock>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials,
                                         unsigned int* arrive) {
    __shared__ bool last;
    block_sum<NV, BS>(v);
    const int G = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partials[k * kMaxGrid + blockIdx.x] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(arrive, 1u);
        last = (t == (unsigned)G - 1u);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < G; i += blockDim.x) acc += __ldcg(&partials[k * kMaxGrid + i]);
        v[k] = acc;
    }
    block_sum<NV, BS>(v);
    if (threadIdx.x == 0) *arrive = 0u;
    return true;
}

}  // namespace cps

// Context and system handles (opaque in the C ABI).
struct cps_ctx_s {
    int device = 0;
    int num_sms = 0;
    int max_threads_per_sm = 2048;
    size_t l2_bytes = 0;
    size_t l2_persist_max = 0;   // cudaDevAttrMaxPersistingL2CacheSize
    size_t l2_persist_set = 0;   // persisting L2 limit this process has set
    std::string last_error;
    std::mutex mu;               // guards last_error and tune_cache (solves may run on threads)
    std::mutex l2_mu;            // guards the persisting-L2 set-aside
    std::unordered_set<cps_sys_s*> systems;   // live systems, freed with the context
    int batch_path = CPS_BATCH_ONE_LAUNCH;   // FP64 cps_solve_batch: one launch or graph chunks
    // Tuned launch choices by mesh size (cells, vertices): a system assembled
    // later on a mesh of the same size starts from them instead of re-timing.
    std::map<std::pair<int64_t, int64_t>, std::array<cps::Tuning, 2>> tune_cache;
};

namespace cps {
// Records the context's last error message (thread-safe).
inline void set_error(cps_ctx_s* ctx, const std::string& msg) {
    std::lock_guard<std::mutex> lock(ctx->mu);
    ctx->last_error = msg;
}
}  // namespace cps

struct cps_sys_s {
    cps_ctx ctx = nullptr;
    int64_t nt = 0, nv = 0;
    int kind = CPS_KIND_CP2;
    int field_loc = CPS_PER_VERTEX;
    int precond = CPS_PC_JACOBI;
    double nu = 0, dt = 0;
    int64_t n_interior = 0;
    double diag_min = 0;
    int is_mmatrix = 0;
    bool iso_cell = false;      // CPS_PER_CELL with isotropic Kinv (adjoint theta chain)
    bool logk = false;          // assembled from CPS_PER_CELL_LOGK (kinv holds theta)
    cps::Cp2Data* cp2 = nullptr;  // CP2 step data (cps_cp2_setup)
    cps::Cp1Data* cp1 = nullptr;  // CP1 step data (cps_cp1_setup, on the x system)
    int64_t assembly_launches = 0;

    // Matrix in symmetrically scaled padded-ELL form: A = S (I + Aoff) S with
    // S = diag(s), s = sqrt(diag(A)); slot-major arrays [3][nt].
    double* s = nullptr;        // [nt]
    double* diag = nullptr;     // [nt] unscaled diagonal (export / info)
    double* a = nullptr;        // [3*nt] scaled off-diagonals (allocation also holds col)
    int32_t* col = nullptr;     // [3*nt] column (= row for an unused slot)
    size_t mat_bytes = 0;       // bytes of the a + col allocation
    float* a32 = nullptr;       // [3*nt] binary32 copy of a (mixed precision)
    float* s32 = nullptr;       // [nt]
    // Adjoint: per slot dT/dxi_e, per cell dxi/dtheta (CP2, cell fields).
    double* gfac = nullptr;     // [3*nt]
    double* dxi = nullptr;      // [nt]
    int32_t* slot_kind = nullptr;   // [3*nt] 0 no-flux, 1 interior, 2 Dirichlet

    // IC(0) in colour order (scaled matrix, unit diagonal), set up on demand.
    int ncolours = 0;
    int64_t colour_start[17] = {0};
    int32_t* perm = nullptr;    // [nt] colour order -> mesh order
    int32_t* iperm = nullptr;   // [nt] mesh order -> colour order
    double* pa = nullptr;       // [3*nt] permuted scaled off-diagonals
    int32_t* pcol = nullptr;    // [3*nt] permuted columns
    double* pl = nullptr;       // [3*nt] IC(0) factor entries per slot
    double* pdinv = nullptr;    // [nt] inverse IC(0) pivots
    double* pdiag = nullptr;    // [nt] the IC(0) pivots themselves
    double* ps = nullptr;       // [nt] s in colour order
    float* pa32 = nullptr;
    float* pl32 = nullptr;
    float* pdinv32 = nullptr;
    float* ps32 = nullptr;

    // PCG workspace (allocated at assembly so that solves never allocate), one
    // allocation of 9 vectors of vec_stride doubles in the order r, p0, q, y,
    // p1, z, b, x, best: r, p0 and q, the vectors every iteration reads and
    // writes, are one contiguous range for an L2 access-policy window.
    double* wvec = nullptr;
    int64_t vec_stride = 0;
    double* wy = nullptr;       // [nt] iterate (scaled)
    double* wr = nullptr;       // [nt] residual
    double* wp0 = nullptr;      // [nt] search direction, even iterations
    double* wp1 = nullptr;      // [nt] search direction, odd iterations
    double* wq = nullptr;       // [nt] A p
    double* wz = nullptr;       // [nt] preconditioned residual (IC0)
    double* wb = nullptr;       // [nt] right-hand side in colour order
    double* wx = nullptr;       // [nt] FP64 iterate in colour order
    double* wbest = nullptr;    // [nt] mixed precision: FP64 iterate with the least residual
    double* partials = nullptr; // [(kNumPartials + 16) * kMaxGrid]
    cps::CgState* st = nullptr; // device state
    cps::CgState* hst = nullptr;  // pinned host mirror (2 slots)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int grid = 0;

    // CUDA graphs of a chunk of iterations, per (precision, preconditioner).
    cudaStream_t cap_stream = nullptr;
    // [precision][0 Jacobi, 1 IC(0), 2 reduced system, 3 single-reduction Jacobi]
    cudaGraphExec_t graph[2][4] = {{nullptr, nullptr, nullptr, nullptr},
                                   {nullptr, nullptr, nullptr, nullptr}};
    int64_t graph_nodes[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    int graph_l2win[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    cps::Tuning tune[2];        // per precision (CPS_FP64, CPS_MIXED)
    int cluster_size = 0;       // CTAs of the last one-cluster solve
    void* gsync = nullptr;      // grid-barrier state of the persistent solves
    int inject = 0;             // one-shot test fault (cps_test_inject)
};

#define CPS_CUDA_TRY(ctx, call)                                                        \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (ctx) {                                                                 \
                cps::set_error((ctx), std::string(#call) + ": " + cudaGetErrorString(e_)); \
            }                                                                          \
            return e_ == cudaErrorMemoryAllocation ? CPS_ERR_NOMEM : CPS_ERR_CUDA;     \
        }                                                                              \
    } while (0)

namespace cps {

inline int grid_for(const cps_ctx_s* ctx, int64_t n, int per_sm = 8) {
    int64_t need = (n + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)ctx->num_sms * per_sm;
    if (cap > kMaxGrid) cap = kMaxGrid;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

int assemble_impl(cps_ctx ctx, const double* xy, int64_t nv, const int32_t* tri, int64_t nt,
                  const int32_t* dirichlet, int64_t nb, const double* eps, const double* kinv,
                  int field_loc, int kind, double nu, double dt, cps_sys* out,
                  cudaStream_t stream);
int precond_impl(cps_sys sys, int precond, cudaStream_t stream);
int solve_impl(cps_sys sys, const double* b, double* x, double rtol, int64_t max_iter,
               int precision, cps_stats* stats, cudaStream_t stream);
int solve_batch_impl(const cps_sys* systems, int nsys, const double* const* b,
                     double* const* x, double rtol, int64_t max_iter, int precision,
                     cps_stats* stats, cudaStream_t stream);
int adjoint_impl(cps_sys sys, const double* x, const double* g, double* lambda, double* dT,
                 double* dtheta, double rtol, int64_t max_iter, cps_stats* stats,
                 cudaStream_t stream);
int matvec_impl(cps_sys sys, const double* x, double* y, cudaStream_t stream);
int64_t cluster_max_rows(cps_ctx ctx, int variant = 0);
int cluster_solve(cps_sys s, const double* b, const double* x, double* y, double rtol,
                  long long max_iter, cudaStream_t stream,
                  int variant = 0);
int persistent_solve(cps_sys s, int reduced, const double* a, const int32_t* col,
                     const double* sc, double* y, double* r, double* p, double* q, double* t,
                     int64_t n, int64_t nR, const void* win_base, size_t win_bytes, int grid,
                     cudaStream_t stream, double* z = nullptr, const double* dinv = nullptr,
                     const double* dpiv = nullptr);
int persistent_max_grid(cps_sys s, int reduced);
bool l2_vectors_fit(cps_sys s);
bool l2_window_fits_mode(cps_sys s, int mode);
void drop_graphs(cps_sys s, int prec);
int export_impl(cps_sys sys, double* diag, int32_t* col, double* val, cudaStream_t stream);
void free_sys(cps_sys sys);
void free_cp2(cps_sys sys);
int cp2_setup_impl(cps_sys sys, const double* xy, const int32_t* tri, const double* eps,
                   const double* kinv, cudaStream_t stream);
int cp2_step_impl(cps_sys sys, const double* u23, const double* g_k, double* eta_tilde,
                  double* eta, double* u_next, double* g_next, double* flux, double rtol,
                  int64_t max_iter, int precision, cps_stats* stats, cudaStream_t stream);
int cp2_kernel_times(cps_sys sys, float* ms);
void free_cp1(cps_sys sys);
int cp1_setup_impl(cps_sys sx, cps_sys sy, const double* xy, const int32_t* tri,
                   const double* eps, const double* kinv, cudaStream_t stream);
int cp1_step_impl(cps_sys sx, cps_sys sy, const double* du_breve, double* du, double toll,
                  int64_t max_outer, double rtol, int64_t max_iter, int precision,
                  cps_cp1_stats* stats, cudaStream_t stream);

}  // namespace cps
