// Preconditioned conjugate gradients on the device (Sec. 3.2.2: the
// corrector systems are solved by PCG; the matrix is assembled and factored
// once and reused for every right-hand side, Sec. 3.1).
//
// Jacobi-PCG on A runs as plain CG on the symmetrically scaled matrix
// Ahat = S^-1 A S^-1 (S = diag(sqrt(a_ee)), unit diagonal): with yhat = S x
// and bhat = S^-1 b its iterates are those of Jacobi-PCG on A, and the
// diagonal is never read inside the loop.  IC(0) runs in a colour order
// (precond.cu) on the same scaled matrix.  The kernels are in
// pcg_kernels.cuh; the scalars of the iteration never leave the device, and
// the host polls a stop flag once per chunk of iterations replayed from a
// CUDA graph.
//
// Mixed precision (CPS_MIXED): binary32 matrix, vectors and SpMV in the
// iteration, FP64 dot products and alpha/beta.  The binary32 recursion's
// residual is replaced by the true FP64 residual r = b - A x each time it has
// dropped by a factor kDelta (reliable updates: the correction is folded into
// the FP64 iterate x and the search direction is kept), until
// ||b - A x||_2 <= rtol ||b||_2 holds in FP64.
#include "cps_internal.cuh"
#include "pcg_kernels.cuh"

#include <cmath>

namespace cps {

namespace {
constexpr int kChunk = 32;          // iterations per graph replay
constexpr int kCheckEvery = 8;      // stop test period inside a chunk
constexpr double kDelta = 0.5;      // residual drop between reliable updates
constexpr int kMaxUpdates = 2000;
constexpr double kDiverge = 1e4;    // mixed: ||r||^2 this far above the best ends the solve
constexpr int64_t kTuneMinRows = 1 << 17;   // smaller systems keep the defaults
constexpr int kTuneIters = 32;               // iterations per timed candidate
}  // namespace

static int ensure_capture_stream(cps_sys s) {
    if (!s->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cps::set_error(s->ctx, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            return CPS_ERR_CUDA;
        }
    }
    return CPS_OK;
}

// Operands of one CG run in working precision V, in solve order.
template <typename V>
struct Run {
    const V* a;
    const int32_t* col;
    const V* s;
    const V* l;        // IC(0) factor (null: Jacobi)
    const V* dinv;
    V* y;
    V* r;
    V* p0;
    V* p1;
    V* q;
    V* z;              // == r for Jacobi
    int64_t n;
};

template <typename V>
static Run<V> make_run(cps_sys s);

template <>
Run<double> make_run<double>(cps_sys s) {
    const bool ic0 = s->precond == CPS_PC_IC0;
    Run<double> v{};
    v.a = ic0 ? s->pa : s->a;
    v.col = ic0 ? s->pcol : s->col;
    v.s = ic0 ? s->ps : s->s;
    v.l = ic0 ? s->pl : nullptr;
    v.dinv = ic0 ? s->pdinv : nullptr;
    v.y = s->wy;
    v.r = s->wr;
    v.p0 = s->wp0;
    v.p1 = s->wp1;
    v.q = s->wq;
    v.z = ic0 ? s->wz : s->wr;
    v.n = s->nt;
    return v;
}

// binary32 vectors reuse the first half of the FP64 work buffers.
template <>
Run<float> make_run<float>(cps_sys s) {
    const bool ic0 = s->precond == CPS_PC_IC0;
    Run<float> v{};
    v.a = ic0 ? s->pa32 : s->a32;
    v.col = ic0 ? s->pcol : s->col;
    v.s = ic0 ? s->ps32 : s->s32;
    v.l = ic0 ? s->pl32 : nullptr;
    v.dinv = ic0 ? s->pdinv32 : nullptr;
    v.y = reinterpret_cast<float*>(s->wy);
    v.r = reinterpret_cast<float*>(s->wr);
    v.p0 = reinterpret_cast<float*>(s->wp0);
    v.p1 = reinterpret_cast<float*>(s->wp1);
    v.q = reinterpret_cast<float*>(s->wq);
    v.z = ic0 ? reinterpret_cast<float*>(s->wz) : v.r;
    v.n = s->nt;
    return v;
}


// ------------------------------------------------------------ launch configs
// Each streaming kernel of the iteration runs with a (rows-per-thread
// unroll U, grid) pair picked by the autotuner below.  (Programmatic
// dependent launch between the iteration kernels was measured slower than
// plain graph edges on GB300 -- 65.6 against 55 us per iteration at 2.1M
// cells -- and is not used.)

template <typename... KArgs, typename... Args>
static void launch_k(void (*kernel)(KArgs...), int grid, cudaStream_t st, Args... args) {
    kernel<<<grid, kBlock, 0, st>>>(static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
static void launch_kb(void (*kernel)(KArgs...), int grid, int block, cudaStream_t st,
                      Args... args) {
    kernel<<<grid, block, 0, st>>>(static_cast<KArgs>(args)...);
}

template <typename V>
static void launch_a(const KCfg& c, const Run<V>& v, cps_sys s, cudaStream_t st);

// FP64 iteration kernels: (unroll, block size) picks the instantiation.
#define CPS_FP64_SHAPES(KERNEL_U_B, ...)                                                  \
    switch (c.unroll * 2048 + c.block) {                                                  \
        case 1 * 2048 + 1024:                                                             \
            launch_kb(KERNEL_U_B(1, 1024), c.grid, 1024, __VA_ARGS__);                    \
            break;                                                                        \
        case 2 * 2048 + 1024:                                                             \
            launch_kb(KERNEL_U_B(2, 1024), c.grid, 1024, __VA_ARGS__);                    \
            break;                                                                        \
        case 4 * 2048 + 1024:                                                             \
            launch_kb(KERNEL_U_B(4, 1024), c.grid, 1024, __VA_ARGS__);                    \
            break;                                                                        \
        case 1 * 2048 + kBlock:                                                           \
            launch_kb(KERNEL_U_B(1, kBlock), c.grid, kBlock, __VA_ARGS__);                \
            break;                                                                        \
        case 4 * 2048 + kBlock:                                                           \
            launch_kb(KERNEL_U_B(4, kBlock), c.grid, kBlock, __VA_ARGS__);                \
            break;                                                                        \
        default:                                                                          \
            launch_kb(KERNEL_U_B(2, kBlock), c.grid, kBlock, __VA_ARGS__);                \
            break;                                                                        \
    }

// The vector kernels (residual and direction updates) also take 8 rows per
// trip: with two or three loads per row they need more rows in flight.
#define CPS_FP64_SHAPES_V(KERNEL_U_B, ...)                                                \
    if (c.unroll == 8 && c.block == 1024)                                                 \
        launch_kb(KERNEL_U_B(8, 1024), c.grid, 1024, __VA_ARGS__);                        \
    else if (c.unroll == 8)                                                               \
        launch_kb(KERNEL_U_B(8, kBlock), c.grid, kBlock, __VA_ARGS__);                    \
    else                                                                                  \
        CPS_FP64_SHAPES(KERNEL_U_B, __VA_ARGS__)

#define CPS_SPMV64(U, B) k_spmv_dot<double, U, B>
template <>
void launch_a<double>(const KCfg& c, const Run<double>& v, cps_sys s, cudaStream_t st) {
    CPS_FP64_SHAPES(CPS_SPMV64, st, v.a, v.col, v.p0, v.q, v.n, s->partials, s->st)
}

template <>
void launch_a<float>(const KCfg& c, const Run<float>& v, cps_sys s, cudaStream_t st) {
    switch (c.unroll) {
        case 1: launch_k(k_cg_a<float, 1>, c.grid, st, v.a, v.col, v.z, v.p0, v.p1, v.y, v.q, v.n, s->partials, s->st); break;
        case 4: launch_k(k_cg_a<float, 4>, c.grid, st, v.a, v.col, v.z, v.p0, v.p1, v.y, v.q, v.n, s->partials, s->st); break;
        default: launch_k(k_cg_a<float, 2>, c.grid, st, v.a, v.col, v.z, v.p0, v.p1, v.y, v.q, v.n, s->partials, s->st); break;
    }
}

template <typename V, bool NORM, bool JACOBI>
static void launch_b_u(const KCfg& c, const Run<V>& v, cps_sys s, cudaStream_t st) {
    if constexpr (sizeof(V) == 8) {
#define CPS_CGB64(U, B) k_cg_b<double, NORM, JACOBI, U, B>
        CPS_FP64_SHAPES_V(CPS_CGB64, st, v.r, v.q, v.s, v.n, s->partials, s->st)
#undef CPS_CGB64
    } else {
        switch (c.unroll) {
            case 1: launch_k(k_cg_b<V, NORM, JACOBI, 1>, c.grid, st, v.r, v.q, v.s, v.n, s->partials, s->st); break;
            case 4: launch_k(k_cg_b<V, NORM, JACOBI, 4>, c.grid, st, v.r, v.q, v.s, v.n, s->partials, s->st); break;
            default: launch_k(k_cg_b<V, NORM, JACOBI, 2>, c.grid, st, v.r, v.q, v.s, v.n, s->partials, s->st); break;
        }
    }
}

template <typename V>
static void launch_b(const KCfg& c, const Run<V>& v, bool norm, cps_sys s, cudaStream_t st) {
    const bool jac = v.l == nullptr;
    if (norm && jac) launch_b_u<V, true, true>(c, v, s, st);
    else if (norm) launch_b_u<V, true, false>(c, v, s, st);
    else if (jac) launch_b_u<V, false, true>(c, v, s, st);
    else launch_b_u<V, false, false>(c, v, s, st);
}

#define CPS_CGC64(U, B) k_cg_c<double, U, B>
static void launch_c(const KCfg& c, const Run<double>& v, cps_sys s, cudaStream_t st) {
    CPS_FP64_SHAPES_V(CPS_CGC64, st, v.y, v.p0, v.z, v.n, s->st)
}

// The update kernel keeps five loaded vectors per row in registers: with
// 1024-thread blocks (64 registers a thread) more than two rows per trip
// spill, so those shapes take two (and are not instantiated).
static void launch_gear_update(const KCfg& c, const Run<double>& v, cps_sys s,
                               cudaStream_t st) {
    if (c.block == 1024) {
        if (c.unroll == 1)
            launch_kb(k_gear_update<1, 1024>, c.grid, 1024, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st);
        else
            launch_kb(k_gear_update<2, 1024>, c.grid, 1024, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st);
        return;
    }
    switch (c.unroll) {
        case 1: launch_kb(k_gear_update<1, kBlock>, c.grid, kBlock, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st); break;
        case 4: launch_kb(k_gear_update<4, kBlock>, c.grid, kBlock, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st); break;
        case 8: launch_kb(k_gear_update<8, kBlock>, c.grid, kBlock, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st); break;
        default: launch_kb(k_gear_update<2, kBlock>, c.grid, kBlock, st, v.y, v.r, v.p0, v.q, v.p1, v.n, s->st); break;
    }
}

static void launch_gear_spmv(const KCfg& c, const Run<double>& v, bool norm, cps_sys s,
                             cudaStream_t st) {
    if (norm) {
#define CPS_GEARS64(U, B) k_gear_spmv<true, U, B>
        CPS_FP64_SHAPES(CPS_GEARS64, st, v.a, v.col, v.r, v.p1, v.s, v.n, s->partials, s->st)
#undef CPS_GEARS64
    } else {
#define CPS_GEARS64(U, B) k_gear_spmv<false, U, B>
        CPS_FP64_SHAPES(CPS_GEARS64, st, v.a, v.col, v.r, v.p1, v.s, v.n, s->partials, s->st)
#undef CPS_GEARS64
    }
}

// One single-reduction FP64 Jacobi iteration: the update kernel with its own
// tuned shape (the residual update's until the path probe has timed it), the
// SpMV with the SpMV's.
static int64_t enqueue_iteration_gear(cps_sys s, const Run<double>& v, bool norm,
                                      cudaStream_t st) {
    const Tuning& t = s->tune[CPS_FP64];
    launch_gear_update(t.kg_set ? t.kg : t.k[1], v, s, st);
    launch_gear_spmv(t.k[0], v, norm, s, st);
    return 2;
}

static Tuning default_tuning(cps_sys s) {
    Tuning t;
    for (auto& k : t.k) {
        k.unroll = 2;
        k.grid = grid_for(s->ctx, s->nt);
    }
    return t;
}

// The context's remembered choices for systems of this mesh size.
// f(entry) runs under the context's lock (solves of different systems may
// run on different host threads).
template <typename F>
static void update_cached_tuning(cps_sys s, int prec, F f) {
    std::lock_guard<std::mutex> lock(s->ctx->mu);
    f(s->ctx->tune_cache[{s->nt, s->nv}][prec]);
}

template <typename V>
static int64_t enqueue_iteration(cps_sys s, const Run<V>& v, int prec, bool norm, cudaStream_t st);

// Picks the launch shape of every iteration kernel by timing whole
// iterations on the system's own matrix: coordinate descent over the
// kernels (SpMV, residual update, direction update), each candidate timed
// as kTuneIters consecutive iterations with the other kernels at their
// current choice.  Timing a kernel alone, with its operands warm in L2 from
// the repetition before, ranks candidates differently from the loop.  The
// vectors are scratch here (a CG run on positive constant data, primed so
// that it never stops); the caller starts the run afresh afterwards.
template <typename V>
static int autotune(cps_sys s, int prec, const Run<V>& v, cudaStream_t stream) {
    Tuning& t = s->tune[prec];
    {
        const Tuning d = default_tuning(s);     // kernel shapes only: a chosen path stays
        for (int k = 0; k < 3; ++k) t.k[k] = d.k[k];
    }
    t.done = true;
    if (s->nt < kTuneMinRows) return CPS_OK;
    const size_t vb = sizeof(V) * (size_t)s->nt;
    // 0x3F bytes: a small positive value in binary32 and in binary64
    V* const scratch[4] = {v.r, v.p0, v.p1, v.z};
    for (int k = 0; k < 4; ++k)
        CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(scratch[k], 0x3F, vb, stream));
    CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(v.y, 0, vb, stream));
    CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(v.q, 0, vb, stream));
    cudaEvent_t e0, e1;
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e0));
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e1));
    int rc = ensure_capture_stream(s);
    if (rc) return rc;
    // kTuneIters iterations as one graph (as the solve replays them), timed
    // three times; the first run warms up
    auto time_loop = [&]() -> float {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t ge = nullptr;
        if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess) {
            rc = CPS_ERR_CUDA;
            return 1e30f;
        }
        for (int k = 0; k < kTuneIters; ++k)
            enqueue_iteration<V>(s, v, prec, (k % kCheckEvery) == kCheckEvery - 1, s->cap_stream);
        const cudaError_t le = cudaGetLastError();
        const cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess ||
            cudaGraphInstantiate(&ge, graph, 0) != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            rc = CPS_ERR_CUDA;
            return 1e30f;
        }
        cudaGraphDestroy(graph);
        float best = 1e30f;
        for (int rep = 0; rep < 3 && rc == CPS_OK; ++rep) {
            k_tune_prime<<<1, 1, 0, stream>>>(s->st);
            cudaEventRecord(e0, stream);
            cudaGraphLaunch(ge, stream);
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = ms < best ? ms : best;
        }
        cudaGraphExecDestroy(ge);
        return best;
    };
    // candidates: rows per thread per trip x (block size, blocks per SM)
    const int unrolls[4] = {1, 2, 4, 8};       // 8: FP64 vector kernels only
    struct Shape {
        int block, per_sm;
    };
    const Shape shapes64[5] = {{kBlock, 4}, {kBlock, 8}, {kBlock, 16}, {1024, 1}, {1024, 2}};
    const int nshapes = sizeof(V) == 8 ? 5 : 3;       // binary32 kernels: 256 threads
    const int nk = sizeof(V) == 8 ? 3 : 2;
    for (int kind = 0; kind < nk && rc == CPS_OK; ++kind) {
        KCfg keep = t.k[kind];
        float best = time_loop();
        const int nu = (sizeof(V) == 8 && kind > 0) ? 4 : 3;
        for (int ui = 0; ui < nu && rc == CPS_OK; ++ui)
            for (int gi = 0; gi < nshapes && rc == CPS_OK; ++gi) {
                const Shape sh = shapes64[gi];
                KCfg c;
                c.unroll = unrolls[ui];
                c.block = sh.block;
                c.grid = grid_for(s->ctx, s->nt * kBlock / sh.block, sh.per_sm);
                if (c.unroll == keep.unroll && c.block == keep.block && c.grid == keep.grid)
                    continue;
                t.k[kind] = c;
                const float ms = time_loop();
                if (ms < best) {
                    best = ms;
                    keep = c;
                }
            }
        t.k[kind] = keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) rc = CPS_ERR_CUDA;
    if (rc) {
        cps::set_error(s->ctx, "autotune: kernel launch failed");
        return rc;
    }
    update_cached_tuning(s, prec, [&](Tuning& c) {
        for (int k = 0; k < 3; ++k) c.k[k] = t.k[k];
        c.done = true;
    });
    return CPS_OK;
}

// z = M^-1 r with the IC(0) colour sweeps; also rho = r.z and beta.
template <typename V>
static int64_t enqueue_precond(cps_sys s, const Run<V>& v, cudaStream_t st) {
    const int C = s->ncolours;
    const int64_t* cs = s->colour_start;
    const int g = s->grid;
    int64_t launches = 0;
    for (int c = 1; c < C; ++c, ++launches)
        launch_k(k_ic0_fwd<V>, g, st, v.l, v.col, v.dinv, v.r, v.z, v.n, cs[c], cs[c + 1], cs[1],
                   c == C - 1 ? 1 : 0, c, s->partials, s->st);
    for (int c = C - 2; c >= 0; --c, ++launches)
        launch_k(k_ic0_bwd<V>, g, st, v.l, v.col, v.dinv, v.r, v.z, v.n, cs[c], cs[c + 1], C, c,
                   s->partials, s->st);
    if (C == 1) {
        launch_k(k_ic0_bwd<V>, g, st, v.l, v.col, v.dinv, v.r, v.z, v.n, cs[0], cs[1], C, 0,
                   s->partials, s->st);
        ++launches;
    }
    return launches;
}

template <typename V>
static int64_t enqueue_iteration(cps_sys s, const Run<V>& v, int prec, bool norm, cudaStream_t st) {
    const Tuning& t = s->tune[prec];
    int64_t nl = 2;
    launch_a<V>(t.k[0], v, s, st);
    launch_b<V>(t.k[1], v, norm, s, st);
    if (v.l) nl += enqueue_precond<V>(s, v, st);
    if constexpr (sizeof(V) == 8) {
        launch_c(t.k[2], v, s, st);
        ++nl;
    }
    return nl;
}

// Persisting L2 access-policy windows of a FP64 Jacobi run: mode 1 holds
// the matrix (values and columns, one allocation; re-read every iteration),
// mode 2 the vectors r, p and q (one contiguous range; each is read and
// written every iteration, 64 of the 117 bytes a row moves).  At a few
// million cells either fits GB300's 129 MB L2 next to the streamed rest.
// Mode 3, for the single-reduction loop, holds r, p, q (= s), y and p1
// (= w): every vector that loop reads and writes (five contiguous slices);
// mode 4, for the single-reduction IC(0) loop, also z (six slices).
static void* l2_window_base(cps_sys s, int mode) {
    return mode == 1 ? (void*)s->a : (void*)s->wr;
}
static size_t l2_window_bytes(cps_sys s, int mode) {
    if (mode == 1) return s->mat_bytes;
    return (size_t)(mode == 4 ? 6 : (mode == 3 ? 5 : 3)) * s->vec_stride * sizeof(double);
}
static bool l2_window_fits(cps_sys s, int mode) {
    return s->ctx->l2_persist_max > 0 && l2_window_bytes(s, mode) <= s->ctx->l2_persist_max;
}

bool l2_vectors_fit(cps_sys s) { return l2_window_fits(s, 2); }
bool l2_window_fits_mode(cps_sys s, int mode) { return l2_window_fits(s, mode); }

// Forgets the chunk graphs of one precision (captured with launch shapes
// that have changed).
void drop_graphs(cps_sys s, int prec) {
    for (int pc = 0; pc < 4; ++pc)
        if (s->graph[prec][pc]) {
            cudaGraphExecDestroy(s->graph[prec][pc]);
            s->graph[prec][pc] = nullptr;
        }
}

// The persisting set-aside is a context-wide reservation that shrinks the L2
// every other kernel sees, so it is held only for the duration of a solve
// that uses the window and given back (set to 0) right after.
// Solves running at the same time on one context (host threads) share the
// set-aside: one may give it back while another's window is in use, which
// costs speed, not correctness (persistence is a cache hint).
static int l2_set_aside(cps_sys s, int mode, cudaStream_t st) {
    const size_t want = mode ? l2_window_bytes(s, mode) : 0;
    std::unique_lock<std::mutex> lock(s->ctx->l2_mu);
    if (s->ctx->l2_persist_set == want) return CPS_OK;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && s->ctx->l2_persist_set) e = cudaCtxResetPersistingL2Cache();
    if (e == cudaSuccess) e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
    if (e != cudaSuccess) {
        lock.unlock();
        cps::set_error(s->ctx, std::string("persisting L2 set-aside: ") + cudaGetErrorString(e));
        return CPS_ERR_CUDA;
    }
    s->ctx->l2_persist_set = want;
    return CPS_OK;
}

static int set_l2_window(cps_sys s, cudaStream_t st, int mode) {
    cudaStreamAttrValue v = {};
    if (mode) {
        v.accessPolicyWindow.base_ptr = l2_window_base(s, mode);
        v.accessPolicyWindow.num_bytes = l2_window_bytes(s, mode);
        v.accessPolicyWindow.hitRatio = 1.0f;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    } else {
        v.accessPolicyWindow.num_bytes = 0;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyNormal;
        v.accessPolicyWindow.missProp = cudaAccessPropertyNormal;
    }
    CPS_CUDA_TRY(s->ctx, cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v));
    return CPS_OK;
}

template <typename V>
static int get_chunk_graph(cps_sys s, int prec, const Run<V>& v, cudaGraphExec_t* out,
                           int64_t* per_chunk, bool gear = false) {
    const int pc = gear ? 3 : (v.l ? 1 : 0);
    const int win = (prec == CPS_FP64 && (pc == 0 || pc == 3)) ? s->tune[CPS_FP64].l2win : 0;
    if (s->graph[prec][pc] && s->graph_l2win[prec][pc] != win) {
        cudaGraphExecDestroy(s->graph[prec][pc]);
        s->graph[prec][pc] = nullptr;
    }
    cudaGraphExec_t& ge = s->graph[prec][pc];
    int64_t nl = 0;
    if (!ge) {
        int rc = ensure_capture_stream(s);
        if (rc) return rc;
        rc = set_l2_window(s, s->cap_stream, win);
        if (rc) return rc;
        s->graph_l2win[prec][pc] = win;
        cudaGraph_t graph = nullptr;
        CPS_CUDA_TRY(s->ctx, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kChunk; ++k) {
            const bool norm = (k % kCheckEvery) == kCheckEvery - 1;
            if constexpr (sizeof(V) == 8) {
                if (gear) {
                    nl += enqueue_iteration_gear(s, v, norm, s->cap_stream);
                    continue;
                }
            }
            nl += enqueue_iteration<V>(s, v, prec, norm, s->cap_stream);
        }
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cps::set_error(s->ctx, std::string("graph capture: ") +
                                 cudaGetErrorString(le != cudaSuccess ? le : ce));
            return CPS_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            ge = nullptr;
            cps::set_error(s->ctx, std::string("graph instantiate: ") + cudaGetErrorString(ie));
            return CPS_ERR_CUDA;
        }
        s->graph_nodes[prec][pc] = nl;
        if (win) {
            rc = set_l2_window(s, s->cap_stream, 0);
            if (rc) return rc;
        }
    }
    *per_chunk = s->graph_nodes[prec][pc];
    *out = ge;
    return CPS_OK;
}

// Replays iteration chunks until the device sets st->done.  One chunk of
// look-ahead keeps the GPU busy while the host reads the previous flag; a
// chunk enqueued after the stop returns at once in every kernel.
template <typename V>
static int run_chunks(cps_sys s, int prec, const Run<V>& v, cudaStream_t stream,
                      CgState* final_state, int64_t* launches, bool gear = false) {
    cudaGraphExec_t ge = nullptr;
    int64_t per_chunk = 0;
    int rc = get_chunk_graph<V>(s, prec, v, &ge, &per_chunk, gear);
    if (rc) return rc;
    for (long long k = 0;; ++k) {
        const int slot = (int)(k & 1);
        CPS_CUDA_TRY(s->ctx, cudaGraphLaunch(ge, stream));
        *launches += per_chunk;
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

static void fill_stats(cps_stats* stats, int64_t iters, double rel, int status, int refinements,
                       int64_t launches) {
    if (!stats) return;
    stats->iters = iters;
    stats->rel_res = rel;
    stats->status = status;
    stats->refinements = refinements;
    stats->launches = launches;
}

// ------------------------------------------------------------------ FP64

// For Jacobi solves, times a short run (64 iterations; 256 on large systems)
// of each path that applies from x = 0 and keeps the fastest: graph-replayed
// streaming kernels, the one-launch cluster solve (systems that fit one
// cluster's shared memory), streaming with the matrix or with the vectors
// r, p, q held in persisting L2 (large systems whose window fits the
// set-aside), and the persistent grid-synchronised launch.
static int choose_fp64_path(cps_sys s, const Run<double>& v, const double* b,
                            cudaStream_t stream) {
    Tuning& t = s->tune[CPS_FP64];
    t.path_done = true;
    t.path = 0;
    t.l2win = 0;
    t.pgrid = 0;
    if (s->precond != CPS_PC_JACOBI) return CPS_OK;
    const bool try_cluster = s->nt <= cluster_max_rows(s->ctx);
    const bool big = !try_cluster && s->nt >= kTuneMinRows;
    const long long probe = s->nt >= kTuneMinRows ? 256 : 64;
    // candidates (slot in probe_us): 0 streaming, 1 one-cluster launch,
    // 2 streaming with the matrix in persisting L2, 3 one persistent
    // grid-synchronised launch, 4 streaming with the vectors r, p, q in
    // persisting L2, 5 persistent with the vectors in persisting L2,
    // 6 single-reduction streaming, 7 the same with its vectors in
    // persisting L2, 8 single-reduction persistent, 9 the same with its five
    // vectors in persisting L2.  The persistent launches are timed at a few
    // grid sizes (fewer blocks synchronise faster; more blocks move more
    // bytes).
    struct Cand {
        int slot, path, win, grid, var;
    };
    Cand cands[24];
    int nc = 0;
    cands[nc++] = {0, 0, 0, 0, 0};
    if (try_cluster) cands[nc++] = {1, 1, 0, 0, 0};
    // the single-reduction cluster solve (one barrier fewer per iteration).
    // Not the pipelined one (CPS_PATH_CLUSTER_PIPE): on the 7,938-cell
    // block it is 1.4% faster per iteration, but its recurrences drift
    // sooner and it needs 4% more iterations to 1e-10, which a per-iteration
    // probe cannot see.
    if (s->nt <= cluster_max_rows(s->ctx, 1)) cands[nc++] = {1, 1, 0, 0, 1};
    if (big && l2_window_fits(s, 1)) cands[nc++] = {2, 0, 1, 0, 0};
    if (big && l2_window_fits(s, 2)) cands[nc++] = {4, 0, 2, 0, 0};
    // single-reduction streaming (two kernels per iteration)
    if (!try_cluster) cands[nc++] = {6, 3, 0, 0, 0};
    if (big && l2_window_fits(s, 2)) cands[nc++] = {7, 3, 2, 0, 0};
    if (big && l2_window_fits(s, 3)) cands[nc++] = {7, 3, 3, 0, 0};
    {
        const int gmax = persistent_max_grid(s, 0);
        int grids[3] = {gmax, (int)((s->nt + 8191) / 8192), (int)((s->nt + 2047) / 2048)};
        for (int i = 0; i < 3; ++i) {
            const int gi = grids[i] < 1 ? 1 : (grids[i] > gmax ? gmax : grids[i]);
            bool dup = gmax <= 0;
            for (int j = 0; j < i; ++j) dup = dup || grids[j] == gi;
            grids[i] = gi;
            if (dup) continue;
            cands[nc++] = {3, 2, 0, gi, 0};
            if (big && l2_window_fits(s, 2)) cands[nc++] = {5, 2, 2, gi, 0};
        }
    }
    if (!try_cluster) {
        const int gmax = persistent_max_grid(s, 2);
        int grids[2] = {gmax, (int)((s->nt + 8191) / 8192)};
        for (int i = 0; i < 2; ++i) {
            const int gi = grids[i] < 1 ? 1 : (grids[i] > gmax ? gmax : grids[i]);
            if (gmax <= 0 || (i == 1 && gi == grids[0])) continue;
            grids[i] = gi;
            cands[nc++] = {8, 4, 0, gi, 0};
            if (big && l2_window_fits(s, 3)) cands[nc++] = {9, 4, 3, gi, 0};
        }
    }
    cudaEvent_t e0, e1;
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e0));
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e1));
    double per_iter[10] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double best_t = 0.0;
    Cand best{0, 0, 0, 0, 0};
    int rc = CPS_OK;
    cudaGraphExec_t ge = nullptr;
    int64_t per_chunk = 0, dummy = 0;
    // microseconds per iteration of one candidate (0: it cannot run here)
    auto time_cand = [&](const Cand& c) -> double {
        t.l2win = c.win;
        rc = l2_set_aside(s, c.win, stream);
        if (rc == CPS_OK && (c.path == 0 || c.path == 3))
            rc = get_chunk_graph<double>(s, CPS_FP64, v, &ge, &per_chunk, c.path == 3);
        double us = 0.0;
        for (int rep = 0; rep < 2 && rc == CPS_OK; ++rep) {   // first one warms up
            if (cudaMemsetAsync(s->wx, 0, sizeof(double) * s->nt, stream) != cudaSuccess ||
                cudaEventRecord(e0, stream) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            CgState h{};
            if (c.path == 2 || c.path == 4) {
                k_init64<<<s->grid, kBlock, 0, stream>>>(b, s->wx, v.s, v.a, v.col, s->nt, v.y, v.r,
                                                         v.p0, 0.0, probe, 1, s->partials, s->st);
                if (c.path == 4)
                    k_gear_start<<<s->grid, kBlock, 0, stream>>>(v.a, v.col, v.r, v.p1, v.p0, v.q,
                                                                 s->nt, s->partials, s->st);
                rc = persistent_solve(s, c.path == 4 ? 2 : 0, v.a, v.col, v.s, v.y, v.r, v.p0, v.q,
                                      c.path == 4 ? v.p1 : nullptr, s->nt,
                                      0, c.win ? l2_window_base(s, c.win) : nullptr,
                                      c.win ? l2_window_bytes(s, c.win) : 0, c.grid, stream);
                if (rc == CPS_OK) rc = read_state(s, stream, &h);
                if (rc == CPS_OK && h.status != CPS_OK) rc = CPS_ERR_ARG;   // not usable here
            } else if (c.path == 0 || c.path == 3) {
                k_init64<<<s->grid, kBlock, 0, stream>>>(b, s->wx, v.s, v.a, v.col, s->nt, v.y, v.r,
                                                         v.p0, 0.0, probe, 1, s->partials, s->st);
                if (c.path == 3)
                    k_gear_start<<<s->grid, kBlock, 0, stream>>>(v.a, v.col, v.r, v.p1, v.p0, v.q,
                                                                 s->nt, s->partials, s->st);
                rc = run_chunks<double>(s, CPS_FP64, v, stream, &h, &dummy, c.path == 3);
            } else {
                rc = cluster_solve(s, b, s->wx, v.y, 0.0, probe, stream, c.var);
                if (rc == CPS_OK) rc = read_state(s, stream, &h);
            }
            if (cudaEventRecord(e1, stream) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            us = rc == CPS_OK ? 1e3 * ms / (double)(h.iter > 0 ? h.iter : 1) : 0.0;
        }
        if (rc == CPS_ERR_ARG) {            // a candidate that cannot run here: skip it
            rc = CPS_OK;
            cudaGetLastError();
            return 0.0;
        }
        return rc == CPS_OK ? us : 0.0;
    };
    for (int ci = 0; ci < nc && rc == CPS_OK; ++ci) {
        const Cand c = cands[ci];
        const double us = time_cand(c);
        if (rc != CPS_OK || us <= 0.0) continue;
        if (per_iter[c.slot] == 0.0 || us < per_iter[c.slot]) per_iter[c.slot] = us;
        if (best_t == 0.0 || us < best_t) {
            best_t = us;
            best = c;
        }
    }
    // The single-reduction update kernel moves 72 bytes a row (the residual
    // update whose tuned shape it starts from moves 24): time a few shapes of
    // its own on the chosen loop and keep the fastest.
    if (rc == CPS_OK && best.path == 3 && big) {
        t.path = 3;
        const KCfg start = t.kg_set ? t.kg : t.k[1];
        const KCfg shapes[5] = {start, t.k[2],
                                {2, grid_for(s->ctx, s->nt, 8), kBlock},
                                {4, grid_for(s->ctx, s->nt, 4), kBlock},
                                {2, grid_for(s->ctx, s->nt * kBlock / 1024, 2), 1024}};
        KCfg keep = start;
        double keep_t = best_t;
        for (int k = 0; k < 5 && rc == CPS_OK; ++k) {
            if (k > 0 && shapes[k].unroll == keep.unroll && shapes[k].grid == keep.grid &&
                shapes[k].block == keep.block)
                continue;
            t.kg = shapes[k];
            t.kg_set = true;
            if (s->graph[CPS_FP64][3]) {
                cudaGraphExecDestroy(s->graph[CPS_FP64][3]);
                s->graph[CPS_FP64][3] = nullptr;
            }
            const double us = time_cand(best);
            if (rc == CPS_OK && us > 0.0 && us < keep_t) {
                keep_t = us;
                keep = shapes[k];
            }
        }
        t.kg = keep;
        t.kg_set = true;
        if (s->graph[CPS_FP64][3]) {
            cudaGraphExecDestroy(s->graph[CPS_FP64][3]);
            s->graph[CPS_FP64][3] = nullptr;
        }
        best_t = keep_t;
        per_iter[best.slot] = keep_t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        const int rc2 = l2_set_aside(s, 0, stream);
        if (rc == CPS_OK) rc = rc2;
    }
    t.l2win = 0;
    if (rc == CPS_OK) {
        t.path = best.path;
        t.l2win = best.win;
        t.pgrid = best.grid;
        t.cluster_variant = best.var;
    }
    for (int k = 0; k < 10; ++k) t.probe_us[k] = per_iter[k];
    if (rc == CPS_OK) {
        update_cached_tuning(s, CPS_FP64, [&](Tuning& c) {
            c.path_done = true;
            c.path = t.path;
            c.l2win = t.l2win;
            c.pgrid = t.pgrid;
            c.cluster_variant = t.cluster_variant;
            c.kg = t.kg;
            c.kg_set = t.kg_set;
            for (int k = 0; k < 10; ++k) c.probe_us[k] = t.probe_us[k];
        });
    }
    return rc;
}

// One persistent single-reduction IC(0) run from the state k_init64 left
// (colour order, two colours), with persisting L2 window `win` (the caller
// holds its set-aside) on `grid` blocks (0: all that stay resident).
static int persistent_ic0(cps_sys s, int win, cudaStream_t stream) {
    return persistent_solve(s, 3, s->pa, s->pcol, s->ps, s->wy, s->wr, s->wp0, s->wq, s->wp1,
                            s->nt, s->colour_start[1], win ? l2_window_base(s, win) : nullptr,
                            win ? l2_window_bytes(s, win) : 0, 0, stream, s->wz, s->pdinv,
                            s->pdiag);
}

// For IC(0) on a two-colour order: times a short run (64 iterations; 256 on
// large systems) of the graph-replayed streaming kernels and of the
// persistent single-reduction launch (without and, where the set-aside holds
// them, with its six vectors in persisting L2) and keeps the fastest.  bb is
// the right-hand side in colour order.
static int choose_ic0_path(cps_sys s, const Run<double>& v, const double* bb,
                           cudaStream_t stream) {
    Tuning& t = s->tune[CPS_FP64];
    t.ic0_done = true;
    t.ic0_path = 0;
    t.ic0_win = 0;
    if (s->ncolours != 2) return CPS_OK;
    const long long probe = s->nt >= kTuneMinRows ? 256 : 64;
    struct Cand {
        int path, win;
    };
    Cand cands[3];
    int nc = 0;
    cands[nc++] = {0, 0};
    if (persistent_max_grid(s, 3) > 0) {
        cands[nc++] = {1, 0};
        // six vectors in persisting L2 where they fit, else the first five
        // (xh, rh, p, s, w: all but v / z)
        if (s->nt >= kTuneMinRows && l2_window_fits(s, 4)) cands[nc++] = {1, 4};
        else if (s->nt >= kTuneMinRows && l2_window_fits(s, 3)) cands[nc++] = {1, 3};
    }
    cudaEvent_t e0, e1;
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e0));
    CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e1));
    double per_iter[2] = {0.0, 0.0};
    double best_t = 0.0;
    Cand best{0, 0};
    int rc = CPS_OK;
    int64_t dummy = 0;
    for (int ci = 0; ci < nc && rc == CPS_OK; ++ci) {
        const Cand c = cands[ci];
        rc = l2_set_aside(s, c.win, stream);
        double us = 0.0;
        for (int rep = 0; rep < 2 && rc == CPS_OK; ++rep) {    // the first one warms up
            if (cudaMemsetAsync(s->wx, 0, sizeof(double) * s->nt, stream) != cudaSuccess ||
                cudaEventRecord(e0, stream) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            k_init64<<<s->grid, kBlock, 0, stream>>>(bb, s->wx, v.s, v.a, v.col, s->nt, v.y, v.r,
                                                     v.p0, 0.0, probe, 0, s->partials, s->st);
            CgState h{};
            if (c.path == 1) {
                rc = persistent_ic0(s, c.win, stream);
                if (rc == CPS_OK) rc = read_state(s, stream, &h);
                if (rc == CPS_OK && h.status != CPS_OK) rc = CPS_ERR_ARG;   // not usable here
            } else {
                enqueue_precond<double>(s, v, stream);
                k_copy<double><<<s->grid, kBlock, 0, stream>>>(v.p0, v.z, s->nt);
                rc = run_chunks<double>(s, CPS_FP64, v, stream, &h, &dummy);
            }
            if (cudaEventRecord(e1, stream) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            us = rc == CPS_OK ? 1e3 * ms / (double)(h.iter > 0 ? h.iter : 1) : 0.0;
        }
        if (rc == CPS_ERR_ARG) {            // a candidate that cannot run here: skip it
            rc = CPS_OK;
            cudaGetLastError();
            continue;
        }
        if (rc != CPS_OK || us <= 0.0) continue;
        if (per_iter[c.path] == 0.0 || us < per_iter[c.path]) per_iter[c.path] = us;
        if (best_t == 0.0 || us < best_t) {
            best_t = us;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        const int rc2 = l2_set_aside(s, 0, stream);
        if (rc == CPS_OK) rc = rc2;
    }
    if (rc != CPS_OK) return rc;
    t.ic0_path = best.path;
    t.ic0_win = best.win;
    t.ic0_probe_us[0] = per_iter[0];
    t.ic0_probe_us[1] = per_iter[1];
    update_cached_tuning(s, CPS_FP64, [&](Tuning& cc) {
        cc.ic0_done = true;
        cc.ic0_path = t.ic0_path;
        cc.ic0_win = t.ic0_win;
        cc.ic0_probe_us[0] = per_iter[0];
        cc.ic0_probe_us[1] = per_iter[1];
    });
    return CPS_OK;
}

static int solve_fp64(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
                      cps_stats* stats, cudaStream_t stream) {
    const int64_t n = s->nt;
    const int g = s->grid;
    const bool ic0 = s->precond == CPS_PC_IC0;
    const Run<double> v = make_run<double>(s);
    const double* bb = b;
    double* xx = x;
    int64_t total = 0, launches = 0;
    if (!s->tune[CPS_FP64].done) {
        int rc = autotune<double>(s, CPS_FP64, v, stream);
        if (rc) return rc;
    }
    if (!ic0 && !s->tune[CPS_FP64].path_done) {
        int rc = choose_fp64_path(s, v, b, stream);
        if (rc) return rc;
    }
    const bool cluster = !ic0 && s->tune[CPS_FP64].path == 1;
    const bool persistent = !ic0 && (s->tune[CPS_FP64].path == 2 || s->tune[CPS_FP64].path == 4);
    const bool pgear = !ic0 && s->tune[CPS_FP64].path == 4;
    const bool gear = !ic0 && s->tune[CPS_FP64].path == 3;
    const int window = (!ic0 && !cluster) ? s->tune[CPS_FP64].l2win : 0;
    if (window) {
        int rc = l2_set_aside(s, window, stream);
        if (rc) return rc;
    }
    if (ic0) {
        k_permute_in<<<g, kBlock, 0, stream>>>(b, x, s->perm, n, s->wb, s->wx);
        ++launches;
        bb = s->wb;
        xx = s->wx;
        if (!s->tune[CPS_FP64].ic0_done) {
            // the probe runs from x = 0 in wx: keep the caller's start in wbest
            CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(s->wbest, s->wx, sizeof(double) * n,
                                                 cudaMemcpyDeviceToDevice, stream));
            int rc = choose_ic0_path(s, v, bb, stream);
            if (rc) return rc;
            CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(s->wx, s->wbest, sizeof(double) * n,
                                                 cudaMemcpyDeviceToDevice, stream));
        }
    }
    const bool pic0 = ic0 && s->ncolours == 2 && s->tune[CPS_FP64].ic0_path == 1;
    const int ic0_window = pic0 ? s->tune[CPS_FP64].ic0_win : 0;
    if (ic0_window) {
        int rc = l2_set_aside(s, ic0_window, stream);
        if (rc) return rc;
    }
    CgState h{};
    int status = CPS_OK;
    // A restart recomputes r = b - A x when the recursively updated residual
    // has met rtol but the true residual has not (rounding drift).
    for (int restart = 0; restart < 8; ++restart) {
        const long long budget = (long long)(max_iter - total);
        if (cluster) {
            int rc = cluster_solve(s, bb, xx, v.y, rtol, budget, stream,
                                   s->tune[CPS_FP64].cluster_variant);
            if (rc) return rc;
            ++launches;
            CgState hc{};
            rc = read_state(s, stream, &hc);
            if (rc) return rc;
            total += hc.iter;
            status = hc.status;
            k_final64<<<g, kBlock, 0, stream>>>(bb, v.y, v.s, v.a, v.col, n, xx, s->partials, s->st);
            ++launches;
            CPS_CUDA_TRY(s->ctx, cudaGetLastError());
            rc = read_state(s, stream, &h);
            if (rc) return rc;
            if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
            continue;
        }
        k_init64<<<g, kBlock, 0, stream>>>(bb, xx, v.s, v.a, v.col, n, v.y, v.r, v.p0, rtol,
                                            budget, ic0 ? 0 : 1, s->partials, s->st);
        ++launches;
        if (pic0) {
            // one launch runs to the stop (it returns at once if init stopped)
            int rc = persistent_ic0(s, ic0_window, stream);
            if (rc) return rc;
            ++launches;
            rc = read_state(s, stream, &h);
            if (rc) return rc;
            total += h.iter;
            status = h.status;
            k_final64<<<g, kBlock, 0, stream>>>(bb, v.y, v.s, v.a, v.col, n, xx, s->partials,
                                                s->st);
            ++launches;
            CPS_CUDA_TRY(s->ctx, cudaGetLastError());
            rc = read_state(s, stream, &h);
            if (rc) return rc;
            if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
            continue;
        }
        if (persistent) {
            if (pgear) {
                k_gear_start<<<g, kBlock, 0, stream>>>(v.a, v.col, v.r, v.p1, v.p0, v.q, n,
                                                       s->partials, s->st);
                ++launches;
            }
            // one launch runs to the stop (it returns at once if init stopped)
            int rc = persistent_solve(s, pgear ? 2 : 0, v.a, v.col, v.s, v.y, v.r, v.p0, v.q,
                                      pgear ? v.p1 : nullptr, n, 0,
                                      window ? l2_window_base(s, window) : nullptr,
                                      window ? l2_window_bytes(s, window) : 0,
                                      s->tune[CPS_FP64].pgrid, stream);
            if (rc) return rc;
            ++launches;
            rc = read_state(s, stream, &h);
            if (rc) return rc;
            total += h.iter;
            status = h.status;
            k_final64<<<g, kBlock, 0, stream>>>(bb, v.y, v.s, v.a, v.col, n, xx, s->partials,
                                                s->st);
            ++launches;
            CPS_CUDA_TRY(s->ctx, cudaGetLastError());
            rc = read_state(s, stream, &h);
            if (rc) return rc;
            if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
            continue;
        }
        if (ic0) {
            launches += enqueue_precond<double>(s, v, stream);
            k_copy<double><<<g, kBlock, 0, stream>>>(v.p0, v.z, n);
            ++launches;
        }
        if (gear) {
            k_gear_start<<<g, kBlock, 0, stream>>>(v.a, v.col, v.r, v.p1, v.p0, v.q, n,
                                                   s->partials, s->st);
            ++launches;
        }
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        int rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (!h.done && budget > 0) {
            rc = run_chunks<double>(s, CPS_FP64, v, stream, &h, &launches, gear);
            if (rc) return rc;
        }
        total += h.iter;
        status = h.status;
        k_final64<<<g, kBlock, 0, stream>>>(bb, v.y, v.s, v.a, v.col, n, xx, s->partials, s->st);
        ++launches;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
    }
    if (ic0) {
        k_permute_out<<<g, kBlock, 0, stream>>>(s->wx, s->perm, n, x);
        ++launches;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    }
    if (window || ic0_window) {
        // release the lines and the set-aside: later work gets the whole L2
        int rc = l2_set_aside(s, 0, stream);
        if (rc) return rc;
    }
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    if (status == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) status = CPS_ERR_NOT_CONVERGED;
    fill_stats(stats, total, rel, status, 1, launches);
    if (status == CPS_ERR_NOT_SPD) cps::set_error(s->ctx, "solve: p.Ap <= 0 (matrix not SPD or NaN input)");
    if (status == CPS_ERR_TIMEOUT) cps::set_error(s->ctx, "solve: a grid barrier wait ran out");
    if (status == CPS_ERR_NOT_CONVERGED)
        cps::set_error(s->ctx, total >= max_iter
                                   ? "solve: max_iter reached"
                                   : "solve: the true residual stays above rtol (FP64 rounding "
                                     "floor of this system and right-hand side)");
    return status;
}

// ------------------------------------------------------------ reduced system

// CG on the black-cell Schur complement of the two-coloured scaled system
// (kernels at the end of pcg_kernels.cuh); the red unknowns are recovered
// exactly at the end, and the true residual of the full system decides.
static int solve_reduced(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
                         cps_stats* stats, cudaStream_t stream) {
    const int64_t n = s->nt, nR = s->colour_start[1], nB = n - nR;
    const int g = s->grid;
    const double* A = s->pa;
    const int32_t* col = s->pcol;
    const double* S = s->ps;
    double *y = s->wy, *r = s->wr, *p = s->wp0, *q = s->wq, *t = s->wz;
    int64_t total = 0, launches = 0;
    k_permute_in<<<g, kBlock, 0, stream>>>(b, x, s->perm, n, s->wb, s->wx);
    ++launches;
    const double* bb = s->wb;
    double* xx = s->wx;
    // black-range views for the shared update kernels
    Run<double> vb{};
    vb.s = S + nR;
    vb.y = y + nR;
    vb.r = r + nR;
    vb.p0 = p + nR;
    vb.q = q + nR;
    vb.z = r + nR;
    vb.n = nB;
    KCfg cb{2, grid_for(s->ctx, nB)};
    cudaGraphExec_t& ge = s->graph[CPS_FP64][2];
    // The chunk graph of the reduced iteration, captured with persisting-L2
    // window `win` (0 none, 2 the vectors r, p, q) on its kernel nodes.
    auto build_graph = [&](int win) -> int {
        if (ge && s->graph_l2win[CPS_FP64][2] == win) return CPS_OK;
        if (ge) {
            cudaGraphExecDestroy(ge);
            ge = nullptr;
        }
        int rc = ensure_capture_stream(s);
        if (rc) return rc;
        rc = set_l2_window(s, s->cap_stream, win);
        if (rc) return rc;
        cudaGraph_t graph = nullptr;
        int64_t nl = 0;
        CPS_CUDA_TRY(s->ctx, cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < kChunk; ++k) {
            launch_k(k_schur_red, g, s->cap_stream, A, col, (const double*)p, t, n, nR, s->st);
            launch_k(k_schur_black, g, s->cap_stream, A, col, (const double*)p,
                       (const double*)t, q, n, nR, s->partials, s->st);
            launch_b<double>(cb, vb, (k % kCheckEvery) == kCheckEvery - 1, s, s->cap_stream);
            launch_c(cb, vb, s, s->cap_stream);
            nl += 4;
        }
        cudaError_t le = cudaGetLastError();
        cudaError_t ce = cudaStreamEndCapture(s->cap_stream, &graph);
        if (win) set_l2_window(s, s->cap_stream, 0);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cps::set_error(s->ctx, std::string("graph capture: ") +
                                 cudaGetErrorString(le != cudaSuccess ? le : ce));
            return CPS_ERR_CUDA;
        }
        cudaError_t ie = cudaGraphInstantiate(&ge, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            ge = nullptr;
            cps::set_error(s->ctx, std::string("graph instantiate: ") + cudaGetErrorString(ie));
            return CPS_ERR_CUDA;
        }
        s->graph_nodes[CPS_FP64][2] = nl;
        s->graph_l2win[CPS_FP64][2] = win;
        return CPS_OK;
    };
    // Runs CG from the state k_black_init left, on the graph-replayed kernels
    // (kind 0) or in one persistent grid-synchronised launch of pgrid blocks
    // (kind 1 the textbook recurrences, 2 the single-reduction ones, with
    // s = S p in q and w = S r in p1), with window win (the caller holds its
    // set-aside); state into *hh.
    auto run_cg = [&](int kind, int win, int pgrid, CgState* hh) -> int {
        if (kind) {
            int rc = persistent_solve(s, kind == 2 ? 4 : 1, A, col, S, y, r, p, q, t, n, nR,
                                      win ? l2_window_base(s, win) : nullptr,
                                      win ? l2_window_bytes(s, win) : 0, pgrid, stream,
                                      kind == 2 ? s->wp1 : nullptr);
            if (rc) return rc;
            ++launches;
            return read_state(s, stream, hh);
        }
        int rc = build_graph(win);
        if (rc) return rc;
        rc = read_state(s, stream, hh);
        if (rc || hh->done) return rc;
        for (long long k = 0;; ++k) {
            const int slot = (int)(k & 1);
            CPS_CUDA_TRY(s->ctx, cudaGraphLaunch(ge, stream));
            launches += s->graph_nodes[CPS_FP64][2];
            CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(&s->hst[slot], s->st, sizeof(CgState),
                                                 cudaMemcpyDeviceToHost, stream));
            CPS_CUDA_TRY(s->ctx, cudaEventRecord(s->ev[slot], stream));
            if (k >= 1) {
                CPS_CUDA_TRY(s->ctx, cudaEventSynchronize(s->ev[1 - slot]));
                if (s->hst[1 - slot].done) break;
            }
        }
        return read_state(s, stream, hh);
    };
    Tuning& tu = s->tune[CPS_FP64];
    if (!tu.red_done) {
        // time a short run of each way from x = 0 and keep the fastest:
        // slot 0 graph, 1 persistent, 2 graph + window, 3 persistent + window,
        // 4 persistent single-reduction, 5 the same + its five vectors in
        // persisting L2 (persistent at a few grid sizes)
        const long long probe = nB >= kTuneMinRows ? 256 : 64;
        const bool try_win = nB >= kTuneMinRows && l2_window_fits(s, 2);
        const bool try_win5 = nB >= kTuneMinRows && l2_window_fits(s, 3);
        struct Cand {
            int slot, win, grid;
        };
        Cand cands[16];
        int nc = 0;
        cands[nc++] = {0, 0, 0};
        if (try_win) cands[nc++] = {2, 2, 0};
        for (int kind = 1; kind <= 2; ++kind) {
            const int gmax = persistent_max_grid(s, kind == 2 ? 4 : 1);
            int grids[3] = {gmax, (int)((nB + 8191) / 8192), (int)((nB + 2047) / 2048)};
            for (int i = 0; i < 3; ++i) {
                const int gi = grids[i] < 1 ? 1 : (grids[i] > gmax ? gmax : grids[i]);
                bool dup = gmax <= 0;
                for (int j = 0; j < i; ++j) dup = dup || grids[j] == gi;
                grids[i] = gi;
                if (dup) continue;
                if (kind == 1) {
                    cands[nc++] = {1, 0, gi};
                    if (try_win) cands[nc++] = {3, 2, gi};
                } else {
                    cands[nc++] = {4, 0, gi};
                    if (try_win5) cands[nc++] = {5, 3, gi};
                }
            }
        }
        cudaEvent_t e0, e1;
        CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e0));
        CPS_CUDA_TRY(s->ctx, cudaEventCreate(&e1));
        double per_iter[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        double best_t = 0.0;
        Cand best{0, 0, 0};
        int rc = CPS_OK;
        auto kind_of = [](int slot) { return slot >= 4 ? 2 : (slot & 1); };
        for (int ci = 0; ci < nc && rc == CPS_OK; ++ci) {
            const Cand c = cands[ci];
            const int kind = kind_of(c.slot);
            const bool pers = kind != 0;
            rc = l2_set_aside(s, c.win, stream);
            double us = 0.0;
            for (int rep = 0; rep < 2 && rc == CPS_OK; ++rep) {
                CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(xx, 0, sizeof(double) * n, stream));
                if (!pers) rc = build_graph(c.win);        // outside the timed region
                if (rc) break;
                CPS_CUDA_TRY(s->ctx, cudaEventRecord(e0, stream));
                k_red_recover<<<g, kBlock, 0, stream>>>(bb, xx, S, A, col, n, nR, 1, y);
                k_black_init<<<g, kBlock, 0, stream>>>(bb, xx, S, A, col, n, nR, y, r, p, 0.0,
                                                       probe, s->partials, s->st);
                CgState hp{};
                rc = run_cg(kind, c.win, c.grid, &hp);
                if (rc == CPS_OK && hp.status != CPS_OK) rc = CPS_ERR_ARG;
                CPS_CUDA_TRY(s->ctx, cudaEventRecord(e1, stream));
                CPS_CUDA_TRY(s->ctx, cudaEventSynchronize(e1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                us = rc == CPS_OK ? 1e3 * ms / (double)(hp.iter > 0 ? hp.iter : 1) : 0.0;
            }
            if (rc == CPS_ERR_ARG) {
                rc = CPS_OK;
                cudaGetLastError();
                continue;
            }
            if (rc != CPS_OK || us <= 0.0) continue;
            if (per_iter[c.slot] == 0.0 || us < per_iter[c.slot]) per_iter[c.slot] = us;
            if (best_t == 0.0 || us < best_t) {
                best_t = us;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        {
            const int rc2 = l2_set_aside(s, 0, stream);
            if (rc == CPS_OK) rc = rc2;
        }
        if (rc != CPS_OK) return rc;
        tu.red_done = true;
        tu.red_path = kind_of(best.slot);
        tu.red_win = best.win;
        tu.red_pgrid = best.grid;
        for (int c = 0; c < 6; ++c) tu.red_probe_us[c] = per_iter[c];
        update_cached_tuning(s, CPS_FP64, [&](Tuning& c) {
            c.red_done = true;
            c.red_path = tu.red_path;
            c.red_win = tu.red_win;
            c.red_pgrid = tu.red_pgrid;
            for (int k = 0; k < 6; ++k) c.red_probe_us[k] = tu.red_probe_us[k];
        });
    }
    const int kind = tu.red_path;
    const int win = tu.red_win;
    if (win) {
        int rc = l2_set_aside(s, win, stream);
        if (rc) return rc;
    }
    CgState h{};
    int status = CPS_OK;
    for (int restart = 0; restart < 8; ++restart) {
        const long long budget = (long long)(max_iter - total);
        k_red_recover<<<g, kBlock, 0, stream>>>(bb, xx, S, A, col, n, nR, 1, y);
        k_black_init<<<g, kBlock, 0, stream>>>(bb, xx, S, A, col, n, nR, y, r, p, rtol, budget,
                                               s->partials, s->st);
        launches += 2;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        int rc = run_cg(kind, win, tu.red_pgrid, &h);
        if (rc) return rc;
        total += h.iter;
        status = h.status;
        k_red_recover<<<g, kBlock, 0, stream>>>(bb, y, S, A, col, n, nR, 0, y);
        k_final64<<<g, kBlock, 0, stream>>>(bb, y, S, A, col, n, xx, s->partials, s->st);
        launches += 2;
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (status != CPS_OK || h.rnorm2 <= h.thresh2 || total >= max_iter) break;
    }
    k_permute_out<<<g, kBlock, 0, stream>>>(s->wx, s->perm, n, x);
    ++launches;
    CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    if (win) {
        int rc = l2_set_aside(s, 0, stream);
        if (rc) return rc;
    }
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    if (status == CPS_OK && h.bnorm2 > 0 && !(rel <= rtol)) status = CPS_ERR_NOT_CONVERGED;
    fill_stats(stats, total, rel, status, 1, launches);
    if (status == CPS_ERR_NOT_SPD) cps::set_error(s->ctx, "solve: p.Sp <= 0 (reduced system)");
    if (status == CPS_ERR_TIMEOUT) cps::set_error(s->ctx, "solve: a grid barrier wait ran out");
    if (status == CPS_ERR_NOT_CONVERGED)
        cps::set_error(s->ctx, total >= max_iter
                                   ? "solve: max_iter reached"
                                   : "solve: the true residual stays above rtol (FP64 rounding "
                                     "floor of this system and right-hand side)");
    return status;
}

// ------------------------------------------------------------------ mixed

static int solve_mixed(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
                       cps_stats* stats, cudaStream_t stream) {
    const int64_t n = s->nt;
    const int g = s->grid;
    const bool ic0 = s->precond == CPS_PC_IC0;
    const Run<float> v = make_run<float>(s);
    if (!s->tune[CPS_MIXED].done) {
        int rc = autotune<float>(s, CPS_MIXED, v, stream);
        if (rc) return rc;
    }
    const double* A64 = ic0 ? s->pa : s->a;
    const double* S64 = ic0 ? s->ps : s->s;
    const double* bb = b;
    double* xx = x;
    int64_t launches = 0;
    if (ic0) {
        k_permute_in<<<g, kBlock, 0, stream>>>(b, x, s->perm, n, s->wb, s->wx);
        ++launches;
        bb = s->wb;
        xx = s->wx;
    }
    int64_t base = 0;          // iterations of runs before the last restart
    int updates = 0, stall = 0, restarts = 0;
    double prev = INFINITY, last = INFINITY;
    // The FP64 iterate with the least true residual so far is kept in wbest:
    // where kappa(A) u_32 approaches 1 the binary32 corrections stop helping
    // and refinement can drive the residual up; the solve then ends with that
    // iterate and CPS_ERR_NOT_CONVERGED.
    double best = INFINITY;
    bool restore = false;
    int first = 1;
    CgState h{};
    int status = CPS_OK;
    for (;;) {
        const long long budget = (long long)(max_iter - base - (first ? 0 : h.iter));
        k_res64<<<g, kBlock, 0, stream>>>(bb, xx, S64, A64, v.col, n, v.r, v.p0, v.y, rtol, kDelta,
                                          budget, first, ic0 ? 0 : 1, s->partials, s->st);
        ++launches;
        if (ic0) launches += enqueue_precond<float>(s, v, stream);
        CPS_CUDA_TRY(s->ctx, cudaGetLastError());
        int rc = read_state(s, stream, &h);
        if (rc) return rc;
        if (h.bnorm2 == 0.0 || h.rnorm2 <= rtol * rtol * h.bnorm2) break;   // converged
        if (h.rnorm2 < best) {
            best = h.rnorm2;
            CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(s->wbest, xx, sizeof(double) * n,
                                                 cudaMemcpyDeviceToDevice, stream));
        } else if (!(h.rnorm2 <= kDiverge * best)) {
            status = CPS_ERR_NOT_CONVERGED;      // refinement diverging
            restore = true;
            break;
        }
        if (base + h.iter >= max_iter || updates >= kMaxUpdates) {
            status = CPS_ERR_NOT_CONVERGED;
            restore = h.rnorm2 > best;
            break;
        }
        // A replaced residual that stops falling (no 10% gain over 8
        // replacements): restart the search directions, at most 4 times.  One
        // that rose since the last replacement restarts them too, without
        // counting against that limit (the stall count still runs).
        if (h.rnorm2 < 0.81 * prev) {
            prev = h.rnorm2;
            stall = 0;
        } else {
            ++stall;
        }
        const bool rose = h.rnorm2 > last;
        last = h.rnorm2;
        if (stall >= 8 && !first) {
            if (++restarts > 4) {
                status = CPS_ERR_NOT_CONVERGED;
                restore = h.rnorm2 > best;
                break;
            }
            base += h.iter;
            first = 1;
            stall = 0;
            continue;
        }
        if (rose && !first) {
            base += h.iter;
            first = 1;
            continue;
        }
        first = 0;
        ++updates;
        if (!h.done) {
            rc = run_chunks<float>(s, CPS_MIXED, v, stream, &h, &launches);
            if (rc) return rc;
        }
        if (h.status != CPS_OK) {
            status = h.status;
            break;
        }
        k_flush_y<float><<<g, kBlock, 0, stream>>>(v.y, v.p0, v.p1, n, s->st);
        k_correct<<<g, kBlock, 0, stream>>>(xx, v.y, S64, n);
        launches += 2;
    }
    if (restore) {
        CPS_CUDA_TRY(s->ctx, cudaMemcpyAsync(xx, s->wbest, sizeof(double) * n,
                                             cudaMemcpyDeviceToDevice, stream));
        h.rnorm2 = best;
    }
    if (ic0) {
        k_permute_out<<<g, kBlock, 0, stream>>>(s->wx, s->perm, n, x);
        ++launches;
    }
    if (h.bnorm2 == 0.0) CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(x, 0, sizeof(double) * n, stream));
    CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    CPS_CUDA_TRY(s->ctx, cudaStreamSynchronize(stream));
    const double rel = h.bnorm2 > 0 ? std::sqrt(h.rnorm2 / h.bnorm2) : 0.0;
    fill_stats(stats, base + h.iter, rel, status, updates, launches);
    if (status == CPS_ERR_NOT_CONVERGED)
        cps::set_error(s->ctx, restore ? "solve: mixed precision did not reach rtol (binary32 "
                                         "refinement stopped reducing the residual; x holds the "
                                         "iterate with the least residual)"
                                       : "solve: mixed precision did not reach rtol");
    if (status == CPS_ERR_NOT_SPD) cps::set_error(s->ctx, "solve: p.Ap <= 0 in the binary32 iteration");
    return status;
}

int solve_impl(cps_sys s, const double* b, double* x, double rtol, int64_t max_iter,
               int precision, cps_stats* stats, cudaStream_t stream) {
    if (!b || !x || !(rtol >= 0.0) || max_iter < 0) {
        cps::set_error(s->ctx, "solve: bad argument");
        return CPS_ERR_ARG;
    }
    if (s->precond == CPS_PC_REDUCED) {
        if (precision != CPS_FP64) {
            cps::set_error(s->ctx, "solve: the reduced-system solve is FP64 only");
            return CPS_ERR_ARG;
        }
        const int rc = solve_reduced(s, b, x, rtol, max_iter, stats, stream);
        l2_set_aside(s, 0, stream);   // error paths: give back a set-aside still held
        return rc;
    }
    if (precision == CPS_FP64) {
        const int rc = solve_fp64(s, b, x, rtol, max_iter, stats, stream);
        l2_set_aside(s, 0, stream);   // error paths: give back a set-aside still held
        return rc;
    }
    if (precision == CPS_MIXED) return solve_mixed(s, b, x, rtol, max_iter, stats, stream);
    cps::set_error(s->ctx, "solve: bad precision");
    return CPS_ERR_ARG;
}

int matvec_impl(cps_sys s, const double* x, double* y, cudaStream_t stream) {
    if (!x || !y) {
        cps::set_error(s->ctx, "matvec: null pointer");
        return CPS_ERR_ARG;
    }
    k_matvec64<<<s->grid, kBlock, 0, stream>>>(x, s->s, s->a, s->col, s->nt, y);
    CPS_CUDA_TRY(s->ctx, cudaGetLastError());
    return CPS_OK;
}

int export_impl(cps_sys s, double* diag, int32_t* col, double* val, cudaStream_t stream) {
    if (!diag || !col || !val) {
        cps::set_error(s->ctx, "export: null pointer");
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
        cps::set_error(s->ctx, "adjoint: null pointer");
        return CPS_ERR_ARG;
    }
    if (dtheta && !s->iso_cell) {
        cps::set_error(s->ctx, "adjoint: dtheta needs a CP2 system with an isotropic per-cell field");
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

}  // namespace cps
