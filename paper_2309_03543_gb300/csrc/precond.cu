// Incomplete Cholesky IC(0) set-up in a multicolour order (Sec. 3.2.2: the
// corrector systems are solved by PCG with an incomplete Cholesky
// factorisation, computed once before the time loop, Sec. 3.1).
//
//   1. colour the cell graph so that no two neighbours share a colour:
//      first try two colours (union-find with parity; the cell graph of the
//      triangular lattice is bipartite), else greedy Jones-Plassmann
//      colouring with hashed priorities (at most 4 colours: every cell has at
//      most 3 neighbours);
//   2. order the cells colour by colour (stable inside a colour) and permute
//      the scaled matrix;
//   3. factor Ahat ~ L D L^T with L unit lower triangular on the pattern of
//      Ahat (no fill), colour by colour:
//        l_ik = (a_ik - sum_{m<k, m~i, m~k} l_im d_m l_km) / d_k,
//        d_i  = 1 - sum_k l_ik^2 d_k,
//      storing l_ik in the lower slots of row i and l_ki in the upper slots.
// On a two-coloured graph no cell has two mutually adjacent neighbours, so
// l_ik = a_ik / d_k and the black pivots are d_i = 1 - sum_red a_ik^2.
#include "cps_internal.cuh"

#include <cstring>
#include <vector>

namespace cps {
namespace {

constexpr int kMaxColours = 16;

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    // lowbias32 integer hash.
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Two-colouring by union-find with parity.  Word w[u] = (parent << 1) | t,
// t = parity of u relative to its parent; a root is its own parent with
// t = 0.  Roots are only ever hooked under a root of smaller index, so
// parents strictly decrease and every walk ends.  For a side (u, v) the two
// roots are joined so that u and v get opposite absolute parities; a side
// whose ends already share a root and a parity proves an odd cycle.
__device__ __forceinline__ int32_t uf_find(long long* w, int32_t u, int* par, int64_t n) {
    int acc = 0;
    int32_t x = u;
    for (int64_t guard = 0; guard <= n; ++guard) {
        const long long wx = __ldcg(&w[x]);
        const int32_t px = (int32_t)(wx >> 1);
        if (px == x) break;
        const long long wp = __ldcg(&w[px]);
        const int32_t gp = (int32_t)(wp >> 1);
        if (gp != px) {
            // path halving: point x at its grandparent, parities composed
            const long long nw = ((long long)gp << 1) | ((wx ^ wp) & 1LL);
            atomicCAS(reinterpret_cast<unsigned long long*>(&w[x]), (unsigned long long)wx,
                      (unsigned long long)nw);
        }
        acc ^= (int)(wx & 1);
        x = px;
    }
    *par = acc;
    return x;
}

__global__ void k_uf_init(long long* w, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        w[e] = (long long)e << 1;
}

__global__ void k_uf_union(const int32_t* __restrict__ col, int64_t n, long long* w, int* flags) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            if (c <= (int32_t)e) continue;           // each side once
            bool ok = false;
            for (int attempt = 0; attempt < (1 << 20); ++attempt) {
                int pu, pv;
                const int32_t ru = uf_find(w, (int32_t)e, &pu, n);
                const int32_t rv = uf_find(w, c, &pv, n);
                if (ru == rv) {
                    if (pu == pv) flags[0] = 1;      // odd cycle
                    ok = true;
                    break;
                }
                const int32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
                const long long t = (long long)(pu ^ pv ^ 1);
                const unsigned long long expect = (unsigned long long)((long long)hi << 1);
                const unsigned long long want = (unsigned long long)(((long long)lo << 1) | t);
                if (atomicCAS(reinterpret_cast<unsigned long long*>(&w[hi]), expect, want) == expect) {
                    ok = true;
                    break;
                }
            }
            if (!ok) flags[1] = 1;                   // gave up: use the general colouring
        }
    }
}

__global__ void k_uf_colour(int64_t n, long long* w, int32_t* __restrict__ colour) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int par;
        uf_find(w, (int32_t)e, &par, n);
        colour[e] = par;
    }
}

__global__ void k_parity_check(const int32_t* __restrict__ col, int64_t n,
                               const int32_t* __restrict__ colour, int* conflict) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            if (c != (int32_t)e && colour[c] == colour[e]) *conflict = 1;
        }
    }
}

// One Jones-Plassmann round: an uncoloured cell whose priority beats every
// uncoloured neighbour takes the smallest colour no coloured neighbour has.
__global__ void k_jp_round(const int32_t* __restrict__ col, int64_t n, int32_t* colour,
                           int* remaining) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (colour[e] >= 0) continue;
        const uint32_t pe = hash32((uint32_t)e);
        bool top = true;
        unsigned used = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = col[j * n + e];
            if (c == (int32_t)e) continue;
            const int32_t cc = __ldcg(&colour[c]);
            if (cc < 0) {
                const uint32_t pc = hash32((uint32_t)c);
                if (pc > pe || (pc == pe && c > (int32_t)e)) top = false;
            } else if (cc < 32) {
                used |= 1u << cc;
            }
        }
        if (top) {
            colour[e] = __ffs(~used) - 1;
        } else {
            *remaining = 1;
        }
    }
}

__global__ void k_colour_max(const int32_t* __restrict__ colour, int64_t n, int* cmax) {
    int m = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        m = max(m, colour[e]);
    atomicMax(cmax, m);
}

// Tile b = cells [b*kBlock, (b+1)*kBlock): counts[c * nblk + b].
__global__ void __launch_bounds__(kBlock) k_colour_count(const int32_t* __restrict__ colour,
                                                         int64_t n, int ncol, int64_t nblk,
                                                         int* __restrict__ counts) {
    const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    const int my = i < n ? colour[i] : -1;
    for (int c = 0; c < ncol; ++c) {
        const int cnt = __syncthreads_count(my == c);
        if (threadIdx.x == 0) counts[c * nblk + blockIdx.x] = cnt;
    }
}

// Exclusive scan of counts (length m) in one block; colour c starts at
// offsets[c * nblk].
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ counts, int64_t m,
                                               long long* __restrict__ offsets) {
    __shared__ long long part[1024];
    const int64_t per = (m + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = threadIdx.x * per;
    const int64_t b1 = b0 + per < m ? b0 + per : m;
    long long s = 0;
    for (int64_t k = b0; k < b1; ++k) s += counts[k];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const long long v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int64_t k = b0; k < b1; ++k) {
        offsets[k] = run;
        run += counts[k];
    }
}

__global__ void __launch_bounds__(kBlock) k_colour_scatter(const int32_t* __restrict__ colour,
                                                           int64_t n, int ncol, int64_t nblk,
                                                           const long long* __restrict__ offsets,
                                                           int32_t* __restrict__ perm,
                                                           int32_t* __restrict__ iperm) {
    __shared__ int wcount[kMaxColours][kBlock / 32];
    const int64_t i = blockIdx.x * (int64_t)kBlock + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int my = i < n ? colour[i] : -1;
    unsigned mine = 0;
    for (int c = 0; c < ncol; ++c) {
        const unsigned m = __ballot_sync(0xffffffffu, my == c);
        if (my == c) mine = m;
        if (lane == 0) wcount[c][warp] = __popc(m);
    }
    __syncthreads();
    if (my >= 0) {
        int rank = __popc(mine & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) rank += wcount[my][w];
        const long long dst = offsets[(int64_t)my * nblk + blockIdx.x] + rank;
        perm[dst] = (int32_t)i;
        iperm[i] = (int32_t)dst;
    }
}

__global__ void k_permute_matrix(const double* __restrict__ a, const int32_t* __restrict__ col,
                                 const double* __restrict__ s, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ iperm, int64_t n,
                                 double* __restrict__ pa, int32_t* __restrict__ pcol,
                                 double* __restrict__ ps, float* __restrict__ pa32,
                                 float* __restrict__ ps32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = perm[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = a[j * n + o];
            pa[j * n + i] = v;
            pa32[j * n + i] = (float)v;
            pcol[j * n + i] = iperm[col[j * n + o]];
        }
        ps[i] = s[o];
        ps32[i] = (float)s[o];
    }
}

// IC(0) rows of one colour [cs, ce): lower slots have pcol < i.
__global__ void k_ic0_factor(const double* __restrict__ pa, const int32_t* __restrict__ pcol,
                             int64_t n, int64_t cs, int64_t ce, double* __restrict__ pl,
                             double* __restrict__ pdinv, double* __restrict__ pdiag, int* err) {
    for (int64_t i = cs + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ce;
         i += (int64_t)gridDim.x * blockDim.x) {
        int kk[3], sl[3], m = 0;
        double av[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t c = pcol[j * n + i];
            pl[j * n + i] = 0.0;
            if (c < i) {
                kk[m] = c;
                sl[m] = j;
                av[m] = pa[j * n + i];
                ++m;
            }
        }
        // ascending column order
        for (int u = 0; u < m; ++u)
            for (int v = u + 1; v < m; ++v)
                if (kk[v] < kk[u]) {
                    int t = kk[u]; kk[u] = kk[v]; kk[v] = t;
                    t = sl[u]; sl[u] = sl[v]; sl[v] = t;
                    double d = av[u]; av[u] = av[v]; av[v] = d;
                }
        double L[3] = {0.0, 0.0, 0.0};
        double dsum = 0.0;
        for (int u = 0; u < m; ++u) {
            const int32_t k = kk[u];
            double v = av[u];
            for (int w = 0; w < u; ++w) {
                const int32_t mm = kk[w];
                for (int t = 0; t < 3; ++t)
                    if (pcol[t * n + k] == mm) v -= L[w] * (1.0 / pdinv[mm]) * pl[t * n + k];
            }
            L[u] = v * pdinv[k];
            pl[sl[u] * n + i] = L[u];
            dsum += L[u] * v;
        }
        const double d = 1.0 - dsum;
        if (!(d > 0.0) || !isfinite(d)) {
            set_error(err, CPS_ERR_NOT_SPD);
            pdinv[i] = 1.0;
            pdiag[i] = 1.0;
        } else {
            pdinv[i] = 1.0 / d;
            pdiag[i] = d;
        }
    }
}

// Upper slots of row i (pcol > i) take l_ki from row k's slot pointing at i;
// also the binary32 copies.
__global__ void k_ic0_upper(const int32_t* __restrict__ pcol, int64_t n, double* __restrict__ pl,
                            const double* __restrict__ pdinv, float* __restrict__ pl32,
                            float* __restrict__ pdinv32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int32_t k = pcol[j * n + i];
            if (k > i) {
                double v = 0.0;
                for (int t = 0; t < 3; ++t)
                    if (pcol[t * n + k] == (int32_t)i) v = pl[t * n + k];
                pl[j * n + i] = v;
            }
        }
        pdinv32[i] = (float)pdinv[i];
    }
}

__global__ void k_to_float(const double* __restrict__ v, int64_t m, float* __restrict__ o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (float)v[i];
}

}  // namespace

static int alloc_ic0(cps_sys s) {
    if (s->pa) return CPS_OK;
    const int64_t n = s->nt;
    struct {
        void** p;
        size_t bytes;
    } req[] = {{(void**)&s->perm, 4 * (size_t)n},       {(void**)&s->iperm, 4 * (size_t)n},
               {(void**)&s->pa, 24 * (size_t)n},        {(void**)&s->pcol, 12 * (size_t)n},
               {(void**)&s->pl, 24 * (size_t)n},        {(void**)&s->pdinv, 8 * (size_t)n},
               {(void**)&s->pdiag, 8 * (size_t)n},
               {(void**)&s->ps, 8 * (size_t)n},         {(void**)&s->pa32, 12 * (size_t)n},
               {(void**)&s->pl32, 12 * (size_t)n},      {(void**)&s->pdinv32, 4 * (size_t)n},
               {(void**)&s->ps32, 4 * (size_t)n}};
    for (auto& r : req) {
        cudaError_t e = cudaMalloc(r.p, r.bytes);
        if (e != cudaSuccess) {
            cps::set_error(s->ctx, std::string("set_precond: cudaMalloc: ") + cudaGetErrorString(e));
            return CPS_ERR_NOMEM;
        }
    }
    return CPS_OK;
}

static int colour_cells(cps_sys s, int32_t* colour, cudaStream_t stream, int* ncol_out) {
    const int64_t n = s->nt;
    const int g = grid_for(s->ctx, n);
    constexpr int kRounds = 16;
    long long* w = nullptr;
    int* flags = nullptr;   // [0] odd cycle, [1] union gave up, [2] parity conflict,
                            // [3] max colour, [4..4+kRounds) JP rounds still colouring
    CPS_CUDA_TRY(s->ctx, cudaMallocAsync((void**)&w, sizeof(long long) * n, stream));
    CPS_CUDA_TRY(s->ctx, cudaMallocAsync((void**)&flags, sizeof(int) * (4 + kRounds), stream));
    int h[4 + kRounds];
    int rc = CPS_OK;
    cudaMemsetAsync(flags, 0, sizeof(int) * (4 + kRounds), stream);
    k_uf_init<<<g, kBlock, 0, stream>>>(w, n);
    k_uf_union<<<g, kBlock, 0, stream>>>(s->col, n, w, flags);
    k_uf_colour<<<g, kBlock, 0, stream>>>(n, w, colour);
    k_parity_check<<<g, kBlock, 0, stream>>>(s->col, n, colour, flags + 2);
    cudaMemcpyAsync(h, flags, sizeof(int) * 3, cudaMemcpyDeviceToHost, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = CPS_ERR_CUDA;
    const bool two = rc == CPS_OK && h[0] == 0 && h[1] == 0 && h[2] == 0;
    if (rc == CPS_OK && !two) {
        // Jones-Plassmann: at most (max degree + 1) = 4 colours.
        cudaMemsetAsync(colour, 0xFF, sizeof(int32_t) * n, stream);
        for (int64_t round = 0; round <= n; round += kRounds) {
            cudaMemsetAsync(flags + 4, 0, sizeof(int) * kRounds, stream);
            for (int r = 0; r < kRounds; ++r)
                k_jp_round<<<g, kBlock, 0, stream>>>(s->col, n, colour, flags + 4 + r);
            cudaMemcpyAsync(h + 4, flags + 4, sizeof(int) * kRounds, cudaMemcpyDeviceToHost, stream);
            if (cudaStreamSynchronize(stream) != cudaSuccess) {
                rc = CPS_ERR_CUDA;
                break;
            }
            if (h[4 + kRounds - 1] == 0) break;
        }
    }
    if (rc == CPS_OK) {
        k_colour_max<<<g, kBlock, 0, stream>>>(colour, n, flags + 3);
        cudaMemcpyAsync(h + 3, flags + 3, sizeof(int), cudaMemcpyDeviceToHost, stream);
        if (cudaStreamSynchronize(stream) != cudaSuccess) rc = CPS_ERR_CUDA;
        *ncol_out = h[3] + 1;
    }
    cudaFreeAsync(w, stream);
    cudaFreeAsync(flags, stream);
    if (rc != CPS_OK) cps::set_error(s->ctx, "set_precond: colouring failed");
    return rc;
}

int precond_impl(cps_sys s, int precond, cudaStream_t stream) {
    if (precond == CPS_PC_JACOBI) {
        s->precond = precond;
        return CPS_OK;
    }
    if (precond != CPS_PC_IC0 && precond != CPS_PC_REDUCED) {
        cps::set_error(s->ctx, "set_precond: unknown preconditioner");
        return CPS_ERR_ARG;
    }
    if (s->ncolours > 0) {   // ordered and factored already (the matrix is fixed)
        if (precond == CPS_PC_REDUCED && s->ncolours != 2) {
            cps::set_error(s->ctx, "set_precond: the cell graph is not two-colourable");
            return CPS_ERR_ARG;
        }
        s->precond = precond;
        return CPS_OK;
    }
    int rc = alloc_ic0(s);
    if (rc) return rc;
    const int64_t n = s->nt;
    const int g = grid_for(s->ctx, n);
    int32_t* colour = nullptr;
    int* counts = nullptr;
    long long* offsets = nullptr;
    int* err = nullptr;
    CPS_CUDA_TRY(s->ctx, cudaMallocAsync((void**)&colour, sizeof(int32_t) * n, stream));
    CPS_CUDA_TRY(s->ctx, cudaMallocAsync((void**)&err, sizeof(int), stream));
    CPS_CUDA_TRY(s->ctx, cudaMemsetAsync(err, 0, sizeof(int), stream));
    int ncol = 0;
    rc = colour_cells(s, colour, stream, &ncol);
    if (rc == CPS_OK && (ncol < 1 || ncol > kMaxColours)) {
        cps::set_error(s->ctx, "set_precond: too many colours");
        rc = CPS_ERR_ARG;
    }
    if (rc == CPS_OK) {
        const int64_t nblk = (n + kBlock - 1) / kBlock;
        const int64_t m = (int64_t)ncol * nblk;
        cudaError_t ce = cudaMallocAsync((void**)&counts, sizeof(int) * m, stream);
        if (ce == cudaSuccess) ce = cudaMallocAsync((void**)&offsets, sizeof(long long) * m, stream);
        if (ce != cudaSuccess) {
            rc = CPS_ERR_NOMEM;
        } else {
            k_colour_count<<<(unsigned)nblk, kBlock, 0, stream>>>(colour, n, ncol, nblk, counts);
            k_scan<<<1, 1024, 0, stream>>>(counts, m, offsets);
            k_colour_scatter<<<(unsigned)nblk, kBlock, 0, stream>>>(colour, n, ncol, nblk, offsets,
                                                                  s->perm, s->iperm);
            std::vector<long long> starts(ncol);
            for (int c = 0; c < ncol; ++c)
                cudaMemcpyAsync(&starts[c], offsets + (int64_t)c * nblk, sizeof(long long),
                                cudaMemcpyDeviceToHost, stream);
            k_permute_matrix<<<g, kBlock, 0, stream>>>(s->a, s->col, s->s, s->perm, s->iperm, n,
                                                       s->pa, s->pcol, s->ps, s->pa32, s->ps32);
            if (cudaStreamSynchronize(stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                rc = CPS_ERR_CUDA;
            } else {
                for (int c = 0; c < ncol; ++c) s->colour_start[c] = starts[c];
                s->colour_start[ncol] = n;
                for (int c = 0; c < ncol; ++c)
                    k_ic0_factor<<<g, kBlock, 0, stream>>>(s->pa, s->pcol, n, s->colour_start[c],
                                                           s->colour_start[c + 1], s->pl, s->pdinv,
                                                           s->pdiag, err);
                k_ic0_upper<<<g, kBlock, 0, stream>>>(s->pcol, n, s->pl, s->pdinv, s->pl32,
                                                      s->pdinv32);
                k_to_float<<<grid_for(s->ctx, 3 * n), kBlock, 0, stream>>>(s->pl, 3 * n, s->pl32);
                int herr = 0;
                cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
                if (cudaStreamSynchronize(stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
                    rc = CPS_ERR_CUDA;
                else if (herr) {
                    cps::set_error(s->ctx, "set_precond: IC(0) pivot <= 0");
                    rc = herr;
                }
            }
        }
    }
    if (counts) cudaFreeAsync(counts, stream);
    if (offsets) cudaFreeAsync(offsets, stream);
    cudaFreeAsync(colour, stream);
    cudaFreeAsync(err, stream);
    cudaStreamSynchronize(stream);
    if (rc != CPS_OK) {
        if (s->ctx->last_error.empty()) cps::set_error(s->ctx, "set_precond: IC(0) set-up failed");
        return rc;
    }
    s->ncolours = ncol;
    if (precond == CPS_PC_REDUCED && ncol != 2) {
        s->precond = CPS_PC_JACOBI;
        cps::set_error(s->ctx, "set_precond: the cell graph is not two-colourable");
        return CPS_ERR_ARG;
    }
    s->precond = precond;
    return CPS_OK;
}

}  // namespace cps
