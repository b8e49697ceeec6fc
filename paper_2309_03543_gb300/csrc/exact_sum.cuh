// Exact, order-independent sums of doubles in integer arithmetic, shared by
// the persistent and the batched solves.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace cps {

// ---- Exact sums in integer arithmetic.  GB300 issues FP64 at 2 per SM per
// clock, and a chain of dependent FP64 adds pays the FP64 latency per add: a
// block sum of 1024 doubles took about 2 us that way.  Here a set of doubles
// is summed by aligning every value to the set's largest exponent E
// (rounding to the nearest multiple of 2^(E - 1075 + h), h bits of headroom)
// and adding the aligned integers exactly, with warp integer reductions on
// 18-20-bit limbs.  The result depends on the set only, not on the order of
// the values (deterministic, bit-identical in every block that sums the same
// set); each value is off by at most half a unit of 2^(E - 1075 + h).

// Biased exponent of v's binade (1 for zero and subnormals).
__device__ __forceinline__ int align_exp(double v) {
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return e > 0 ? e : 1;
}

// round(v / 2^(E - 1075 + h)) for |v| < 2^(E - 1022), h >= 1: at most 2^(53 - h)
// in magnitude.
__device__ __forceinline__ long long align_fixed(double v, int E, int h) {
    const long long bits = __double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7FF);
    long long m = bits & 0xFFFFFFFFFFFFFLL;
    if (e) m |= 1LL << 52;
    const int sh = E - (e > 0 ? e : 1) + h;
    const long long f = sh > 62 ? 0 : ((m + (1LL << (sh - 1))) >> sh);
    return bits < 0 ? -f : f;
}

// T 2^(E - 1075 + h) as a double (NaN if the set held an infinity or NaN).
__device__ __forceinline__ double fixed_to_double(long long T, int E, int h) {
    if (E >= 2047) return __longlong_as_double(0x7FF8000000000000LL);
    return ldexp(__ll2double_rn(T), E - 1075 + h);
}

// Exact sum over the warp of x, |x| <= 2^B (B <= 57): the biased value
// x + 2^B is split into three limbs whose 32-lane sums fit 32 bits; the
// recombination runs modulo 2^64, exact because the true sum (at most
// 2^(B + 5)) fits a signed 64-bit integer.
template <int B>
__device__ __forceinline__ long long warp_sum_fixed(long long x) {
    constexpr int L = (B + 4) / 3;
    static_assert(B <= 57 && L <= 26 && 3 * L >= B + 2, "limbs of the biased value");
    const unsigned long long u = (unsigned long long)x + (1ULL << B);
    const unsigned mask = (1u << L) - 1u;
    const unsigned long long s0 = __reduce_add_sync(0xffffffffu, (unsigned)(u & mask));
    const unsigned long long s1 = __reduce_add_sync(0xffffffffu, (unsigned)((u >> L) & mask));
    const unsigned long long s2 = __reduce_add_sync(0xffffffffu, (unsigned)(u >> (2 * L)));
    return (long long)(s0 + (s1 << L) + (s2 << (2 * L)) - (32ULL << B));
}


// Exact sum over a block of BS threads (BS a multiple of 32, at most 1024) of
// v[0..NV): every thread receives the totals in v.  Per quantity, the warps
// align their values to the block's largest exponent and sum them, then warp 0
// sums the warps' totals.  Three barriers.
template <int NV, int BS>
__device__ __forceinline__ void block_sum_exact(double (&v)[NV]) {
    static_assert(BS % 32 == 0 && BS <= 1024, "block shape");
    constexpr int W = BS / 32;
    __shared__ int s_e[NV][32];
    __shared__ long long s_w[NV][32];
    __shared__ double s_t[NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int em = __reduce_max_sync(0xffffffffu, align_exp(v[k]));
        if (lane == 0) s_e[k][warp] = em;
    }
    __syncthreads();
    int E[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        E[k] = __reduce_max_sync(0xffffffffu, lane < W ? s_e[k][lane] : 1);
        const long long w = warp_sum_fixed<52>(align_fixed(v[k], E[k], 1));
        if (lane == 0) s_w[k][warp] = w;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const long long T = warp_sum_fixed<57>(lane < W ? s_w[k][lane] : 0LL);
            if (lane == 0) s_t[k] = fixed_to_double(T, E[k], 1);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = s_t[k];
}

}  // namespace cps
