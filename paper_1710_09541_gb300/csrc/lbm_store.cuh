// lbm_store.cuh -- population storage formats.  All arithmetic is FP32; the
// formats differ only in how the two population sets sit in HBM.
//
//   FP32 (LBM_STORE_FP32): f and g as 9 FP32 planes each (36 B + 36 B / node);
//     f_0 is written as phi - sum_{i>0} f_i (see below).
//
//   FP16 / BF16 shifted (LBM_STORE_FP16_SHIFTED, LBM_STORE_BF16_SHIFTED):
//     f_0          FP32, written as phi - sum_{i>0} decode(encode(f_i)): the
//                  rest population absorbs the rounding of the eight moving
//                  ones, so the stored populations of a node sum to its phi up
//                  to FP32 round-off and sum phi stays conserved.
//     f_1..f_8     16-bit codes of f_i / w_i - 1/2: the offset from the
//                  weight-scaled rest state at phi_ref = 1/2 (phi lies in [0, 1]).
//     g_0..g_8     16-bit codes of S g_i / w_i (p_ref = 0), with S = 2^10 for
//                  FP16 so pressures and momenta of O(1e-6) stay above the
//                  FP16 subnormal range; S = 1 for BF16 (FP32 exponent range).
//   Layout: the f buffer holds the f_0 plane (N floats) and then 8 planes of
//   N 32-bit words; word (i - 1, node) packs the codes of f_i (low half) and
//   g_i (high half), which are pulled from the same neighbour, so one load
//   serves both and one packed conversion encodes both.  The g buffer holds
//   the g_0 codes (N 16-bit values).
//   Bytes per node: 4 + 32 + 2 = 38 per set (92 B read + written per update
//   with phi u).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_kernels.cuh"

// 16-bit pulls of kernels compiled for walls: per-lane selects (0) or the
// warp-uniform branch the run-time-wall kernels use (1).  With 32 x 8 tiles
// the selects were 5% faster; with the 32 x 4 tiles the branch is (walled
// impact 2400 x 600, FP16: 39.1 k -> 40.1-41.0 k MLUPS).
// FP32 population stores with the evict-first (streaming) cache hint
#ifndef LBM_STORE_STREAMING
#define LBM_STORE_STREAMING 0
#endif
#ifndef LBM_WALL_BRANCH
#define LBM_WALL_BRANCH 1
#endif

namespace lbmpf {

enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2 };

template <int ST>
struct Pop;

template <>
struct Pop<ST_FP32> {
    static size_t f_bytes(size_t N) { return 36 * N; }
    static size_t g_bytes(size_t N) { return 36 * N; }
    // store the post-collision set of node idx; f_0 is written as the
    // remainder phi - sum_{i>0} f_i, so the stored populations of a node sum
    // to its phi up to one rounding and sum phi does not drift with the
    // rounding of the collision.  Stores of f_i and g_i interleaved (as
    // measured fastest).
    __device__ static void stfg(void* fb, void* gb, int N, int idx, const float f[9],
                                const float g[9], float phi) {
        float* F = static_cast<float*>(fb);
        float* G = static_cast<float*>(gb);
#if LBM_STORE_STREAMING
        __stcs(F + idx, sub(phi, sum8(f)));
        __stcs(G + idx, g[0]);
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            __stcs(F + (i * N + idx), f[i]);
            __stcs(G + (i * N + idx), g[i]);
        }
#else
        F[idx] = sub(phi, sum8(f));
        G[idx] = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            F[i * N + idx] = f[i];
            G[i * N + idx] = g[i];
        }
#endif
    }
    // one plane entry (checkpoint and initial-state permutations); the rest
    // population's correction is zero in FP32
    __device__ static void putf(void* b, int N, int i, int idx, float v) {
        static_cast<float*>(b)[i * N + idx] = v;
    }
    __device__ static void putg(void*, void* b, int N, int i, int idx, float v) {
        static_cast<float*>(b)[i * N + idx] = v;
    }
    __device__ static float round_f(int, float v) { return v; }
    // population planes, and the address of entry idx of plane k (prefetches)
    static constexpr int PLANES = 18;
    __device__ static const void* plane_addr(const void* fb, const void* gb, int N, int k, int idx) {
        return k < 9 ? static_cast<const float*>(fb) + (k * N + idx)
                     : static_cast<const float*>(gb) + ((k - 9) * N + idx);
    }
};

template <typename H>
struct Half16;
template <>
struct Half16<__half> {
    static constexpr float GS = 1024.f;
    __device__ static float to_f(unsigned short u) { return __half2float(__ushort_as_half(u)); }
    __device__ static unsigned short from_f(float v) { return __half_as_ushort(__float2half_rn(v)); }
    // (from_f(lo), from_f(hi)) in one word, one packed conversion
    __device__ static unsigned int pack(float lo, float hi) {
        const __half2 h = __floats2half2_rn(lo, hi);
        return (unsigned int)__half_as_ushort(__low2half(h)) |
               ((unsigned int)__half_as_ushort(__high2half(h)) << 16);
    }
};
template <>
struct Half16<__nv_bfloat16> {
    static constexpr float GS = 1.f;
    __device__ static float to_f(unsigned short u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
    __device__ static unsigned short from_f(float v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
    __device__ static unsigned int pack(float lo, float hi) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return (unsigned int)__bfloat16_as_ushort(__low2bfloat16(h)) |
               ((unsigned int)__bfloat16_as_ushort(__high2bfloat16(h)) << 16);
    }
};

template <typename H>
struct Shifted16 {
    using C = Half16<H>;
    static size_t f_bytes(size_t N) { return 4 * N + 32 * N; }
    static size_t g_bytes(size_t N) { return 2 * N; }
    __device__ static const unsigned int* pw(const void* fb, int N) {
        return reinterpret_cast<const unsigned int*>(static_cast<const float*>(fb) + N);
    }
    __device__ static unsigned int* pw(void* fb, int N) {
        return reinterpret_cast<unsigned int*>(static_cast<float*>(fb) + N);
    }
    __device__ static unsigned short lo(unsigned int w) { return (unsigned short)(w & 0xffffu); }
    __device__ static unsigned short hi(unsigned int w) { return (unsigned short)(w >> 16); }
    // f_i = w_i (v + 1/2) for i > 0
    __device__ static float dec_f(int i, unsigned short u) {
        return fma_rn(C::to_f(u), w_of(i), 0.5f * w_of(i));
    }
    __device__ static unsigned short enc_f(int i, float v) {
        return C::from_f(fma_rn(v, 1.f / w_of(i), -0.5f));
    }
    __device__ static float dec_g(int i, unsigned short u) {
        return mul(C::to_f(u), w_of(i) / C::GS);
    }
    __device__ static unsigned short enc_g(int i, float v) {
        return C::from_f(mul(v, C::GS / w_of(i)));
    }
    // the word of direction i > 0: the codes enc_f(i, f) | enc_g(i, g) << 16
    __device__ static unsigned int enc_pair(int i, float f, float g) {
        return C::pack(fma_rn(f, 1.f / w_of(i), -0.5f), mul(g, C::GS / w_of(i)));
    }
    // store the post-collision set of node idx (f_0 as the remainder)
    __device__ static void stfg(void* fb, void* gb, int N, int idx, const float f[9],
                                const float g[9], float phi) {
        unsigned int* P = pw(fb, N);
        float d[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const unsigned int w = enc_pair(i, f[i], g[i]);
            P[(i - 1) * N + idx] = w;
            d[i] = dec_f(i, lo(w));
        }
        static_cast<float*>(fb)[idx] = sub(phi, sum8(d));
        static_cast<unsigned short*>(gb)[idx] = enc_g(0, g[0]);
    }
    // one entry (checkpoint and initial-state permutations)
    __device__ static void putf(void* fb, int N, int i, int idx, float v) {
        if (i == 0)
            static_cast<float*>(fb)[idx] = v;
        else
            reinterpret_cast<unsigned short*>(pw(fb, N))[2 * ((i - 1) * N + idx)] = enc_f(i, v);
    }
    __device__ static void putg(void* fb, void* gb, int N, int i, int idx, float v) {
        if (i == 0)
            static_cast<unsigned short*>(gb)[idx] = enc_g(0, v);
        else
            reinterpret_cast<unsigned short*>(pw(fb, N))[2 * ((i - 1) * N + idx) + 1] = enc_g(i, v);
    }
    // the value a moving population takes after storage
    __device__ static float round_f(int i, float v) { return i == 0 ? v : dec_f(i, enc_f(i, v)); }
    // planes: f_0, the 8 word planes, g_0; address of entry idx of plane k
    static constexpr int PLANES = 10;
    __device__ static const void* plane_addr(const void* fb, const void* gb, int N, int k, int idx) {
        if (k == 0) return static_cast<const float*>(fb) + idx;
        if (k == 9) return static_cast<const unsigned short*>(gb) + idx;
        return pw(fb, N) + ((k - 1) * N + idx);
    }
};

template <>
struct Pop<ST_FP16> : Shifted16<__half> {};
template <>
struct Pop<ST_BF16> : Shifted16<__nv_bfloat16> {};

// Pull (stream) node q through a 16-bit storage format: the nine loads first
// (f_0 and g_0, and one word of (f_i, g_i) codes per moving direction), then
// the decodes.  The six wall-dependent loads sit in a branch that is uniform
// across a warp (BR; a warp covers part of one tile row), or are per-lane
// selects.  G: decode g as well.
template <int ST, bool BR, bool G>
__device__ __forceinline__ void pull_16(const void* fs, const void* gs, int N, const Nbr& q,
                                        float f[9], float g[9]) {
    using P = Pop<ST>;
    const unsigned int* W = P::pw(fs, N);
    auto raw = [&](int i, int idx) { return __ldg(W + ((i - 1) * N + idx)); };
    unsigned int w[9];
    const float f0 = __ldg(static_cast<const float*>(fs) + (q.r0 + q.x));
    unsigned short g0 = 0;
    if (G) g0 = __ldg(static_cast<const unsigned short*>(gs) + (q.r0 + q.x));
    w[1] = raw(1, q.r0 + q.xm);
    w[3] = raw(3, q.r0 + q.xp);
    if (!BR || q.lo || q.hi) {
        w[2] = q.lo ? raw(4, q.r0 + q.x) : raw(2, q.rm + q.x);
        w[4] = q.hi ? raw(2, q.r0 + q.x) : raw(4, q.rp + q.x);
        w[5] = q.lo ? raw(7, q.r0 + q.x) : raw(5, q.rm + q.xm);
        w[6] = q.lo ? raw(8, q.r0 + q.x) : raw(6, q.rm + q.xp);
        w[7] = q.hi ? raw(5, q.r0 + q.x) : raw(7, q.rp + q.xp);
        w[8] = q.hi ? raw(6, q.r0 + q.x) : raw(8, q.rp + q.xm);
    } else {
        w[2] = raw(2, q.rm + q.x);
        w[4] = raw(4, q.rp + q.x);
        w[5] = raw(5, q.rm + q.xm);
        w[6] = raw(6, q.rm + q.xp);
        w[7] = raw(7, q.rp + q.xp);
        w[8] = raw(8, q.rp + q.xm);
    }
    // a bounce-back link decodes with the stored direction's weight: opposite
    // directions share w_i, so the stored and the pulled index agree on it
    f[0] = f0;
#pragma unroll
    for (int i = 1; i < 9; ++i) f[i] = P::dec_f(i, P::lo(w[i]));
    if (G) {
        g[0] = P::dec_g(0, g0);
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = P::dec_g(i, P::hi(w[i]));
    }
}

// Pull both population sets of node q in any storage format (WALLS as in
// make_nbr: < 0 when the wall flag is a run-time value).
template <int ST, int WALLS = -1>
__device__ __forceinline__ void pull18(const void* fs, const void* gs, int N, const Nbr& q,
                                       float f[9], float g[9]) {
    if constexpr (ST == ST_FP32) {
        pull9(static_cast<const float*>(fs), (size_t)N, q, f);
        pull9(static_cast<const float*>(gs), (size_t)N, q, g);
    } else {
        pull_16<ST, (WALLS < 0) || LBM_WALL_BRANCH, true>(fs, gs, N, q, f, g);
    }
}
// the f set only
template <int ST, int WALLS = -1>
__device__ __forceinline__ void pull9f(const void* fs, int N, const Nbr& q, float v[9]) {
    if constexpr (ST == ST_FP32) {
        pull9(static_cast<const float*>(fs), (size_t)N, q, v);
    } else {
        float unused[9];
        pull_16<ST, (WALLS < 0) || LBM_WALL_BRANCH, false>(fs, nullptr, N, q, v, unused);
    }
}

template <int ST, int WALLS = -1>
__device__ __forceinline__ float phi_at_st(const void* fs, int N, int x, int y, int nx, int ny,
                                           int walls) {
    float v[9];
    pull9f<ST, WALLS>(fs, N, make_nbr<WALLS>(x, y, nx, ny, walls), v);
    return sum9(v);
}

}  // namespace lbmpf
