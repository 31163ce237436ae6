// lbm_store.cuh -- population storage formats.  All arithmetic is FP32; the
// formats differ only in how the two population sets sit in HBM.
//
//   FP32 (LBM_STORE_FP32): f and g as 9 FP32 planes each (36 B + 36 B / node);
//     f_0 is written as phi - sum_{i>0} f_i (see below).
//
//   FP16 / BF16 shifted (LBM_STORE_FP16_SHIFTED, LBM_STORE_BF16_SHIFTED):
//     f_0          FP32 plane, written as phi - sum_{i>0} decode(encode(f_i)):
//                  the rest population absorbs the rounding of the eight
//                  moving ones, so the stored populations of a node sum to its
//                  phi up to FP32 round-off and sum phi stays conserved.
//     f_1..f_8     16-bit planes of f_i / w_i - 1/2: the offset from the
//                  weight-scaled rest state at phi_ref = 1/2 (phi lies in [0, 1]).
//     g_0..g_8     16-bit planes of S g_i / w_i (p_ref = 0), with S = 2^10 for
//                  FP16 so pressures and momenta of O(1e-6) stay above the
//                  FP16 subnormal range; S = 1 for BF16 (FP32 exponent range).
//   Bytes per node: f 4 + 16, g 18 (92 B read + written per update with phi u).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_kernels.cuh"

namespace lbmpf {

enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2 };

template <int ST>
struct Pop;

template <>
struct Pop<ST_FP32> {
    static size_t f_bytes(size_t N) { return 36 * N; }
    static size_t g_bytes(size_t N) { return 36 * N; }
    __device__ static float ldf(const void* b, int N, int i, int idx) {
        return __ldg(static_cast<const float*>(b) + (i * N + idx));
    }
    __device__ static float ldg(const void* b, int N, int i, int idx) { return ldf(b, N, i, idx); }
    // store the post-collision set of node idx; f_0 is written as the
    // remainder phi - sum_{i>0} f_i, so the stored populations of a node sum
    // to its phi up to one rounding and sum phi does not drift with the
    // rounding of the collision
    __device__ static void stf(void* b, int N, int idx, const float f[9], float phi) {
#pragma unroll
        for (int i = 1; i < 9; ++i) static_cast<float*>(b)[i * N + idx] = f[i];
        static_cast<float*>(b)[idx] = sub(phi, sum8(f));
    }
    __device__ static void stg(void* b, int N, int idx, const float g[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) static_cast<float*>(b)[i * N + idx] = g[i];
    }
    // both sets, stores of f_i and g_i interleaved (as measured fastest)
    __device__ static void stfg(void* fb, void* gb, int N, int idx, const float f[9],
                                const float g[9], float phi) {
        float* F = static_cast<float*>(fb);
        float* G = static_cast<float*>(gb);
        F[idx] = sub(phi, sum8(f));
        G[idx] = g[0];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            F[i * N + idx] = f[i];
            G[i * N + idx] = g[i];
        }
    }
    // one plane entry (checkpoint and initial-state permutations); the rest
    // population's correction is zero in FP32
    __device__ static void putf(void* b, int N, int i, int idx, float v) {
        static_cast<float*>(b)[i * N + idx] = v;
    }
    __device__ static void putg(void* b, int N, int i, int idx, float v) {
        static_cast<float*>(b)[i * N + idx] = v;
    }
    __device__ static float round_f(int, float v) { return v; }
    // address of entry idx of plane i (for prefetches)
    __device__ static const void* addr_f(const void* b, int N, int i, int idx) {
        return static_cast<const float*>(b) + (i * N + idx);
    }
    __device__ static const void* addr_g(const void* b, int N, int i, int idx) {
        return addr_f(b, N, i, idx);
    }
};

template <typename H>
struct Half16;
template <>
struct Half16<__half> {
    static constexpr float GS = 1024.f;
    __device__ static float to_f(unsigned short u) { return __half2float(__ushort_as_half(u)); }
    __device__ static unsigned short from_f(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <>
struct Half16<__nv_bfloat16> {
    static constexpr float GS = 1.f;
    __device__ static float to_f(unsigned short u) { return __bfloat162float(__ushort_as_bfloat16(u)); }
    __device__ static unsigned short from_f(float v) {
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
};

template <typename H>
struct Shifted16 {
    using C = Half16<H>;
    static size_t f_bytes(size_t N) { return 4 * N + 16 * N; }
    static size_t g_bytes(size_t N) { return 18 * N; }
    __device__ static const unsigned short* fh(const void* b, int N) {
        return reinterpret_cast<const unsigned short*>(static_cast<const float*>(b) + N);
    }
    __device__ static unsigned short* fh(void* b, int N) {
        return reinterpret_cast<unsigned short*>(static_cast<float*>(b) + N);
    }
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
    __device__ static float ldf(const void* b, int N, int i, int idx) {
        if (i == 0) return __ldg(static_cast<const float*>(b) + idx);
        return dec_f(i, __ldg(fh(b, N) + ((i - 1) * N + idx)));
    }
    __device__ static float ldg(const void* b, int N, int i, int idx) {
        return dec_g(i, __ldg(static_cast<const unsigned short*>(b) + (i * N + idx)));
    }
    // undecoded 16-bit words (f: i > 0), so a pull can issue all its loads
    // before the first decode waits on one
    __device__ static unsigned short rawf(const void* b, int N, int i, int idx) {
        return __ldg(fh(b, N) + ((i - 1) * N + idx));
    }
    __device__ static unsigned short rawg(const void* b, int N, int i, int idx) {
        return __ldg(static_cast<const unsigned short*>(b) + (i * N + idx));
    }
    __device__ static void stf(void* b, int N, int idx, const float f[9], float phi) {
        float d[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const unsigned short e = enc_f(i, f[i]);
            fh(b, N)[(i - 1) * N + idx] = e;
            d[i] = dec_f(i, e);
        }
        static_cast<float*>(b)[idx] = sub(phi, sum8(d));
    }
    __device__ static void stg(void* b, int N, int idx, const float g[9]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) static_cast<unsigned short*>(b)[i * N + idx] = enc_g(i, g[i]);
    }
    __device__ static void stfg(void* fb, void* gb, int N, int idx, const float f[9],
                                const float g[9], float phi) {
        stf(fb, N, idx, f, phi);
        stg(gb, N, idx, g);
    }
    __device__ static void putf(void* b, int N, int i, int idx, float v) {
        if (i == 0)
            static_cast<float*>(b)[idx] = v;
        else
            fh(b, N)[(i - 1) * N + idx] = enc_f(i, v);
    }
    __device__ static void putg(void* b, int N, int i, int idx, float v) {
        static_cast<unsigned short*>(b)[i * N + idx] = enc_g(i, v);
    }
    // the value a moving population takes after storage
    __device__ static float round_f(int i, float v) { return i == 0 ? v : dec_f(i, enc_f(i, v)); }
    // address of entry idx of plane i (for prefetches)
    __device__ static const void* addr_f(const void* b, int N, int i, int idx) {
        if (i == 0) return static_cast<const float*>(b) + idx;
        return fh(b, N) + ((i - 1) * N + idx);
    }
    __device__ static const void* addr_g(const void* b, int N, int i, int idx) {
        return static_cast<const unsigned short*>(b) + (i * N + idx);
    }
};

template <>
struct Pop<ST_FP16> : Shifted16<__half> {};
template <>
struct Pop<ST_BF16> : Shifted16<__nv_bfloat16> {};

// Pull (stream) the 9 populations of node q through a 16-bit storage format:
// all nine loads first, then the decodes.  The six wall-dependent loads sit
// in a branch that is uniform across a warp when the wall flag is a run-time
// value (BR, the batched kernel: fewer instructions), and are per-lane
// selects when the kernel is compiled for walls (measured 5% faster there).
template <int ST, bool F, bool BR>
__device__ __forceinline__ void pull9_16(const void* s, int N, const Nbr& q, float v[9]) {
    using P = Pop<ST>;
    auto raw = [&](int i, int idx) { return F ? P::rawf(s, N, i, idx) : P::rawg(s, N, i, idx); };
    unsigned short u[9];
    float v0 = 0.f;
    if (F)
        v0 = __ldg(static_cast<const float*>(s) + (q.r0 + q.x));
    else
        u[0] = raw(0, q.r0 + q.x);
    u[1] = raw(1, q.r0 + q.xm);
    u[3] = raw(3, q.r0 + q.xp);
    if (!BR || q.lo || q.hi) {
        u[2] = q.lo ? raw(4, q.r0 + q.x) : raw(2, q.rm + q.x);
        u[4] = q.hi ? raw(2, q.r0 + q.x) : raw(4, q.rp + q.x);
        u[5] = q.lo ? raw(7, q.r0 + q.x) : raw(5, q.rm + q.xm);
        u[6] = q.lo ? raw(8, q.r0 + q.x) : raw(6, q.rm + q.xp);
        u[7] = q.hi ? raw(5, q.r0 + q.x) : raw(7, q.rp + q.xp);
        u[8] = q.hi ? raw(6, q.r0 + q.x) : raw(8, q.rp + q.xm);
    } else {
        u[2] = raw(2, q.rm + q.x);
        u[4] = raw(4, q.rp + q.x);
        u[5] = raw(5, q.rm + q.xm);
        u[6] = raw(6, q.rm + q.xp);
        u[7] = raw(7, q.rp + q.xp);
        u[8] = raw(8, q.rp + q.xm);
    }
    // a bounce-back link decodes with the stored direction's weight: opposite
    // directions share w_i, so the stored and the pulled index agree on it
    if (F) {
        v[0] = v0;
#pragma unroll
        for (int i = 1; i < 9; ++i) v[i] = P::dec_f(i, u[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = P::dec_g(i, u[i]);
    }
}

// Pull the 9 populations of node q in any storage format (WALLS as in
// make_nbr: < 0 when the wall flag is a run-time value).
template <int ST, int WALLS = -1>
__device__ __forceinline__ void pull9f(const void* s, int N, const Nbr& q, float v[9]) {
    if constexpr (ST == ST_FP32)
        pull9(static_cast<const float*>(s), (size_t)N, q, v);
    else
        pull9_16<ST, true, (WALLS < 0)>(s, N, q, v);
}
template <int ST, int WALLS = -1>
__device__ __forceinline__ void pull9g(const void* s, int N, const Nbr& q, float v[9]) {
    if constexpr (ST == ST_FP32)
        pull9(static_cast<const float*>(s), (size_t)N, q, v);
    else
        pull9_16<ST, false, (WALLS < 0)>(s, N, q, v);
}

template <int ST, int WALLS = -1>
__device__ __forceinline__ float phi_at_st(const void* fs, int N, int x, int y, int nx, int ny,
                                           int walls) {
    float v[9];
    if constexpr (ST == ST_FP32)  // the plain float pull (its address arithmetic measured faster)
        pull9(static_cast<const float*>(fs), (size_t)N, make_nbr<WALLS>(x, y, nx, ny, walls), v);
    else
        pull9f<ST, WALLS>(fs, N, make_nbr<WALLS>(x, y, nx, ny, walls), v);
    return sum9(v);
}

}  // namespace lbmpf
