// lbm_store.cuh -- population storage formats.  All arithmetic is FP32; the
// formats differ only in how the two population sets sit in HBM.
//
//   FP32 (LBM_STORE_FP32): f and g as 9 FP32 planes each (36 B + 36 B / node);
//     f_0 is written as phi - sum_{i>0} f_i (see below).
//
//   FP16 / BF16 shifted (LBM_STORE_FP16_SHIFTED, LBM_STORE_BF16_SHIFTED); the
//   step works on the stored codes themselves (see Shifted16), so a pull
//   needs one conversion per population and a store one packed conversion
//   per pair:
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
//
//   BF16 shifted with stochastic rounding (LBM_STORE_BF16_SHIFTED_SR): the
//   BF16 layout; the step rounds the nine g codes stochastically (the f codes
//   and the read-back, initialisation and checkpoints as BF16_SHIFTED).
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

enum { ST_FP32 = 0, ST_FP16 = 1, ST_BF16 = 2, ST_BF16_SR = 3 };

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
                                const float g[9], float phi, unsigned int = 0) {
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
    // the step's hooks (the 16-bit formats work on codes instead): phi from
    // the pulled f (Eq. 12), the moments of g (Eq. 22), the pulled values as
    // populations, and the rest population f_0 that makes the stored
    // populations of an initial state sum to phi
    __device__ static float phi_of(const float f[9]) { return sum9(f); }
    __device__ static GMom gmom(const float g[9]) { return gmoments(g); }
    __device__ static void canon(float*, float*) {}
    __device__ static float init_rest(float phi, const float fe[9]) { return sub(phi, sum8(fe)); }
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

// Stochastic rounding of the g codes (LBM_STORE_BF16_SHIFTED_SR).  BF16 keeps
// 8 significant bits, and where tau_g is large (low Reynolds numbers) the
// change a collision makes to a g code each step is a small fraction of its
// spacing: rounding to nearest then returns the same code step after step and
// the slow viscous evolution stalls.  Rounding up with probability equal to
// the discarded fraction makes the stored code right on average, E[code] = v.
//
// The uniform 16-bit dithers come from a counter-based hash of (node, step):
// a 32-bit base per node, lowbias32 (C. Wellons, "Prospecting for hash
// functions", 2018: x ^= x >> 16; x *= 0x7feb352d; x ^= x >> 15;
// x *= 0x846ca68b; x ^= x >> 16) of the node index xor the step seed, then
// for j = 0..4 the product (base + j * 0x9e3779b9) * 0x85ebca6b, whose upper
// and lower halves serve directions 2j + 1 and 2j + 2 (j < 4) and the rest
// direction (the upper half of j = 4).  For a fixed node and
// direction each half is uniform, and independent from step to step through
// the seed; the dithers of one node's directions are correlated, which leaves
// each direction's rounding unbiased.
__device__ __forceinline__ unsigned int lowbias32(unsigned int x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// (hi, lo) rounded stochastically to a BF16 pair, hi in the upper half: the
// conversion with random bits (cvt.rs), which adds r[31:16] to the discarded
// half of hi and r[15:0] to that of lo and truncates, so each carries into
// the kept half with probability (discarded half) / 2^16.  (Checked on GB300
// against that integer definition on 2^20 random finite pairs: equal bit for
// bit.)
__device__ __forceinline__ unsigned int bf16x2_sr(float hi, float lo, unsigned int r) {
    unsigned int d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}

// The 16-bit formats store codes: h_i = f_i / w_i - 1/2 for the moving f_i
// and k_i = GS g_i / w_i for every g_i.  The step reads them as codes (one
// conversion each, no scaling), forms phi and the moments of g with the
// weights factored out per weight class, collides in code units
// (collide_code) and writes the new codes with one packed conversion per
// direction: decode and encode cost no arithmetic.  f_0 stays an FP32 value.
// SR (BF16 only): the step's stores round the g codes stochastically.
template <typename H, bool SR = false>
struct Shifted16 {
    using C = Half16<H>;
    static constexpr float GS = C::GS;
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
    // population <-> code (initialisation, checkpoints): f_i = w_i (h + 1/2)
    // for i > 0, g_i = w_i k / GS
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
    // sum_{i>0} f_i = sum_{i>0} w_i (h_i + 1/2), the weights factored out per
    // weight class; phi (Eq. 12) and the rest population written as the
    // remainder both use this one association order, so in uniform bulk
    // f_0 + s8 gives phi back exactly (f_0 = phi - s8 is exact by Sterbenz's
    // lemma) and their roundings cannot drift sum phi in one direction
    static constexpr float HALF_MOVING = 0.5f * (4.f * w_of(1) + 4.f * w_of(5));
    __device__ static float s8(const float h[9]) {
        const float a = add(add(h[1], h[3]), add(h[2], h[4]));
        const float d = add(add(h[5], h[7]), add(h[6], h[8]));
        return fma_rn(w_of(1), a, fma_rn(w_of(5), d, HALF_MOVING));
    }
    __device__ static float phi_of(const float h[9]) { return add(h[0], s8(h)); }
    // the moments of g (Eq. 22) from the codes k_i
    __device__ static GMom gmom(const float k[9]) {
        constexpr float a1 = w_of(1) / GS, a5 = w_of(5) / GS;  // exact: GS is a power of 2
        GMom o;
        o.mx = fma_rn(a1, sub(k[1], k[3]), mul(a5, add(sub(k[5], k[6]), sub(k[8], k[7]))));
        o.my = fma_rn(a1, sub(k[2], k[4]), mul(a5, add(sub(k[5], k[8]), sub(k[6], k[7]))));
        o.snz = fma_rn(a1, add(add(k[1], k[3]), add(k[2], k[4])),
                       mul(a5, add(add(k[5], k[7]), add(k[6], k[8]))));
        return o;
    }
    // codes -> populations (checkpoint read-out)
    __device__ static void canon(float f[9], float g[9]) {
#pragma unroll
        for (int i = 1; i < 9; ++i) f[i] = fma_rn(f[i], w_of(i), 0.5f * w_of(i));
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = mul(g[i], w_of(i) / GS);
    }
    // f_0 of an initial state whose moving populations fe_1..8 are stored as codes
    __device__ static float init_rest(float phi, const float fe[9]) {
        float h[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) h[i] = C::to_f(enc_f(i, fe[i]));
        return sub(phi, s8(h));
    }
    // store the post-collision codes of node idx: h_i | k_i << 16 per moving
    // direction, k_0, and f_0 as the remainder phi - s8(stored codes); seed
    // (SR only) is the step's seed of the dithers
    __device__ static void stfg(void* fb, void* gb, int N, int idx, const float h[9],
                                const float k[9], float phi, unsigned int seed = 0) {
        static_assert(!SR || C::GS == 1.f, "stochastic rounding is a BF16 format");
        unsigned int* P = pw(fb, N);
        float d[9];
        if constexpr (SR) {
            const unsigned int base = lowbias32((unsigned int)idx ^ seed);
#pragma unroll
            for (int i = 1; i < 9; i += 2) {
                // directions i and i + 1 take the upper and lower halves of
                // product (i - 1) / 2: one conversion rounds both g codes, one
                // packs both f codes, and two byte permutations make the words
                const unsigned int r = (base + (unsigned int)(i >> 1) * 0x9e3779b9u) * 0x85ebca6bu;
                const unsigned int kk = bf16x2_sr(k[i], k[i + 1], r);
                const unsigned int hh = C::pack(h[i], h[i + 1]);
                const unsigned int wi = __byte_perm(hh, kk, 0x7610);
                const unsigned int wj = __byte_perm(hh, kk, 0x5432);
                P[(i - 1) * N + idx] = wi;
                P[i * N + idx] = wj;
                d[i] = C::to_f(lo(wi));
                d[i + 1] = C::to_f(lo(wj));
            }
            static_cast<float*>(fb)[idx] = sub(phi, s8(d));
            static_cast<unsigned short*>(gb)[idx] =
                (unsigned short)(bf16x2_sr(k[0], 0.f, (base + 4u * 0x9e3779b9u) * 0x85ebca6bu) >> 16);
        } else {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const unsigned int w = C::pack(h[i], k[i]);
                P[(i - 1) * N + idx] = w;
                d[i] = C::to_f(lo(w));
            }
            static_cast<float*>(fb)[idx] = sub(phi, s8(d));
            static_cast<unsigned short*>(gb)[idx] = C::from_f(k[0]);
        }
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
template <>
struct Pop<ST_BF16_SR> : Shifted16<__nv_bfloat16, true> {};

// Both collisions of one node in the code units of a 16-bit format (the
// same update as collide, Eqs. 2, 3, 8, 9, 11 and 15-17, 20, divided through
// by the weights): h[1..8] hold the codes h_i = f_i / w_i - 1/2 and k[0..8]
// the codes k_i = GS g_i / w_i, and are overwritten with the post-collision
// codes.  With V as in collide, (f_i^eq + tau_f F_i) / w_i - 1/2 =
// phi - 1/2 + 3 c_i . V and (g_i^eq + tau_g G_i) GS / w_i = GS (rho s_i / w_i
// + 3 nu [3 c_i . F + 3 (rho_l - rho_g)(c_i . u)(c_i . grad phi)] + 3 p) for
// i > 0, GS (rho s_0 / w_0 + 3 p (w_0 - 1) / w_0) for i = 0, with s_i / w_i =
// 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 |u|^2.  f_0 is not collided: the store writes
// it as the remainder.  Returns (phi ux, phi uy).
template <class P>
__device__ __forceinline__ float2 collide_code(const Model& m, float h[9], float k[9], float phi,
                                               const Stencil& st, const Macro& M, float2 phiu_prev) {
    constexpr float GS = P::GS;
    const float ux = M.ux, uy = M.uy;
    const float nu = viscosity(m, phi, M.inv_rho);                     // Eqs. 23-26
    const float omega_g = rcp_approx(fma_rn(3.f, nu, 0.5f));
    float cu[9];
    cdot9(ux, uy, cu);
    const float2 phiu = make_float2(mul(phi, ux), mul(phi, uy));
    const float Dx = sub(phiu.x, phiu_prev.x);                          // d_t(phi u), Eq. 11
    const float Dy = sub(phiu.y, phiu_prev.y);
    const float lam = mul(mul(m.four_over_W, phi), sub(1.f, phi));      // Eq. 3
    const float phm = sub(phi, 0.5f);
    float nx_ = 0.f, ny_ = 0.f;
    if (!m.local_normal) {  // Eq. 2 with the gradient of Eq. 27
        const float g2 = fma_rn(st.gx, st.gx, mul(st.gy, st.gy));
        if (g2 > 1e-12f) {
            const float inv = rsqrt_approx(g2);
            nx_ = mul(st.gx, inv);
            ny_ = mul(st.gy, inv);
        }
    } else {  // Eq. 29: C = sum c_i (f_i - f_i^eq) + d_t(phi u)/2, n = -C/|C|
        float ne[9];  // (f_i - f_i^eq) / w_i
#pragma unroll
        for (int i = 1; i < 9; ++i) ne[i] = sub(h[i], fma_rn(3.f, cu[i], phm));
        const float Cx = add(mul(0.5f, Dx), fma_rn(w_of(1), sub(ne[1], ne[3]),
                                                   mul(w_of(5), add(sub(ne[5], ne[6]), sub(ne[8], ne[7])))));
        const float Cy = add(mul(0.5f, Dy), fma_rn(w_of(1), sub(ne[2], ne[4]),
                                                   mul(w_of(5), add(sub(ne[5], ne[8]), sub(ne[6], ne[7])))));
        const float c2 = fma_rn(Cx, Cx, mul(Cy, Cy));
        if (c2 > 1e-12f) {
            const float inv = rsqrt_approx(c2);
            nx_ = -mul(Cx, inv);
            ny_ = -mul(Cy, inv);
        }
    }
    // Allen-Cahn, Eqs. 8, 9, 11 (first, so c_i . V is dead before the g terms)
    {
        const float l3 = mul(lam, 1.f / 3.f);
        float cv[9];
        cdot9(fma_rn(m.tau_f_mh, fma_rn(l3, nx_, Dx), phiu.x),
              fma_rn(m.tau_f_mh, fma_rn(l3, ny_, Dy), phiu.y), cv);   // c_i . V
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float he = fma_rn(3.f, cv[i], phm);
            h[i] = fma_rn(m.inv_tau_f, sub(he, h[i]), h[i]);
        }
    }
    // Navier-Stokes, Eqs. 15-17, 20
    float ch[9], ce[9];
    const float nu9 = mul(9.f * GS, nu);                          // GS scalings are exact
    cdot9(mul(nu9, M.Fx), mul(nu9, M.Fy), ch);                    // GS c_i . 3 nu 3F
    const float e9 = mul(nu9, m.drho);
    cdot9(mul(e9, st.gx), mul(e9, st.gy), ce);                    // GS c_i . 3 nu 3 (rho_l - rho_g) grad phi
    const float p3 = mul(3.f * GS, M.p);
    const float rho = mul(GS, M.rho);
    const float m15 = mul(-1.5f, M.usq);
    {
        const float ke0 = fma_rn(rho, m15, mul(p3, (w_of(0) - 1.f) / w_of(0)));
        k[0] = fma_rn(omega_g, sub(ke0, k[0]), k[0]);
    }
    // Opposite directions i, o(i) share the part of the target even in c_i,
    // A = rho (4.5 (c_i.u)^2 - 1.5 |u|^2) + (c_i.u)(c_i . 3 nu 3 (rho_l -
    // rho_g) grad phi) + 3p, and take the odd part B = 3 rho c_i.u + c_i . 3 nu
    // 3F with opposite signs: A + B and A - B.
    const float rho3 = mul(3.f, rho);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // done with its opposite
        const int o = opp_of(i);
        const float c = cu[i];
        const float A = fma_rn(rho, fma_rn(mul(4.5f, c), c, m15), fma_rn(c, ce[i], p3));
        const float B = fma_rn(rho3, c, ch[i]);
        k[i] = fma_rn(omega_g, sub(add(A, B), k[i]), k[i]);
        k[o] = fma_rn(omega_g, sub(sub(A, B), k[o]), k[o]);
    }
    return phiu;
}

// The collision of the storage format ST: on populations (FP32) or on codes.
template <int ST>
__device__ __forceinline__ float2 collide_st(const Model& m, float f[9], float g[9], float phi,
                                             const Stencil& st, const Macro& M, float2 prev) {
    if constexpr (ST == ST_FP32)
        return collide(m, f, g, phi, st, M, prev);
    else
        return collide_code<Pop<ST>>(m, f, g, phi, st, M, prev);
}

// Pull (stream) node q through a 16-bit storage format: the nine loads (f_0
// and g_0, and one word of (f_i, g_i) codes per moving direction; w[i] holds
// direction i's word).  The six wall-dependent loads sit in a branch that is
// uniform across a warp (BR; a warp covers part of one tile row), or are
// per-lane selects.  G: load g_0 as well.  pull_16 adds the conversions of
// the codes to FP32 (f[0] is the FP32 value of f_0, f[1..8] and g[0..8] the
// codes h_i and k_i).
template <int ST, bool BR, bool G>
__device__ __forceinline__ void pull_words16(const void* fs, const void* gs, int N, const Nbr& q,
                                             unsigned int w[9], float& f0, unsigned short& g0) {
    using P = Pop<ST>;
    const unsigned int* W = P::pw(fs, N);
    auto raw = [&](int i, int idx) { return __ldg(W + ((i - 1) * N + idx)); };
    f0 = __ldg(static_cast<const float*>(fs) + (q.r0 + q.x));
    g0 = 0;
    if (G) g0 = __ldg(static_cast<const unsigned short*>(gs) + (q.r0 + q.x));
    w[0] = 0u;
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
}

// the codes as floats: h[0] = f_0 (an FP32 value), h[1..8] the f codes; k[0..8]
// the g codes.  A bounce-back link takes the code of the stored direction,
// which has the pulled direction's weight (opposite directions share w_i), so
// the code means the same population in either.
template <int ST>
__device__ __forceinline__ void codes_f(const unsigned int w[9], float f0, float h[9]) {
    using P = Pop<ST>;
    h[0] = f0;
#pragma unroll
    for (int i = 1; i < 9; ++i) h[i] = P::C::to_f(P::lo(w[i]));
}
template <int ST>
__device__ __forceinline__ void codes_g(const unsigned int w[9], unsigned short g0, float k[9]) {
    using P = Pop<ST>;
    k[0] = P::C::to_f(g0);
#pragma unroll
    for (int i = 1; i < 9; ++i) k[i] = P::C::to_f(P::hi(w[i]));
}

template <int ST, bool BR, bool G>
__device__ __forceinline__ void pull_16(const void* fs, const void* gs, int N, const Nbr& q,
                                        float f[9], float g[9]) {
    unsigned int w[9];
    float f0;
    unsigned short g0;
    pull_words16<ST, BR, G>(fs, gs, N, q, w, f0, g0);
    codes_f<ST>(w, f0, f);
    if (G) codes_g<ST>(w, g0, g);
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
    return Pop<ST>::phi_of(v);
}

}  // namespace lbmpf
