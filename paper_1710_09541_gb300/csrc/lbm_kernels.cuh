// lbm_kernels.cuh -- device code of the phase-field lattice Boltzmann step
// (Liang et al., arXiv:1710.09541, Sec. II) for sm_103a.
//
// Data layout in HBM (structure of arrays): population set s in {f, g} is
// 9 planes of N = nx*ny FP32 values, plane i holding direction i (order of
// Eq. 10), node (x, y) at y*nx + x.  Two such buffers per set alternate each
// step (pull scheme: a step reads buffer A and writes buffer B at the node's
// own address).  A buffer holds post-collision values of the previous step;
// pulling f_i from x - c_i yields the pre-collision f_i(x, t) of Eq. 8.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmpf {

// D2Q9 velocities and weights, Eq. 10
__host__ __device__ constexpr int cx_of(int i) {
    return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy_of(int i) {
    return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
// Weights 4/9, 1/9, 1/36 rounded to FP32 sum to 1 + 2^-27, which makes every
// collision add 7.5e-9 phi to sum f_i^eq and drifts sum phi by ~1e-5 per
// 1000 steps.  w_5..8 is taken one ulp below RN(1/36) so that the FP32
// weights sum to exactly 1: w0 = 14913081 2^-25, w1 = 14913081 2^-27,
// w5 = 14913080 2^-29.
__host__ __device__ constexpr float w_of(int i) {
    return i == 0 ? 0x1.c71c72p-2f : (i < 5 ? 0x1.c71c72p-4f : 0x1.c71c70p-6f);
}
static_assert(0x1.c71c72p-2f + 4 * 0x1.c71c72p-4f + 4 * 0x1.c71c70p-6f == 1.0f, "weights");
__host__ __device__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i < 5 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 && opp_of(4) == 2, "opp");
static_assert(opp_of(5) == 7 && opp_of(6) == 8 && opp_of(7) == 5 && opp_of(8) == 6, "opp");

// Model constants in FP32, derived on the host from lbm_params.
struct Model {
    float rho_g, drho;      // rho_g, rho_l - rho_g               (Eq. 13)
    float beta4, kappa;     // 4 beta = 48 sigma / W, k = 1.5 sigma W (Eqs. 6, 7)
    float Gx, Gy;           // body force density                (Eq. 19)
    float inv_tau_f;        // 1 / tau_f                         (Eq. 8)
    float tau_f_mh;         // tau_f - 1/2 = tau_f (1 - 1/(2 tau_f)) (Eq. 11)
    float four_over_W;      // lambda = (4/W) phi (1 - phi)     (Eq. 3)
    float nu_l, nu_g;       // Eq. 24
    float inv_nu_l, inv_nu_g; // Eq. 25
    float mu_l, mu_g;       // Eq. 26
    int visc_mode;
    int walls;              // y boundary: 0 periodic, 1 bounce-back walls at both
                            // ends, 2 bounce-back wall at y = 0 and an open top
    int local_normal;       // Eq. 29 instead of Eq. 2 with Eq. 27
    int check_nonfinite;    // record non-finite nodes in the status flag (check_every > 0)
    unsigned int seed;      // this step's seed of the stochastic-rounding dithers (BF16_SHIFTED_SR)
};

// Neighbour addressing of one node: row offsets and wrapped columns.
struct Nbr {
    int r0, rm, rp;   // y*nx, (y-1)*nx, (y+1)*nx (periodic wrap in y)
    int x, xm, xp;    // x, x-1, x+1 (periodic wrap in x)
    bool lo, hi;      // node touches the wall at y = -1/2 / y = ny - 1/2
};

// `walls` is the y-boundary code of Model::walls.  WALLS < 0: everything
// decided at run time; 0: periodic, fixed at compile time; 1: a wall at y = 0
// fixed at compile time, the kind of top (wall or open) read from `walls`.
// At the open top the links that would enter from outside (c_y = -1) pull
// from the top row itself, i.e. they take the values the row below pulls
// (zero-gradient outflow); links leaving through it are not pulled by anyone.
template <int WALLS = -1>
__device__ __forceinline__ Nbr make_nbr(int x, int y, int nx, int ny, int walls) {
    const bool walled = WALLS >= 0 ? WALLS != 0 : walls != 0;
    const bool open_top = walled && walls == 2;
    Nbr q;
    q.x = x;
    q.xm = (x == 0) ? nx - 1 : x - 1;
    q.xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? (open_top ? y : 0) : y + 1;
    q.r0 = y * nx;
    q.rm = ym * nx;
    q.rp = yp * nx;
    q.lo = walled && (y == 0);
    q.hi = walled && !open_top && (y == ny - 1);
    return q;
}

// Pull (stream) the 9 populations of one node from buffer s:
// v_i = s_i(x - c_i); a link that crosses a wall returns the node's own
// post-collision value of the opposite direction (half-way bounce-back).
__device__ __forceinline__ void pull9(const float* __restrict__ s, size_t Nz, const Nbr& q,
                                      float v[9]) {
    const int N = (int)Nz;  // 20 N < 2^31 (checked at create): 32-bit offsets
    v[0] = __ldg(s + (q.r0 + q.x));
    v[1] = __ldg(s + (N + q.r0 + q.xm));
    v[3] = __ldg(s + (3 * N + q.r0 + q.xp));
    // A wall row is uniform across a warp (a warp covers part of one tile
    // row), so this is a branch, not a per-lane select of two loads.
    if (q.lo || q.hi) {
        v[2] = q.lo ? __ldg(s + (4 * N + q.r0 + q.x)) : __ldg(s + (2 * N + q.rm + q.x));
        v[4] = q.hi ? __ldg(s + (2 * N + q.r0 + q.x)) : __ldg(s + (4 * N + q.rp + q.x));
        v[5] = q.lo ? __ldg(s + (7 * N + q.r0 + q.x)) : __ldg(s + (5 * N + q.rm + q.xm));
        v[6] = q.lo ? __ldg(s + (8 * N + q.r0 + q.x)) : __ldg(s + (6 * N + q.rm + q.xp));
        v[7] = q.hi ? __ldg(s + (5 * N + q.r0 + q.x)) : __ldg(s + (7 * N + q.rp + q.xp));
        v[8] = q.hi ? __ldg(s + (6 * N + q.r0 + q.x)) : __ldg(s + (8 * N + q.rp + q.xm));
    } else {
        v[2] = __ldg(s + (2 * N + q.rm + q.x));
        v[4] = __ldg(s + (4 * N + q.rp + q.x));
        v[5] = __ldg(s + (5 * N + q.rm + q.xm));
        v[6] = __ldg(s + (6 * N + q.rm + q.xp));
        v[7] = __ldg(s + (7 * N + q.rp + q.xp));
        v[8] = __ldg(s + (8 * N + q.rp + q.xm));
    }
}

// Explicitly rounded FP32 operations.  All arithmetic of the step goes
// through these, so no multiply-add contraction is left to the compiler and
// every kernel that inlines the functions below (single-case and batched
// steps, field read-back, initialisation, probes) produces the same bits for
// the same inputs.  Additions, multiplications and fused multiply-adds are IEEE
// round-to-nearest.  The step has no division or square root: the five
// reciprocals it needs, 1/rho (Eq. 22a), 1/tau_g (Eq. 23), 1/(interpolated
// 1/nu) (Eq. 25), 1/|grad phi| (Eq. 2) and 1/|C| (Eq. 29), use the hardware
// approximations below.
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
// Hardware reciprocal and reciprocal square root (one instruction each,
// relative error below 2^-22; operands here are never subnormal: rho >= rho_g,
// tau_g >= 1/2, |grad phi|^2 > 1e-12).  Deterministic, so every kernel still
// produces the same bits.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Programmatic dependent launch.  A step kernel launched with programmatic
// stream serialisation may be scheduled while the previous step is still
// finishing: it waits here, before its first access to the state that step
// reads and writes, until the previous grid has completed and its writes are
// visible, and then lets the next step's CTAs be scheduled into the SM slots
// its own last wave leaves free.  For a kernel launched without the
// attribute both are no-ops.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

#ifndef LBM_FLAG_READ_FIRST
#define LBM_FLAG_READ_FIRST 1
#endif
// Record a non-finite node in the status flag: the lowest lane of those that
// reach this call (the offending ones) reports for its warp, and only while
// the bit is not yet set, so a blown-up state does not serialise on one
// address (measured at 2048^2 with 58% of the nodes NaN: FP32 19.3 k MLUPS with
// one atomic per warp, 39.3 k with the read first, against 40.4 k healthy).
__device__ __forceinline__ void report_nonfinite(unsigned int* flag) {
    const unsigned int lanes = __activemask();
    unsigned int lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
#if LBM_FLAG_READ_FIRST
    // once the bit is set, later warps read it (from L2) instead of queueing atomics
    if (lane == (unsigned int)(__ffs(lanes) - 1) && !(__ldcg(flag) & 1u)) atomicOr(flag, 1u);
#else
    if (lane == (unsigned int)(__ffs(lanes) - 1)) atomicOr(flag, 1u);
#endif
}

// c_i . v for the nine directions of Eq. 10; opposite directions get exactly
// opposite values (one rounding per pair).
__device__ __forceinline__ void cdot9(float vx, float vy, float c[9]) {
    const float s = add(vx, vy), d = sub(vy, vx);
    c[0] = 0.f;
    c[1] = vx;
    c[2] = vy;
    c[3] = -vx;
    c[4] = -vy;
    c[5] = s;
    c[6] = d;
    c[7] = -s;
    c[8] = -d;
}

// sum of the eight moving populations, in the association order used both
// for phi below and for the rest population written as the remainder
// phi - sum8 after the collision
__device__ __forceinline__ float sum8(const float v[9]) {
    return add(add(add(v[1], v[3]), add(v[2], v[4])), add(add(v[5], v[7]), add(v[6], v[8])));
}

// The one-node ring around a TX x TY tile: slot r -> tile-relative (lx, ly),
// -1 <= lx <= TX, -1 <= ly <= TY (top and bottom rows first, then the sides).
template <int TX, int TY>
struct Ring {
    static constexpr int count = 2 * (TX + 2) + 2 * TY;
    __device__ static void pos(int r, int& lx, int& ly) {
        if (r < TX + 2) {
            lx = r - 1;
            ly = -1;
        } else if (r < 2 * (TX + 2)) {
            lx = r - (TX + 2) - 1;
            ly = TY;
        } else if (r < 2 * (TX + 2) + TY) {
            lx = -1;
            ly = r - 2 * (TX + 2);
        } else {
            lx = TX;
            ly = r - 2 * (TX + 2) - TY;
        }
    }
};

// phi = sum_i f_i (Eq. 12), in one fixed association order everywhere so a
// node's phi is bit-identical whichever block computes it.  The rest
// population is added last, to the same tree of the moving ones that the
// remainder subtracts: where the pulled moving populations equal the node's
// own (uniform bulk), f_0 + sum8 then gives back phi exactly (f_0 = phi - sum8
// is exact by Sterbenz's lemma when sum8 lies in [phi/2, 2 phi]), so the
// rounding of the two sums cannot drift sum phi in one direction.
__device__ __forceinline__ float sum9(const float v[9]) { return add(v[0], sum8(v)); }

// coordinate of a tile/halo slot folded into the grid: periodic wrap in x;
// in y wrap, or clamp at a wall or the open top (ghost row = edge row).
__device__ __forceinline__ int fold_x(int x, int nx) {
    if ((unsigned)x >= (unsigned)nx) x = ((x % nx) + nx) % nx;
    return x;
}
__device__ __forceinline__ int fold_y(int y, int ny, int walls) {
    if ((unsigned)y >= (unsigned)ny) {
        if (walls) y = y < 0 ? 0 : ny - 1;
        else y = ((y % ny) + ny) % ny;
    }
    return y;
}

template <int WALLS = -1>
__device__ __forceinline__ float phi_at(const float* __restrict__ fs, size_t N, int x, int y,
                                        int nx, int ny, int walls) {
    float v[9];
    pull9(fs, N, make_nbr<WALLS>(x, y, nx, ny, walls), v);
    return sum9(v);
}

// nu(phi) by Eq. 24, 25 or 26 (inv_rho = 1/rho(phi) for Eq. 26)
__device__ __forceinline__ float viscosity(const Model& m, float phi, float inv_rho) {
    if (m.visc_mode == 1) return rcp_approx(fma_rn(phi, sub(m.inv_nu_l, m.inv_nu_g), m.inv_nu_g));
    if (m.visc_mode == 2) return mul(phi >= 0.5f ? m.mu_l : m.mu_g, inv_rho);
    return fma_rn(phi, sub(m.nu_l, m.nu_g), m.nu_g);
}

// Macroscopic state of one node from its pulled g_i and the phi stencil.
struct Macro {
    float rho, inv_rho, Fx, Fy, ux, uy, p, usq;
};

// The moments of g a node's recovery needs (Eq. 22): sum c_i g_i and the sum
// of the moving populations sum_{i != 0} g_i.
struct GMom {
    float mx, my, snz;
};
__device__ __forceinline__ GMom gmoments(const float g[9]) {
    GMom o;
    o.mx = add(sub(g[1], g[3]), add(sub(g[5], g[6]), sub(g[8], g[7])));
    o.my = add(sub(g[2], g[4]), add(sub(g[5], g[8]), sub(g[6], g[7])));
    o.snz = add(add(add(g[1], g[3]), add(g[2], g[4])), add(add(g[5], g[7]), add(g[6], g[8])));
    return o;
}

__device__ __forceinline__ Macro macro_from(const Model& m, const GMom& gm, float phi, float gx,
                                            float gy, float lap) {
    Macro o;
    o.rho = fma_rn(phi, m.drho, m.rho_g);                                      // Eq. 13
    const float bulk = mul(mul(mul(m.beta4, phi), sub(phi, 1.f)), sub(phi, 0.5f));
    const float mu = fma_rn(-m.kappa, lap, bulk);                              // Eq. 6
    o.Fx = fma_rn(mu, gx, m.Gx);                                               // Eqs. 5, 19
    o.Fy = fma_rn(mu, gy, m.Gy);
    o.inv_rho = rcp_approx(o.rho);
    o.ux = mul(fma_rn(0.5f, o.Fx, gm.mx), o.inv_rho);                         // Eq. 22a
    o.uy = mul(fma_rn(0.5f, o.Fy, gm.my), o.inv_rho);
    o.usq = fma_rn(o.ux, o.ux, mul(o.uy, o.uy));
    // Eq. 22b with c_s^2/(1 - w_0) = 3/5 and rho s_0(u) = -(2/3) rho |u|^2
    const float ugrad = fma_rn(o.ux, gx, mul(o.uy, gy));
    const float t = fma_rn(mul(0.5f, m.drho), ugrad, gm.snz);
    o.p = mul(0.6f, fma_rn(mul(-2.f / 3.f, o.rho), o.usq, t));
    return o;
}

__device__ __forceinline__ Macro macroscopic(const Model& m, const float g[9], float phi,
                                             float gx, float gy, float lap) {
    return macro_from(m, gmoments(g), phi, gx, gy, lap);
}

// Isotropic stencils of Eqs. 27 and 28 from the 3x3 neighbourhood
// (pE = phi(x+1, y), pN = phi(x, y+1), pNE = phi(x+1, y+1), ...).
struct Stencil {
    float gx, gy, lap;
};
__device__ __forceinline__ Stencil stencil(float pC, float pE, float pW, float pN, float pS,
                                           float pNE, float pNW, float pSW, float pSE) {
    Stencil s;
    const float dd = sub(pNE, pSW);
    const float da = sub(pSE, pNW);
    s.gx = fma_rn(sub(pE, pW), 1.f / 3.f, mul(add(dd, da), 1.f / 12.f));
    s.gy = fma_rn(sub(pN, pS), 1.f / 3.f, mul(sub(dd, da), 1.f / 12.f));
    // differences to the centre first: nearly exact in FP32 for neighbouring
    // values (Sterbenz), so the Laplacian carries no O(ulp(phi)) cancellation
    const float axis = add(add(sub(pE, pC), sub(pW, pC)), add(sub(pN, pC), sub(pS, pC)));
    const float diag = add(add(sub(pNE, pC), sub(pSW, pC)), add(sub(pNW, pC), sub(pSE, pC)));
    s.lap = fma_rn(axis, 2.f / 3.f, mul(diag, 1.f / 6.f));
    return s;
}

// f_i^eq (Eq. 9) formed as w phi + 3 w phi (c_i.u): opposite directions round
// symmetrically about the representable w phi, so each pair sums to 2 w phi
// exactly (writing w phi (1 +- 3 c.u) rounds 1+x and 1-x on different grids
// and drifts sum phi).
__device__ __forceinline__ float feq_i(int i, float phi, float cu) {
    const float wphi = mul(w_of(i), phi);
    return fma_rn(mul(3.f, wphi), cu, wphi);
}

// g_i^eq (Eqs. 16, 17): p/c_s^2 (w_i - [i == 0]) + rho w_i (3 cu + 4.5 cu^2 - 1.5 |u|^2)
__device__ __forceinline__ float geq_i(int i, float p3, float rho, float cu, float usq) {
    const float w = w_of(i);
    const float s = mul(w, fma_rn(cu, fma_rn(4.5f, cu, 3.f), mul(-1.5f, usq)));
    return fma_rn(rho, s, mul(p3, i == 0 ? w - 1.f : w));
}

// Both collisions of one node (Eqs. 2, 3, 8, 9, 11 and 15-17, 20); f and g are
// overwritten with the post-collision values.  phiu_prev = (phi u) of the
// previous step.  Returns (phi ux, phi uy) of this step.
__device__ __forceinline__ float2 collide(const Model& m, float f[9], float g[9], float phi,
                                          const Stencil& st, const Macro& M, float2 phiu_prev) {
    const float ux = M.ux, uy = M.uy;
    // relaxation time of the flow field, Eq. 23: tau_g = 3 nu + 1/2
    const float nu = viscosity(m, phi, M.inv_rho);
    const float omega_g = rcp_approx(fma_rn(3.f, nu, 0.5f));

    float cu[9];
    cdot9(ux, uy, cu);

    // d_t(phi u) by the backward difference, Eq. 11
    const float2 phiu = make_float2(mul(phi, ux), mul(phi, uy));
    const float Dx = sub(phiu.x, phiu_prev.x);
    const float Dy = sub(phiu.y, phiu_prev.y);
    const float lam = mul(mul(m.four_over_W, phi), sub(1.f, phi));  // Eq. 3
    float nx_ = 0.f, ny_ = 0.f;
    if (!m.local_normal) {  // Eq. 2 with the gradient of Eq. 27
        const float g2 = fma_rn(st.gx, st.gx, mul(st.gy, st.gy));
        if (g2 > 1e-12f) {  // |grad phi| > 1e-6: n is 0/0 below FP32 resolution
            const float inv = rsqrt_approx(g2);
            nx_ = mul(st.gx, inv);
            ny_ = mul(st.gy, inv);
        }
    } else {  // Eq. 29: C = sum c_i (f_i - f_i^eq) + d_t(phi u)/2, n = -C/|C|
        float ne[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) ne[i] = sub(f[i], feq_i(i, phi, cu[i]));
        const float Cx = add(mul(0.5f, Dx), add(sub(ne[1], ne[3]), add(sub(ne[5], ne[6]), sub(ne[8], ne[7]))));
        const float Cy = add(mul(0.5f, Dy), add(sub(ne[2], ne[4]), add(sub(ne[5], ne[8]), sub(ne[6], ne[7]))));
        const float c2 = fma_rn(Cx, Cx, mul(Cy, Cy));
        if (c2 > 1e-12f) {
            const float inv = rsqrt_approx(c2);
            nx_ = -mul(Cx, inv);
            ny_ = -mul(Cy, inv);
        }
    }

    // Each BGK update is x + (x^eq + tau S - x) / tau: the delta form, with
    // the source S (Eq. 11 or 20) folded into the equilibrium it relaxes to,
    //   f_i^eq + tau_f F_i = w_i phi + 3 w_i c_i . V,
    //       V = phi u + (tau_f - 1/2) (d_t(phi u) + lambda n / 3)    (Eqs. 9, 11)
    //   g_i^eq + tau_g G_i = p/c_s^2 (w_i - [i = 0]) + w_i [rho s_i(u)
    //       + 3 nu (3 c_i.F + 3 (rho_l - rho_g)(c_i.u)(c_i.grad phi))]
    //                           (Eqs. 16, 17, 20 with tau_g - 1/2 = 3 nu).
    // A node at equilibrium with no source stays bit-identical from step to
    // step, and opposite f directions round symmetrically about w_i phi
    // (c_i . V is exactly odd in c_i).  Against adding S after the update
    // this saves two operations per direction (FP16 storage at 2048^2:
    // 47.6 k -> 49.4 k MLUPS).  The form (1 - 1/tau) x + x^eq / tau + S is not
    // used: it moves every bulk value by an ulp each step, which drifted
    // sum phi 400x more on the layered Poiseuille run (4e-5 over 2e5 steps)
    // and shifted the FP16-stored Laplace jump by 4.6%.
    const float l3 = mul(lam, 1.f / 3.f);
    float cv[9], ch[9], ce[9];
    cdot9(fma_rn(m.tau_f_mh, fma_rn(l3, nx_, Dx), phiu.x),
          fma_rn(m.tau_f_mh, fma_rn(l3, ny_, Dy), phiu.y), cv);   // c_i . V
    const float nu9 = mul(9.f, nu);
    cdot9(mul(nu9, M.Fx), mul(nu9, M.Fy), ch);                    // c_i . 3 nu 3F
    const float e9 = mul(nu9, m.drho);
    cdot9(mul(e9, st.gx), mul(e9, st.gy), ce);                    // c_i . 3 nu 3 (rho_l - rho_g) grad phi
    const float p3 = mul(3.f, M.p);
    const float m15 = mul(-1.5f, M.usq);

    // i = 0 (c_0 = 0): F_0 = G_0 = 0 and the velocity-linear parts vanish;
    // written out because the explicitly rounded operations cannot fold the
    // products with zero away.  The results are the same bits as the general
    // form below would give.
    f[0] = fma_rn(m.inv_tau_f, sub(mul(w_of(0), phi), f[0]), f[0]);
    {
        const float geq0 = fma_rn(M.rho, mul(w_of(0), m15), mul(p3, w_of(0) - 1.f));
        g[0] = fma_rn(omega_g, sub(geq0, g[0]), g[0]);
    }
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        // Allen-Cahn, Eqs. 8, 9, 11
        const float fe = fma_rn(cv[i], 3.f * w_of(i), mul(w_of(i), phi));
        f[i] = fma_rn(m.inv_tau_f, sub(fe, f[i]), f[i]);
        // Navier-Stokes, Eqs. 15-17, 20
        const float s = fma_rn(cu[i], fma_rn(4.5f, cu[i], 3.f), m15);   // s_i / w_i
        const float t = fma_rn(cu[i], ce[i], ch[i]);
        const float ge = fma_rn(w_of(i), fma_rn(M.rho, s, t), mul(p3, w_of(i)));
        g[i] = fma_rn(omega_g, sub(ge, g[i]), g[i]);
    }
    return phiu;
}

}  // namespace lbmpf
