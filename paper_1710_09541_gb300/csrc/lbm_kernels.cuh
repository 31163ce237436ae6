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
    float src_f;            // 1 - 1/(2 tau_f)                   (Eq. 11)
    float four_over_W;      // lambda = (4/W) phi (1 - phi)     (Eq. 3)
    float nu_l, nu_g;       // Eq. 24
    float inv_nu_l, inv_nu_g; // Eq. 25
    float mu_l, mu_g;       // Eq. 26
    int visc_mode;
    int walls;              // half-way bounce-back walls in y
    int local_normal;       // Eq. 29 instead of Eq. 2 with Eq. 27
};

// Neighbour addressing of one node: row offsets and wrapped columns.
struct Nbr {
    int r0, rm, rp;   // y*nx, (y-1)*nx, (y+1)*nx (periodic wrap in y)
    int x, xm, xp;    // x, x-1, x+1 (periodic wrap in x)
    bool lo, hi;      // node touches the wall at y = -1/2 / y = ny - 1/2
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int nx, int ny, int walls) {
    Nbr q;
    q.x = x;
    q.xm = (x == 0) ? nx - 1 : x - 1;
    q.xp = (x == nx - 1) ? 0 : x + 1;
    const int ym = (y == 0) ? ny - 1 : y - 1;
    const int yp = (y == ny - 1) ? 0 : y + 1;
    q.r0 = y * nx;
    q.rm = ym * nx;
    q.rp = yp * nx;
    q.lo = walls && (y == 0);
    q.hi = walls && (y == ny - 1);
    return q;
}

// Pull (stream) the 9 populations of one node from buffer s:
// v_i = s_i(x - c_i); a link that crosses a wall returns the node's own
// post-collision value of the opposite direction (half-way bounce-back).
__device__ __forceinline__ void pull9(const float* __restrict__ s, size_t N, const Nbr& q,
                                      float v[9]) {
    v[0] = __ldg(s + q.r0 + q.x);
    v[1] = __ldg(s + N + q.r0 + q.xm);
    v[3] = __ldg(s + 3 * N + q.r0 + q.xp);
    v[2] = q.lo ? __ldg(s + 4 * N + q.r0 + q.x) : __ldg(s + 2 * N + q.rm + q.x);
    v[4] = q.hi ? __ldg(s + 2 * N + q.r0 + q.x) : __ldg(s + 4 * N + q.rp + q.x);
    v[5] = q.lo ? __ldg(s + 7 * N + q.r0 + q.x) : __ldg(s + 5 * N + q.rm + q.xm);
    v[6] = q.lo ? __ldg(s + 8 * N + q.r0 + q.x) : __ldg(s + 6 * N + q.rm + q.xp);
    v[7] = q.hi ? __ldg(s + 5 * N + q.r0 + q.x) : __ldg(s + 7 * N + q.rp + q.xp);
    v[8] = q.hi ? __ldg(s + 6 * N + q.r0 + q.x) : __ldg(s + 8 * N + q.rp + q.xm);
}

// phi = sum_i f_i (Eq. 12), in one fixed association order everywhere so a
// node's phi is bit-identical whichever block computes it.
__device__ __forceinline__ float sum9(const float v[9]) {
    return ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
}

// coordinate of a tile/halo slot folded into the grid: periodic wrap in x;
// in y wrap, or clamp at a wall (mirror ghost phi(-1) = phi(0)).
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

__device__ __forceinline__ float phi_at(const float* __restrict__ fs, size_t N, int x, int y,
                                        int nx, int ny, int walls) {
    float v[9];
    pull9(fs, N, make_nbr(x, y, nx, ny, walls), v);
    return sum9(v);
}

// nu(phi) by Eq. 24, 25 or 26
__device__ __forceinline__ float viscosity(const Model& m, float phi, float rho) {
    if (m.visc_mode == 1) return 1.f / fmaf(phi, m.inv_nu_l - m.inv_nu_g, m.inv_nu_g);
    if (m.visc_mode == 2) return (phi >= 0.5f ? m.mu_l : m.mu_g) / rho;
    return fmaf(phi, m.nu_l - m.nu_g, m.nu_g);
}

// Macroscopic state of one node from its pulled g_i and the phi stencil.
struct Macro {
    float rho, Fx, Fy, ux, uy, p;
};

__device__ __forceinline__ Macro macroscopic(const Model& m, const float g[9], float phi,
                                             float gx, float gy, float lap) {
    Macro o;
    o.rho = fmaf(phi, m.drho, m.rho_g);                                     // Eq. 13
    const float mu = m.beta4 * phi * (phi - 1.f) * (phi - 0.5f) - m.kappa * lap; // Eq. 6
    o.Fx = fmaf(mu, gx, m.Gx);                                              // Eqs. 5, 19
    o.Fy = fmaf(mu, gy, m.Gy);
    const float mx = (g[1] - g[3]) + ((g[5] - g[6]) + (g[8] - g[7]));
    const float my = (g[2] - g[4]) + ((g[5] - g[8]) + (g[6] - g[7]));
    o.ux = (mx + 0.5f * o.Fx) / o.rho;                                      // Eq. 22a
    o.uy = (my + 0.5f * o.Fy) / o.rho;
    const float snz = ((g[1] + g[3]) + (g[2] + g[4])) + ((g[5] + g[7]) + (g[6] + g[8]));
    const float usq = o.ux * o.ux + o.uy * o.uy;
    // Eq. 22b with c_s^2/(1 - w_0) = 3/5 and rho s_0(u) = -(2/3) rho |u|^2
    o.p = 0.6f * (snz + 0.5f * m.drho * (o.ux * gx + o.uy * gy) - (2.f / 3.f) * o.rho * usq);
    return o;
}

// Isotropic stencils of Eqs. 27 and 28 from the 3x3 neighbourhood
// (pE = phi(x+1, y), pN = phi(x, y+1), pNE = phi(x+1, y+1), ...).
struct Stencil {
    float gx, gy, lap;
};
__device__ __forceinline__ Stencil stencil(float pC, float pE, float pW, float pN, float pS,
                                           float pNE, float pNW, float pSW, float pSE) {
    Stencil s;
    const float dd = (pNE - pSW);
    const float da = (pSE - pNW);
    s.gx = (pE - pW) * (1.f / 3.f) + (dd + da) * (1.f / 12.f);
    s.gy = (pN - pS) * (1.f / 3.f) + (dd - da) * (1.f / 12.f);
    // differences to the centre first: nearly exact in FP32 for neighbouring
    // values (Sterbenz), so the Laplacian carries no O(ulp(phi)) cancellation
    s.lap = (((pE - pC) + (pW - pC)) + ((pN - pC) + (pS - pC))) * (2.f / 3.f) +
            (((pNE - pC) + (pSW - pC)) + ((pNW - pC) + (pSE - pC))) * (1.f / 6.f);
    return s;
}

// Both collisions of one node (Eqs. 2, 3, 8, 9, 11 and 15-17, 20); f and g are
// overwritten with the post-collision values.  phiu_prev = (phi u) of the
// previous step.  Returns (phi ux, phi uy) of this step.
__device__ __forceinline__ float2 collide(const Model& m, float f[9], float g[9], float phi,
                                          const Stencil& st, const Macro& M, float2 phiu_prev) {
    const float ux = M.ux, uy = M.uy;
    const float usq = ux * ux + uy * uy;
    // relaxation time of the flow field, Eq. 23
    const float nu = viscosity(m, phi, M.rho);
    const float omega_g = 1.f / fmaf(3.f, nu, 0.5f);
    const float src_g = fmaf(-0.5f, omega_g, 1.f);

    // d_t(phi u) by the backward difference, Eq. 11
    const float2 phiu = make_float2(phi * ux, phi * uy);
    const float Dx = phiu.x - phiu_prev.x;
    const float Dy = phiu.y - phiu_prev.y;
    const float lam = m.four_over_W * phi * (1.f - phi); // Eq. 3
    float nx_ = 0.f, ny_ = 0.f;
    if (!m.local_normal) {  // Eq. 2 with the gradient of Eq. 27
        const float g2 = st.gx * st.gx + st.gy * st.gy;
        if (g2 > 1e-12f) {  // |grad phi| > 1e-6: n is 0/0 below FP32 resolution
            const float inv = 1.f / sqrtf(g2);
            nx_ = st.gx * inv;
            ny_ = st.gy * inv;
        }
    } else {  // Eq. 29: C = sum c_i (f_i - f_i^eq) + d_t(phi u)/2, n = -C/|C|
        float Cx = 0.5f * Dx, Cy = 0.5f * Dy;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float cu = cx_of(i) * ux + cy_of(i) * uy;
            const float wphi = w_of(i) * phi;
            const float neq = f[i] - fmaf(3.f * wphi, cu, wphi);
            Cx += cx_of(i) * neq;
            Cy += cy_of(i) * neq;
        }
        const float c2 = Cx * Cx + Cy * Cy;
        if (c2 > 1e-12f) {
            const float inv = 1.f / sqrtf(c2);
            nx_ = -Cx * inv;
            ny_ = -Cy * inv;
        }
    }
    // F_i = (1 - 1/2tau_f) w_i 3 c_i . (D + lambda n / 3)           Eq. 11
    const float ax = fmaf(lam * (1.f / 3.f), nx_, Dx);
    const float ay = fmaf(lam * (1.f / 3.f), ny_, Dy);
    const float p3 = 3.f * M.p;
    const float hx = 3.f * M.Fx, hy = 3.f * M.Fy;              // 3 F
    const float ex = 3.f * m.drho * st.gx, ey = 3.f * m.drho * st.gy;

#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float w = w_of(i);
        const float cu = cx_of(i) * ux + cy_of(i) * uy;
        // Allen-Cahn: f_i^eq (Eq. 9) as w phi + 3 w phi (c_i.u): opposite
        // directions round symmetrically about the representable w phi, so
        // the pair sums to 2 w phi exactly (no drift of sum phi from 1 +- x
        // rounding on the two grids around 1.0), then source (Eq. 11), BGK (Eq. 8)
        const float wphi = w * phi;
        const float feq = fmaf(3.f * wphi, cu, wphi);
        const float Fi = m.src_f * 3.f * w * (cx_of(i) * ax + cy_of(i) * ay);
        f[i] = fmaf(m.inv_tau_f, feq - f[i], f[i]) + Fi;
        // Navier-Stokes: g_i^eq (Eqs. 16, 17), forcing (Eq. 20), BGK (Eq. 15)
        const float s = w * (cu * fmaf(4.5f, cu, 3.f) - 1.5f * usq);
        const float geq = (i == 0 ? p3 * (w - 1.f) : p3 * w) + M.rho * s;
        const float cF = cx_of(i) * hx + cy_of(i) * hy;
        const float cg = cx_of(i) * ex + cy_of(i) * ey;
        const float Gi = src_g * w * fmaf(cu, cg, cF);
        g[i] = fmaf(omega_g, geq - g[i], g[i]) + Gi;
    }
    return phiu;
}

}  // namespace lbmpf
