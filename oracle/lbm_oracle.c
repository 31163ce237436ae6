/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle of the phase-field lattice
 * Boltzmann time step of Liang, Xu, Chen, Wang, Chai & Shi,
 * "Phase-field-based lattice Boltzmann modeling of large-density-ratio
 * two-phase flows" (arXiv:1710.09541).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Everything is double precision, evaluated node by node in the order the
 * paper states the model (Sec. II):
 *   state at time t  = pre-collision populations f_i(x,t), g_i(x,t) (the left
 *                      hand sides of Eqs. 8 and 15 after streaming) plus the
 *                      product phi*u of the previous step (for d_t(phi u)).
 *   one step         = phi (Eq. 12) -> rho (Eq. 13) -> grad phi, lap phi
 *                      (Eqs. 27, 28) -> mu_phi, F (Eqs. 5-7, 19) -> u, p
 *                      (Eq. 22) -> nu, tau_g (Eqs. 23-26) -> Allen-Cahn
 *                      collision (Eqs. 2, 3, 8, 9, 11) -> Navier-Stokes
 *                      collision (Eqs. 15-17, 20) -> streaming with periodic
 *                      or half-way bounce-back boundaries.
 *
 * Readings of points the paper leaves open (each is used identically by the
 * CUDA library, which implements them separately):
 *   - Eq. 27 prints c_k inside a sum over i: read c_i.
 *   - d_t(phi u) in Eq. 11 is the first-order backward difference
 *     (phi u)^t - (phi u)^{t-1}; the history starts as phi0*u0.
 *   - n = grad phi / |grad phi| when |grad phi| > 1e-6, else n = 0.  Where
 *     grad phi vanishes (a symmetry point, a far tail) n is 0/0; the cut-off
 *     sits above the round-off of an FP32 stencil of an O(1) field (~1e-7)
 *     so single- and double-precision evaluations take the same branch.
 *   - At a half-way bounce-back wall the phi stencil uses a mirror ghost
 *     phi(y=-1) = phi(0), phi(ny) = phi(ny-1) (neutral wall).
 *   - The "open" top boundary of the impact case (Sec. III D names it without
 *     a rule) is a zero-gradient outflow: populations leaving through the top
 *     are lost, the unknown incoming ones of the top row (c_y = -1) equal the
 *     row below's after streaming, and the phi stencil's ghost row equals the
 *     top row.  The initial state obeys the same rule.
 *   - The step-function viscosity of Eq. 26 takes the liquid value at
 *     phi >= 0.5 and converts to kinematic viscosity with nu = mu/rho(phi).
 *   - Initial populations are the equilibria of Eqs. 9 and 16.
 *   - The local normal of Eq. 29 uses C = sum c_i (f_i - f_i^eq)
 *     + 0.5 d_t(phi u) (the Chapman-Enskog expansion of Eq. 8 with the
 *     source of Eq. 11 fixes the last term as the time derivative).  As
 *     A < 0 < B, Eq. 29 gives n = -C/|C|.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- D2Q9 lattice, Eq. 10 (velocity order of the paper) ----------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WGT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c = dx/dt = 1 */

/* opposite direction: c_opp(i) = -c_i */
static int opposite(int i) {
    for (int j = 0; j < 9; ++j)
        if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
    return -1;
}

typedef struct {
    double rho_l, rho_g;   /* Eq. 13 */
    double nu_l, nu_g;     /* Eqs. 24-26 (kinematic) */
    int visc_mode;         /* 0: Eq. 24, 1: Eq. 25, 2: Eq. 26 */
    double sigma, W;       /* Eq. 7 */
    double tau_h;          /* Allen-Cahn relaxation time (tau_f of Eq. 8) */
    double Gx, Gy;         /* body force density G, Eq. 4b / 19 */
    int bc_y;              /* 0: periodic in y, 1: half-way bounce-back walls,
                              2: bounce-back wall at y = 0, open top */
    int normal_scheme;     /* 0: central gradient (Eq. 27), 1: local (Eq. 29) */
} orc_params;

typedef struct {
    int nx, ny;
    orc_params p;
    double *f, *g;         /* pre-collision populations [9][ny][nx] */
    double *fs, *gs;       /* streamed (next) populations */
    double *phiu_x, *phiu_y; /* (phi u) of the previous step */
    double *phi, *gpx, *gpy, *lap; /* per-step work fields */
} orc_lattice;

void orc_lattice_constants(int* cx, int* cy, double* w, int* opp) {
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = WGT[i];
        opp[i] = opposite(i);
    }
}

/* ---- per-node model terms -------------------------------------------- */

/* Eq. 9: f_i^eq = w_i phi (1 + c_i.u / c_s^2) */
void orc_feq(double phi, double ux, double uy, double* feq) {
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = WGT[i] * phi * (1.0 + cu / CS2);
    }
}

/* Eq. 17: s_i(u) = w_i [c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)] */
static double s_i(int i, double ux, double uy) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return WGT[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Eq. 16: g_0^eq = p/c_s^2 (w_0 - 1) + rho s_0;  g_i^eq = p/c_s^2 w_i + rho s_i */
void orc_geq(double p, double rho, double ux, double uy, double* geq) {
    for (int i = 0; i < 9; ++i) {
        double pterm = (i == 0) ? (p / CS2) * (WGT[0] - 1.0) : (p / CS2) * WGT[i];
        geq[i] = pterm + rho * s_i(i, ux, uy);
    }
}

/* Eq. 11: F_i = (1 - 1/(2 tau_f)) w_i c_i.[d_t(phi u) + c_s^2 lambda n] / c_s^2 */
void orc_source_f(double tau_f, double lambda, double nx, double ny,
                  double dtx, double dty, double* Fi) {
    double ax = dtx + CS2 * lambda * nx;
    double ay = dty + CS2 * lambda * ny;
    for (int i = 0; i < 9; ++i)
        Fi[i] = (1.0 - 1.0 / (2.0 * tau_f)) * WGT[i] * (CX[i] * ax + CY[i] * ay) / CS2;
}

/* Eq. 20: G_i = (1 - 1/(2 tau_g)) w_i [c_i.(mu_phi grad phi + G)/c_s^2
 *               + (rho_l - rho_g) u grad phi : c_i c_i / c_s^2]
 * (Fx, Fy) is the total force mu_phi grad phi + G of Eq. 19. */
void orc_force_g(double tau_g, double drho, double ux, double uy,
                 double gpx, double gpy, double Fx, double Fy, double* Gi) {
    for (int i = 0; i < 9; ++i) {
        double cF = CX[i] * Fx + CY[i] * Fy;
        double cu = CX[i] * ux + CY[i] * uy;
        double cg = CX[i] * gpx + CY[i] * gpy;
        Gi[i] = (1.0 - 1.0 / (2.0 * tau_g)) * WGT[i] * (cF / CS2 + drho * cu * cg / CS2);
    }
}

/* Eqs. 24-26: kinematic viscosity at order parameter phi */
double orc_viscosity(const orc_params* P, double phi) {
    if (P->visc_mode == 1) /* Eq. 25 */
        return 1.0 / (phi * (1.0 / P->nu_l - 1.0 / P->nu_g) + 1.0 / P->nu_g);
    if (P->visc_mode == 2) { /* Eq. 26, nu = mu / rho(phi) */
        double rho = phi * (P->rho_l - P->rho_g) + P->rho_g;
        double mu = (phi >= 0.5) ? P->rho_l * P->nu_l : P->rho_g * P->nu_g;
        return mu / rho;
    }
    return phi * (P->nu_l - P->nu_g) + P->nu_g; /* Eq. 24 */
}

/* ---- finite differences, Eqs. 27 and 28 --------------------------------- */

/* phi at (x, y) with periodic wrap in x and, in y, either wrap (bc_y = 0) or
 * the ghost row equal to the edge row (a neutral wall, or zero gradient at an
 * open boundary). */
static double phi_at(const double* phi, int nx, int ny, int bc_y, int x, int y) {
    x = ((x % nx) + nx) % nx;
    if (bc_y == 0) {
        y = ((y % ny) + ny) % ny;
    } else {
        if (y < 0) y = 0;
        if (y > ny - 1) y = ny - 1;
    }
    return phi[(size_t)y * nx + x];
}

/* grad phi = sum_{i!=0} w_i c_i phi(x + c_i) / c_s^2               (Eq. 27)
 * lap phi  = sum_{i!=0} 2 w_i [phi(x + c_i) - phi(x)] / c_s^2       (Eq. 28) */
void orc_grad_lap(int nx, int ny, int bc_y, const double* phi,
                  double* gpx, double* gpy, double* lap) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double c = phi[(size_t)y * nx + x];
            double sx = 0.0, sy = 0.0, sl = 0.0;
            for (int i = 1; i < 9; ++i) {
                double nb = phi_at(phi, nx, ny, bc_y, x + CX[i], y + CY[i]);
                sx += WGT[i] * CX[i] * nb / CS2;
                sy += WGT[i] * CY[i] * nb / CS2;
                sl += 2.0 * WGT[i] * (nb - c) / CS2;
            }
            size_t n = (size_t)y * nx + x;
            gpx[n] = sx;
            gpy[n] = sy;
            lap[n] = sl;
        }
}

/* Open top (bc_y = 2): the populations that would enter the top row from
 * outside (c_y = -1) take the values the row below holds for the same
 * direction after streaming (zero normal gradient). */
static void open_top_fill(double* f, double* g, int nx, int ny) {
    const size_t N = (size_t)nx * ny;
    for (int i = 0; i < 9; ++i) {
        if (CY[i] != -1) continue;
        for (int x = 0; x < nx; ++x) {
            size_t top = (size_t)(ny - 1) * nx + x, below = (size_t)(ny - 2) * nx + x;
            f[i * N + top] = f[i * N + below];
            g[i * N + top] = g[i * N + below];
        }
    }
}

/* ---- lattice object ------------------------------------------------------ */

int orc_create(int nx, int ny, const orc_params* p, orc_lattice** out) {
    if (nx < 1 || ny < 1 || !p || !out) return -1;
    if (p->normal_scheme != 0 && p->normal_scheme != 1) return -1;
    if (p->bc_y < 0 || p->bc_y > 2) return -1;
    if (p->bc_y == 2 && ny < 2) return -1; /* the open top copies the row below */
    orc_lattice* L = (orc_lattice*)calloc(1, sizeof(orc_lattice));
    if (!L) return -5;
    size_t N = (size_t)nx * ny;
    L->nx = nx;
    L->ny = ny;
    L->p = *p;
    L->f = (double*)calloc(9 * N, sizeof(double));
    L->g = (double*)calloc(9 * N, sizeof(double));
    L->fs = (double*)calloc(9 * N, sizeof(double));
    L->gs = (double*)calloc(9 * N, sizeof(double));
    L->phiu_x = (double*)calloc(N, sizeof(double));
    L->phiu_y = (double*)calloc(N, sizeof(double));
    L->phi = (double*)calloc(N, sizeof(double));
    L->gpx = (double*)calloc(N, sizeof(double));
    L->gpy = (double*)calloc(N, sizeof(double));
    L->lap = (double*)calloc(N, sizeof(double));
    if (!L->f || !L->g || !L->fs || !L->gs || !L->phiu_x || !L->phiu_y ||
        !L->phi || !L->gpx || !L->gpy || !L->lap) {
        free(L->f); free(L->g); free(L->fs); free(L->gs); free(L->phiu_x);
        free(L->phiu_y); free(L->phi); free(L->gpx); free(L->gpy); free(L->lap);
        free(L);
        return -5;
    }
    *out = L;
    return 0;
}

void orc_destroy(orc_lattice* L) {
    if (!L) return;
    free(L->f); free(L->g); free(L->fs); free(L->gs); free(L->phiu_x);
    free(L->phiu_y); free(L->phi); free(L->gpx); free(L->gpy); free(L->lap);
    free(L);
}

/* Initial state: f = f^eq(phi0, u0) (Eq. 9), g = g^eq(p0, rho(phi0), u0)
 * (Eqs. 13, 16), (phi u)_prev = phi0 u0.  ux0, uy0, p0 may be NULL (zero). */
int orc_init(orc_lattice* L, const double* phi0, const double* ux0,
             const double* uy0, const double* p0) {
    size_t N = (size_t)L->nx * L->ny;
    const orc_params* P = &L->p;
    for (size_t n = 0; n < N; ++n) {
        double phi = phi0[n];
        double ux = ux0 ? ux0[n] : 0.0;
        double uy = uy0 ? uy0[n] : 0.0;
        double p = p0 ? p0[n] : 0.0;
        double rho = phi * (P->rho_l - P->rho_g) + P->rho_g;
        double feq[9], geq[9];
        orc_feq(phi, ux, uy, feq);
        orc_geq(p, rho, ux, uy, geq);
        for (int i = 0; i < 9; ++i) {
            L->f[i * N + n] = feq[i];
            L->g[i * N + n] = geq[i];
        }
        L->phiu_x[n] = phi * ux;
        L->phiu_y[n] = phi * uy;
    }
    if (P->bc_y == 2) open_top_fill(L->f, L->g, L->nx, L->ny);
    return 0;
}

/* phi over the whole grid (Eq. 12) and its stencils (Eqs. 27, 28) */
static void order_parameter_and_stencils(orc_lattice* L) {
    size_t N = (size_t)L->nx * L->ny;
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < (long long)N; ++n) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += L->f[i * N + n];
        L->phi[n] = s;
    }
    orc_grad_lap(L->nx, L->ny, L->p.bc_y, L->phi, L->gpx, L->gpy, L->lap);
}

/* Macroscopic quantities at node n from the current populations:
 * rho (Eq. 13), mu_phi (Eqs. 6, 7), F (Eqs. 5, 19), u (Eq. 22a), p (Eq. 22b). */
static void macroscopic(const orc_lattice* L, size_t n, double* rho_o,
                        double* mu_o, double* Fx_o, double* Fy_o, double* ux_o,
                        double* uy_o, double* p_o) {
    const orc_params* P = &L->p;
    size_t N = (size_t)L->nx * L->ny;
    double phi = L->phi[n];
    double drho = P->rho_l - P->rho_g;
    double rho = phi * drho + P->rho_g;
    double k = 1.5 * P->sigma * P->W;   /* Eq. 7 */
    double beta = 12.0 * P->sigma / P->W;
    double mu = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - k * L->lap[n]; /* Eq. 6 */
    double Fx = mu * L->gpx[n] + P->Gx; /* Eqs. 5, 19 */
    double Fy = mu * L->gpy[n] + P->Gy;
    double mx = 0.0, my = 0.0, sum_nz = 0.0;
    for (int i = 0; i < 9; ++i) {
        double gi = L->g[i * N + n];
        mx += CX[i] * gi;
        my += CY[i] * gi;
        if (i != 0) sum_nz += gi;
    }
    double ux = (mx + 0.5 * Fx) / rho; /* Eq. 22a */
    double uy = (my + 0.5 * Fy) / rho;
    double s0 = s_i(0, ux, uy);
    double p = CS2 / (1.0 - WGT[0]) *
               (sum_nz + 0.5 * drho * (ux * L->gpx[n] + uy * L->gpy[n]) + rho * s0); /* Eq. 22b */
    *rho_o = rho;
    *mu_o = mu;
    *Fx_o = Fx;
    *Fy_o = Fy;
    *ux_o = ux;
    *uy_o = uy;
    *p_o = p;
}

/* Unit normal n (Eq. 2 with Eq. 27, or Eq. 29) */
static void unit_normal(const orc_lattice* L, size_t n, const double* fpre,
                        double phi, double ux, double uy, double dtx, double dty,
                        double* nx_o, double* ny_o) {
    if (L->p.normal_scheme == 0) {
        double gx = L->gpx[n], gy = L->gpy[n];
        double mag = sqrt(gx * gx + gy * gy);
        if (mag > 1e-6) {
            *nx_o = gx / mag;
            *ny_o = gy / mag;
        } else {
            *nx_o = 0.0;
            *ny_o = 0.0;
        }
        return;
    }
    /* Eq. 29: C = sum c_i (f_i - f_i^eq) + 0.5 d_t(phi u);  n = -C/|C| */
    double feq[9];
    orc_feq(phi, ux, uy, feq);
    double Cx = 0.5 * dtx, Cy = 0.5 * dty;
    for (int i = 0; i < 9; ++i) {
        Cx += CX[i] * (fpre[i] - feq[i]);
        Cy += CY[i] * (fpre[i] - feq[i]);
    }
    double mag = sqrt(Cx * Cx + Cy * Cy);
    if (mag > 1e-6) {
        *nx_o = -Cx / mag;
        *ny_o = -Cy / mag;
    } else {
        *nx_o = 0.0;
        *ny_o = 0.0;
    }
}

/* One time step (Eqs. 8 and 15 with everything they use). */
static void one_step(orc_lattice* L) {
    const orc_params* P = &L->p;
    const int nx = L->nx, ny = L->ny;
    const size_t N = (size_t)nx * ny;
    const double tau_f = P->tau_h;
    const double drho = P->rho_l - P->rho_g;

    order_parameter_and_stencils(L);

#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            size_t n = (size_t)y * nx + x;
            double rho, mu, Fx, Fy, ux, uy, p;
            macroscopic(L, n, &rho, &mu, &Fx, &Fy, &ux, &uy, &p);
            double phi = L->phi[n];

            /* relaxation time of the flow field, Eq. 23 with Eqs. 24-26 */
            double nu = orc_viscosity(P, phi);
            double tau_g = nu / CS2 + 0.5;

            /* Allen-Cahn collision, Eqs. 2, 3, 8, 9, 11 */
            double fpre[9], gpre[9];
            for (int i = 0; i < 9; ++i) {
                fpre[i] = L->f[i * N + n];
                gpre[i] = L->g[i * N + n];
            }
            double lambda = 4.0 * phi * (1.0 - phi) / P->W;
            double dtx = phi * ux - L->phiu_x[n];
            double dty = phi * uy - L->phiu_y[n];
            double nxv, nyv;
            unit_normal(L, n, fpre, phi, ux, uy, dtx, dty, &nxv, &nyv);
            double feq[9], Fi[9];
            orc_feq(phi, ux, uy, feq);
            orc_source_f(tau_f, lambda, nxv, nyv, dtx, dty, Fi);

            /* Navier-Stokes collision, Eqs. 15-17, 20 */
            double geq[9], Gi[9];
            orc_geq(p, rho, ux, uy, geq);
            orc_force_g(tau_g, drho, ux, uy, L->gpx[n], L->gpy[n], Fx, Fy, Gi);

            for (int i = 0; i < 9; ++i) {
                double fpost = fpre[i] - (fpre[i] - feq[i]) / tau_f + Fi[i];
                double gpost = gpre[i] - (gpre[i] - geq[i]) / tau_g + Gi[i];
                /* streaming: f_i(x + c_i, t + 1) = f_i*(x, t); a link that
                 * leaves through a wall returns to x as the opposite
                 * direction (half-way bounce-back). */
                int xd = ((x + CX[i]) % nx + nx) % nx;
                int yd = y + CY[i];
                int id = i;
                if (P->bc_y == 0) {
                    yd = ((yd % ny) + ny) % ny;
                } else if (P->bc_y == 2 && yd > ny - 1) {
                    continue; /* leaves through the open top */
                } else if (yd < 0 || yd > ny - 1) {
                    xd = x;
                    yd = y;
                    id = opposite(i);
                }
                size_t m = (size_t)yd * nx + xd;
                L->fs[id * N + m] = fpost;
                L->gs[id * N + m] = gpost;
            }
            L->phiu_x[n] = phi * ux;
            L->phiu_y[n] = phi * uy;
        }
    }
    if (P->bc_y == 2) open_top_fill(L->fs, L->gs, nx, ny);
    double* t;
    t = L->f; L->f = L->fs; L->fs = t;
    t = L->g; L->g = L->gs; L->gs = t;
}

/* Threads of the OpenMP loops (n >= 1); returns the count in use, 1 without
 * OpenMP.  The results do not depend on it (every node is independent and
 * the only global sum is serial). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_step(orc_lattice* L, int nsteps) {
    if (nsteps < 0) return -1;
    for (int s = 0; s < nsteps; ++s) one_step(L);
    return 0;
}

/* phi, rho, u, p (and mu_phi) of the current state, by the formulas the step
 * uses.  Any output may be NULL. */
int orc_get_fields(orc_lattice* L, double* phi, double* rho, double* ux,
                   double* uy, double* p, double* mu) {
    size_t N = (size_t)L->nx * L->ny;
    order_parameter_and_stencils(L);
#pragma omp parallel for schedule(static)
    for (long long n = 0; n < (long long)N; ++n) {
        double r, m, Fx, Fy, vx, vy, pp;
        macroscopic(L, n, &r, &m, &Fx, &Fy, &vx, &vy, &pp);
        if (phi) phi[n] = L->phi[n];
        if (rho) rho[n] = r;
        if (ux) ux[n] = vx;
        if (uy) uy[n] = vy;
        if (p) p[n] = pp;
        if (mu) mu[n] = m;
    }
    return 0;
}

/* State: f[9][ny][nx], g[9][ny][nx], phiu_x[ny][nx], phiu_y[ny][nx] (doubles) */
int orc_get_state(const orc_lattice* L, double* buf) {
    size_t N = (size_t)L->nx * L->ny;
    memcpy(buf, L->f, 9 * N * sizeof(double));
    memcpy(buf + 9 * N, L->g, 9 * N * sizeof(double));
    memcpy(buf + 18 * N, L->phiu_x, N * sizeof(double));
    memcpy(buf + 19 * N, L->phiu_y, N * sizeof(double));
    return 0;
}

int orc_set_state(orc_lattice* L, const double* buf) {
    size_t N = (size_t)L->nx * L->ny;
    memcpy(L->f, buf, 9 * N * sizeof(double));
    memcpy(L->g, buf + 9 * N, 9 * N * sizeof(double));
    memcpy(L->phiu_x, buf + 18 * N, N * sizeof(double));
    memcpy(L->phiu_y, buf + 19 * N, N * sizeof(double));
    return 0;
}

/* sum of phi over the grid (plain running sum in node order) */
double orc_sum_phi(const orc_lattice* L) {
    size_t N = (size_t)L->nx * L->ny;
    double s = 0.0;
    for (size_t n = 0; n < N; ++n)
        for (int i = 0; i < 9; ++i) s += L->f[i * N + n];
    return s;
}
