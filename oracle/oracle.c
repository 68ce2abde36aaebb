/*
 * FP64 CPU oracle for the D2Q9 two-relaxation-time regularized lattice
 * Boltzmann (TRT-RLB) scheme of Yu, Qin, Chen, Shu and Yuan,
 * "Two-relaxation-time regularized lattice Boltzmann model for Navier-Stokes
 * equations" (arXiv 2312.10318).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the
 * GPU library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Equation names are the paper's equation labels (eq2, eq3, eq4, eq6, eq9,
 * eq11, eq_Gi, eq_a20, ...); sections are those of the paper.
 *
 * Everything is written the way the paper states it, without D2Q9 shortcuts:
 *   - Hermite tensors are built from their definition (eq3) and contracted with
 *     full alpha, beta, gamma loops;
 *   - the equilibrium is the third-order Hermite expansion (eq4);
 *   - the non-equilibrium moments are literal projections of f - f^eq (eq9);
 *   - the post-collision state is the right-hand side of eq2, term by term;
 *   - streaming is the left-hand side of eq2 in push form, with half-way
 *     bounce-back (eq_a20) at walls.
 * Compiled with -ffp-contract=off so that no fused multiply-add changes the
 * rounding of the plain expressions.
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the project's design notes):
 *   R1  d_gamma Phi_abg is discretised by second-order central differences on
 *       the node lattice; Phi is taken at the current time level (CURRENT), at
 *       the previous one (LAGGED, with Phi^{-1} := Phi^0), or dropped (OFF).
 *   R2  Phi at non-fluid neighbours: 0 at stationary walls and outside a
 *       non-periodic edge, rho_w u_w^3 at a moving (inlet) wall node, and the
 *       inward neighbour's value at an outlet ghost node.
 *   R4  f is initialised as f^eq(rho,u) - (1/2) w_i e_i.F / c_s^2, so that the
 *       zeroth and first moments satisfy eq11 and the initial second- and
 *       third-order non-equilibrium parts vanish.
 *   R5  The body force is F = rho g with the local density (eq_a2).
 *   R11 A moving wall reflects with Ladd's correction
 *       -2 w_i rho_w (e_i.u_w)/c_s^2 (e_i pointing into the wall); an outlet
 *       ghost node does not collide and re-emits the post-collision populations
 *       of its inward neighbour (x-1, y) (zero-gradient outlet).
 *   R15 Zou-He constant-pressure outlet (Sec. III D): a class-4 node on the
 *       last column of a lattice that is not periodic in x collides like a
 *       fluid node; the populations entering it across the edge (e_x = -1)
 *       are rebuilt from the others so that sum f = outlet_rho, sum e_y f = 0
 *       and the normal non-equilibrium part bounces back:
 *         f_i = f_ibar + (f^eq_i - f^eq_ibar)(outlet_rho, (u_x, 0))
 *               - 1/2 e_iy (f_(0,1) - f_(0,-1)),
 *       u_x = [sum_{e_x=0} f + 2 sum_{e_x=1} f] / outlet_rho - 1.  The rebuild
 *       is applied to every state the step reads or returns.  Phi beyond the
 *       edge is the outlet node's own value (zero gradient); the links that
 *       leave across the edge are open, not walls.
 *   R18 The vorticity compared in the error norms is omega = d_x u_y - d_y u_x
 *       by central differences on the node lattice, at fluid nodes whose four
 *       axis neighbours are fluid nodes of the domain.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9
#define ND 2

/* Node classes of the boundary mask. */
enum { ORC_FLUID = 0, ORC_SOLID = 1, ORC_INLET = 2, ORC_OUTLET = 3, ORC_PRESSURE = 4 };
/* Time level of Phi in G_i (reading R1). */
enum { ORC_G_LAGGED = 0, ORC_G_CURRENT = 1, ORC_G_OFF = 2 };

typedef struct {
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    double tau1;      /* tau_{s,1}: relaxes first and second order (eq2) */
    double tau2;      /* tau_{s,2}: relaxes the third order (eq2)        */
    double gx, gy;    /* body acceleration, F = rho g (eq_a2)            */
    double wall_ux, wall_uy, wall_rho; /* moving-wall state (inlet)      */
    double outlet_rho; /* density of Zou-He pressure outlet nodes (R15)  */
    int32_t g_mode;   /* ORC_G_LAGGED / CURRENT / OFF                    */
} orc_params;

/* ---- D2Q9 lattice, Sec. II B: velocity matrix, weights, c_s = c/sqrt(3) -- */
static const int EV[NQ][ND] = {
    {0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
static const double WV[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 with c = dx/dt = 1 */

static double kron(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Hermite tensors, eq3. */
static double herm1(int i, int a) { return (double)EV[i][a]; }
static double herm2(int i, int a, int b) {
    return (double)(EV[i][a] * EV[i][b]) - CS2 * kron(a, b);
}
static double herm3(int i, int a, int b, int c) {
    return (double)(EV[i][a] * EV[i][b] * EV[i][c]) -
           CS2 * ((double)EV[i][a] * kron(b, c) + (double)EV[i][b] * kron(c, a) +
                  (double)EV[i][c] * kron(a, b));
}

/* Index of the velocity opposite to e_i, found by search (not tabulated). */
static int opposite(int i) {
    for (int j = 0; j < NQ; ++j)
        if (EV[j][0] == -EV[i][0] && EV[j][1] == -EV[i][1]) return j;
    return -1;
}

/* Threads the collision loop runs on. */
int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the threads of the following loops (n >= 1); for timing on one core. */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- exported lattice description, for the identity tests ------------- */
void orc_lattice(int32_t* e /* [9][2] */, double* w /* [9] */, double* cs2) {
    for (int i = 0; i < NQ; ++i) {
        e[2 * i] = EV[i][0];
        e[2 * i + 1] = EV[i][1];
        w[i] = WV[i];
    }
    *cs2 = CS2;
}

/* All Hermite tensors of velocity i: h1[2], h2[2][2], h3[2][2][2] (eq3). */
void orc_hermite(int i, double* h1, double* h2, double* h3) {
    for (int a = 0; a < ND; ++a) {
        h1[a] = herm1(i, a);
        for (int b = 0; b < ND; ++b) {
            h2[a * ND + b] = herm2(i, a, b);
            for (int c = 0; c < ND; ++c) h3[(a * ND + b) * ND + c] = herm3(i, a, b, c);
        }
    }
}

/* ---- per-node pieces of the scheme ------------------------------------- */

/* Third-order Hermite equilibrium, eq4. */
void orc_equilibrium(double rho, const double* u, double* feq) {
    const double cs4 = CS2 * CS2, cs6 = CS2 * CS2 * CS2;
    for (int i = 0; i < NQ; ++i) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int a = 0; a < ND; ++a) {
            t1 += herm1(i, a) * u[a];
            for (int b = 0; b < ND; ++b) {
                t2 += herm2(i, a, b) * u[a] * u[b];
                for (int c = 0; c < ND; ++c) t3 += herm3(i, a, b, c) * u[a] * u[b] * u[c];
            }
        }
        feq[i] = WV[i] * rho * (1.0 + t1 / CS2 + t2 / (2.0 * cs4) + t3 / (6.0 * cs6));
    }
}

/* Forcing term of Luo, eq6. */
void orc_forcing(const double* F, const double* u, double* Fi) {
    const double cs4 = CS2 * CS2;
    for (int i = 0; i < NQ; ++i) {
        double t1 = 0.0, t2 = 0.0;
        for (int a = 0; a < ND; ++a) {
            t1 += herm1(i, a) * F[a];
            for (int b = 0; b < ND; ++b) t2 += herm2(i, a, b) * (F[a] * u[b] + u[a] * F[b]);
        }
        Fi[i] = WV[i] * (t1 / CS2 + t2 / (2.0 * cs4));
    }
}

/* Cubic-error compensation, eq_Gi.  dphi[a][b] = d_gamma Phi_{a b gamma}. */
void orc_compensation(double tau1, const double* dphi, double* G) {
    const double cs6 = CS2 * CS2 * CS2;
    for (int i = 0; i < NQ; ++i) {
        double t = 0.0;
        for (int a = 0; a < ND; ++a)
            for (int b = 0; b < ND; ++b) t += herm2(i, a, b) * dphi[a * ND + b];
        G[i] = -WV[i] * t / (6.0 * cs6) * (1.0 - 1.0 / (2.0 * tau1));
    }
}

/* Non-equilibrium projections, eq9: A1[2], A2[2][2], A3[2][2][2]. */
void orc_projections(const double* f, const double* feq, double* A1, double* A2, double* A3) {
    for (int a = 0; a < ND; ++a) {
        A1[a] = 0.0;
        for (int i = 0; i < NQ; ++i) A1[a] += herm1(i, a) * (f[i] - feq[i]);
        for (int b = 0; b < ND; ++b) {
            double s2 = 0.0;
            for (int i = 0; i < NQ; ++i) s2 += herm2(i, a, b) * (f[i] - feq[i]);
            A2[a * ND + b] = s2;
            for (int c = 0; c < ND; ++c) {
                double s3 = 0.0;
                for (int i = 0; i < NQ; ++i) s3 += herm3(i, a, b, c) * (f[i] - feq[i]);
                A3[(a * ND + b) * ND + c] = s3;
            }
        }
    }
}

/* Density and velocity with He's half-force shift, eq11 and the mass sum
 * before it: rho = sum f, rho u = sum e f + F/2, F = rho g (eq_a2). */
void orc_macroscopic(const double* f, const double* g, double* rho, double* u) {
    double r = 0.0;
    for (int i = 0; i < NQ; ++i) r += f[i];
    for (int a = 0; a < ND; ++a) {
        double j = 0.0;
        for (int i = 0; i < NQ; ++i) j += (double)EV[i][a] * f[i];
        u[a] = (j + 0.5 * r * g[a]) / r;
    }
    *rho = r;
}

/* Post-collision populations: the right-hand side of eq2 at one node.
 * dphi[a][b] = d_gamma Phi_{a b gamma} at the node (ignored when g_mode is
 * OFF).  Optional outputs (may be NULL): feq, G, Fi, rho, u. */
void orc_collide_node(const orc_params* p, const double* f, const double* dphi, double* fstar,
                      double* feq_out, double* G_out, double* Fi_out, double* rho_out,
                      double* u_out) {
    const double cs4 = CS2 * CS2, cs6 = CS2 * CS2 * CS2;
    const double g[ND] = {p->gx, p->gy};
    double rho, u[ND], F[ND], feq[NQ], G[NQ], Fi[NQ];
    double A1[ND], A2[ND * ND], A3[ND * ND * ND];
    orc_macroscopic(f, g, &rho, u);
    for (int a = 0; a < ND; ++a) F[a] = rho * g[a];
    orc_equilibrium(rho, u, feq);
    orc_projections(f, feq, A1, A2, A3);
    if (p->g_mode == ORC_G_OFF) {
        for (int i = 0; i < NQ; ++i) G[i] = 0.0;
    } else {
        orc_compensation(p->tau1, dphi, G);
    }
    orc_forcing(F, u, Fi);
    for (int i = 0; i < NQ; ++i) {
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < ND; ++a) {
            s1 += herm1(i, a) * A1[a];
            for (int b = 0; b < ND; ++b) {
                s2 += herm2(i, a, b) * A2[a * ND + b];
                for (int c = 0; c < ND; ++c) s3 += herm3(i, a, b, c) * A3[(a * ND + b) * ND + c];
            }
        }
        fstar[i] = feq[i] + (1.0 - 1.0 / p->tau1) * WV[i] * s1 / CS2 +
                   (1.0 - 1.0 / p->tau1) * WV[i] * s2 / (2.0 * cs4) +
                   (1.0 - 1.0 / p->tau2) * WV[i] * s3 / (6.0 * cs6) + G[i] +
                   (1.0 - 1.0 / (2.0 * p->tau1)) * Fi[i];
    }
    if (feq_out) memcpy(feq_out, feq, sizeof feq);
    if (G_out) memcpy(G_out, G, sizeof G);
    if (Fi_out) memcpy(Fi_out, Fi, sizeof Fi);
    if (rho_out) *rho_out = rho;
    if (u_out) memcpy(u_out, u, sizeof u);
}

/* ---- lattice-wide helpers ---------------------------------------------- */

static size_t node(const orc_params* p, int x, int y) { return (size_t)y * p->nx + x; }

/* Wraps (x, y) for periodic directions.  Returns 0 when the point lies outside
 * a non-periodic edge. */
static int wrap(const orc_params* p, int* x, int* y) {
    if (*x < 0 || *x >= p->nx) {
        if (!p->periodic_x) return 0;
        *x = ((*x % p->nx) + p->nx) % p->nx;
    }
    if (*y < 0 || *y >= p->ny) {
        if (!p->periodic_y) return 0;
        *y = ((*y % p->ny) + p->ny) % p->ny;
    }
    return 1;
}

static int cls(const uint8_t* mask, const orc_params* p, int x, int y) {
    return mask ? mask[node(p, x, y)] : ORC_FLUID;
}

/* Nodes that collide: fluid nodes and pressure outlet nodes. */
static int colliding(int c) { return c == ORC_FLUID || c == ORC_PRESSURE; }

/* Mask validity: classes in 0..4, every outlet ghost's inward neighbour
 * (x-1, y) exists and is a fluid node, and pressure outlet nodes lie on the
 * last column of a lattice that is not periodic in x.  Returns 0 when valid. */
int orc_check_mask(const orc_params* p, const uint8_t* mask) {
    if (!mask) return 0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            int c = mask[node(p, x, y)];
            if (c > ORC_PRESSURE) return 1;
            if (c == ORC_OUTLET) {
                int xs = x - 1, ys = y;
                if (!wrap(p, &xs, &ys) || cls(mask, p, xs, ys) != ORC_FLUID) return 2;
            }
            if (c == ORC_PRESSURE && (p->periodic_x || x != p->nx - 1)) return 3;
        }
    return 0;
}

/* Zou-He rebuild (reading R15) of the populations entering every pressure
 * outlet node across the x = nx edge, in place. */
static void zou_he_outlet(const orc_params* p, const uint8_t* mask, double* f) {
    if (!mask) return;
    const size_t n = (size_t)p->nx * p->ny;
    const int x = p->nx - 1;
    for (int y = 0; y < p->ny; ++y) {
        const size_t k = node(p, x, y);
        if (mask[k] != ORC_PRESSURE) continue;
        double fk[NQ];
        for (int i = 0; i < NQ; ++i) fk[i] = f[(size_t)i * n + k];
        double tangential = 0.0, outgoing = 0.0, fn = 0.0, fs = 0.0;
        for (int i = 0; i < NQ; ++i) {
            if (EV[i][0] == 0) tangential += fk[i];
            if (EV[i][0] == 1) outgoing += fk[i];
            if (EV[i][0] == 0 && EV[i][1] == 1) fn = fk[i];
            if (EV[i][0] == 0 && EV[i][1] == -1) fs = fk[i];
        }
        const double rho = p->outlet_rho;
        const double u[ND] = {(tangential + 2.0 * outgoing) / rho - 1.0, 0.0};
        double feq[NQ];
        orc_equilibrium(rho, u, feq);
        for (int i = 0; i < NQ; ++i) {
            if (EV[i][0] != -1) continue;
            const int j = opposite(i);
            f[(size_t)i * n + k] = fk[j] + (feq[i] - feq[j]) - 0.5 * EV[i][1] * (fn - fs);
        }
    }
}

/* The rebuild on its own (for tests). */
void orc_zou_he(const orc_params* p, const uint8_t* mask, double* f) { zou_he_outlet(p, mask, f); }

/* Phi_xxx = rho u_x^3 and Phi_yyy = rho u_y^3 (eq_Gi) on every node, with
 * the non-fluid values of reading R2.  rho, ux, uy hold fluid-node moments. */
static void phi_field(const orc_params* p, const uint8_t* mask, const double* rho,
                      const double* ux, const double* uy, double* phi /* [2][ny][nx] */) {
    const size_t n = (size_t)p->nx * p->ny;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t k = node(p, x, y);
            int c = cls(mask, p, x, y);
            if (colliding(c)) {
                phi[k] = rho[k] * ux[k] * ux[k] * ux[k];
                phi[n + k] = rho[k] * uy[k] * uy[k] * uy[k];
            } else if (c == ORC_INLET) {
                phi[k] = p->wall_rho * p->wall_ux * p->wall_ux * p->wall_ux;
                phi[n + k] = p->wall_rho * p->wall_uy * p->wall_uy * p->wall_uy;
            } else {
                phi[k] = 0.0;
                phi[n + k] = 0.0;
            }
        }
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x)
            if (cls(mask, p, x, y) == ORC_OUTLET) {
                int xs = x - 1, ys = y;
                wrap(p, &xs, &ys);
                phi[node(p, x, y)] = phi[node(p, xs, ys)];
                phi[n + node(p, x, y)] = phi[n + node(p, xs, ys)];
            }
}

/* Phi component c at (x, y); 0 outside a non-periodic edge (reading R2). */
static double phi_at(const orc_params* p, const double* phi, int c, int x, int y) {
    if (!wrap(p, &x, &y)) return 0.0;
    return phi[(size_t)c * p->nx * p->ny + node(p, x, y)];
}

/* Phi component c at the neighbour (xn, yn) of node (x, y): beyond the edge
 * next to a pressure outlet node it is that node's own value (reading R15). */
static double phi_nb(const orc_params* p, const uint8_t* mask, const double* phi, int c, int x,
                     int y, int xn, int yn) {
    int xw = xn, yw = yn;
    if (!wrap(p, &xw, &yw) && xn == p->nx && cls(mask, p, x, y) == ORC_PRESSURE)
        return phi_at(p, phi, c, x, y);
    return phi_at(p, phi, c, xn, yn);
}

/* Moments (eq11) of every fluid node; non-fluid nodes get rho = u = 0. */
void orc_moments(const orc_params* p, const uint8_t* mask, const double* f, double* rho,
                 double* ux, double* uy) {
    const size_t n = (size_t)p->nx * p->ny;
    const double g[ND] = {p->gx, p->gy};
    for (size_t k = 0; k < n; ++k) {
        if (mask && !colliding(mask[k])) {
            rho[k] = ux[k] = uy[k] = 0.0;
            continue;
        }
        double fk[NQ], r, u[ND];
        for (int i = 0; i < NQ; ++i) fk[i] = f[(size_t)i * n + k];
        orc_macroscopic(fk, g, &r, u);
        rho[k] = r;
        ux[k] = u[0];
        uy[k] = u[1];
    }
}

/* Phi field (eq_Gi, reading R2) of the state f. */
void orc_phi_of_state(const orc_params* p, const uint8_t* mask, const double* f, double* phi) {
    const size_t n = (size_t)p->nx * p->ny;
    double* m = (double*)malloc(3 * n * sizeof(double));
    orc_moments(p, mask, f, m, m + n, m + 2 * n);
    phi_field(p, mask, m, m + n, m + 2 * n, phi);
    free(m);
}

/* Initial populations (reading R4) from rho, u on fluid nodes, and the
 * initial Phi (Phi^{-1} := Phi^0, reading R1).  rho may be NULL (then 1).
 * Non-fluid entries of f are set to 0. */
int orc_init(const orc_params* p, const uint8_t* mask, const double* rho, const double* ux,
             const double* uy, double* f, double* phi) {
    if (orc_check_mask(p, mask)) return 1;
    const size_t n = (size_t)p->nx * p->ny;
    double* r = (double*)malloc(n * sizeof(double));
    for (size_t k = 0; k < n; ++k) {
        r[k] = rho ? rho[k] : 1.0;
        if (mask && !colliding(mask[k])) {
            for (int i = 0; i < NQ; ++i) f[(size_t)i * n + k] = 0.0;
            continue;
        }
        double u[ND] = {ux[k], uy[k]}, F[ND] = {r[k] * p->gx, r[k] * p->gy}, feq[NQ];
        orc_equilibrium(r[k], u, feq);
        for (int i = 0; i < NQ; ++i) {
            double eF = 0.0;
            for (int a = 0; a < ND; ++a) eF += herm1(i, a) * F[a];
            f[(size_t)i * n + k] = feq[i] - 0.5 * WV[i] * eF / CS2;
        }
    }
    zou_he_outlet(p, mask, f);
    if (phi) phi_field(p, mask, r, ux, uy, phi);
    free(r);
    return 0;
}

/* Advances f by nsteps steps of eq2.  phi holds Phi of the previous step
 * (LAGGED mode; updated in place); it is ignored by CURRENT and OFF and may
 * then be NULL.  Returns 0 on success. */
int orc_step(const orc_params* p, const uint8_t* mask, double* f, double* phi, int nsteps) {
    if (orc_check_mask(p, mask)) return 1;
    if (p->g_mode == ORC_G_LAGGED && !phi) return 2;
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    double* fstar = (double*)calloc((size_t)NQ * n, sizeof(double));
    double* fnew = (double*)calloc((size_t)NQ * n, sizeof(double));
    double* mom = (double*)malloc(3 * n * sizeof(double));
    double* phi_t = (double*)malloc(2 * n * sizeof(double));
    if (!fstar || !fnew || !mom || !phi_t) {
        free(fstar); free(fnew); free(mom); free(phi_t);
        return 3;
    }
    double *rho = mom, *ux = mom + n, *uy = mom + 2 * n;

    for (int s = 0; s < nsteps; ++s) {
        /* 0. pressure outlet populations of the state at time t (R15) */
        zou_he_outlet(p, mask, f);
        /* 1. macroscopic fields at time t (eq11) */
        orc_moments(p, mask, f, rho, ux, uy);
        /* 2. Phi at time t (eq_Gi, reading R2) */
        phi_field(p, mask, rho, ux, uy, phi_t);
        const double* phi_use =
            p->g_mode == ORC_G_CURRENT ? phi_t : (p->g_mode == ORC_G_LAGGED ? phi : NULL);

        /* 3. collision of every fluid node: right-hand side of eq2 */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = node(p, x, y);
                if (!colliding(cls(mask, p, x, y))) continue;
                double fk[NQ], fs[NQ], dphi[ND * ND];
                for (int i = 0; i < NQ; ++i) fk[i] = f[(size_t)i * n + k];
                /* d_gamma Phi_{a b gamma}: Phi_{a b gamma} is rho u_a^3 when
                 * a = b = gamma and 0 otherwise; d_gamma by central
                 * differences (reading R1). */
                for (int a = 0; a < ND; ++a)
                    for (int b = 0; b < ND; ++b) {
                        double d = 0.0;
                        if (phi_use)
                            for (int c = 0; c < ND; ++c) {
                                if (!(a == b && b == c)) continue;
                                int xp = x + (c == 0), yp = y + (c == 1);
                                int xm = x - (c == 0), ym = y - (c == 1);
                                d += 0.5 * (phi_nb(p, mask, phi_use, c, x, y, xp, yp) -
                                            phi_nb(p, mask, phi_use, c, x, y, xm, ym));
                            }
                        dphi[a * ND + b] = d;
                    }
                orc_collide_node(p, fk, dphi, fs, NULL, NULL, NULL, NULL, NULL);
                for (int i = 0; i < NQ; ++i) fstar[(size_t)i * n + k] = fs[i];
            }

        /* 4. streaming, left-hand side of eq2 in push form, with half-way
         * bounce-back (eq_a20), the moving-wall correction and outlet ghosts
         * (reading R11). */
        for (size_t q = 0; q < (size_t)NQ * n; ++q) fnew[q] = 0.0;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c0 = cls(mask, p, x, y);
                if (!colliding(c0) && c0 != ORC_OUTLET) continue;
                size_t k = node(p, x, y), ksrc = k;
                if (c0 == ORC_OUTLET) {
                    int xs = x - 1, ys = y;
                    wrap(p, &xs, &ys);
                    ksrc = node(p, xs, ys);
                }
                for (int i = 0; i < NQ; ++i) {
                    double fs = fstar[(size_t)i * n + ksrc];
                    int xt = x + EV[i][0], yt = y + EV[i][1];
                    int inside = wrap(p, &xt, &yt);
                    /* a pressure outlet's links across the edge are open */
                    if (!inside && c0 == ORC_PRESSURE && EV[i][0] == 1) continue;
                    int ct = inside ? cls(mask, p, xt, yt) : ORC_SOLID;
                    if (colliding(ct)) {
                        fnew[(size_t)i * n + node(p, xt, yt)] = fs;
                    } else if (colliding(c0) && ct == ORC_SOLID) {
                        fnew[(size_t)opposite(i) * n + k] = fs;
                    } else if (colliding(c0) && ct == ORC_INLET) {
                        double eu = EV[i][0] * p->wall_ux + EV[i][1] * p->wall_uy;
                        fnew[(size_t)opposite(i) * n + k] =
                            fs - 2.0 * WV[i] * p->wall_rho * eu / CS2;
                    }
                    /* links ending in an outlet ghost, and any link leaving a
                     * ghost that does not end in a fluid node, are dropped */
                }
            }
        memcpy(f, fnew, (size_t)NQ * n * sizeof(double));
        zou_he_outlet(p, mask, f);
        /* 5. LAGGED: Phi^t becomes the previous level of the next step */
        if (p->g_mode == ORC_G_LAGGED) memcpy(phi, phi_t, 2 * n * sizeof(double));
    }
    free(fstar);
    free(fnew);
    free(mom);
    free(phi_t);
    return 0;
}

/* ---- diagnostics -------------------------------------------------------- */

/* Relative L2 error of eq_n1: sqrt(sum (qn - qa)^2 / sum qa^2). */
double orc_l2(const double* qn, const double* qa, int64_t n) {
    double num = 0.0, den = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double d = qn[k] - qa[k];
        num += d * d;
        den += qa[k] * qa[k];
    }
    return sqrt(num / den);
}

/* Largest local change of eq_n2's steady-state test, before the division by
 * the characteristic speed: max over colliding nodes of |u - u_ref|. */
double orc_max_change(const orc_params* p, const uint8_t* mask, const double* ux, const double* uy,
                      const double* rx, const double* ry) {
    const size_t n = (size_t)p->nx * p->ny;
    double m = 0.0;
    for (size_t k = 0; k < n; ++k) {
        if (mask && !colliding(mask[k])) continue;
        const double dx = ux[k] - rx[k], dy = uy[k] - ry[k];
        const double d = sqrt(dx * dx + dy * dy);
        if (d > m) m = d;
    }
    return m;
}

/* Vorticity omega = d_x u_y - d_y u_x by second-order central differences on
 * the node lattice (reading R18), at colliding nodes whose four axis
 * neighbours are colliding nodes of the domain (wrapped across periodic
 * edges); there valid[k] = 1, elsewhere valid[k] = 0 and w[k] = 0. */
void orc_vorticity(const orc_params* p, const uint8_t* mask, const double* ux, const double* uy,
                   double* w, uint8_t* valid) {
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const size_t k = node(p, x, y);
            w[k] = 0.0;
            valid[k] = 0;
            if (!colliding(cls(mask, p, x, y))) continue;
            int xp = x + 1, yp = y, xm = x - 1, ym = y, xs = x, ysp = y + 1, xs2 = x, ysm = y - 1;
            if (!wrap(p, &xp, &yp) || !wrap(p, &xm, &ym) || !wrap(p, &xs, &ysp) || !wrap(p, &xs2, &ysm))
                continue;
            if (!colliding(cls(mask, p, xp, yp)) || !colliding(cls(mask, p, xm, ym)) ||
                !colliding(cls(mask, p, xs, ysp)) || !colliding(cls(mask, p, xs2, ysm)))
                continue;
            const double duy_dx = 0.5 * (uy[node(p, xp, yp)] - uy[node(p, xm, ym)]);
            const double dux_dy = 0.5 * (ux[node(p, xs, ysp)] - ux[node(p, xs2, ysm)]);
            w[k] = duy_dx - dux_dy;
            valid[k] = 1;
        }
}

/* Momentum-exchange force on the walls (solid class-1 nodes and the
 * stationary walls outside non-periodic edges), Sec. III D:
 * F = sum over wall links of e_i [f*_ibar(x_s) + f*_i(x_f)].  Under half-way
 * bounce-back the population returned by the wall, f*_ibar(x_s), is the
 * reflected one, which the state after the step holds as f_ibar(x_f, t+1) =
 * f*_i(x_f, t) (reading R12), so each link contributes 2 e_i f_ibar(x_f).
 * f is the state after the step.  Writes force[2]. */
void orc_drag(const orc_params* p, const uint8_t* mask, const double* f, double* force) {
    const size_t n = (size_t)p->nx * p->ny;
    force[0] = force[1] = 0.0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const int c = cls(mask, p, x, y);
            if (!colliding(c)) continue;
            for (int i = 1; i < NQ; ++i) {
                int xt = x + EV[i][0], yt = y + EV[i][1];
                const int inside = wrap(p, &xt, &yt);
                if (inside && cls(mask, p, xt, yt) != ORC_SOLID) continue;
                if (!inside && c == ORC_PRESSURE && EV[i][0] == 1) continue;  /* open (R15) */
                double fr = f[(size_t)opposite(i) * n + node(p, x, y)];
                force[0] += 2.0 * EV[i][0] * fr;
                force[1] += 2.0 * EV[i][1] * fr;
            }
        }
}
