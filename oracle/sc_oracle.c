/*
 * sc_oracle.c -- plain, slow FP64 CPU oracle of the two-component Shan-Chen
 * D3Q19 lattice Boltzmann step with wall adhesion and half-way bounce-back.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: the lattice, the voxeliser and the measurements are written out here
 * a second time, from the paper's equations, in double precision, one cell at a
 * time, in the order the method states them.
 *
 * Passages followed (paper: Montella, Yuan, Chareyre, Gens, "A hybrid multiphase
 * model based on lattice Boltzmann method direct simulations"):
 *   Eq. 1   lattice Boltzmann equation, BGK collision + streaming (Sec. 2.1)
 *   Eqs. 2-3 moments rho = sum f, rho u = sum f e                  (Sec. 2.1)
 *   Eq. 4   Shan-Chen inter-component force                        (Sec. 2.1)
 *   Eq. 5   non-ideal equation of state p = cs2 (r1+r2) + cs2 G r1 r2 (Sec. 2.1)
 *   Sec. 2.2.2  throat domain = triangular prism through the sphere centres,
 *               inlet/outlet densities adjusted to raise p_c, p_c^e = max p_c.
 * Readings taken where the paper is silent or garbled (each is listed in the
 * design notes):
 *   - Eq. 4 is read with psi = rho and the D3Q19 weights w_k inside the sum,
 *     G_12 = G_21 = G, no self-interaction.
 *   - the force enters through the velocity shift of Shan & Chen (1993), the
 *     paper's cited model: common velocity u' = sum(j/tau)/sum(rho/tau),
 *     u_eq = u' + tau F / rho.
 *   - wall adhesion F_ads = -G_ads rho(x) sum_k w_k s(x+e_k) e_k, s = 1 on
 *     adhesive (grain) solid cells; solid cells carry rho = 0 in the cohesion sum.
 *   - walls are half-way bounce-back; cells beyond a non-periodic box edge are
 *     neutral (non-adhesive) solid.
 *   - reservoir layers: after collision their populations are replaced by the
 *     rest equilibrium of the imposed densities.
 *   - membrane cells are fluid for the wetting component and solid for the
 *     non-wetting one.
 *
 * Memory layout: f[s][k][cell], cell = (z*ny + y)*nx + x, s = 0 wetting,
 * s = 1 non-wetting.  Masks are uint8 with the bits below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OQ 19
#define M_SOLID 1u
#define M_ADHESIVE 2u
#define M_MEMBRANE 4u
#define M_INLET 8u
#define M_OUTLET 16u

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    double tau[2];
    double G;
    double G_ads[2];
    double g[3];           /* body-force acceleration: F_body = rho_s * g   */
    double rho_in[2];      /* (w, nw) densities imposed on inlet cells      */
    double rho_out[2];     /* (w, nw) densities imposed on outlet cells     */
} orc_params;

typedef struct {
    double mass[2];
    double p_w, p_nw, p_c;
    double p_in, p_out, p_c_res;
    double S_w;
    long long n_fluid, n_w, n_interface, n_bulk_w, n_bulk_nw, n_in, n_out;
    long long n_nonfinite, n_negative;
} orc_measurement;

/* ---------------------------------------------------------------- lattice */
/* D3Q19: the rest velocity, the 6 face neighbours, the 12 edge neighbours.
 * The paper names the model (Sec. 2.1) but not its weights; these are the
 * standard ones with cs^2 = 1/3. */
static const int OE[OQ][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight(int k) {
    int n2 = OE[k][0] * OE[k][0] + OE[k][1] * OE[k][1] + OE[k][2] * OE[k][2];
    if (n2 == 0) return 1.0 / 3.0;
    if (n2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* opposite direction found by search, not by a table */
static int opposite_search(int k) {
    for (int j = 0; j < OQ; ++j)
        if (OE[j][0] == -OE[k][0] && OE[j][1] == -OE[k][1] && OE[j][2] == -OE[k][2]) return j;
    return -1;
}

/* memo of weight() and opposite_search(), filled on first use */
static double W_[OQ];
static int OPP_[OQ];
static int tables_ready = 0;
static void tables(void) {
    if (tables_ready) return;
    for (int k = 0; k < OQ; ++k) { W_[k] = weight(k); OPP_[k] = opposite_search(k); }
    tables_ready = 1;
}
static int opposite(int k) { return OPP_[k]; }

void orc_lattice(int* e_out, double* w_out, int* opp_out) {
    for (int k = 0; k < OQ; ++k) {
        for (int d = 0; d < 3; ++d) e_out[3 * k + d] = OE[k][d];
        w_out[k] = weight(k);
        opp_out[k] = opposite_search(k);
    }
}

/* second-order equilibrium f_k^eq(rho, u) = w_k rho (1 + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u) */
void orc_equilibrium(double rho, const double* u, double* feq) {
    tables();
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < OQ; ++k) {
        double eu = OE[k][0] * u[0] + OE[k][1] * u[1] + OE[k][2] * u[2];
        feq[k] = W_[k] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* ----------------------------------------------------------- cell helpers */
static long long cell_index(const orc_params* p, int x, int y, int z) {
    return ((long long)z * p->ny + y) * p->nx + x;
}

/* Neighbour lookup with periodic wrap. Returns -1 when the neighbour lies
 * beyond a non-periodic edge of the box. */
static long long neighbour(const orc_params* p, int x, int y, int z, int dx, int dy, int dz) {
    int c[3] = {x + dx, y + dy, z + dz};
    int n[3] = {p->nx, p->ny, p->nz};
    if (c[0] >= 0 && c[0] < n[0] && c[1] >= 0 && c[1] < n[1] && c[2] >= 0 && c[2] < n[2])
        return cell_index(p, c[0], c[1], c[2]);
    for (int d = 0; d < 3; ++d) {
        if (c[d] < 0 || c[d] >= n[d]) {
            if (!p->periodic[d]) return -1;
            c[d] = ((c[d] % n[d]) + n[d]) % n[d];
        }
    }
    return cell_index(p, c[0], c[1], c[2]);
}

/* fluid for component s: not solid, and for the non-wetting one not membrane */
static int fluid_for(uint8_t m, int s) {
    if (m & M_SOLID) return 0;
    if (s == 1 && (m & M_MEMBRANE)) return 0;
    return 1;
}

static int adhesive_solid(uint8_t m) { return (m & M_SOLID) && (m & M_ADHESIVE); }

/* ------------------------------------------------------------ init, moments */
/* f = f^eq(rho0, 0) on cells where the component is fluid, 0 elsewhere */
void orc_init(const orc_params* p, const uint8_t* mask, const double* rho0, double* f) {
    tables();
    long long N = (long long)p->nx * p->ny * p->nz;
    double zero[3] = {0, 0, 0}, feq[OQ];
    for (int s = 0; s < 2; ++s)
        for (long long c = 0; c < N; ++c) {
            int fl = fluid_for(mask[c], s);
            orc_equilibrium(fl ? rho0[s * N + c] : 0.0, zero, feq);
            for (int k = 0; k < OQ; ++k) f[((long long)s * OQ + k) * N + c] = fl ? feq[k] : 0.0;
        }
}

/* Eq. 2: rho_s = sum_k f_k^s (0 where the component is not fluid) */
void orc_density(const orc_params* p, const uint8_t* mask, const double* f, double* rho) {
    long long N = (long long)p->nx * p->ny * p->nz;
    for (int s = 0; s < 2; ++s)
#pragma omp parallel for schedule(static)
        for (long long c = 0; c < N; ++c) {
            double r = 0.0;
            if (fluid_for(mask[c], s))
                for (int k = 0; k < OQ; ++k) r += f[((long long)s * OQ + k) * N + c];
            rho[s * N + c] = r;
        }
}

/* Eq. 4 (cohesion, psi = rho, weights w_k), adhesion and body force, per
 * component, at every cell where the component is fluid. F[s][d][cell]. */
void orc_force(const orc_params* p, const uint8_t* mask, const double* rho, double* F) {
    tables();
    long long N = (long long)p->nx * p->ny * p->nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long long c = cell_index(p, x, y, z);
                for (int s = 0; s < 2; ++s) {
                    int sb = 1 - s;
                    double coh[3] = {0, 0, 0}, adh[3] = {0, 0, 0};
                    if (fluid_for(mask[c], s)) {
                        for (int k = 1; k < OQ; ++k) {
                            long long nb = neighbour(p, x, y, z, OE[k][0], OE[k][1], OE[k][2]);
                            double rb = 0.0, sol = 0.0;
                            if (nb >= 0) {
                                rb = fluid_for(mask[nb], sb) ? rho[sb * N + nb] : 0.0;
                                sol = adhesive_solid(mask[nb]) ? 1.0 : 0.0;
                            }
                            for (int d = 0; d < 3; ++d) {
                                coh[d] += W_[k] * rb * OE[k][d];
                                adh[d] += W_[k] * sol * OE[k][d];
                            }
                        }
                    }
                    double rs = fluid_for(mask[c], s) ? rho[s * N + c] : 0.0;
                    for (int d = 0; d < 3; ++d) {
                        double fc = -p->G * rs * coh[d];
                        double fa = -p->G_ads[s] * rs * adh[d];
                        double fb = rs * p->g[d];
                        F[((long long)s * 3 + d) * N + c] = fc + fa + fb;
                    }
                }
            }
}

/* ---------------------------------------------------------------- the step */
/* One time step on the pre-collision state f(t) -> f(t+1), in the order:
 * moments (Eqs. 2-3), force (Eq. 4 + adhesion + body), common velocity and
 * velocity shift, BGK collision towards f^eq (Eq. 1 right-hand side),
 * reservoir override, pull streaming with half-way bounce-back (Eq. 1
 * left-hand side).  fpost is scratch of the same size as f. */
static void one_step(const orc_params* p, const uint8_t* mask, double* f, double* fpost,
                     double* rho, double* F) {
    long long N = (long long)p->nx * p->ny * p->nz;
    orc_density(p, mask, f, rho);
    orc_force(p, mask, rho, F);

    /* collision */
#pragma omp parallel for schedule(static)
    for (long long c = 0; c < N; ++c) {
        double j[2][3], rs[2];
        int fl[2];
        double fc[2][OQ];
        for (int s = 0; s < 2; ++s) {
            fl[s] = fluid_for(mask[c], s);
            rs[s] = rho[s * N + c];
            for (int k = 0; k < OQ; ++k) fc[s][k] = f[((long long)s * OQ + k) * N + c];
            /* Eq. 3: j_s = sum_k f_k e_k */
            for (int d = 0; d < 3; ++d) {
                double acc = 0.0;
                if (fl[s])
                    for (int k = 0; k < OQ; ++k) acc += fc[s][k] * OE[k][d];
                j[s][d] = acc;
            }
        }
        /* common velocity u' = (sum_s j_s / tau_s) / (sum_s rho_s / tau_s) */
        double num[3] = {0, 0, 0}, den = 0.0, up[3] = {0, 0, 0};
        for (int s = 0; s < 2; ++s) {
            if (!fl[s]) continue;
            for (int d = 0; d < 3; ++d) num[d] += j[s][d] / p->tau[s];
            den += rs[s] / p->tau[s];
        }
        if (den != 0.0)
            for (int d = 0; d < 3; ++d) up[d] = num[d] / den;

        for (int s = 0; s < 2; ++s) {
            if (!fl[s]) {
                for (int k = 0; k < OQ; ++k) fpost[((long long)s * OQ + k) * N + c] = 0.0;
                continue;
            }
            double ueq[3], feq[OQ];
            for (int d = 0; d < 3; ++d) {
                double shift = 0.0;
                if (rs[s] != 0.0) shift = p->tau[s] * F[((long long)s * 3 + d) * N + c] / rs[s];
                ueq[d] = up[d] + shift;
            }
            if (mask[c] & (M_INLET | M_OUTLET)) {
                /* reservoir layer: rest equilibrium of the imposed density */
                double zero[3] = {0, 0, 0};
                double rr = (mask[c] & M_INLET) ? p->rho_in[s] : p->rho_out[s];
                orc_equilibrium(rr, zero, feq);
                for (int k = 0; k < OQ; ++k) fpost[((long long)s * OQ + k) * N + c] = feq[k];
                continue;
            }
            orc_equilibrium(rs[s], ueq, feq);
            for (int k = 0; k < OQ; ++k) {
                double fk = fc[s][k];
                fpost[((long long)s * OQ + k) * N + c] = fk - (fk - feq[k]) / p->tau[s];
            }
        }
    }

    /* pull streaming with half-way bounce-back */
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long long c = cell_index(p, x, y, z);
                for (int s = 0; s < 2; ++s) {
                    if (!fluid_for(mask[c], s)) continue;
                    for (int k = 0; k < OQ; ++k) {
                        long long src = neighbour(p, x, y, z, -OE[k][0], -OE[k][1], -OE[k][2]);
                        double v;
                        if (src >= 0 && fluid_for(mask[src], s))
                            v = fpost[((long long)s * OQ + k) * N + src];
                        else
                            v = fpost[((long long)s * OQ + opposite(k)) * N + c];
                        f[((long long)s * OQ + k) * N + c] = v;
                    }
                }
            }
}

/* Advance nsteps time steps in place. Returns 0, or -1 on allocation failure. */
int orc_step(const orc_params* p, const uint8_t* mask, double* f, int nsteps) {
    tables();
    long long N = (long long)p->nx * p->ny * p->nz;
    double* fpost = (double*)calloc((size_t)(2 * OQ * N), sizeof(double));
    double* rho = (double*)calloc((size_t)(2 * N), sizeof(double));
    double* F = (double*)calloc((size_t)(6 * N), sizeof(double));
    if (!fpost || !rho || !F) {
        free(fpost); free(rho); free(F);
        return -1;
    }
    for (int t = 0; t < nsteps; ++t) one_step(p, mask, f, fpost, rho, F);
    free(fpost); free(rho); free(F);
    return 0;
}

/* ------------------------------------------------------------ measurement */
typedef struct { double s, c; } kahan;
static void kadd(kahan* k, double v) {
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* Eq. 5 pressure */
static double eos_pressure(const orc_params* p, double rw, double rn) {
    return (rw + rn) / 3.0 + p->G * rw * rn / 3.0;
}

/* Observables of the pre-collision state f(t):
 *   mass per component over cells where it is fluid (reservoirs included);
 *   interior fluid = not solid, not membrane, not a reservoir layer;
 *   S_w = #(interior, rho_w > rho_nw) / #interior   (a tie counts as nw);
 *   interface cells: |phi| < 0.5, phi = (rho_w - rho_nw)/(rho_w + rho_nw);
 *   bulk phase pressures: Eq. 5 averaged over phi > 0.9 (w) and phi < -0.9 (nw);
 *   p_c = p_nw - p_w, p_c_res = mean p(inlet) - mean p(outlet).
 * Sums are compensated (Kahan) in cell order. */
void orc_measure(const orc_params* p, const uint8_t* mask, const double* f, orc_measurement* out) {
    tables();
    long long N = (long long)p->nx * p->ny * p->nz;
    double* rho = (double*)calloc((size_t)(2 * N), sizeof(double));
    memset(out, 0, sizeof(*out));
    if (!rho) return;
    orc_density(p, mask, f, rho);
    kahan mass[2] = {{0, 0}, {0, 0}}, pw = {0, 0}, pn = {0, 0}, pin = {0, 0}, pout = {0, 0};
    for (long long c = 0; c < N; ++c) {
        uint8_t m = mask[c];
        double rw = rho[c], rn = rho[N + c];
        for (int s = 0; s < 2; ++s) {
            if (!fluid_for(m, s)) continue;
            double r = rho[s * N + c];
            kadd(&mass[s], r);
            if (!isfinite(r)) out->n_nonfinite++;
            else if (r < 0.0) out->n_negative++;
        }
        if (m & M_SOLID) continue;
        if (m & M_INLET) { kadd(&pin, eos_pressure(p, rw, rn)); out->n_in++; continue; }
        if (m & M_OUTLET) { kadd(&pout, eos_pressure(p, rw, rn)); out->n_out++; continue; }
        if (m & M_MEMBRANE) continue;
        out->n_fluid++;
        if (rw > rn) out->n_w++;
        double phi = (rw - rn) / (rw + rn);
        if (fabs(phi) < 0.5) out->n_interface++;
        if (phi > 0.9) { kadd(&pw, eos_pressure(p, rw, rn)); out->n_bulk_w++; }
        if (phi < -0.9) { kadd(&pn, eos_pressure(p, rw, rn)); out->n_bulk_nw++; }
    }
    out->mass[0] = mass[0].s;
    out->mass[1] = mass[1].s;
    out->p_w = out->n_bulk_w ? pw.s / (double)out->n_bulk_w : NAN;
    out->p_nw = out->n_bulk_nw ? pn.s / (double)out->n_bulk_nw : NAN;
    out->p_c = out->p_nw - out->p_w;
    out->p_in = out->n_in ? pin.s / (double)out->n_in : NAN;
    out->p_out = out->n_out ? pout.s / (double)out->n_out : NAN;
    out->p_c_res = out->p_in - out->p_out;
    out->S_w = out->n_fluid ? (double)out->n_w / (double)out->n_fluid : NAN;
    free(rho);
}

/* Physical velocity of the mixture, u = (sum_s j_s + F_total/2) / sum_s rho_s,
 * per cell, for the channel-flow check. */
void orc_velocity(const orc_params* p, const uint8_t* mask, const double* f, double* u) {
    tables();
    long long N = (long long)p->nx * p->ny * p->nz;
    double* rho = (double*)calloc((size_t)(2 * N), sizeof(double));
    double* F = (double*)calloc((size_t)(6 * N), sizeof(double));
    if (!rho || !F) { free(rho); free(F); return; }
    orc_density(p, mask, f, rho);
    orc_force(p, mask, rho, F);
    for (long long c = 0; c < N; ++c) {
        double rt = 0.0, m[3] = {0, 0, 0};
        for (int s = 0; s < 2; ++s) {
            if (!fluid_for(mask[c], s)) continue;
            rt += rho[s * N + c];
            for (int k = 0; k < OQ; ++k)
                for (int d = 0; d < 3; ++d) m[d] += f[((long long)s * OQ + k) * N + c] * OE[k][d];
            for (int d = 0; d < 3; ++d) m[d] += 0.5 * F[((long long)s * 3 + d) * N + c];
        }
        for (int d = 0; d < 3; ++d) u[(long long)d * N + c] = rt != 0.0 ? m[d] / rt : 0.0;
    }
    free(rho); free(F);
}

/* -------------------------------------------------------------- geometry */
/* Cell (i,j,k) has its centre at (i,j,k) in lattice units.  A cell is
 * grain solid when its centre lies within a sphere, |x - c| <= r, tested as
 * dx*dx + dy*dy + dz*dz <= r*r summed left to right. */
static int in_sphere(double px, double py, double pz, const double* sph) {
    double dx = px - sph[0];
    double dy = py - sph[1];
    double dz = pz - sph[2];
    double d2 = dx * dx + dy * dy + dz * dz;
    return d2 <= sph[3] * sph[3];
}

static void vsub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double vdot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void vcross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Prism test for a throat of three sphere centres c0, c1, c2 (Sec. 2.2.2):
 * the three walls are orthogonal to the plane of the centres and each passes
 * through two centres.  A point is inside when it lies on the inner side of all
 * three walls (on a wall counts as inside). */
static int in_prism(const double* pt, const double* c0, const double* c1, const double* c2) {
    const double* c[3] = {c0, c1, c2};
    double a[3], b[3], nrm[3];
    vsub(c1, c0, a);
    vsub(c2, c0, b);
    vcross(a, b, nrm);
    for (int i = 0; i < 3; ++i) {
        const double* p0 = c[i];
        const double* p1 = c[(i + 1) % 3];
        double edge[3], inward[3], rel[3];
        vsub(p1, p0, edge);
        vcross(nrm, edge, inward);
        vsub(pt, p0, rel);
        if (vdot(rel, inward) < 0.0) return 0;
    }
    return 1;
}

/* Box-frame voxeliser.  spheres: n x (cx, cy, cz, r).  flags: bit 0 = clip to
 * the prism of the first three spheres (outside -> neutral solid); bit 1 =
 * reservoir layers at z = 0 (inlet) and z = nz-1 (outlet); membrane_layers > 0
 * marks that many fluid layers just above the outlet layer as membrane. */
void orc_voxelise(int nx, int ny, int nz, const double* spheres, int n_spheres, int flags,
                  int membrane_layers, uint8_t* mask) {
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                long long c = ((long long)z * ny + y) * nx + x;
                uint8_t m = 0;
                double pt[3] = {(double)x, (double)y, (double)z};
                for (int i = 0; i < n_spheres; ++i)
                    if (in_sphere(pt[0], pt[1], pt[2], spheres + 4 * i)) { m = M_SOLID | M_ADHESIVE; break; }
                if (!m && (flags & 1) && n_spheres >= 3)
                    if (!in_prism(pt, spheres, spheres + 4, spheres + 8)) m = M_SOLID;
                if (!m && (flags & 2)) {
                    if (z == 0) m = M_INLET;
                    else if (z == nz - 1) m = M_OUTLET;
                    else if (z >= nz - 1 - membrane_layers) m = M_MEMBRANE;
                }
                mask[c] = m;
            }
}

/* Throat frame (Sec. 2.2.2 domain, fitted box): for centres c0, c1, c2
 *   e1 = (c1 - c0)/|c1 - c0|, e3 = (c1 - c0) x (c2 - c0) normalised, e2 = e3 x e1;
 * local coordinates of a point q are ((q-c0).e1, (q-c0).e2, (q-c0).e3).
 * The box spans floor(min) .. ceil(max) of the local x and y of the centres and
 * z in [-ceil(H), ceil(H)], H the largest radius.  Cell (i,j,k) sits at local
 * (x0 + i, y0 + j, z0 + k).  dims_out = (nx, ny, nz), origin_out = (x0, y0, z0),
 * local_out = 3 x 4 local sphere records (x, y, z, r). */
void orc_throat_frame(const double* spheres3, int* dims_out, double* origin_out, double* local_out) {
    const double* c0 = spheres3;
    const double* c1 = spheres3 + 4;
    const double* c2 = spheres3 + 8;
    double a[3], b[3], e1[3], e2[3], e3[3], n3[3];
    vsub(c1, c0, a);
    vsub(c2, c0, b);
    double la = sqrt(vdot(a, a));
    for (int d = 0; d < 3; ++d) e1[d] = a[d] / la;
    vcross(a, b, n3);
    double ln = sqrt(vdot(n3, n3));
    for (int d = 0; d < 3; ++d) e3[d] = n3[d] / ln;
    vcross(e3, e1, e2);
    double H = 0.0;
    double lx[3], ly[3];
    for (int i = 0; i < 3; ++i) {
        const double* ci = spheres3 + 4 * i;
        double rel[3];
        vsub(ci, c0, rel);
        lx[i] = vdot(rel, e1);
        ly[i] = vdot(rel, e2);
        local_out[4 * i + 0] = lx[i];
        local_out[4 * i + 1] = ly[i];
        local_out[4 * i + 2] = vdot(rel, e3);
        local_out[4 * i + 3] = ci[3];
        if (ci[3] > H) H = ci[3];
    }
    double xmin = lx[0], xmax = lx[0], ymin = ly[0], ymax = ly[0];
    for (int i = 1; i < 3; ++i) {
        if (lx[i] < xmin) xmin = lx[i];
        if (lx[i] > xmax) xmax = lx[i];
        if (ly[i] < ymin) ymin = ly[i];
        if (ly[i] > ymax) ymax = ly[i];
    }
    double x0 = floor(xmin), y0 = floor(ymin), hz = ceil(H);
    dims_out[0] = (int)(ceil(xmax) - x0) + 1;
    dims_out[1] = (int)(ceil(ymax) - y0) + 1;
    dims_out[2] = 2 * (int)hz + 1;
    origin_out[0] = x0;
    origin_out[1] = y0;
    origin_out[2] = -hz;
}

/* Throat-box voxeliser: grain solid inside the spheres, neutral solid outside
 * the prism, inlet layer at k = 0 and outlet layer at k = nz-1. */
void orc_voxelise_throat(const double* spheres3, uint8_t* mask) {
    int dims[3];
    double org[3], loc[12];
    orc_throat_frame(spheres3, dims, org, loc);
    for (int k = 0; k < dims[2]; ++k)
        for (int j = 0; j < dims[1]; ++j)
            for (int i = 0; i < dims[0]; ++i) {
                long long c = ((long long)k * dims[1] + j) * dims[0] + i;
                double pt[3] = {org[0] + (double)i, org[1] + (double)j, org[2] + (double)k};
                uint8_t m = 0;
                for (int s = 0; s < 3; ++s)
                    if (in_sphere(pt[0], pt[1], pt[2], loc + 4 * s)) { m = M_SOLID | M_ADHESIVE; break; }
                if (!m && !in_prism(pt, loc, loc + 4, loc + 8)) m = M_SOLID;
                if (!m) {
                    if (k == 0) m = M_INLET;
                    else if (k == dims[2] - 1) m = M_OUTLET;
                }
                mask[c] = m;
            }
}
