/*
 * lbref.c -- FP64 CPU oracle (test infrastructure; see lbref.h).
 *
 * One time step follows the paper in this order:
 *   1. remap particles onto the lattice: covered nodes lose their fluid to
 *      the particle, uncovered nodes are refilled (Sec. III, Sec. IV:
 *      Eqs. eqn_rho_neu, eqn_ladd_vernichtenunderzeugen, masscorr);
 *   2. densities; shell nodes get the virtual fluid density plus colour
 *      (Sec. IV, Eqs. for rho_new^r / rho_new^b); Psi (Eq. eqn_ref_dens);
 *   3. Shan-Chen force on fluid and shell nodes (Eq. eqn_shan-chen-F);
 *   4. Shan-Chen force of the shell nodes onto the particle
 *      (Eq. eqn_shan_chen_particle);
 *   5. BGK collision with the cubic equilibrium (Eqs. eq:boltz, Equil) at
 *      the velocity shifted by tau F / rho;
 *   6. streaming with moving-wall bounce-back and momentum exchange
 *      (Eqs. eqn_bounce-back, eqn_ladd_bewegtewand);
 *   7. particle MD: Hertz contact (Eq. eq:hertz), lubrication
 *      (Eq. eqn_ladd_lubrikation), leap-frog for U, omega, X (or, with
 *      implicit_update, the implicit velocity update of reading #18).
 * Readings of places where the paper is silent or garbled are listed where
 * they are used.
 */
#include "lbref.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocity set and weights (Sec. II; the paper does not print the
 * weights, the standard D3Q19 set with c_s^2 = 1/3 is used). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static double WT[Q];
static int OPPI[Q];
static int tables_ready = 0;

static void init_tables(void) {
    if (tables_ready) return;
    for (int i = 0; i < Q; i++) {
        int s = abs(CV[i][0]) + abs(CV[i][1]) + abs(CV[i][2]);
        WT[i] = (s == 0) ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int j = 0; j < Q; j++)
            if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) OPPI[i] = j;
    }
    tables_ready = 1;
}

void orc_lattice(int32_t c[19][3], double w[19], int32_t opp[19]) {
    init_tables();
    for (int i = 0; i < Q; i++) {
        for (int a = 0; a < 3; a++) c[i][a] = CV[i][a];
        w[i] = WT[i];
        opp[i] = OPPI[i];
    }
}

/* Eq. Equil: zeta_i rho [1 + cu/cs2 + (cu)^2/(2cs4) - u^2/(2cs2)
 *                        + (cu)^3/(6cs6) - u^2 cu/(2cs4)], cs2 = 1/3. */
void orc_feq(double rho, const double u[3], double out[19]) {
    init_tables();
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        out[i] = WT[i] * rho *
                 (1.0 + cu / cs2 + (cu * cu) / (2.0 * cs2 * cs2) - uu / (2.0 * cs2) +
                  (cu * cu * cu) / (6.0 * cs2 * cs2 * cs2) - uu * cu / (2.0 * cs2 * cs2));
    }
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the
 * golden-ratio increment; each output is the mixed state.  Counter form:
 * output n of a generator seeded with s is mix(s + (n+1) * gamma). */
static uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t orc_splitmix64(uint64_t s, uint64_t n) { return sm_mix(s + (n + 1) * 0x9E3779B97F4A7C15ULL); }
/* uniform double in [0, 1) from the top 53 bits */
double orc_unit(uint64_t s, uint64_t n) { return (double)(orc_splitmix64(s, n) >> 11) * (1.0 / 9007199254740992.0); }

struct orc_state {
    orc_params p;
    int nx, ny, nz;
    int64_t N;
    int64_t t;
    int np;
    double *f, *fs;     /* [2][Q][N] */
    int32_t* owner;     /* [N] */
    int32_t* newown;    /* [N] */
    double* best;       /* [N] claim distance */
    double *rho, *psi;  /* [2][N] */
    double* force;      /* [2][3][N] */
    uint8_t* shell;     /* [N] */
    double *X, *U, *W, *F, *T, *color; /* [np][3] / [np] */
    double* E;          /* [np][3] body axis of a spheroid (unit vector) */
    double Flast[1], *Fsave, *Tsave;
    double *Z, *dV;     /* implicit update: [np][6][6] link drag tensor, [np][6] velocity change */
    double mass0[2];
    int64_t n_cover, n_uncover;
};

void orc_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static inline int64_t nidx(const orc_state* s, int x, int y, int z) {
    return (int64_t)x + (int64_t)s->nx * ((int64_t)y + (int64_t)s->ny * z);
}
static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static inline void ncoord(const orc_state* s, int64_t n, int* x, int* y, int* z) {
    *x = (int)(n % s->nx);
    *y = (int)((n / s->nx) % s->ny);
    *z = (int)(n / ((int64_t)s->nx * s->ny));
}
static inline int64_t nbr(const orc_state* s, int64_t n, int i) {
    int x, y, z;
    ncoord(s, n, &x, &y, &z);
    return nidx(s, wrap(x + CV[i][0], s->nx), wrap(y + CV[i][1], s->ny), wrap(z + CV[i][2], s->nz));
}
/* minimum image of a displacement along an axis of length L */
static inline double mimg(double d, double L) {
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}
static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
#define FIDX(s, c, i, n) (((int64_t)(c) * Q + (i)) * (s)->N + (n))

/* Non-spherical particles (the generality the paper claims for its
 * coupling, Secs. I and III; reading): spheroids with semi-axes R, R and
 * c = aspect R about a body axis e.  aspect = 1 is the sphere, which keeps
 * the plain distance test and the scalar moment of inertia, so sphere runs
 * are unchanged.  The coupling itself (bounce-back, momentum exchange,
 * cover/uncover, virtual fluid) only needs the set of solid nodes and
 * u_s = U + omega x r, whatever the shape. */
static inline int is_sphere(const orc_params* p) { return p->aspect == 1.0; }
static inline double bound_radius(const orc_params* p) {
    return p->aspect > 1.0 ? p->aspect * p->radius : p->radius;
}
static inline double particle_volume(const orc_params* p) {
    return 4.0 / 3.0 * M_PI * p->radius * p->radius * (p->aspect * p->radius);
}

/* Inside test of a displacement d from the centre: R^2 (d.e)^2 +
 * c^2 (|d|^2 - (d.e)^2) <= R^2 c^2, each product and sum rounded in this
 * order (no contraction) so that both implementations decide alike. */
static int inside_spheroid(const orc_params* p, const double d[3], const double e[3]) {
    const double R2 = p->radius * p->radius, c = p->aspect * p->radius, c2 = c * c;
    const double s = ((d[0] * e[0]) + (d[1] * e[1])) + (d[2] * e[2]);
    const double d2 = ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2]);
    const double s2 = s * s;
    return (R2 * s2) + (c2 * (d2 - s2)) <= R2 * c2;
}
int32_t orc_inside(const orc_params* p, const double d[3], const double e[3]) {
    if (is_sphere(p)) {
        const double d2 = ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2]);
        return d2 <= p->radius * p->radius;
    }
    return inside_spheroid(p, d, e);
}

/* Distance from the centre to the surface along the unit vector n:
 * (n_par^2 / c^2 + n_perp^2 / R^2)^(-1/2). */
static double support_radius(const orc_params* p, const double n[3], const double e[3]) {
    const double R = p->radius, c = p->aspect * p->radius;
    double t = dot3(n, e);
    double t2 = t * t;
    if (t2 > 1.0) t2 = 1.0;
    return 1.0 / sqrt(t2 / (c * c) + (1.0 - t2) / (R * R));
}
/* Contact distance of two particles along the line of centres r_hat
 * (reading: the paper's Hertz and lubrication laws are for spheres; for
 * spheroids the surfaces are taken to meet along the line of centres at
 * sigma = rho_p(r_hat) + rho_q(r_hat), and the laws use the gap r - sigma
 * with the sphere radius replaced by sigma / 2). */
double orc_contact_distance(const orc_params* p, const double rh[3], const double ep[3], const double eq[3]) {
    if (is_sphere(p)) return 2.0 * p->radius;
    return support_radius(p, rh, ep) + support_radius(p, rh, eq);
}

/* Rotational update of one particle with torque T (leap-frog, reading):
 * angular momentum L = I(e) omega, L += T; the symmetry axis of a spheroid
 * moves as de/dt = omega x e = (L x e) / I_perp (the part of omega along e
 * does not move it), so it is turned about L by |L| / I_perp (Rodrigues),
 * which is exact for torque-free motion; then omega = I(e_new)^-1 L.
 * I(e) = I_perp (1 - e e) + I_par e e with I_par = 2/5 m R^2 and I_perp =
 * 1/5 m (R^2 + c^2).  Spheres keep omega += T / J and a fixed axis. */
static void apply_inertia(double Ipar, double Iperp, const double e[3], const double v[3], double o[3], int inv) {
    const double a = inv ? 1.0 / Iperp : Iperp, b = inv ? 1.0 / Ipar : Ipar;
    const double t = dot3(e, v);
    for (int k = 0; k < 3; k++) o[k] = a * v[k] + (b - a) * t * e[k];
}
static void rotate_particle(const orc_params* p, double m, double W[3], double e[3], const double T[3]) {
    const double R = p->radius;
    if (is_sphere(p)) {
        const double J = 0.4 * m * R * R;
        for (int a = 0; a < 3; a++) W[a] += T[a] / J;
        return;
    }
    const double c = p->aspect * R;
    const double Ipar = 0.4 * m * R * R, Iperp = 0.2 * m * (R * R + c * c);
    double L[3];
    apply_inertia(Ipar, Iperp, e, W, L, 0);
    for (int a = 0; a < 3; a++) L[a] += T[a];
    const double Lm = sqrt(dot3(L, L));
    if (Lm > 0.0) {
        const double k[3] = {L[0] / Lm, L[1] / Lm, L[2] / Lm};
        const double th = Lm / Iperp;
        double kxe[3];
        cross3(k, e, kxe);
        const double ct = cos(th), st = sin(th), ke = dot3(k, e);
        double en[3];
        for (int a = 0; a < 3; a++) en[a] = e[a] * ct + kxe[a] * st + k[a] * ke * (1.0 - ct);
        const double nn = sqrt(dot3(en, en));
        for (int a = 0; a < 3; a++) e[a] = en[a] / nn;
    }
    apply_inertia(Ipar, Iperp, e, L, W, 1);
}
void orc_rotate(const orc_params* p, double W[3], double e[3], const double T[3]) {
    rotate_particle(p, p->particle_density * particle_volume(p), W, e, T);
}

static double particle_mass(const orc_state* s) {
    if (is_sphere(&s->p)) return s->p.particle_density * 4.0 / 3.0 * M_PI * s->p.radius * s->p.radius * s->p.radius;
    return s->p.particle_density * particle_volume(&s->p);
}

static int derive_np(const orc_params* p) {
    if (p->n_particles >= 0) return p->n_particles;
    double N = (double)p->nx * p->ny * p->nz;
    double v = is_sphere(p) ? 4.0 / 3.0 * M_PI * p->radius * p->radius * p->radius : particle_volume(p);
    return (int)floor(p->volume_fraction * N / v + 0.5);
}

orc_state* orc_create(const orc_params* p, int32_t n_particles) {
    init_tables();
    if (p->implicit_update && !is_sphere(p)) return NULL;
    orc_state* s = (orc_state*)calloc(1, sizeof(orc_state));
    s->p = *p;
    s->nx = p->nx; s->ny = p->ny; s->nz = p->nz;
    s->N = (int64_t)p->nx * p->ny * p->nz;
    s->np = n_particles >= 0 ? n_particles : derive_np(p);
    size_t N = (size_t)s->N;
    s->f = (double*)calloc(2 * Q * N, sizeof(double));
    s->fs = (double*)calloc(2 * Q * N, sizeof(double));
    s->owner = (int32_t*)malloc(N * sizeof(int32_t));
    s->newown = (int32_t*)malloc(N * sizeof(int32_t));
    s->best = (double*)malloc(N * sizeof(double));
    s->rho = (double*)calloc(2 * N, sizeof(double));
    s->psi = (double*)calloc(2 * N, sizeof(double));
    s->force = (double*)calloc(6 * N, sizeof(double));
    s->shell = (uint8_t*)calloc(N, 1);
    int np = s->np > 0 ? s->np : 1;
    s->X = (double*)calloc(3 * np, sizeof(double));
    s->U = (double*)calloc(3 * np, sizeof(double));
    s->W = (double*)calloc(3 * np, sizeof(double));
    s->F = (double*)calloc(3 * np, sizeof(double));
    s->T = (double*)calloc(3 * np, sizeof(double));
    s->Fsave = (double*)calloc(3 * np, sizeof(double));
    s->Tsave = (double*)calloc(3 * np, sizeof(double));
    s->color = (double*)calloc(np, sizeof(double));
    s->E = (double*)calloc(3 * np, sizeof(double));
    s->Z = (double*)calloc(36 * np, sizeof(double));
    s->dV = (double*)calloc(6 * np, sizeof(double));
    for (int q = 0; q < s->np; q++) s->color[q] = p->color;
    for (int q = 0; q < s->np; q++) s->E[3 * q + 2] = 1.0;
    for (size_t n = 0; n < N; n++) s->owner[n] = -1;
    return s;
}

void orc_destroy(orc_state* s) {
    if (!s) return;
    free(s->f); free(s->fs); free(s->owner); free(s->newown); free(s->best);
    free(s->rho); free(s->psi); free(s->force); free(s->shell);
    free(s->X); free(s->U); free(s->W); free(s->F); free(s->T); free(s->Fsave); free(s->Tsave);
    free(s->color);
    free(s->E);
    free(s->Z); free(s->dV);
    free(s);
}

int32_t orc_n_particles(const orc_state* s) { return s->np; }

void orc_set_particle_colors(orc_state* s, const double* colors) {
    for (int q = 0; q < s->np; q++) s->color[q] = colors[q];
}

void orc_get_axes(const orc_state* s, double* e) { memcpy(e, s->E, sizeof(double) * 3 * (size_t)s->np); }
void orc_set_axes(orc_state* s, const double* e) { memcpy(s->E, e, sizeof(double) * 3 * (size_t)s->np); }

/* Squared minimum-image distance from node (x,y,z) to the centre of
 * particle q, evaluated without contraction so that both implementations
 * reach the same inside/outside decision. */
static double node_dist2(const orc_state* s, int x, int y, int z, int q) {
    double dx = mimg((double)x - s->X[3 * q + 0], (double)s->nx);
    double dy = mimg((double)y - s->X[3 * q + 1], (double)s->ny);
    double dz = mimg((double)z - s->X[3 * q + 2], (double)s->nz);
    double a = dx * dx;
    double b = dy * dy;
    double c = dz * dz;
    return (a + b) + c;
}

/* Node ownership: a node is solid when it lies inside a sphere
 * (|x - X_p|^2 <= R^2, minimum image) or spheroid (inside_spheroid); the
 * nearer centre wins; ties go to the lower particle index (reading: the
 * paper only says "inside").  Static walls never change.  Result in
 * s->newown. */
static void claim_nodes(orc_state* s) {
    const double R = bound_radius(&s->p), R2 = s->p.radius * s->p.radius;
    const int sphere = is_sphere(&s->p);
    for (int64_t n = 0; n < s->N; n++) {
        s->newown[n] = (s->owner[n] == -2) ? -2 : -1;
        s->best[n] = 0.0;
    }
    int dims[3] = {s->nx, s->ny, s->nz};
    for (int q = 0; q < s->np; q++) {
        int lo[3], cnt[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = (int)floor(s->X[3 * q + a] - R);
            int hi = (int)floor(s->X[3 * q + a] + R);
            cnt[a] = hi - lo[a] + 1;
            if (cnt[a] > dims[a]) cnt[a] = dims[a];
        }
        for (int kz = 0; kz < cnt[2]; kz++)
            for (int ky = 0; ky < cnt[1]; ky++)
                for (int kx = 0; kx < cnt[0]; kx++) {
                    int x = wrap(lo[0] + kx, s->nx), y = wrap(lo[1] + ky, s->ny), z = wrap(lo[2] + kz, s->nz);
                    int64_t n = nidx(s, x, y, z);
                    if (s->newown[n] == -2) continue;
                    double d2 = node_dist2(s, x, y, z, q);
                    if (sphere) {
                        if (d2 > R2) continue;
                    } else {
                        const double d[3] = {mimg((double)x - s->X[3 * q + 0], (double)s->nx),
                                             mimg((double)y - s->X[3 * q + 1], (double)s->ny),
                                             mimg((double)z - s->X[3 * q + 2], (double)s->nz)};
                        if (!inside_spheroid(&s->p, d, &s->E[3 * q])) continue;
                    }
                    int cur = s->newown[n];
                    if (cur == -1 || d2 < s->best[n] || (d2 == s->best[n] && q < cur)) {
                        s->newown[n] = q;
                        s->best[n] = d2;
                    }
                }
    }
}

/* displacement of point (px,py,pz) from particle q's centre, minimum image */
static void rel_pos(const orc_state* s, double px, double py, double pz, int q, double r[3]) {
    r[0] = mimg(px - s->X[3 * q + 0], (double)s->nx);
    r[1] = mimg(py - s->X[3 * q + 1], (double)s->ny);
    r[2] = mimg(pz - s->X[3 * q + 2], (double)s->nz);
}

/* surface velocity of particle q at point r from its centre: U + omega x r */
static void surf_vel(const orc_state* s, int q, const double r[3], double us[3]) {
    double wxr[3];
    cross3(&s->W[3 * q], r, wxr);
    for (int a = 0; a < 3; a++) us[a] = s->U[3 * q + a] + wxr[a];
}

static void add_force(orc_state* s, int q, const double r[3], const double dF[3]) {
    double tq[3];
    cross3(r, dF, tq);
    for (int a = 0; a < 3; a++) {
        s->F[3 * q + a] += dF[a];
        s->T[3 * q + a] += tq[a];
    }
}

/* Implicit update (reading #18).  The wall term of a link from the fluid
 * node x to particle q in direction j is k a.V, with k = 6 zeta_j rho^c(x),
 * V = (U, omega) and a = (c_j, r x c_j) (u_s . c_j = c_j . U + (r x c_j) .
 * omega).  The link's force and torque on q are (2 f* - k a.V) a, so they
 * change by -k a a^T dV when V does: Z = sum over links of k a a^T. */
static void link_dir(const double r[3], int j, double a[6]) {
    const double cj[3] = {CV[j][0], CV[j][1], CV[j][2]};
    a[0] = cj[0];
    a[1] = cj[1];
    a[2] = cj[2];
    cross3(r, cj, &a[3]);
}
static void add_drag(orc_state* s, int q, const double r[3], int j, double k) {
    double a[6];
    link_dir(r, j, a);
    for (int u = 0; u < 6; u++)
        for (int v = 0; v < 6; v++) s->Z[36 * q + 6 * u + v] += k * a[u] * a[v];
}

/* densities rho^c = sum_i f_i^c on fluid nodes (rho0 = 1 in the density
 * definition; the paper uses rho0 = 1 throughout), 0 elsewhere */
static void fluid_densities(orc_state* s) {
    const int64_t N = s->N;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        for (int c = 0; c < 2; c++) {
            double r = 0.0;
            if (s->owner[n] == -1)
                for (int i = 0; i < Q; i++) r += s->f[FIDX(s, c, i, n)];
            s->rho[(int64_t)c * N + n] = r;
        }
    }
}

/* Step 1: particles move over the lattice (Sec. III and IV). */
static void remap(orc_state* s) {
    const int64_t N = s->N;
    fluid_densities(s); /* rho(t) on the old fluid nodes */
    double mass_now[2] = {0.0, 0.0};
    for (int c = 0; c < 2; c++)
        for (int64_t n = 0; n < N; n++) mass_now[c] += s->rho[(int64_t)c * N + n];
    claim_nodes(s);
    double corr[2] = {1.0, 1.0};
    if (s->p.mass_corr_c0 != 0.0) {
        /* Eq. masscorr: scale by 1 - C0 (sum_c' rho_init^c' / rho_init^c) dM^c / N,
         * dM^c = current total fluid mass minus the initial one. */
        double rsum = s->p.rho_init[0] + s->p.rho_init[1];
        for (int c = 0; c < 2; c++)
            corr[c] = 1.0 - s->p.mass_corr_c0 * (rsum / s->p.rho_init[c]) * (mass_now[c] - s->mass0[c]) / (double)N;
    }
    for (int64_t n = 0; n < N; n++) {
        int old = s->owner[n], nw = s->newown[n];
        int x, y, z;
        ncoord(s, n, &x, &y, &z);
        if (old == -1 && nw >= 0) {
            /* covered: the fluid is deleted and its momentum sum_c sum_i f c
             * goes to the particle (reading of the printed F = -rho u: the
             * sign that conserves total momentum). */
            double mom[3] = {0, 0, 0};
            for (int c = 0; c < 2; c++)
                for (int i = 0; i < Q; i++) {
                    double fv = s->f[FIDX(s, c, i, n)];
                    for (int a = 0; a < 3; a++) mom[a] += fv * CV[i][a];
                    s->f[FIDX(s, c, i, n)] = 0.0;
                }
            double r[3];
            rel_pos(s, x, y, z, nw, r);
            add_force(s, nw, r, mom);
            s->n_cover++;
        } else if (old >= 0 && nw == -1) {
            /* uncovered: refill with rho_new^c = mean rho^c over the
             * neighbours that were fluid (Eq. eqn_rho_neu, optionally scaled
             * by Eq. masscorr), f = f^eq(rho_new, u_surf); the particle
             * loses the created momentum sum_c rho_new u_surf
             * (Eq. eqn_ladd_vernichtenunderzeugen, sign from momentum
             * conservation). */
            double r[3], us[3];
            rel_pos(s, x, y, z, old, r);
            surf_vel(s, old, r, us);
            double mom[3] = {0, 0, 0};
            for (int c = 0; c < 2; c++) {
                double sum = 0.0;
                int cntn = 0;
                for (int i = 1; i < Q; i++) {
                    int64_t m = nbr(s, n, i);
                    if (s->owner[m] == -1) {
                        sum += s->rho[(int64_t)c * N + m];
                        cntn++;
                    }
                }
                double rbar = cntn ? sum / cntn : s->p.rho_init[c];
                double rnew = rbar * corr[c];
                double fe[Q];
                orc_feq(rnew, us, fe);
                for (int i = 0; i < Q; i++) s->f[FIDX(s, c, i, n)] = fe[i];
                for (int a = 0; a < 3; a++) mom[a] -= rnew * us[a];
            }
            add_force(s, old, r, mom);
            s->n_uncover++;
        }
    }
    memcpy(s->owner, s->newown, (size_t)N * sizeof(int32_t));
}

/* Step 2: densities on the new status, virtual fluid on the shell
 * (Sec. IV), Psi = rho0 (1 - exp(-rho/rho0)) (Eq. eqn_ref_dens). */
static void densities_and_psi(orc_state* s) {
    const int64_t N = s->N;
    fluid_densities(s);
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        int own = s->owner[n];
        s->shell[n] = 0;
        if (own == -1) continue;
        double sum[2] = {0.0, 0.0};
        int cnt = 0;
        for (int i = 1; i < Q; i++) {
            int64_t m = nbr(s, n, i);
            if (s->owner[m] == -1) {
                sum[0] += s->rho[m];
                sum[1] += s->rho[N + m];
                cnt++;
            }
        }
        if (cnt > 0) {
            s->shell[n] = 1;
            if (s->p.virtual_fluid) {
                double r0 = sum[0] / cnt, r1 = sum[1] / cnt;
                double col = own >= 0 ? s->color[own] : 0.0;
                if (col > 0.0) r0 += col;          /* positive colour: red added */
                else if (col < 0.0) r1 += -col;    /* negative colour: blue added */
                s->rho[n] = r0;
                s->rho[N + n] = r1;
            }
        }
    }
    const double r0 = s->p.rho0;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++)
        for (int c = 0; c < 2; c++) s->psi[(int64_t)c * N + n] = r0 * (1.0 - exp(-s->rho[(int64_t)c * N + n] / r0));
}

/* Step 3: F^c(x) = -Psi^c(x) g_{c cbar} sum_x' W(x'-x) Psi^cbar(x') (x' - x)
 * over the 18 D3Q19 neighbours (Eq. eqn_shan-chen-F with g_rr = g_bb = 0;
 * the link weights W are a parameter, default 1). */
static void sc_forces(orc_state* s) {
    const int64_t N = s->N;
    const double g = s->p.g_br;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        for (int c = 0; c < 2; c++)
            for (int a = 0; a < 3; a++) s->force[((int64_t)c * 3 + a) * N + n] = 0.0;
        if (!(s->owner[n] == -1 || s->shell[n])) continue;
        for (int c = 0; c < 2; c++) {
            int cb = 1 - c;
            double acc[3] = {0, 0, 0};
            for (int i = 1; i < Q; i++) {
                int s1 = abs(CV[i][0]) + abs(CV[i][1]) + abs(CV[i][2]);
                double wl = s1 == 1 ? s->p.sc_weight[0] : s->p.sc_weight[1];
                double pn = s->psi[(int64_t)cb * N + nbr(s, n, i)];
                for (int a = 0; a < 3; a++) acc[a] += wl * pn * CV[i][a];
            }
            double pc = s->psi[(int64_t)c * N + n];
            for (int a = 0; a < 3; a++) s->force[((int64_t)c * 3 + a) * N + n] = -g * pc * acc[a];
        }
    }
}

/* Step 4: force and torque of the shell nodes onto their particle
 * (Eq. eqn_shan_chen_particle; interior nodes have Psi = 0, so F = 0). */
static void particle_sc_force(orc_state* s) {
    const int64_t N = s->N;
    for (int64_t n = 0; n < N; n++) {
        int q = s->owner[n];
        if (q < 0 || !s->shell[n]) continue;
        double dF[3];
        for (int a = 0; a < 3; a++) dF[a] = s->force[(0 * 3 + a) * N + n] + s->force[(1 * 3 + a) * N + n];
        int x, y, z;
        ncoord(s, n, &x, &y, &z);
        double r[3];
        rel_pos(s, x, y, z, q, r);
        add_force(s, q, r, dF);
    }
}

/* Step 5: BGK collision (Sec. II).  The equilibrium of component c is
 * taken at u' + tau^c F^c / rho^c, u' the Shan-Chen common velocity
 * sum_c(j^c/tau^c) / sum_c(rho^c/tau^c) (vel_mode 0) or the component's
 * own velocity j^c/rho^c (vel_mode 1). */
static void collide(orc_state* s) {
    const int64_t N = s->N;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        if (s->owner[n] != -1) {
            for (int c = 0; c < 2; c++)
                for (int i = 0; i < Q; i++) s->fs[FIDX(s, c, i, n)] = 0.0;
            continue;
        }
        double rho[2], j[2][3];
        for (int c = 0; c < 2; c++) {
            rho[c] = 0.0;
            j[c][0] = j[c][1] = j[c][2] = 0.0;
            for (int i = 0; i < Q; i++) {
                double fv = s->f[FIDX(s, c, i, n)];
                rho[c] += fv;
                for (int a = 0; a < 3; a++) j[c][a] += fv * CV[i][a];
            }
        }
        double up[3];
        {
            double den = rho[0] / s->p.tau[0] + rho[1] / s->p.tau[1];
            for (int a = 0; a < 3; a++) up[a] = (j[0][a] / s->p.tau[0] + j[1][a] / s->p.tau[1]) / den;
        }
        for (int c = 0; c < 2; c++) {
            double ueq[3];
            for (int a = 0; a < 3; a++) {
                double base = s->p.vel_mode ? j[c][a] / rho[c] : up[a];
                double Fa = s->force[((int64_t)c * 3 + a) * N + n] + rho[c] * s->p.body_force[a];
                ueq[a] = base + s->p.tau[c] * Fa / rho[c];
            }
            double fe[Q];
            orc_feq(rho[c], ueq, fe);
            for (int i = 0; i < Q; i++) {
                double fv = s->f[FIDX(s, c, i, n)];
                s->fs[FIDX(s, c, i, n)] = fv - (fv - fe[i]) / s->p.tau[c];
            }
        }
    }
}

/* Step 6: pull streaming; a link whose source x - c_i is solid is bounced
 * back with the moving-wall term (Eq. after eqn_bounce-back-force):
 *   f_i(x,t+1) = f*_j(x) - 6 zeta_j rho^c(x) u_s . c_j,   j = opposite(i),
 * where u_s is the surface velocity at the link midpoint x + c_j/2.  The
 * printed "1/6" is read as 2 zeta_j / c_s^2 = 6 zeta_j (Ladd), and the
 * printed "2 rho" as 2 f*_j; the particle receives
 *   dF = (2 f*_j - 6 zeta_j rho u_s . c_j) c_j  (Eq. eqn_ladd_bewegtewand)
 * and the torque r x dF with r from the centre to the link midpoint. */
static void stream_bounce(orc_state* s) {
    const int64_t N = s->N;
    /* fluid-fluid links: independent per destination */
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; n++) {
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < Q; i++) {
                double v = 0.0;
                if (s->owner[n] == -1) {
                    int64_t src = (i == 0) ? n : nbr(s, n, OPPI[i]);
                    if (s->owner[src] == -1) v = s->fs[FIDX(s, c, i, src)];
                }
                s->f[FIDX(s, c, i, n)] = v;
            }
    }
    /* solid links, in node order so the particle sums are reproducible */
    for (int64_t n = 0; n < N; n++) {
        if (s->owner[n] != -1) continue;
        int x, y, z;
        ncoord(s, n, &x, &y, &z);
        for (int i = 1; i < Q; i++) {
            int j = OPPI[i];
            int64_t src = nbr(s, n, j); /* x - c_i = x + c_j */
            int q = s->owner[src];
            if (q == -1) continue;
            double r[3] = {0, 0, 0}, us[3] = {0, 0, 0};
            if (q >= 0) {
                rel_pos(s, x + 0.5 * CV[j][0], y + 0.5 * CV[j][1], z + 0.5 * CV[j][2], q, r);
                surf_vel(s, q, r, us);
            }
            double cu = us[0] * CV[j][0] + us[1] * CV[j][1] + us[2] * CV[j][2];
            for (int c = 0; c < 2; c++) {
                double fsj = s->fs[FIDX(s, c, j, n)];
                double wall = 6.0 * WT[j] * s->rho[(int64_t)c * N + n] * cu;
                s->f[FIDX(s, c, i, n)] = fsj - wall;
                if (q >= 0) {
                    double mag = 2.0 * fsj - wall;
                    double dF[3] = {mag * CV[j][0], mag * CV[j][1], mag * CV[j][2]};
                    add_force(s, q, r, dF);
                    if (s->p.implicit_update) add_drag(s, q, r, j, 6.0 * WT[j] * s->rho[(int64_t)c * N + n]);
                }
            }
        }
    }
}

/* Step 7: particle MD (Sec. III).  Pair forces with r = X_p - X_q:
 *   Hertz: F_p = -dV/dr r_hat = 5/2 K_H (2R - r)^{3/2} r_hat for r < 2R;
 *   lubrication: F_p = -6 pi nu R^4/(2R)^2 r_hat [r_hat.(U_p - U_q)]
 *                 (1/h - 1/h_c) for gap h = r - 2R < h_c, h clamped at
 *                 h_min (reading: the printed "-1" would make the force jump
 *                 at the stated cut-off 2/3; 1/h_c keeps it continuous);
 *   nu = c_s^2 (tau - 1/2) with tau the mean of the two components.
 * (Spheroids: 2R becomes the contact distance sigma, R becomes sigma / 2.)
 * Then leap-frog: U += F/m, the rotation of rotate_particle, X += U. */
/* Pair force on particle p from particle q (Hertz + lubrication, see
 * md_update); r = X_p - X_q with the minimum image. */
static void pair_force(const orc_params* P, const double Lb[3], const double* Xp, const double* Xq,
                       const double* Up, const double* Uq, const double* ep, const double* eq, double Fp[3]) {
    double nu = (1.0 / 3.0) * (0.5 * (P->tau[0] + P->tau[1]) - 0.5);
    double r[3];
    Fp[0] = Fp[1] = Fp[2] = 0.0;
    for (int a = 0; a < 3; a++) r[a] = mimg(Xp[a] - Xq[a], Lb[a]);
    double d = sqrt(dot3(r, r));
    if (d <= 0.0) return;
    double rh[3] = {r[0] / d, r[1] / d, r[2] / d};
    /* contact distance: 2R for spheres; for spheroids the sum of the
     * support radii along r_hat, with sigma / 2 in place of R below */
    const double sigma = orc_contact_distance(P, rh, ep, eq), R = 0.5 * sigma;
    if (d < sigma) {
        double mag = 2.5 * P->k_hertz * pow(sigma - d, 1.5);
        for (int a = 0; a < 3; a++) Fp[a] += mag * rh[a];
    }
    double h = d - sigma;
    if (h < P->lub_cut) {
        double he = h < P->lub_min ? P->lub_min : h;
        double du[3] = {Up[0] - Uq[0], Up[1] - Uq[1], Up[2] - Uq[2]};
        double mag = -6.0 * M_PI * nu * pow(R, 4) / (4.0 * R * R) * dot3(rh, du) * (1.0 / he - 1.0 / P->lub_cut);
        for (int a = 0; a < 3; a++) Fp[a] += mag * rh[a];
    }
}

void orc_pair_force(const orc_params* P, const double Xp[3], const double Xq[3], const double Up[3],
                    const double Uq[3], double Fp[3]) {
    double Lb[3] = {(double)P->nx, (double)P->ny, (double)P->nz};
    const double ez[3] = {0.0, 0.0, 1.0};
    pair_force(P, Lb, Xp, Xq, Up, Uq, ez, ez, Fp);
}

/* Solve A x = b for a 6 x 6 system (Gaussian elimination, partial
 * pivoting); A is row-major, both are overwritten. */
static void solve6(double A[36], double b[6], double x[6]) {
    for (int col = 0; col < 6; col++) {
        int piv = col;
        for (int r = col + 1; r < 6; r++)
            if (fabs(A[6 * r + col]) > fabs(A[6 * piv + col])) piv = r;
        if (piv != col) {
            for (int v = 0; v < 6; v++) {
                const double t = A[6 * col + v];
                A[6 * col + v] = A[6 * piv + v];
                A[6 * piv + v] = t;
            }
            const double t = b[col];
            b[col] = b[piv];
            b[piv] = t;
        }
        for (int r = col + 1; r < 6; r++) {
            const double f = A[6 * r + col] / A[6 * col + col];
            for (int v = col; v < 6; v++) A[6 * r + v] -= f * A[6 * col + v];
            b[r] -= f * b[col];
        }
    }
    for (int r = 5; r >= 0; r--) {
        double t = b[r];
        for (int v = r + 1; v < 6; v++) t -= A[6 * r + v] * x[v];
        x[r] = t / A[6 * r + r];
    }
}

/* Reading #18, implicit particle velocity update (the cited particle
 * method, Ladd & Verberg 2001, discusses implicit updates for light
 * particles).  The links' wall term is taken at the new velocity: with the
 * force and torque (F, T) of this step, computed at the old velocity, and
 * the drag tensor Z of add_drag,
 *     (M + Z) dV = (F, T),  M = diag(m, m, m, J, J, J),  J = 2/5 m R^2.
 * The fluid gets the same change of the wall term, -k a.dV on every link's
 * bounce-back population, so fluid plus particle momentum stays exact.
 * Then U += dU, omega += d omega, X += U.  Spheres only. */
static void implicit_velocity_update(orc_state* s, double m, const double Lb[3]) {
    const int np = s->np;
    const int64_t N = s->N;
    const double J = 0.4 * m * s->p.radius * s->p.radius;
    const int moving = !s->p.fixed_particles;
    for (int p = 0; p < np; p++) {
        double A[36], b[6];
        for (int u = 0; u < 36; u++) A[u] = s->Z[36 * p + u];
        for (int u = 0; u < 3; u++) {
            A[7 * u] += m;
            A[7 * (u + 3)] += J;
            b[u] = s->F[3 * p + u];
            b[u + 3] = s->T[3 * p + u];
        }
        if (moving) solve6(A, b, &s->dV[6 * p]);
        else
            for (int u = 0; u < 6; u++) s->dV[6 * p + u] = 0.0;
    }
    if (moving) {
        /* the fluid's share: links as in stream_bounce, with the positions
         * the step used */
        for (int64_t n = 0; n < N; n++) {
            if (s->owner[n] != -1) continue;
            int x, y, z;
            ncoord(s, n, &x, &y, &z);
            for (int i = 1; i < Q; i++) {
                const int j = OPPI[i];
                const int q = s->owner[nbr(s, n, j)];
                if (q < 0) continue;
                double r[3], a[6];
                rel_pos(s, x + 0.5 * CV[j][0], y + 0.5 * CV[j][1], z + 0.5 * CV[j][2], q, r);
                link_dir(r, j, a);
                double ad = 0.0;
                for (int u = 0; u < 6; u++) ad += a[u] * s->dV[6 * q + u];
                for (int c = 0; c < 2; c++) s->f[FIDX(s, c, i, n)] -= 6.0 * WT[j] * s->rho[(int64_t)c * N + n] * ad;
            }
        }
        for (int p = 0; p < np; p++)
            for (int a = 0; a < 3; a++) {
                s->U[3 * p + a] += s->dV[6 * p + a];
                s->W[3 * p + a] += s->dV[6 * p + 3 + a];
                double xn = s->X[3 * p + a] + s->U[3 * p + a];
                xn -= Lb[a] * floor(xn / Lb[a]);
                if (xn >= Lb[a]) xn -= Lb[a];
                s->X[3 * p + a] = xn;
            }
    }
    for (int p = 0; p < np; p++) {
        for (int a = 0; a < 3; a++) s->F[3 * p + a] = s->T[3 * p + a] = 0.0;
        for (int u = 0; u < 36; u++) s->Z[36 * p + u] = 0.0;
    }
}

static void md_update(orc_state* s) {
    const int np = s->np;
    memcpy(s->Fsave, s->F, 3 * sizeof(double) * (np > 0 ? np : 1));
    memcpy(s->Tsave, s->T, 3 * sizeof(double) * (np > 0 ? np : 1));
    if (np == 0) return;
    double Lb[3] = {(double)s->nx, (double)s->ny, (double)s->nz};
    for (int p = 0; p < np; p++)
        for (int q = p + 1; q < np; q++) {
            double Fp[3];
            pair_force(&s->p, Lb, &s->X[3 * p], &s->X[3 * q], &s->U[3 * p], &s->U[3 * q], &s->E[3 * p], &s->E[3 * q],
                       Fp);
            for (int a = 0; a < 3; a++) {
                s->F[3 * p + a] += Fp[a];
                s->F[3 * q + a] -= Fp[a];
            }
        }
    double m = particle_mass(s);
    if (s->p.implicit_update) {
        implicit_velocity_update(s, m, Lb);
        return;
    }
    for (int p = 0; p < np; p++) {
        if (!s->p.fixed_particles) {
            rotate_particle(&s->p, m, &s->W[3 * p], &s->E[3 * p], &s->T[3 * p]);
            for (int a = 0; a < 3; a++) {
                s->U[3 * p + a] += s->F[3 * p + a] / m;
                double xn = s->X[3 * p + a] + s->U[3 * p + a];
                xn -= Lb[a] * floor(xn / Lb[a]);
                if (xn >= Lb[a]) xn -= Lb[a];
                s->X[3 * p + a] = xn;
            }
        }
        for (int a = 0; a < 3; a++) s->F[3 * p + a] = s->T[3 * p + a] = 0.0;
    }
}

/* test hook: only step 1 (particle remap with cover/uncover) */
void orc_debug_remap(orc_state* s) { remap(s); }

int orc_step(orc_state* s, int32_t nsteps) {
    for (int k = 0; k < nsteps; k++) {
        remap(s);
        densities_and_psi(s);
        sc_forces(s);
        particle_sc_force(s);
        collide(s);
        stream_bounce(s);
        md_update(s);
        s->t++;
    }
    return 0;
}

static double fluid_mass(const orc_state* s, int c) {
    double m = 0.0;
    for (int64_t n = 0; n < s->N; n++)
        if (s->owner[n] == -1)
            for (int i = 0; i < Q; i++) m += s->f[FIDX(s, c, i, n)];
    return m;
}

/* f = f^eq(rho, u) on fluid nodes, nodes inside spheres solid (no fluid) */
int orc_init_fields(orc_state* s, const double* rho, const double* u, const double* particles, const int32_t* walls) {
    const int64_t N = s->N;
    for (int q = 0; q < s->np; q++)
        for (int a = 0; a < 3; a++) {
            s->X[3 * q + a] = particles[9 * q + a];
            s->U[3 * q + a] = particles[9 * q + 3 + a];
            s->W[3 * q + a] = particles[9 * q + 6 + a];
            s->F[3 * q + a] = s->T[3 * q + a] = 0.0;
        }
    for (int64_t n = 0; n < N; n++) s->owner[n] = (walls && walls[n] == -2) ? -2 : -1;
    claim_nodes(s);
    memcpy(s->owner, s->newown, (size_t)N * sizeof(int32_t));
    for (int64_t n = 0; n < N; n++) {
        double uu[3] = {0, 0, 0};
        if (u)
            for (int a = 0; a < 3; a++) uu[a] = u[(int64_t)a * N + n];
        for (int c = 0; c < 2; c++) {
            double fe[Q];
            orc_feq(rho[(int64_t)c * N + n], uu, fe);
            for (int i = 0; i < Q; i++) s->f[FIDX(s, c, i, n)] = s->owner[n] == -1 ? fe[i] : 0.0;
        }
    }
    s->mass0[0] = fluid_mass(s, 0);
    s->mass0[1] = fluid_mass(s, 1);
    s->t = 0;
    s->n_cover = s->n_uncover = 0;
    return 0;
}

/* Seeded init.  Stream 0 of SplitMix64(seed) drives random sequential
 * addition: candidate centres X = L * u (three draws), accepted when the
 * minimum-image distance to every earlier centre is at least 2R (2 c for
 * prolate spheroids); at most 10^6 candidates.  Spheroids take their axes
 * from stream 3: z = 2 u - 1, phi = 2 pi u' (draws 2q, 2q + 1), e =
 * (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z).  Stream 1 + c gives the node noise of component c:
 * rho^c(n) = rho_init^c + a (2 u - 1) with u the n-th draw.  Stream seeds
 * are the first outputs of SplitMix64(seed): s_k = splitmix64(seed, k). */
int orc_init_from_seed(orc_state* s, uint64_t seed) {
    const int64_t N = s->N;
    uint64_t s0 = orc_splitmix64(seed, 0);
    uint64_t sc[2] = {orc_splitmix64(seed, 1), orc_splitmix64(seed, 2)};
    double Lb[3] = {(double)s->nx, (double)s->ny, (double)s->nz};
    double* parts = (double*)calloc(9 * (size_t)(s->np > 0 ? s->np : 1), sizeof(double));
    uint64_t draw = 0;
    int placed = 0;
    const double dmin2 = 4.0 * bound_radius(&s->p) * bound_radius(&s->p);
    for (int64_t attempt = 0; placed < s->np; attempt++) {
        if (attempt >= 1000000) {
            free(parts);
            return -5;
        }
        double c[3];
        for (int a = 0; a < 3; a++) c[a] = Lb[a] * orc_unit(s0, draw++);
        int ok = 1;
        for (int q = 0; q < placed && ok; q++) {
            double dx = mimg(c[0] - parts[9 * q + 0], Lb[0]);
            double dy = mimg(c[1] - parts[9 * q + 1], Lb[1]);
            double dz = mimg(c[2] - parts[9 * q + 2], Lb[2]);
            double a2 = dx * dx, b2 = dy * dy, c2 = dz * dz;
            if ((a2 + b2) + c2 < dmin2) ok = 0;
        }
        if (!ok) continue;
        for (int a = 0; a < 3; a++) parts[9 * placed + a] = c[a];
        placed++;
    }
    if (!is_sphere(&s->p)) {
        const uint64_t se = orc_splitmix64(seed, 3);
        for (int q = 0; q < s->np; q++) {
            const double zc = 2.0 * orc_unit(se, 2 * (uint64_t)q) - 1.0;
            const double ph = 2.0 * M_PI * orc_unit(se, 2 * (uint64_t)q + 1);
            const double rr = sqrt(1.0 - zc * zc);
            s->E[3 * q + 0] = rr * cos(ph);
            s->E[3 * q + 1] = rr * sin(ph);
            s->E[3 * q + 2] = zc;
        }
    }
    double* rho = (double*)malloc(2 * (size_t)N * sizeof(double));
    for (int c = 0; c < 2; c++)
        for (int64_t n = 0; n < N; n++)
            rho[(int64_t)c * N + n] = s->p.rho_init[c] + s->p.noise_amp * (2.0 * orc_unit(sc[c], (uint64_t)n) - 1.0);
    int rc = orc_init_fields(s, rho, NULL, parts, NULL);
    free(rho);
    free(parts);
    return rc;
}

void orc_get_state(const orc_state* s, double* f, int32_t* owner, double* particles, double meta[4]) {
    if (f) memcpy(f, s->f, sizeof(double) * 2 * Q * (size_t)s->N);
    if (owner) memcpy(owner, s->owner, sizeof(int32_t) * (size_t)s->N);
    if (particles)
        for (int q = 0; q < s->np; q++)
            for (int a = 0; a < 3; a++) {
                particles[9 * q + a] = s->X[3 * q + a];
                particles[9 * q + 3 + a] = s->U[3 * q + a];
                particles[9 * q + 6 + a] = s->W[3 * q + a];
            }
    if (meta) {
        meta[0] = (double)s->t;
        meta[1] = s->mass0[0];
        meta[2] = s->mass0[1];
        meta[3] = (double)s->np;
    }
}

int orc_set_state(orc_state* s, const double* f, const int32_t* owner, const double* particles, const double meta[4]) {
    memcpy(s->f, f, sizeof(double) * 2 * Q * (size_t)s->N);
    memcpy(s->owner, owner, sizeof(int32_t) * (size_t)s->N);
    for (int q = 0; q < s->np; q++)
        for (int a = 0; a < 3; a++) {
            s->X[3 * q + a] = particles[9 * q + a];
            s->U[3 * q + a] = particles[9 * q + 3 + a];
            s->W[3 * q + a] = particles[9 * q + 6 + a];
            s->F[3 * q + a] = s->T[3 * q + a] = 0.0;
        }
    s->t = (int64_t)meta[0];
    s->mass0[0] = meta[1];
    s->mass0[1] = meta[2];
    return 0;
}

void orc_get_rho(const orc_state* s, double* rho) {
    for (int c = 0; c < 2; c++)
        for (int64_t n = 0; n < s->N; n++) {
            double r = 0.0;
            if (s->owner[n] == -1)
                for (int i = 0; i < Q; i++) r += s->f[FIDX(s, c, i, n)];
            rho[(int64_t)c * s->N + n] = r;
        }
}

void orc_get_forces(const orc_state* s, double* F, double* T) {
    memcpy(F, s->Fsave, 3 * sizeof(double) * (size_t)s->np);
    memcpy(T, s->Tsave, 3 * sizeof(double) * (size_t)s->np);
}

void orc_last_psi(const orc_state* s, double* psi) { memcpy(psi, s->psi, sizeof(double) * 2 * (size_t)s->N); }
void orc_last_sc_force(const orc_state* s, double* F) { memcpy(F, s->force, sizeof(double) * 6 * (size_t)s->N); }

void orc_observe(const orc_state* s, orc_obs* o) {
    memset(o, 0, sizeof(*o));
    o->step = s->t;
    double mu = 0.0;
    for (int64_t n = 0; n < s->N; n++) {
        if (s->owner[n] != -1) continue;
        double rt = 0.0, jt[3] = {0, 0, 0};
        for (int c = 0; c < 2; c++)
            for (int i = 0; i < Q; i++) {
                double fv = s->f[FIDX(s, c, i, n)];
                o->mass[c] += fv;
                rt += fv;
                for (int a = 0; a < 3; a++) {
                    o->mom_fluid[a] += fv * CV[i][a];
                    jt[a] += fv * CV[i][a];
                }
            }
        double um = sqrt(dot3(jt, jt)) / rt;
        if (um > mu) mu = um;
    }
    o->max_u = mu;
    double m = particle_mass(s);
    if (!s->p.fixed_particles)
        for (int q = 0; q < s->np; q++)
            for (int a = 0; a < 3; a++) o->mom_part[a] += m * s->U[3 * q + a];
    o->n_cover = s->n_cover;
    o->n_uncover = s->n_uncover;
}
