/*
 * lbref.h -- FP64 CPU oracle for the two-component Shan-Chen D3Q19 BGK
 * lattice Boltzmann fluid with suspended spheres (Jansen & Harting,
 * "From Bijels to Pickering emulsions: a lattice Boltzmann study",
 * arXiv:1004.4414).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference that the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product never does.
 * It shares no code, header or constant table with the CUDA library.
 *
 * Conventions (interface, shared by value with the library's canonical
 * export format, not by code):
 *   node index   n = x + nx*(y + ny*z)
 *   populations  f[c][i][n], c = 0 red, 1 blue; i = 0..18 in the order
 *                0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the 12 face
 *                diagonals in opposite pairs (odd i, i+1).
 *   owner[n]     -1 fluid, -2 static wall, p >= 0 solid node of particle p.
 *   particle     9 doubles: X[3], U[3], omega[3]; spheroids also carry a
 *                body axis e[3] (orc_get_axes / orc_set_axes).
 */
#ifndef LBREF_H
#define LBREF_H
#include <stdint.h>

typedef struct {
    int32_t nx, ny, nz;
    int32_t n_particles;        /* exact count used by the seeded init; <0: from volume_fraction */
    double tau[2];              /* BGK relaxation time per component (Sec. II) */
    double g_br;                /* Shan-Chen coupling g_br = g_rb (Eq. eqn_shan-chen-F) */
    double rho0;                /* reference density in Psi (Eq. eqn_ref_dens) */
    double sc_weight[2];        /* stencil weights for axis / diagonal links */
    double rho_init[2];         /* initial mean density per component */
    double noise_amp;           /* seeded init: rho = rho_init + U(-a, a) */
    double volume_fraction;     /* seeded init: alpha */
    double radius;              /* r_par, same for every particle */
    double particle_density;    /* m = rho_p 4/3 pi R^3 */
    double color;               /* particle colour Delta rho (Sec. IV) */
    double k_hertz;             /* K_Hertz (Eq. eq:hertz); the paper gives no value: parity unpinned */
    double lub_cut;             /* lubrication acts below this gap (2/3) */
    double lub_min;             /* gap at which it is clamped (1/10) */
    double mass_corr_c0;        /* C0 of Eq. masscorr; 0 = off */
    double body_force[3];       /* test-only acceleration on the fluid */
    int32_t vel_mode;           /* 0: Shan-Chen common velocity, 1: own velocity u^c */
    int32_t virtual_fluid;      /* 1: shell filled with virtual fluid (Sec. IV); 0: empty (Fig. 1b) */
    int32_t fixed_particles;    /* 1: particles never move (test-only) */
    int32_t pad_;
    uint64_t seed;
    double aspect;              /* spheroid: semi-axes R, R, aspect R about the body axis e; 1 = sphere */
    int32_t implicit_update;    /* 1: implicit particle velocity update (reading #18; spheres only) */
    int32_t pad2_;
} orc_params;

typedef struct orc_state orc_state;

typedef struct {
    int64_t step;
    double mass[2];
    double mom_fluid[3];
    double mom_part[3];
    double max_u;
    int64_t n_cover, n_uncover;
} orc_obs;

/* lattice tables (for tests) */
void orc_lattice(int32_t c[19][3], double w[19], int32_t opp[19]);
/* equilibrium, Eq. Equil */
void orc_feq(double rho, const double u[3], double out[19]);
/* SplitMix64: the n-th output (n = 0, 1, ...) of the generator seeded with s */
uint64_t orc_splitmix64(uint64_t s, uint64_t n);
double orc_unit(uint64_t s, uint64_t n);

/* NULL for implicit_update with a non-spherical particle shape */
orc_state* orc_create(const orc_params* p, int32_t n_particles);
void orc_destroy(orc_state* s);
int32_t orc_n_particles(const orc_state* s);

/* Seeded synthetic init: node noise + random sequential addition of spheres. */
int orc_init_from_seed(orc_state* s, uint64_t seed);
/* Init from macroscopic fields: rho[2][N], u[3][N] (may be NULL), particles
 * [np][9], owner_walls[N] (may be NULL; -2 marks a static wall node). */
int orc_init_fields(orc_state* s, const double* rho, const double* u,
                    const double* particles, const int32_t* walls);
int orc_step(orc_state* s, int32_t n);

/* Full state in canonical order; also the checkpoint format. */
void orc_get_state(const orc_state* s, double* f, int32_t* owner, double* particles, double meta[4]);
int orc_set_state(orc_state* s, const double* f, const int32_t* owner, const double* particles, const double meta[4]);
void orc_get_rho(const orc_state* s, double* rho);     /* rho[2][N]: sum of populations, 0 on solid */
void orc_get_forces(const orc_state* s, double* F, double* T); /* last step's particle F, T before MD */
void orc_set_particle_colors(orc_state* s, const double* colors);
/* body axes e[np][3] of the particles (unit vectors; (0,0,1) by default) */
void orc_get_axes(const orc_state* s, double* e);
void orc_set_axes(orc_state* s, const double* e);
/* test hooks for spheroids: inside test of a displacement d (minimum image)
 * for a particle with axis e; contact distance of two particles along r_hat.
 * Parity unpinned for the contact distance: the paper gives no contact law
 * for non-spherical particles.  The sum of the two support radii along the
 * line of centres is a reading, pinned only to its closed-form limits
 * (spheres: 2R; aligned spheroids: sums of semi-axes). */
int32_t orc_inside(const orc_params* p, const double d[3], const double e[3]);
double orc_contact_distance(const orc_params* p, const double rh[3], const double ep[3], const double eq[3]);
/* one rotational MD update of a free particle: omega (in/out), e (in/out), torque T */
void orc_rotate(const orc_params* p, double W[3], double e[3], const double T[3]);
void orc_observe(const orc_state* s, orc_obs* o);
/* per-step internals exposed for pins */
void orc_last_psi(const orc_state* s, double* psi);    /* Psi[2][N] of the last step */
void orc_last_sc_force(const orc_state* s, double* F); /* F^c[2][3][N] of the last step */
void orc_set_threads(int32_t n);
/* test hooks */
void orc_pair_force(const orc_params* p, const double Xp[3], const double Xq[3], const double Up[3],
                    const double Uq[3], double Fp[3]);
void orc_debug_remap(orc_state* s);

#endif
