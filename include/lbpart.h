/*
 * lbpart.h -- C ABI of the GB300 (sm_103a) library for the two-component
 * Shan-Chen D3Q19 BGK lattice Boltzmann fluid with suspended spherical
 * particles of Jansen & Harting, "From Bijels to Pickering emulsions: a
 * lattice Boltzmann study" (arXiv:1004.4414).
 *
 * What one time step computes (lb_step), in the paper's order:
 *   - particle remap: nodes a sphere newly covers lose their fluid and its
 *     momentum to the particle; nodes it uncovers are refilled with the mean
 *     density of their fluid neighbours at the surface velocity
 *     (Sec. III; Sec. IV, Eqs. eqn_rho_neu, eqn_ladd_vernichtenunderzeugen,
 *     optional Eq. masscorr);
 *   - virtual fluid on the outer solid shell with the particle colour
 *     (Sec. IV, the rho_new^r / rho_new^b equations);
 *   - Shan-Chen force with Psi = rho0 (1 - exp(-rho / rho0))
 *     (Eqs. eqn_shan-chen-F, eqn_ref_dens) and its sum on each particle
 *     (Eq. eqn_shan_chen_particle);
 *   - BGK collision with the cubic equilibrium at the shifted velocity
 *     (Eqs. eq:boltz, Equil, Sec. II), streaming with moving-wall
 *     bounce-back and momentum exchange (Eqs. eqn_bounce-back,
 *     eqn_ladd_bewegtewand);
 *   - particle MD with Hertz contact and lubrication, leap-frog
 *     (Eqs. eq:hertz, eqn_ladd_lubrikation, Sec. III).
 *
 * Conventions
 *   - Every call returns LB_OK (0) or a negative LB_E* code; no call aborts
 *     or prints.  lb_strerror gives a text.
 *   - Node index n = x + nx*(y + ny*z); populations f[c][i][n] with
 *     c = 0 red, 1 blue and the direction order 0 rest; 1..6 = +x,-x,+y,-y,
 *     +z,-z; 7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),
 *     (-1,0,-1),(+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 *   - Particles: 9 doubles each, X[3], U[3], omega[3]; particle indices are
 *     per box, 0..n_particles-1.  owner[n] = -1 fluid, -2 static wall,
 *     p >= 0 solid node of particle p.
 *   - Host pointers are plain host memory (pageable or pinned); the library
 *     copies what it needs before the call returns unless stated otherwise.
 *   - A handle is not thread-safe; one host thread drives it at a time.
 *   - All device work is ordered on the CUDA stream given to lb_create: the
 *     handle's own second streams (state copies, the MD pair forces) fork
 *     from it and join it again within the same call or step.
 */
#ifndef LBPART_H
#define LBPART_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define LB_OK 0
#define LB_EINVAL (-1)     /* invalid argument or configuration */
#define LB_ENOMEM (-2)     /* workspace too small */
#define LB_ECUDA (-3)      /* a CUDA runtime call failed */
#define LB_EUNSTABLE (-4)  /* device detected a non-finite density or |u| >= 0.5 */
#define LB_EPLACE (-5)     /* random sequential addition could not place the spheres */
#define LB_ETIMEOUT (-6)   /* reserved: a bounded device wait gave up */
#define LB_EOVERFLOW (-7)  /* a fixed-capacity device list overflowed */

/* population storage (the collision always runs in FP32, or FP64 for LB_FP64) */
#define LB_FP64 0      /* FP64 populations and arithmetic (parity mode) */
#define LB_FP32 1      /* FP32 populations and arithmetic */
#define LB_FP16_DEV 2  /* f_i (i>0) stored as FP16 deviations (f_i - zeta_i rho_ref)/zeta_i, density FP32 */
#define LB_BF16_DEV 3  /* as LB_FP16_DEV with BF16 */

/* One periodic box.  Densities follow the paper's symbols. */
typedef struct {
    int32_t nx, ny, nz;          /* lattice size, each >= 1 */
    int32_t n_particles;         /* exact particle count (<= N); < 0: round(volume_fraction N / (4/3 pi R^3)) */
    double tau[2];               /* BGK relaxation times tau^r, tau^b (> 1/2) */
    double g_br;                 /* Shan-Chen coupling g_br = g_rb; g_rr = g_bb = 0 */
    double rho0;                 /* reference density of Psi */
    double sc_weight[2];         /* link weights of the force stencil: axis, diagonal */
    double rho_init[2];          /* mean initial density per component */
    double noise_amp;            /* seeded init: rho^c = rho_init^c + U(-a, a) per node (a >= 0) */
    double volume_fraction;      /* alpha in [0, 1), used when n_particles < 0 */
    double radius;               /* sphere radius r_par (all particles); for spheroids the equatorial semi-axis R */
    double particle_density;     /* m = rho_p 4/3 pi R^3 (spheroids: R^2 c), J = 2/5 m R^2 */
    double color;                /* particle colour Delta rho; used when contact_angle_deg is NaN */
    double contact_angle_deg;    /* if finite: Delta rho = (theta - 90) / 442 (fit of Fig. 4b) */
    double k_hertz;              /* K_Hertz of Eq. eq:hertz (>= 0) */
    double lub_cut;              /* lubrication below this gap (> lub_min) */
    double lub_min;              /* gap where lubrication is clamped (> 0) */
    double mass_corr_c0;         /* C0 of Eq. masscorr (>= 0; 0 = off) */
    double body_force[3];        /* uniform acceleration of the fluid (tests; 0 in the paper's runs) */
    int32_t vel_mode;            /* 0: Shan-Chen common velocity in f^eq, 1: each component's own velocity */
    int32_t fixed_particles;     /* 1: particles keep X, U, omega (prescribed motion; tests) */
    int32_t precision;           /* LB_FP64 / LB_FP32 / LB_FP16_DEV / LB_BF16_DEV, same for all boxes */
    int32_t implicit_update;     /* 0: the paper's explicit particle velocity update (Sec. III); 1: the
                                    moving-wall term of the links taken at the new velocity, (M + Z) dV =
                                    (F, T) with Z the links' drag tensor, and the fluid given the same
                                    change, which keeps momentum exact (a reading; needed for light
                                    particles in contact, e.g. density 1 in fluid of density 0.7);
                                    spheres only */
    double aspect;               /* particle shape: 0 or 1 sphere; otherwise a spheroid with semi-axes
                                    R, R, c = aspect R about a body axis (0.1 <= aspect <= 10); see lb_set_axes */
} lb_params;

/* Observables of one box (lb_observables). */
typedef struct {
    int64_t step;                /* time steps taken since init */
    double mass[2];              /* sum of the densities rho^c over fluid nodes, per component */
    double mom_fluid[3];         /* sum over fluid nodes of sum_c sum_i f_i c_i */
    double mom_part[3];          /* sum over particles of m U (0 when particles are fixed) */
    double max_u;                /* max over fluid nodes of |j| / rho (both components) */
    int64_t n_cover, n_uncover;  /* cover / uncover events since init */
    int64_t n_fluid, n_solid;    /* current node counts */
    int32_t error;               /* sticky device error (LB_OK or LB_E*) */
    int32_t n_particles;
    double L[3];                 /* domain size L_i = 2 pi / sqrt(<k_i^2>) (Sec. VI, Eq. eq:domsize): <k_i^2>
                                    the second moment along axis i of the structure function
                                    S(k) = |phi'_k|^2 / N of phi = rho^r - rho^b (0 on solid nodes),
                                    phi' = phi - <phi>; NaN for a uniform phi */
    double coverage;             /* fraction of the box's particles whose fluid D3Q19 neighbours (the fluid
                                    nodes linked to their solid nodes) include phi > 0 and phi < 0; the
                                    paper names the interface coverage but does not define it, this is
                                    the reading used; 0 without particles */
} lb_obs;

typedef struct lb_handle lb_handle;

/* Device workspace needed for n_boxes boxes: bytes out.  LB_EINVAL on bad
 * parameters: a value outside the range stated in lb_params, a non-finite
 * real (contact_angle_deg excepted; volume_fraction only when it is used),
 * or mixed precisions.  The caller allocates it (e.g. torch.empty on the device) and
 * keeps it alive until lb_destroy; the library never allocates device
 * memory for the lattice. */
int lb_workspace_bytes(const lb_params* boxes, int32_t n_boxes, size_t* bytes);

/* Create a handle for n_boxes independent boxes stepped together (the
 * batched sweep).  d_workspace: device pointer, 256-byte aligned, at least
 * lb_workspace_bytes bytes.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  The parameters are copied.  No state is initialised
 * until lb_init_from_seed / lb_init_fields / lb_import_state. */
int lb_create(const lb_params* boxes, int32_t n_boxes, void* d_workspace, size_t bytes,
              void* cuda_stream, lb_handle** out);

/* Seeded synthetic initial state of every box (box b uses seed + b):
 * particles by random sequential addition (minimum-image centre distance
 * >= 2R, for spheroids twice the bounding radius; at most 10^6 candidates,
 * LB_EPLACE otherwise; spheroid axes from stream 3), node densities
 * rho_init^c + U(-a, a), f = f^eq(rho, 0) on fluid nodes.  The random
 * numbers come from SplitMix64 (Steele, Lea & Flood 2014): stream k of seed
 * s is seeded with output k of SplitMix64(s); stream 0 places spheres
 * (three draws per candidate centre), stream 1 + c gives the noise of
 * component c at node n (its n-th output).  Synchronous. */
int lb_init_from_seed(lb_handle* h, uint64_t seed);

/* Initial state of one box from macroscopic fields (host arrays):
 * rho[2][N], u[3][N] (NULL: fluid at rest), particles[n_particles][9],
 * walls[N] (NULL: none; -2 marks a static wall node).  f = f^eq(rho, u) on
 * fluid nodes; nodes inside a particle (within R of a sphere's centre, or
 * inside a spheroid with the axes of lb_set_axes) are solid.  Synchronous. */
int lb_init_fields(lb_handle* h, int32_t box, const double* rho, const double* u,
                   const double* particles, const int32_t* walls);

/* Advance every box by n >= 0 steps; asynchronous on the stream (CUDA-graph
 * replays).  Returns launch errors, or the sticky device error seen by an
 * earlier call that has completed. */
int lb_step(lb_handle* h, int64_t n);

/* Wait for the stream; return the sticky device error (LB_OK if none). */
int lb_sync(lb_handle* h);

/* Observables of one box; synchronises the stream.  The domain size and the
 * coverage are computed on the device: one FP64 mixed-radix FFT per lattice
 * line and axis (Parseval reduces the three-dimensional moment to line
 * transforms; any box size, lines longer than 2048 nodes are slower), about
 * 10 ms for a 256^3 box, so call it between steps, not every step. */
int lb_observables(lb_handle* h, int32_t box, lb_obs* out);

/* The order parameter phi = rho^r - rho^b of one box (Sec. VI; 0 on solid
 * nodes), phi[N] in canonical node order (host array, may be NULL), with
 * the domain size L[3] and the coverage of lb_observables (either may be
 * NULL).  LB_EINVAL before an init.  Synchronises the stream. */
int lb_export_phi(lb_handle* h, int32_t box, double* phi, double* L, double* coverage);

/* Full state of one box in canonical order (host arrays, any may be NULL):
 * f[2][19][N] FP64 (0 on solid nodes), owner[N], particles[np][9],
 * meta[4] = {step, initial mass red, initial mass blue, n_particles}.
 * The device keeps each fluid node's density rho^c and its 18 moving
 * populations; the exported rest population is rho^c - sum_{i>0} f_i
 * (so after lb_import_state it returns to within rounding).
 * Synchronises the stream. */
int lb_export_state(lb_handle* h, int32_t box, double* f, int32_t* owner, double* particles,
                    double* meta);

/* Replace the state of one box (same layout as lb_export_state; f, owner,
 * particles and meta are required).  Each fluid node's density becomes the
 * sum of its 19 imported populations.  An owner entry outside [-2,
 * n_particles) returns LB_EINVAL before anything of the box changes.
 * Spheroid axes are not part of this format: a box that was stepped keeps
 * its current axes, otherwise those of the last lb_set_axes.  Host-device
 * copies overlap the per-direction conversion (two staging halves, a second
 * stream).  Synchronous. */
int lb_import_state(lb_handle* h, int32_t box, const double* f, const int32_t* owner,
                    const double* particles, const double* meta);

/* State of one box in the handle's storage format, for checkpoints that
 * skip the conversion to FP64 and move half (FP32 storage) or a quarter
 * (16-bit storage) of lb_export_state's population bytes.  state (host,
 * lb_state_native_bytes bytes): the 18 stored population pairs of every
 * node exactly as the device holds them for the current step (in-place
 * streaming order, so the bytes depend on the step's parity), then the
 * density field rho^c of the current step.  owner and particles as in
 * lb_export_state (either may be NULL); meta[LB_NATIVE_META]: step, the two
 * initial component masses, n_particles, the storage type (lb_params
 * precision), the node count, and the fluid mass of each component that
 * the current step starts from.  LB_EINVAL before an init or for a wrong
 * byte count.  Pinned host buffers give the full host-link rate.
 * Synchronises the stream. */
#define LB_NATIVE_META 8
int lb_state_native_bytes(lb_handle* h, int32_t box, size_t* bytes);
int lb_export_state_native(lb_handle* h, int32_t box, void* state, size_t bytes, int32_t* owner,
                           double* particles, double* meta);

/* Replace the state of one box from lb_export_state_native of a box with
 * the same parameters (state, owner, particles and meta are required): the
 * bytes are copied back as they are.  The particle shell, cell and
 * neighbour lists are rebuilt, so stepping on agrees with the exporting run
 * up to the summation order of the particle forces.
 * LB_EINVAL for a byte count, storage type or node count that differs from
 * this box's, and, before anything of the box changes, for an owner entry
 * outside [-2, n_particles).  Synchronous. */
int lb_import_state_native(lb_handle* h, int32_t box, const void* state, size_t bytes,
                           const int32_t* owner, const double* particles, const double* meta);

/* Densities rho[2][N] of one box (rho^c = sum of the populations on fluid
 * nodes, 0 on solid nodes). */
int lb_export_rho(lb_handle* h, int32_t box, double* rho);

/* Per-particle colour Delta rho of one box (host array of n_particles).
 * lb_init_from_seed, lb_init_fields, lb_import_state and
 * lb_import_state_native give every particle the box colour, so call this
 * after them. */
int lb_set_particle_colors(lb_handle* h, int32_t box, const double* colors);

/* Body axes of the particles of one box, e[n_particles][3] unit vectors
 * (spheroids; spheres ignore them).  The paper's coupling is written for any
 * particle shape (Secs. I and III); for spheroids the node claims use the
 * spheroid inside test, the contact laws the distance at which the surfaces
 * meet along the line of centres, and the MD turns the axis about the
 * angular momentum (exact for torque-free motion).  lb_init_from_seed draws
 * the axes (stream 3 of the box seed); lb_init_fields uses the last axes set
 * here ((0, 0, 1) by default), so call lb_set_axes before it; after an init
 * it also updates the running state.  lb_get_axes reads the current axes.
 * LB_EINVAL for a vector whose length differs from 1 by 1e-6 or more.
 * Synchronise. */
int lb_set_axes(lb_handle* h, int32_t box, const double* e);
int lb_get_axes(lb_handle* h, int32_t box, double* e);

/* Fluid-coupling force and torque on each particle of one box in the last
 * step (momentum exchange, cover/uncover, Shan-Chen), before the MD pair
 * forces: F[np][3], T[np][3].  Synchronises. */
int lb_particle_forces(lb_handle* h, int32_t box, double* F, double* T);

/* Number of particles and lattice nodes of a box. */
int lb_box_info(lb_handle* h, int32_t box, int32_t* n_particles, int64_t* n_nodes);

/* Block shape of the fused step kernel, used by the autotuner.  split = 0:
 * one thread per node, ty rows of 32 nodes per CTA (4, 8 or 16).  split = 1:
 * one thread per node and component (the two components on the two halves
 * of a warp), ty rows of 16 nodes per CTA (8 or 16).  cz planes are marched
 * per CTA (>= 1).  Both give the same results to rounding order.  Rebuilds
 * the launch plan and graphs; other values return LB_EINVAL. */
int lb_set_tiling(lb_handle* h, int32_t ty, int32_t cz, int32_t split);

/* Kernel timing.  When enabled, lb_step launches the kernels one by one and
 * brackets every launch of the fused stream-collide kernel with CUDA events
 * on the handle's stream; lb_kernel_time returns the summed milliseconds and
 * the launch count since the last reset and resets them.  Synchronises. */
int lb_set_profiling(lb_handle* h, int32_t on);
int lb_kernel_time(lb_handle* h, double* ms_fused, int64_t* launches_fused, int64_t* launches_total);

/* Phase times of the steps measured by the last lb_kernel_time (profiling
 * mode: CUDA events at every phase boundary, kernels launched one by one):
 * ms[k] for the first n of the LB_NPHASES phases of a step, in order
 *   0 cell and neighbour lists, 1 remap detection, 2 cover / uncover
 *   (marks, refills, shell flags), 3 shell virtual densities, 4 fused
 *   stream-collide kernel, 5 coupling pass (links, momentum exchange,
 *   Shan-Chen force on the particles), 6 MD velocity and position update.
 * The MD pair forces run on a second stream of the handle beside phases
 * 1-5 and are counted in none of them.
 * Each phase also carries its share of launch gaps. */
#define LB_NPHASES 7
int lb_phase_times(lb_handle* h, double* ms, int32_t n);

/* Destroy the handle (does not free the caller's workspace). */
void lb_destroy(lb_handle* h);

/* Field sums of a population field held on the device, computed without
 * allocating any memory.  The paper has no counterpart to this call; it is
 * for callers that cannot allocate device memory at the point of the call,
 * such as a monitor run between the steps of a long job: cudaMalloc and
 * cudaFree can synchronise the whole device and can fail once the job has
 * committed nearly all device memory.  It calls no allocating routine.
 *
 * d_f      device, f[2][19][n_nodes] FP64 in the layout of lb_export_state
 *          (populations of solid nodes are ignored); caller-owned.
 * d_owner  device, owner[n_nodes] int32 as in lb_export_state (-1 fluid,
 *          anything else solid); caller-owned.
 * n_nodes  0 <= n_nodes <= LB_FIELD_MOMENTS_MAX_NODES (2^27 = 512^3);
 *          larger sizes return LB_EINVAL without touching the device.
 * stream   cudaStream_t to run on (NULL: the legacy default stream).
 * d_out    device, 8 doubles, caller-owned: {mass_r, mass_b, j_x, j_y, j_z,
 *          max |j|/rho, n_fluid, n_solid} -- the same sums lb_observables
 *          reports as mass, mom_fluid, max_u, n_fluid and n_solid.
 *
 * Asynchronous on the stream: read d_out after synchronising it.  Pointers
 * that are not device memory of the current device, or misaligned, return
 * LB_EINVAL; launch failures return LB_ECUDA.
 *
 * Scratch: the library holds one fixed array of LB_FIELD_MOMENTS_MAX_BLOCKS
 * partial sums (256 KB) on every device that loads it, until the process
 * exits.  Every call shares that array and overwrites what the previous call
 * left there, so calls that overlap on the GPU (on different streams, or
 * from different host threads) race and give wrong sums: serialise them.
 * The first call on each device looks up the array's device address with
 * the device current; make that first call before any stream capture. */
#define LB_FIELD_MOMENTS_MAX_BLOCKS 1024
#define LB_FIELD_MOMENTS_MAX_NODES 134217728LL
int lb_field_moments(const double* d_f, const int32_t* d_owner, int64_t n_nodes, void* stream, double* d_out);

const char* lb_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
